// LBVH construction on the GPU.  Not part of the paper (Sionna RT relies on
// Mitsuba's acceleration structure); the tree is the binary radix tree of
// Karras, "Maximizing parallelism in the construction of BVHs, octrees and
// k-d trees" (HPG 2012), over 63-bit Morton codes of the doubled triangle
// centroids, with duplicate keys ordered by their sorted position.
//
// Every floating-point step that decides an integer (the Morton quantisation)
// uses explicitly rounded FP32 intrinsics, and every min / max is the
// comparison-select (b < a ? b : a), so the tree is identical bit for bit on
// any run and to any other IEEE implementation of the same definition.
//
// Node layout (64 bytes = 4 x float4) of internal node i:
//   [0] lo0.x lo0.y lo0.z hi0.x   [1] hi0.y hi0.z lo1.x lo1.y
//   [2] lo1.z hi1.x hi1.y hi1.z   [3] child0 child1 (int bits) 0 0
// Triangles whose largest AABB extent is at least a quarter of the scene's
// (the ground of a city; at most 16 of them) stay out of the tree: they sort
// last (key 2^64 - 1) and the tracer tests them from a short list, so their
// huge boxes do not inflate every node on their path to the root.
// child >= 0: internal node; child < 0: leaf ~p, the triangle at sorted
// position p, whose 48-byte record is trirec[3p .. 3p+2]:
//   [0] a.x a.y a.z b.x   [1] b.y b.z c.x c.y   [2] c.z mat(int) orig(int) 0
#include <algorithm>

#include "common.cuh"

namespace rmsbr {
namespace {

constexpr int MAX_LARGE = MAX_LARGE_TRIS;
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int SORT_WARPS = SORT_THREADS / 32;

__device__ __forceinline__ float fmin_sel(float a, float b) { return (b < a) ? b : a; }
__device__ __forceinline__ float fmax_sel(float a, float b) { return (a < b) ? b : a; }

__global__ void k_check_indices(const int32_t* tris, const int32_t* tri_mat, int64_t nt, int64_t nv,
                                int32_t nm, int32_t* flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    bool bad = false;
    for (int j = 0; j < 3; ++j) {
        int32_t v = tris[3 * i + j];
        bad |= (v < 0) || ((int64_t)v >= nv);
    }
    int32_t m = tri_mat[i];
    bad |= (m < 0) || (m >= nm);
    if (bad) atomicOr(flag, 1);
}

// Per-triangle AABB and doubled centroid c2 = lo + hi; per-block scene bounds
// (min of the lower and max of the upper AABB corners).
__global__ void k_tri_aabb(const float* __restrict__ verts, const int32_t* __restrict__ tris, int64_t nt,
                           float* __restrict__ aabb, float* __restrict__ c2, float* __restrict__ blk) {
    __shared__ float smin[3][256], smax[3][256];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + tid;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < nt) {
        const int32_t i0 = tris[3 * i], i1 = tris[3 * i + 1], i2 = tris[3 * i + 2];
        for (int a = 0; a < 3; ++a) {
            const float v0 = verts[3 * (int64_t)i0 + a], v1 = verts[3 * (int64_t)i1 + a],
                        v2 = verts[3 * (int64_t)i2 + a];
            const float lo = fmin_sel(v0, fmin_sel(v1, v2));
            const float hi = fmax_sel(v0, fmax_sel(v1, v2));
            const float c = __fadd_rn(lo, hi);
            aabb[6 * i + a] = lo;
            aabb[6 * i + 3 + a] = hi;
            c2[3 * i + a] = c;
            mn[a] = lo;
            mx[a] = hi;
        }
    }
    for (int a = 0; a < 3; ++a) { smin[a][tid] = mn[a]; smax[a][tid] = mx[a]; }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s)
            for (int a = 0; a < 3; ++a) {
                smin[a][tid] = fmin_sel(smin[a][tid], smin[a][tid + s]);
                smax[a][tid] = fmax_sel(smax[a][tid], smax[a][tid + s]);
            }
        __syncthreads();
    }
    if (tid == 0)
        for (int a = 0; a < 3; ++a) { blk[6 * blockIdx.x + a] = smin[a][0]; blk[6 * blockIdx.x + 3 + a] = smax[a][0]; }
}

__global__ void k_minmax_final(const float* __restrict__ blk, int nblk, float* __restrict__ out) {
    __shared__ float smin[3][256], smax[3][256];
    const int tid = threadIdx.x;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = tid; b < nblk; b += 256)
        for (int a = 0; a < 3; ++a) { mn[a] = fmin_sel(mn[a], blk[6 * b + a]); mx[a] = fmax_sel(mx[a], blk[6 * b + 3 + a]); }
    for (int a = 0; a < 3; ++a) { smin[a][tid] = mn[a]; smax[a][tid] = mx[a]; }
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (tid < s)
            for (int a = 0; a < 3; ++a) {
                smin[a][tid] = fmin_sel(smin[a][tid], smin[a][tid + s]);
                smax[a][tid] = fmax_sel(smax[a][tid], smax[a][tid + s]);
            }
        __syncthreads();
    }
    if (tid == 0)
        for (int a = 0; a < 3; ++a) { out[a] = smin[a][0]; out[3 + a] = smax[a][0]; }
}

__device__ __forceinline__ float extent3(const float* lo, const float* hi) {
    return fmax_sel(fmax_sel(__fsub_rn(hi[0], lo[0]), __fsub_rn(hi[1], lo[1])), __fsub_rn(hi[2], lo[2]));
}

// Large triangles: largest AABB extent >= 0.25 x the scene's largest extent.
// They are kept out of the tree (tested from a short list) when there are at
// most MAX_LARGE of them; the count (in device memory) decides that.
__global__ void k_flag_large(const float* __restrict__ aabb, const float* __restrict__ sb, int64_t nt,
                             int8_t* __restrict__ large, int32_t* __restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const float thr = __fmul_rn(0.25f, extent3(sb, sb + 3));
    const bool l = extent3(aabb + 6 * i, aabb + 6 * i + 3) >= thr;
    large[i] = l ? 1 : 0;
    if (l) atomicAdd(count, 1);
}

// per-block min / max of the doubled centroids of the triangles that stay in the tree
// the large-triangle list is used when 1..MAX_LARGE triangles are large (decided on the device)
__device__ __forceinline__ bool use_large_list(const int32_t* count) {
    const int32_t c = *count;
    return c > 0 && c <= MAX_LARGE;
}
__device__ __forceinline__ int64_t tree_size(const int32_t* count, int64_t n) {
    return use_large_list(count) ? n - *count : n;
}

__global__ void k_c2_bounds(const float* __restrict__ c2, const int8_t* __restrict__ large,
                            const int32_t* __restrict__ count, int64_t nt, float* __restrict__ blk) {
    const bool use_large = use_large_list(count);
    __shared__ float smin[3][256], smax[3][256];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + tid;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (i < nt && !(use_large && large[i]))
        for (int a = 0; a < 3; ++a) { mn[a] = c2[3 * i + a]; mx[a] = c2[3 * i + a]; }
    for (int a = 0; a < 3; ++a) { smin[a][tid] = mn[a]; smax[a][tid] = mx[a]; }
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (tid < st)
            for (int a = 0; a < 3; ++a) {
                smin[a][tid] = fmin_sel(smin[a][tid], smin[a][tid + st]);
                smax[a][tid] = fmax_sel(smax[a][tid], smax[a][tid + st]);
            }
        __syncthreads();
    }
    if (tid == 0)
        for (int a = 0; a < 3; ++a) { blk[6 * blockIdx.x + a] = smin[a][0]; blk[6 * blockIdx.x + 3 + a] = smax[a][0]; }
}

// spread the low 21 bits of v to every third bit of a 64-bit word
__device__ __forceinline__ uint64_t spread21(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffULL;
    x = (x | x << 16) & 0x1f0000ff0000ffULL;
    x = (x | x << 8) & 0x100f00f00f00f00fULL;
    x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
    x = (x | x << 2) & 0x1249249249249249ULL;
    return x;
}

// One scale for the three axes, so that the Morton order splits space
// isotropically (a flat city does not spend a third of its top splits on height):
// e = max_a (cmax_a - cmin_a),  q_a = min(trunc((c2_a - cmin_a) * (2097151 / e)), 2097151)
// key = interleave(qx, qy, qz) with x on bit 3i+2, y on 3i+1, z on 3i.
__global__ void k_morton(const float* __restrict__ c2, const float* __restrict__ bounds, int64_t nt,
                         const int8_t* __restrict__ large, const int32_t* __restrict__ count,
                         uint64_t* __restrict__ keys, int32_t* __restrict__ vals) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const bool use_large = use_large_list(count);
    vals[i] = (int32_t)i;
    if (use_large && large[i]) {  // after every Morton code: the large triangles end the sorted order
        keys[i] = ~0ULL;
        return;
    }
    const float e = extent3(bounds, bounds + 3);
    const float scale = (e > 0.0f) ? __fdiv_rn(2097151.0f, e) : 0.0f;
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        const float f = __fmul_rn(__fsub_rn(c2[3 * i + a], bounds[a]), scale);
        const uint32_t u = __float2uint_rz(f);
        q[a] = u > 2097151u ? 2097151u : u;
    }
    keys[i] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
}

// ---------------- stable LSD radix sort of (key, value), 8-bit digits ----------------
__global__ void k_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
                       int nblk) {
    __shared__ uint32_t s_h[256];
    const int tid = threadIdx.x;
    s_h[tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const int64_t idx = base + (int64_t)j * SORT_THREADS + tid;
        if (idx < n) atomicAdd(&s_h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)tid * nblk + blockIdx.x] = s_h[tid];
}

// exclusive scan of hist[0 .. total) in place (one block of 1024 threads)
__global__ void k_scan(uint32_t* __restrict__ hist, int64_t total) {
    __shared__ uint32_t s[1024];
    const int tid = threadIdx.x;
    const int64_t len = (total + 1023) / 1024;
    const int64_t b = (int64_t)tid * len, e = min(total, b + len);
    uint32_t sum = 0;
    for (int64_t i = b; i < e; ++i) sum += hist[i];
    s[tid] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = (tid >= off) ? s[tid - off] : 0u;
        __syncthreads();
        s[tid] += v;
        __syncthreads();
    }
    uint32_t run = s[tid] - sum;  // exclusive prefix of this chunk
    for (int64_t i = b; i < e; ++i) {
        uint32_t v = hist[i];
        hist[i] = run;
        run += v;
    }
}

__global__ void k_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin, int64_t n,
                          int shift, const uint32_t* __restrict__ offs, int nblk, uint64_t* __restrict__ kout,
                          int32_t* __restrict__ vout) {
    __shared__ uint32_t s_wc[SORT_WARPS][256];
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_base[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    s_run[tid] = 0;
    s_base[tid] = offs[(int64_t)tid * nblk + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    for (int r = 0; r < SORT_ITEMS; ++r) {
        for (int j = tid; j < SORT_WARPS * 256; j += SORT_THREADS) (&s_wc[0][0])[j] = 0;
        __syncthreads();
        const int64_t idx = base + (int64_t)r * SORT_THREADS + tid;
        const bool valid = idx < n;
        uint64_t key = 0;
        int32_t val = 0;
        uint32_t d = 256;
        if (valid) {
            key = kin[idx];
            val = vin[idx];
            d = (uint32_t)((key >> shift) & 255u);
        }
        const unsigned peers = __match_any_sync(FULL_MASK, d);
        const int rank = __popc(peers & lt);
        if (valid && rank == 0) s_wc[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t off = s_run[d];
            for (int w = 0; w < warp; ++w) off += s_wc[w][d];
            const uint32_t dst = s_base[d] + off + rank;
            kout[dst] = key;
            vout[dst] = val;
        }
        __syncthreads();
        uint32_t tot = 0;
        for (int w = 0; w < SORT_WARPS; ++w) tot += s_wc[w][tid];
        s_run[tid] += tot;
        __syncthreads();
    }
}

// ---------------- one-block sort of small meshes ----------------
// Bitonic sort of (key, position) pairs in shared memory: ordering by the pair
// is the stable order by key, so the result equals the radix sort's.  One
// launch instead of 24 for meshes of at most SMALL_SORT triangles.
constexpr int SMALL_SORT = 2048;
__global__ void __launch_bounds__(1024) k_sort_small(uint64_t* __restrict__ keys, int32_t* __restrict__ vals,
                                                     int n) {
    __shared__ uint64_t sk[SMALL_SORT];
    __shared__ int32_t sv[SMALL_SORT];
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        sk[i] = i < n ? keys[i] : ~0ULL;
        sv[i] = i < n ? vals[i] : INT32_MAX;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));   // lower element of the pair
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const uint64_t ki = sk[i], kj = sk[j];
                const int32_t vi = sv[i], vj = sv[j];
                const bool gt = ki > kj || (ki == kj && vi > vj);
                if (gt == up) {
                    sk[i] = kj; sk[j] = ki;
                    sv[i] = vj; sv[j] = vi;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        keys[i] = sk[i];
        vals[i] = sv[i];
    }
}

// ---------------- Karras hierarchy ----------------
__device__ __forceinline__ int delta(const uint64_t* __restrict__ k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    const uint64_t a = k[i], b = k[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

__global__ void k_karras(const uint64_t* __restrict__ k, int64_t nt, const int32_t* __restrict__ count,
                         float4* __restrict__ nodes, int32_t* __restrict__ parent_leaf,
                         int32_t* __restrict__ parent_node) {
    const int64_t n = tree_size(count, nt);   // the tree covers sorted positions [0, n)
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (delta(k, n, i, i + 1) - delta(k, n, i, i - 1)) > 0 ? 1 : -1;
    const int dmin = delta(k, n, i, i - d);
    int64_t lmax = 2;
    while (delta(k, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(k, n, i, i + (l + t) * d) > dmin) l += t;
    const int64_t j = i + l * d;
    const int dnode = delta(k, n, i, j);
    int64_t s = 0;
    int64_t div = 2;
    int64_t t = (l + div - 1) / div;
    while (true) {
        if (delta(k, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
        div <<= 1;
        t = (l + div - 1) / div;
    }
    const int64_t g = i + s * d + (d < 0 ? -1 : 0);
    const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    const int32_t c0 = (lo == g) ? ~(int32_t)g : (int32_t)g;
    const int32_t c1 = (hi == g + 1) ? ~(int32_t)(g + 1) : (int32_t)(g + 1);
    nodes[4 * i + 3] = make_float4(__int_as_float(c0), __int_as_float(c1), 0.0f, 0.0f);
    if (c0 < 0) parent_leaf[g] = (int32_t)i; else parent_node[g] = (int32_t)i;
    if (c1 < 0) parent_leaf[g + 1] = (int32_t)i; else parent_node[g + 1] = (int32_t)i;
}

// Bottom-up refit: each leaf writes its triangle box into its parent's
// child slot; the second child to arrive at a node (atomic visit counter)
// forms the node's box and carries on upward.  No thread ever waits.
__global__ void k_refit(const float* __restrict__ tri_aabb, const int32_t* __restrict__ order, int64_t nt,
                        const int32_t* __restrict__ count, const int32_t* __restrict__ parent_leaf,
                        const int32_t* __restrict__ parent_node, float4* nodes, int32_t* visit) {
    const int64_t n = tree_size(count, nt);
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < 2 || p >= n) return;
    float box[6];
    const int32_t tri = order[p];
    for (int a = 0; a < 6; ++a) box[a] = tri_aabb[6 * (int64_t)tri + a];
    int32_t me = ~(int32_t)p;
    int32_t node = parent_leaf[p];
    float* nf = reinterpret_cast<float*>(nodes);
    // the path to the root of a valid tree is shorter than n nodes
    for (int64_t step = 0; step < n; ++step) {
        const float4 c = __ldcg(&nodes[4 * (int64_t)node + 3]);
        const int slot = (__float_as_int(c.x) == me) ? 0 : 1;
        float* dst = nf + 16 * (int64_t)node + 6 * slot;
        for (int a = 0; a < 6; ++a) __stcg(dst + a, box[a]);
        __threadfence();
        if (atomicAdd(&visit[node], 1) == 0) return;
        __threadfence();
        const float* src = nf + 16 * (int64_t)node;
        float lb[6], rb[6];
        for (int a = 0; a < 6; ++a) { lb[a] = __ldcg(src + a); rb[a] = __ldcg(src + 6 + a); }
        for (int a = 0; a < 3; ++a) {
            box[a] = fmin_sel(lb[a], rb[a]);
            box[3 + a] = fmax_sel(lb[3 + a], rb[3 + a]);
        }
        if (node == 0) return;
        me = node;
        node = parent_node[node];
    }
}

__global__ void k_trirec(const float* __restrict__ verts, const int32_t* __restrict__ tris,
                         const int32_t* __restrict__ tri_mat, const int32_t* __restrict__ order, int64_t n,
                         float4* __restrict__ rec) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int32_t t = order[p];
    const float* a = verts + 3 * (int64_t)tris[3 * (int64_t)t];
    const float* b = verts + 3 * (int64_t)tris[3 * (int64_t)t + 1];
    const float* c = verts + 3 * (int64_t)tris[3 * (int64_t)t + 2];
    rec[3 * p + 0] = make_float4(a[0], a[1], a[2], b[0]);
    rec[3 * p + 1] = make_float4(b[1], b[2], c[0], c[1]);
    rec[3 * p + 2] = make_float4(c[2], __int_as_float(tri_mat[t]), __int_as_float(t), 0.0f);
}

// ---------------- binned-SAH tree, top down, level by level ----------------
// The same leaves as the LBVH (one triangle per leaf, the large triangles out
// of the tree) under splits that minimise the surface-area heuristic
// (MacDonald & Booth 1990) over 32 centroid bins per axis (Wald 2007).
// Definition, for a range [lo, hi) of positions at depth d, in the Morton
// order to start with (FP32 rounded to nearest, no fused operations, left
// to right):
//   cl, ch = min / max of the doubled centroids c2 over the range;
//   axis a is binned if d < SAH_DEPTH_CAP, e = ch_a - cl_a > 0 and
//   k = 32 / e is finite; bin(t) = min(31, trunc((c2_a(t) - cl_a) k));
//   split b in 1..31: bins < b left; cost = H(L) nL + H(R) nR with
//   H = dx dy + dy dz + dz dx of the side's AABB, its extents scaled by
//   s = 2^-E, max_a e_a = f 2^E with f in [0.5, 1) (exact, so neither an
//   overflow nor a different rounding at any scale; skipped if a side is empty);
//   the first minimum over (a = 0..2, b = 1..31) wins; stable partition,
//   mid = lo + nL; no binned axis: mid = lo + (hi - lo) / 2, order kept.
// Node numbers: the node split at mid is g = mid - 1 (distinct for every
// node), the root is 0 and the node with g = 0 takes the root's g.  The
// child boxes come from the LBVH's refit afterwards.
//
// Level L holds the ranges at depth L, each with its centroid bounds (the
// root's are the Morton bounds; a split computes its children's while it
// partitions).  A range reads its positions from buffer L & 1 and writes
// its stable partition to the other buffer; a child of one position writes
// the final order.  Ranges of at most SAH_BIG positions are split by one
// warp each (bins, sweep, partition); larger ones by every block together in
// chunks of SAH_CHUNK positions: plan (chunk bases, cleared bins), bin (per
// chunk histograms merged into the range's bins), decide (sweep, split, each
// chunk's left offset from its histograms), scatter (partition, children's
// centroid bounds); the next level's plan writes their nodes and children.
constexpr int SAH_BINS = 32;
constexpr int SAH_NB3 = 3 * SAH_BINS;
constexpr int SAH_DEPTH_CAP = 32;     // from this depth on: middle splits (depth <= 32 + log2 n)
constexpr int SAH_BIG = 2048;         // larger ranges: chunked over all blocks; others: one warp
constexpr int SAH_CHUNK = 4096;
constexpr int SAH_BLOCK = 512;        // threads of the chunk kernels
constexpr int SAH_PLAN = 1024;        // threads of the plan kernel (one block)
constexpr int SAH_WARPS = 8;          // warps per block of the warp kernel

struct SahTask {
    int32_t lo, hi, parent, meta;     // meta = depth << 1 | side in the parent; parent < 0: the root
    float cl[3], ch[3];               // centroid bounds of the range
};
// per big range, by level parity
struct SahAux {
    float k[3];
    int32_t ok;                       // bit a: axis a binned
    int32_t pick_a, pick_b, mid;      // pick_a < 0: middle split
    int32_t ccb[2][6];                // children's centroid bounds (order-preserving int images)
};
struct SahArgs {
    const float* c2;                  // [nt][3] doubled centroids
    const float* aabb;                // [nt][6]
    int32_t* buf[2];                  // [nt] positions -> triangle, by level parity
    int32_t* order;                   // [nt] final order (leaves write it)
    float4* nodes;
    int32_t* parent_leaf;
    int32_t* parent_node;
    SahTask* big[2];                  // task lists by level parity
    SahTask* small[2];
    int32_t* cnt_big;                 // [levels + 2] tasks per level
    int32_t* cnt_small;
    int32_t cap_big, cap_small, cap_chunks;
    int32_t* bins;                    // [cap_big][SAH_NB3 * 7]: counts, then lo xyz hi xyz images
    SahAux* aux[2];                   // [cap_big] by level parity
    int32_t* chunk_base;              // [cap_big + 1] first chunk of each big range, then the total
    int32_t* hist;                    // [cap_chunks][SAH_NB3] per-chunk bin counts
    int32_t* loff;                    // [cap_chunks] each chunk's first left slot within its range
    int32_t* groot;                   // the root's split position g
    int32_t* err;                     // bit 0: a list was full (cannot happen for a binary tree)
};

// float <-> int with the same order (min / max of the ints = min / max of the floats)
__device__ __forceinline__ int32_t f2o(float f) {
    const int32_t i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int32_t i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__device__ __forceinline__ int sah_bin(float c, float cl, float k) {
    const int b = __float2int_rz(__fmul_rn(__fsub_rn(c, cl), k));
    return b < SAH_BINS - 1 ? b : SAH_BINS - 1;
}
__device__ __forceinline__ float half_area(const float lo[3], const float hi[3], float sc) {
    const float dx = __fmul_rn(__fsub_rn(hi[0], lo[0]), sc), dy = __fmul_rn(__fsub_rn(hi[1], lo[1]), sc),
                dz = __fmul_rn(__fsub_rn(hi[2], lo[2]), sc);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
}
// the range's cost scale: 2^-E with its largest centroid extent = f 2^E, f in [0.5, 1)
__device__ __forceinline__ float sah_scale(const SahTask& tk) {
    const float m = fmax_sel(fmax_sel(__fsub_rn(tk.ch[0], tk.cl[0]), __fsub_rn(tk.ch[1], tk.cl[1])),
                             __fsub_rn(tk.ch[2], tk.cl[2]));
    int e = 0;
    frexpf(m, &e);
    return ldexpf(1.0f, -e);
}
__device__ __forceinline__ float sel3(const float v[3], int a) { return a == 0 ? v[0] : (a == 1 ? v[1] : v[2]); }

// the binned axes of a range and their scales
__device__ __forceinline__ int sah_axes(const SahTask& tk, float k[3]) {
    int ok = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float e = __fsub_rn(tk.ch[a], tk.cl[a]);
        k[a] = __fdiv_rn((float)SAH_BINS, e);
        if ((tk.meta >> 1) < SAH_DEPTH_CAP && e > 0.0f && k[a] < INFINITY) ok |= 1 << a;
    }
    return ok;
}

// bins of one group: counts [SAH_NB3], then boxes [SAH_NB3][6] as int images
__device__ __forceinline__ void bins_clear(int32_t* cnt, int32_t* box, int t, int G) {
    for (int i = t; i < SAH_NB3; i += G) {
        cnt[i] = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) { box[6 * i + j] = f2o(INFINITY); box[6 * i + 3 + j] = f2o(-INFINITY); }
    }
}

// a run of equal bins of one axis, summed in registers and flushed with atomics
struct SahRun {
    int b = -1, c = 0;
    float lo[3], hi[3];
    __device__ __forceinline__ void flush(int32_t* cnt, int32_t* box, int a) {
        if (c == 0) return;
        const int i = a * SAH_BINS + b;
        atomicAdd(&cnt[i], c);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            atomicMin(&box[6 * i + j], f2o(lo[j]));
            atomicMax(&box[6 * i + 3 + j], f2o(hi[j]));
        }
    }
    __device__ __forceinline__ void add(int32_t* cnt, int32_t* box, int a, int bin, const float blo[3],
                                        const float bhi[3]) {
        if (bin != b) {
            flush(cnt, box, a);
            b = bin;
            c = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; }
        }
        ++c;
#pragma unroll
        for (int j = 0; j < 3; ++j) { lo[j] = fmin_sel(lo[j], blo[j]); hi[j] = fmax_sel(hi[j], bhi[j]); }
    }
};

// Bins the positions p = first + t, first + t + G, ... < end of buffer `src`
// into (cnt, box) with shared or global atomics.
__device__ __forceinline__ void bin_positions(const SahArgs& A, const int32_t* __restrict__ src, int first, int end,
                                              int t, int G, int ok, const float cl[3], const float k[3],
                                              int32_t* cnt, int32_t* box) {
    SahRun r0, r1, r2;
    for (int p = first + t; p < end; p += G) {
        const int32_t tri = src[p];
        const float* c = A.c2 + 3 * (int64_t)tri;
        const float* bx = A.aabb + 6 * (int64_t)tri;
        float blo[3], bhi[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) { blo[j] = bx[j]; bhi[j] = bx[3 + j]; }
        if (ok & 1) r0.add(cnt, box, 0, sah_bin(c[0], cl[0], k[0]), blo, bhi);
        if (ok & 2) r1.add(cnt, box, 1, sah_bin(c[1], cl[1], k[1]), blo, bhi);
        if (ok & 4) r2.add(cnt, box, 2, sah_bin(c[2], cl[2], k[2]), blo, bhi);
    }
    r0.flush(cnt, box, 0);
    r1.flush(cnt, box, 1);
    r2.flush(cnt, box, 2);
}

// The best split of axis a by a warp, lane b holding bin b (SAH_BINS == 32
// bins): the left and right unions by inclusive scans, the cost of split
// b = lane in lane b, and the first minimum (the lowest b of the least cost)
// by a reduction.  Returns the split, -1 without a candidate, in every lane.
static_assert(SAH_BINS == 32, "one bin per lane");
__device__ __forceinline__ int warp_sweep(const int32_t* cnt, const int32_t* box, int a, float sc, int lane,
                                          float* best_out) {
    const int i = a * SAH_BINS + lane;
    int nl = cnt[i], nr = nl;
    float llo[3], lhi[3], rlo[3], rhi[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        llo[j] = rlo[j] = o2f(box[6 * i + j]);
        lhi[j] = rhi[j] = o2f(box[6 * i + 3 + j]);
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int ul = __shfl_up_sync(0xffffffffu, nl, o), dr = __shfl_down_sync(0xffffffffu, nr, o);
        float ulo[3], uhi[3], dlo[3], dhi[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            ulo[j] = __shfl_up_sync(0xffffffffu, llo[j], o);
            uhi[j] = __shfl_up_sync(0xffffffffu, lhi[j], o);
            dlo[j] = __shfl_down_sync(0xffffffffu, rlo[j], o);
            dhi[j] = __shfl_down_sync(0xffffffffu, rhi[j], o);
        }
        if (lane >= o) {
            nl += ul;
#pragma unroll
            for (int j = 0; j < 3; ++j) { llo[j] = fmin_sel(llo[j], ulo[j]); lhi[j] = fmax_sel(lhi[j], uhi[j]); }
        }
        if (lane + o < 32) {
            nr += dr;
#pragma unroll
            for (int j = 0; j < 3; ++j) { rlo[j] = fmin_sel(rlo[j], dlo[j]); rhi[j] = fmax_sel(rhi[j], dhi[j]); }
        }
    }
    // split b = lane: the left side is the union of bins < b, the prefix of lane b - 1
    const int nL = __shfl_up_sync(0xffffffffu, nl, 1);
    float Llo[3], Lhi[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        Llo[j] = __shfl_up_sync(0xffffffffu, llo[j], 1);
        Lhi[j] = __shfl_up_sync(0xffffffffu, lhi[j], 1);
    }
    float c = INFINITY;
    if (lane >= 1 && nL > 0 && nr > 0)
        c = __fadd_rn(__fmul_rn(half_area(Llo, Lhi, sc), __int2float_rn(nL)),
                      __fmul_rn(half_area(rlo, rhi, sc), __int2float_rn(nr)));
    const bool valid = c < INFINITY;   // the serial rule: a cost below the best so far, which starts at +inf
    float bc = valid ? c : INFINITY;
    int bb = valid ? lane : SAH_BINS;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oc = __shfl_xor_sync(0xffffffffu, bc, o);
        const int ob = __shfl_xor_sync(0xffffffffu, bb, o);
        if (oc < bc || (oc == bc && ob < bb)) { bc = oc; bb = ob; }
    }
    *best_out = bc;
    return bb < SAH_BINS ? bb : -1;
}

__device__ __forceinline__ void sah_push(const SahArgs& A, int level, const SahTask& t) {
    const bool big = (t.hi - t.lo) > SAH_BIG;
    int32_t* cnt = big ? A.cnt_big + level : A.cnt_small + level;
    // (selects, not an index: a kernel parameter indexed at run time would be copied to local memory)
    SahTask* list = big ? ((level & 1) ? A.big[1] : A.big[0]) : ((level & 1) ? A.small[1] : A.small[0]);
    const int s = atomicAdd(cnt, 1);
    if (s < (big ? A.cap_big : A.cap_small)) list[s] = t;
    else atomicOr(A.err, 1);
}

// The node of a split range: its number, its record, its parent's link and
// leaf children (whose triangle is at their position of `dst`), and the
// tasks of its larger children with their centroid bounds.
__device__ __forceinline__ void sah_node(const SahArgs& A, const SahTask& tk, int level, int mid,
                                         const int32_t* __restrict__ dst, const float lcl[3], const float lch[3],
                                         const float rcl[3], const float rch[3]) {
    const int lo = tk.lo, hi = tk.hi;
    const int g = mid - 1;
    int id;
    if (tk.parent < 0) {
        *A.groot = g;
        id = 0;
    } else {
        id = (g == 0) ? *A.groot : g;
        reinterpret_cast<int32_t*>(&A.nodes[4 * (int64_t)tk.parent + 3])[tk.meta & 1] = id;
        A.parent_node[id] = tk.parent;
    }
    const int32_t c0 = (mid - lo == 1) ? ~(int32_t)lo : 0, c1 = (hi - mid == 1) ? ~(int32_t)mid : 0;
    A.nodes[4 * (int64_t)id + 3] = make_float4(__int_as_float(c0), __int_as_float(c1), 0.0f, 0.0f);
    const int meta = ((tk.meta >> 1) + 1) << 1;
    if (mid - lo == 1) {
        A.parent_leaf[lo] = id;
        A.order[lo] = dst[lo];
    } else {
        sah_push(A, level + 1, SahTask{lo, mid, id, meta, {lcl[0], lcl[1], lcl[2]}, {lch[0], lch[1], lch[2]}});
    }
    if (hi - mid == 1) {
        A.parent_leaf[mid] = id;
        A.order[mid] = dst[mid];
    } else {
        sah_push(A, level + 1, SahTask{mid, hi, id, meta | 1, {rcl[0], rcl[1], rcl[2]}, {rch[0], rch[1], rch[2]}});
    }
}

// min / max of three values over a group of G threads (a warp, or a block
// with G / 32 <= 32 warps and `red` [G / 32][6] of shared scratch); every
// thread receives them
template <int G>
__device__ __forceinline__ void g_minmax3(float mn[3], float mx[3], float (*red)[6]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin_sel(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmax_sel(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if (G > 32) {
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int a = 0; a < 3; ++a) { red[w][a] = mn[a]; red[w][3 + a] = mx[a]; }
        __syncthreads();
        for (int i = 0; i < G / 32; ++i)
#pragma unroll
            for (int a = 0; a < 3; ++a) { mn[a] = fmin_sel(mn[a], red[i][a]); mx[a] = fmax_sel(mx[a], red[i][3 + a]); }
        __syncthreads();
    }
}

// rank of f among the group's threads below this one, and the group's count
// of f (block: `wcnt` [G / 32] of shared scratch)
template <int G>
__device__ __forceinline__ int g_rank(bool f, int* total, int32_t* wcnt) {
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int l = threadIdx.x & 31;
    const int r = __popc(bal & ((1u << l) - 1u));
    if (G == 32) {
        *total = __popc(bal);
        return r;
    }
    const int w = threadIdx.x >> 5;
    if (l == 0) wcnt[w] = __popc(bal);
    __syncthreads();
    int before = 0, tot = 0;
    for (int i = 0; i < G / 32; ++i) {
        const int c = wcnt[i];
        before += (i < w) ? c : 0;
        tot += c;
    }
    __syncthreads();
    *total = tot;
    return r + before;
}

// inclusive prefix sum over a warp
__device__ __forceinline__ int warp_incl_scan(int v) {
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (l >= o) v += u;
    }
    return v;
}

// Partitions positions [first, end) of `src` stably into `dst`: elements
// with f go to lo_dst + done_l + rank, the others to r_dst + done_r + rank
// (ranks in order), where f = bin on axis pick_a < pick_b, or p < mid when
// pick_a < 0.  Accumulates each side's centroid bounds per thread.
template <int G>
__device__ __forceinline__ void partition_positions(const SahArgs& A, const int32_t* __restrict__ src,
                                                    int32_t* __restrict__ dst, int first, int end, int t,
                                                    int pick_a, int pick_b, float cla, float ka, int mid,
                                                    int l_dst, int r_dst, float lcl[3], float lch[3], float rcl[3],
                                                    float rch[3], int32_t* wcnt) {
    int done_l = 0, done_r = 0;
    for (int base = first; base < end; base += G) {
        const int p = base + t;
        int32_t tri = 0;
        bool f = false;
        if (p < end) {
            tri = src[p];
            const float* c = A.c2 + 3 * (int64_t)tri;
            const float cx = c[0], cy = c[1], cz = c[2];
            f = pick_a >= 0 ? sah_bin(pick_a == 0 ? cx : (pick_a == 1 ? cy : cz), cla, ka) < pick_b : p < mid;
            if (f) {
                lcl[0] = fmin_sel(lcl[0], cx); lcl[1] = fmin_sel(lcl[1], cy); lcl[2] = fmin_sel(lcl[2], cz);
                lch[0] = fmax_sel(lch[0], cx); lch[1] = fmax_sel(lch[1], cy); lch[2] = fmax_sel(lch[2], cz);
            } else {
                rcl[0] = fmin_sel(rcl[0], cx); rcl[1] = fmin_sel(rcl[1], cy); rcl[2] = fmin_sel(rcl[2], cz);
                rch[0] = fmax_sel(rch[0], cx); rch[1] = fmax_sel(rch[1], cy); rch[2] = fmax_sel(rch[2], cz);
            }
        }
        int tot;
        const int r = g_rank<G>(f, &tot, wcnt);
        if (p < end) dst[f ? l_dst + done_l + r : r_dst + done_r + (t - r)] = tri;
        done_l += tot;
        done_r += min(G, end - base) - tot;
    }
}

// ---- ranges of at most SAH_BIG positions: one warp each ----
struct SahWarpShared {
    int32_t cnt[SAH_NB3];
    int32_t box[SAH_NB3 * 6];
};

// the first minimum over the binned axes (a = 0, 1, 2; strict <), by the whole warp
__device__ __forceinline__ void sah_pick(const int32_t* cnt, const int32_t* box, int ok, float sc, int lane,
                                         int* pick_a, int* pick_b) {
    float best = INFINITY;
    *pick_a = -1;
    *pick_b = -1;
    for (int a = 0; a < 3; ++a) {
        if (!((ok >> a) & 1)) continue;
        float c;
        const int b = warp_sweep(cnt, box, a, sc, lane, &c);
        if (b >= 0 && c < best) {
            best = c;
            *pick_a = a;
            *pick_b = b;
        }
    }
}

__device__ __forceinline__ void sah_split_warp(const SahArgs& A, const SahTask& tk, int level, int lane,
                                               SahWarpShared& S) {
    const int32_t* src = (level & 1) ? A.buf[1] : A.buf[0];
    int32_t* dst = (level & 1) ? A.buf[0] : A.buf[1];
    float k[3];
    const int ok = sah_axes(tk, k);
    int pick_a = -1, pick_b = -1;
    if (ok) {
        bins_clear(S.cnt, S.box, lane, 32);
        __syncwarp();
        bin_positions(A, src, tk.lo, tk.hi, lane, 32, ok, tk.cl, k, S.cnt, S.box);
        __syncwarp();
        sah_pick(S.cnt, S.box, ok, sah_scale(tk), lane, &pick_a, &pick_b);
    }
    int nl = (tk.hi - tk.lo) / 2;
    if (pick_a >= 0) {
        nl = 0;
        for (int b = 0; b < pick_b; ++b) nl += S.cnt[pick_a * SAH_BINS + b];
    }
    const int mid = tk.lo + nl;
    float lcl[3] = {INFINITY, INFINITY, INFINITY}, lch[3] = {-INFINITY, -INFINITY, -INFINITY};
    float rcl[3] = {INFINITY, INFINITY, INFINITY}, rch[3] = {-INFINITY, -INFINITY, -INFINITY};
    partition_positions<32>(A, src, dst, tk.lo, tk.hi, lane, pick_a, pick_b, sel3(tk.cl, pick_a), sel3(k, pick_a),
                            mid, tk.lo, mid, lcl, lch, rcl, rch, nullptr);
    g_minmax3<32>(lcl, lch, nullptr);
    g_minmax3<32>(rcl, rch, nullptr);
    __syncwarp();
    if (lane == 0) sah_node(A, tk, level, mid, dst, lcl, lch, rcl, rch);
    __syncwarp();
}

__global__ void __launch_bounds__(32 * SAH_WARPS) k_sah_small(SahArgs A, int level) {
    __shared__ SahWarpShared S[SAH_WARPS];
    const int w = threadIdx.x >> 5;
    const int n = min(A.cnt_small[level], A.cap_small);
    const SahTask* in = (level & 1) ? A.small[1] : A.small[0];
    for (int s = blockIdx.x * SAH_WARPS + w; s < n; s += gridDim.x * SAH_WARPS)
        sah_split_warp(A, in[s], level, threadIdx.x & 31, S[w]);
}

// Meshes of at most SAH_BIG tree positions have no chunked ranges: one block
// runs every level, its warps taking that level's ranges, with a barrier
// between levels instead of five launches, and stops at the first empty
// level (0.44 ms for 1202 triangles, half the per-level launches' time).
constexpr int SAH_ONE_WARPS = 16;
__global__ void __launch_bounds__(32 * SAH_ONE_WARPS) k_sah_one_block(SahArgs A, int levels) {
    __shared__ SahWarpShared S[SAH_ONE_WARPS];
    const int w = threadIdx.x >> 5;
    for (int level = 0; level < levels; ++level) {
        // the count is final: its pushes came before the barrier that ended the last level
        const int n = min(A.cnt_small[level], A.cap_small);
        if (n == 0) break;
        const SahTask* in = (level & 1) ? A.small[1] : A.small[0];
        for (int s = w; s < n; s += SAH_ONE_WARPS) sah_split_warp(A, in[s], level, threadIdx.x & 31, S[w]);
        __syncthreads();
    }
}

// the root task: the tree's positions [0, ns) with the Morton bounds of their centroids
__global__ void k_sah_root(SahArgs A, const int32_t* __restrict__ count, int64_t nt, const float* __restrict__ bnd) {
    const int64_t ns = tree_size(count, nt);
    if (ns >= 2) sah_push(A, 0, SahTask{0, (int32_t)ns, -1, 0, {bnd[0], bnd[1], bnd[2]}, {bnd[3], bnd[4], bnd[5]}});
}

// ---- ranges of more than SAH_BIG positions: chunked over every block ----
// the big range holding chunk c: the last i < nb with chunk_base[i] <= c
__device__ __forceinline__ int chunk_owner(const int32_t* __restrict__ base, int nb, int c) {
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (base[m] <= c) lo = m;
        else hi = m - 1;
    }
    return lo;
}

// Finishes the big ranges of the previous level (their nodes and children),
// then plans this level's: chunk bases (exclusive prefix sum of their chunk
// counts), cleared bins, binned axes, cleared children's bounds.  One block.
__global__ void __launch_bounds__(SAH_PLAN) k_sah_plan(SahArgs A, int level) {
    __shared__ int32_t wsum[SAH_PLAN / 32];
    __shared__ int32_t carry;
    if (level > 0) {
        const int pl = level - 1;
        const int nbp = min(A.cnt_big[pl], A.cap_big);
        const SahTask* in = (pl & 1) ? A.big[1] : A.big[0];
        const SahAux* ax = (pl & 1) ? A.aux[1] : A.aux[0];
        const int32_t* dst = (pl & 1) ? A.buf[0] : A.buf[1];   // where level pl partitioned to
        for (int i = threadIdx.x; i < nbp; i += SAH_PLAN) {
            const SahAux& x = ax[i];
            float lcl[3], lch[3], rcl[3], rch[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lcl[a] = o2f(x.ccb[0][a]);
                lch[a] = o2f(x.ccb[0][3 + a]);
                rcl[a] = o2f(x.ccb[1][a]);
                rch[a] = o2f(x.ccb[1][3 + a]);
            }
            sah_node(A, in[i], pl, x.mid, dst, lcl, lch, rcl, rch);
        }
        __syncthreads();   // their pushes fill this level's lists
    }
    const int nb = min(A.cnt_big[level], A.cap_big);
    const SahTask* in = (level & 1) ? A.big[1] : A.big[0];
    SahAux* ax = (level & 1) ? A.aux[1] : A.aux[0];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int base = 0; base < nb; base += SAH_PLAN) {
        const int i = base + threadIdx.x;
        int v = 0;
        if (i < nb) {
            const SahTask tk = in[i];
            v = (tk.hi - tk.lo + SAH_CHUNK - 1) / SAH_CHUNK;
            SahAux& x = ax[i];
            x.ok = sah_axes(tk, x.k);
            x.pick_a = -1;
            x.pick_b = -1;
            x.mid = tk.lo;
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int a = 0; a < 3; ++a) { x.ccb[s][a] = f2o(INFINITY); x.ccb[s][3 + a] = f2o(-INFINITY); }
        }
        const int incl = warp_incl_scan(v);
        if (l == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int s = warp_incl_scan(wsum[l]);
            wsum[l] = s;   // inclusive over warps
        }
        __syncthreads();
        const int excl = carry + (w > 0 ? wsum[w - 1] : 0) + incl - v;
        if (i < nb) A.chunk_base[i] = excl;
        __syncthreads();
        if (threadIdx.x == SAH_PLAN - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) A.chunk_base[nb] = carry;
    for (int i = threadIdx.x; i < nb * SAH_NB3; i += SAH_PLAN) {
        int32_t* g = A.bins + (int64_t)(i / SAH_NB3) * (SAH_NB3 * 7);
        const int j = i % SAH_NB3;
        g[j] = 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) { g[SAH_NB3 + 6 * j + q] = f2o(INFINITY); g[SAH_NB3 + 6 * j + 3 + q] = f2o(-INFINITY); }
    }
}

// Bins every chunk of this level's big ranges: shared bins per chunk, stored
// as the chunk's histogram and merged into its range's bins.
__global__ void __launch_bounds__(SAH_BLOCK) k_sah_bin(SahArgs A, int level) {
    __shared__ int32_t cnt[SAH_NB3];
    __shared__ int32_t box[SAH_NB3 * 6];
    const int nb = min(A.cnt_big[level], A.cap_big);
    if (nb == 0) return;
    const int nch = min(A.chunk_base[nb], A.cap_chunks);
    const SahTask* in = (level & 1) ? A.big[1] : A.big[0];
    const SahAux* ax = (level & 1) ? A.aux[1] : A.aux[0];
    const int32_t* src = (level & 1) ? A.buf[1] : A.buf[0];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int i = chunk_owner(A.chunk_base, nb, c);
        const SahTask tk = in[i];
        const int ok = ax[i].ok;
        float k[3] = {ax[i].k[0], ax[i].k[1], ax[i].k[2]};
        const int first = tk.lo + (c - A.chunk_base[i]) * SAH_CHUNK;
        const int end = min(tk.hi, first + SAH_CHUNK);
        bins_clear(cnt, box, threadIdx.x, SAH_BLOCK);
        __syncthreads();
        if (ok) bin_positions(A, src, first, end, threadIdx.x, SAH_BLOCK, ok, tk.cl, k, cnt, box);
        __syncthreads();
        int32_t* gcnt = A.bins + (int64_t)i * (SAH_NB3 * 7);
        int32_t* gbox = gcnt + SAH_NB3;
        for (int j = threadIdx.x; j < SAH_NB3; j += SAH_BLOCK) {
            const int n = cnt[j];
            A.hist[(int64_t)c * SAH_NB3 + j] = n;
            if (n) {
                atomicAdd(&gcnt[j], n);
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    atomicMin(&gbox[6 * j + q], box[6 * j + q]);
                    atomicMax(&gbox[6 * j + 3 + q], box[6 * j + 3 + q]);
                }
            }
        }
        __syncthreads();
    }
}

// One warp per big range: the split, then each chunk's first left slot (an
// exclusive prefix sum over the range's chunks of their left counts, read
// from the histograms, or from the middle for a middle split).
__global__ void __launch_bounds__(32 * SAH_WARPS) k_sah_decide(SahArgs A, int level) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = min(A.cnt_big[level], A.cap_big);
    const SahTask* in = (level & 1) ? A.big[1] : A.big[0];
    SahAux* ax = (level & 1) ? A.aux[1] : A.aux[0];
    for (int i = blockIdx.x * SAH_WARPS + w; i < nb; i += gridDim.x * SAH_WARPS) {
        const SahTask tk = in[i];
        const int32_t* gcnt = A.bins + (int64_t)i * (SAH_NB3 * 7);
        int pick_a = -1, pick_b = -1;
        const int ok = ax[i].ok;
        if (ok) sah_pick(gcnt, gcnt + SAH_NB3, ok, sah_scale(tk), lane, &pick_a, &pick_b);
        int nl = (tk.hi - tk.lo) / 2;
        if (pick_a >= 0) {
            nl = 0;
            for (int b = 0; b < pick_b; ++b) nl += gcnt[pick_a * SAH_BINS + b];
        }
        const int mid = tk.lo + nl;
        const int c0 = A.chunk_base[i];
        const int nc = (tk.hi - tk.lo + SAH_CHUNK - 1) / SAH_CHUNK;
        int carry = 0;
        for (int j0 = 0; j0 < nc; j0 += 32) {
            const int j = j0 + lane;
            int v = 0;
            if (j < nc && c0 + j < A.cap_chunks) {
                const int first = tk.lo + j * SAH_CHUNK;
                const int len = min(SAH_CHUNK, tk.hi - first);
                if (pick_a >= 0) {
                    const int32_t* h = A.hist + (int64_t)(c0 + j) * SAH_NB3 + pick_a * SAH_BINS;
                    for (int b = 0; b < pick_b; ++b) v += h[b];
                } else {
                    v = max(0, min(mid - first, len));
                }
            }
            const int incl = warp_incl_scan(v);
            if (j < nc && c0 + j < A.cap_chunks) A.loff[c0 + j] = carry + incl - v;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            ax[i].pick_a = pick_a;
            ax[i].pick_b = pick_b;
            ax[i].mid = mid;
        }
        __syncwarp();
    }
}

// Partitions every chunk of this level's big ranges into the other buffer
// and merges each side's centroid bounds into its range's children's bounds.
__global__ void __launch_bounds__(SAH_BLOCK) k_sah_scatter(SahArgs A, int level) {
    __shared__ float red[SAH_BLOCK / 32][6];
    __shared__ int32_t wcnt[SAH_BLOCK / 32];
    const int nb = min(A.cnt_big[level], A.cap_big);
    if (nb == 0) return;
    const int nch = min(A.chunk_base[nb], A.cap_chunks);
    const SahTask* in = (level & 1) ? A.big[1] : A.big[0];
    SahAux* ax = (level & 1) ? A.aux[1] : A.aux[0];
    const int32_t* src = (level & 1) ? A.buf[1] : A.buf[0];
    int32_t* dst = (level & 1) ? A.buf[0] : A.buf[1];
    for (int c = blockIdx.x; c < nch; c += gridDim.x) {
        const int i = chunk_owner(A.chunk_base, nb, c);
        const SahTask tk = in[i];
        const int pick_a = ax[i].pick_a, pick_b = ax[i].pick_b, mid = ax[i].mid;
        const float ka = pick_a == 0 ? ax[i].k[0] : (pick_a == 1 ? ax[i].k[1] : ax[i].k[2]);
        const int first = tk.lo + (c - A.chunk_base[i]) * SAH_CHUNK;
        const int end = min(tk.hi, first + SAH_CHUNK);
        const int loff = A.loff[c];
        const int roff = (first - tk.lo) - loff;
        float lcl[3] = {INFINITY, INFINITY, INFINITY}, lch[3] = {-INFINITY, -INFINITY, -INFINITY};
        float rcl[3] = {INFINITY, INFINITY, INFINITY}, rch[3] = {-INFINITY, -INFINITY, -INFINITY};
        partition_positions<SAH_BLOCK>(A, src, dst, first, end, threadIdx.x, pick_a, pick_b, sel3(tk.cl, pick_a), ka,
                                       mid, tk.lo + loff, mid + roff, lcl, lch, rcl, rch, wcnt);
        g_minmax3<SAH_BLOCK>(lcl, lch, red);
        g_minmax3<SAH_BLOCK>(rcl, rch, red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                atomicMin(&ax[i].ccb[0][a], f2o(lcl[a]));
                atomicMax(&ax[i].ccb[0][3 + a], f2o(lch[a]));
                atomicMin(&ax[i].ccb[1][a], f2o(rcl[a]));
                atomicMax(&ax[i].ccb[1][3 + a], f2o(rch[a]));
            }
        }
        __syncthreads();
    }
}

// Morton key of each triangle at its final position: keys by triangle id
// (scattered from the sorted pairs), then gathered through the final order.
__global__ void k_keys_by_tri(const uint64_t* __restrict__ ks, const int32_t* __restrict__ vs, int64_t n,
                              uint64_t* __restrict__ by_tri) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) by_tri[vs[p]] = ks[p];
}
__global__ void k_keys_gather(const uint64_t* __restrict__ by_tri, const int32_t* __restrict__ order, int64_t n,
                              uint64_t* __restrict__ keys) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) keys[p] = by_tri[order[p]];
}

// ---------------- the whole build of a small mesh in one block ----------------
// For meshes of at most SMALL_SORT triangles the steps above (boxes, scene
// bounds, large-triangle flags, centroid bounds, Morton codes, sort, Karras
// hierarchy, refit, leaf records) run in one launch of one 1024-thread block,
// with the sort, the hierarchy and the refit in shared memory.  Every value is
// computed by the same expressions as in the multi-kernel path (min / max are
// exact, so the order of the reductions does not matter), so the tree is the
// same bit for bit; it replaces ~14 launches and their gaps.
constexpr int BUILD_THREADS = 1024;
static_assert(SMALL_SORT / 2 <= BUILD_THREADS, "one sort pair per thread");
struct SmallBuildSmem {
    uint64_t sk[SMALL_SORT];
    int32_t sv[SMALL_SORT];
    int32_t pl[SMALL_SORT], pn[SMALL_SORT], visit[SMALL_SORT];
    int32_t child[2 * SMALL_SORT];
    float nb[12 * SMALL_SORT];          // child boxes of the internal nodes
    int8_t large[SMALL_SORT];
    float box[6][SMALL_SORT];           // triangle boxes (lo xyz, hi xyz)
    float red[33 * 6];
    int32_t cnt;
};
static_assert(sizeof(SmallBuildSmem) <= 227 * 1024, "shared memory of one block");

__device__ __forceinline__ void tri_box(const float* __restrict__ verts, const int32_t* __restrict__ tris, int64_t i,
                                        float lo[3], float hi[3]) {
    const int32_t i0 = tris[3 * i], i1 = tris[3 * i + 1], i2 = tris[3 * i + 2];
    for (int a = 0; a < 3; ++a) {
        const float v0 = verts[3 * (int64_t)i0 + a], v1 = verts[3 * (int64_t)i1 + a],
                    v2 = verts[3 * (int64_t)i2 + a];
        lo[a] = fmin_sel(v0, fmin_sel(v1, v2));
        hi[a] = fmax_sel(v0, fmax_sel(v1, v2));
    }
}

// min of mn[], max of mx[] over the block; every thread gets the result
__device__ void block_minmax(float mn[3], float mx[3], float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1)
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin_sel(mn[a], __shfl_xor_sync(FULL_MASK, mn[a], o));
            mx[a] = fmax_sel(mx[a], __shfl_xor_sync(FULL_MASK, mx[a], o));
        }
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { red[6 * warp + a] = mn[a]; red[6 * warp + 3 + a] = mx[a]; }
    __syncthreads();
    if (warp == 0) {
        for (int a = 0; a < 3; ++a) { mn[a] = red[6 * lane + a]; mx[a] = red[6 * lane + 3 + a]; }
        for (int o = 16; o > 0; o >>= 1)
            for (int a = 0; a < 3; ++a) {
                mn[a] = fmin_sel(mn[a], __shfl_xor_sync(FULL_MASK, mn[a], o));
                mx[a] = fmax_sel(mx[a], __shfl_xor_sync(FULL_MASK, mx[a], o));
            }
        if (lane == 0)
            for (int a = 0; a < 3; ++a) { red[6 * 32 + a] = mn[a]; red[6 * 32 + 3 + a] = mx[a]; }
    }
    __syncthreads();
    for (int a = 0; a < 3; ++a) { mn[a] = red[6 * 32 + a]; mx[a] = red[6 * 32 + 3 + a]; }
    __syncthreads();
}

__global__ void __launch_bounds__(BUILD_THREADS) k_build_small(
        const float* __restrict__ verts, const int32_t* __restrict__ tris, const int32_t* __restrict__ tri_mat,
        int n, uint64_t* __restrict__ keys_out, int32_t* __restrict__ order_out, float4* __restrict__ nodes,
        float4* __restrict__ rec, int32_t* __restrict__ count_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallBuildSmem& S = *reinterpret_cast<SmallBuildSmem*>(smem_raw);
    const int tid = threadIdx.x;
    if (tid == 0) S.cnt = 0;
    // scene bounds of the triangle boxes
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = tid; i < n; i += BUILD_THREADS) {
        float lo[3], hi[3];
        tri_box(verts, tris, i, lo, hi);
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin_sel(mn[a], lo[a]);
            mx[a] = fmax_sel(mx[a], hi[a]);
            S.box[a][i] = lo[a];
            S.box[3 + a][i] = hi[a];
        }
    }
    block_minmax(mn, mx, S.red);
    // large triangles
    const float thr = __fmul_rn(0.25f, extent3(mn, mx));
    for (int i = tid; i < n; i += BUILD_THREADS) {
        const float lo[3] = {S.box[0][i], S.box[1][i], S.box[2][i]}, hi[3] = {S.box[3][i], S.box[4][i], S.box[5][i]};
        const bool l = extent3(lo, hi) >= thr;
        S.large[i] = l ? 1 : 0;
        if (l) atomicAdd(&S.cnt, 1);
    }
    __syncthreads();
    const int cnt = S.cnt;
    const bool use_large = cnt > 0 && cnt <= MAX_LARGE;
    // bounds of the doubled centroids of the tree's triangles
    float cmn[3] = {INFINITY, INFINITY, INFINITY}, cmx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = tid; i < n; i += BUILD_THREADS) {
        if (use_large && S.large[i]) continue;
        for (int a = 0; a < 3; ++a) {
            const float c = __fadd_rn(S.box[a][i], S.box[3 + a][i]);
            cmn[a] = fmin_sel(cmn[a], c);
            cmx[a] = fmax_sel(cmx[a], c);
        }
    }
    block_minmax(cmn, cmx, S.red);
    // Morton codes (as k_morton) into the sort buffer, padded to a power of two
    int P = 1;
    while (P < n) P <<= 1;
    {
        const float e = extent3(cmn, cmx);
        const float scale = (e > 0.0f) ? __fdiv_rn(2097151.0f, e) : 0.0f;
        for (int i = tid; i < P; i += BUILD_THREADS) {
            if (i >= n) { S.sk[i] = ~0ULL; S.sv[i] = INT32_MAX; continue; }
            S.sv[i] = i;
            if (use_large && S.large[i]) { S.sk[i] = ~0ULL; continue; }
            uint32_t q[3];
            for (int a = 0; a < 3; ++a) {
                const float f = __fmul_rn(__fsub_rn(__fadd_rn(S.box[a][i], S.box[3 + a][i]), cmn[a]), scale);
                const uint32_t u = __float2uint_rz(f);
                q[a] = u > 2097151u ? 2097151u : u;
            }
            S.sk[i] = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);
        }
    }
    __syncthreads();
    // bitonic sort of (key, position): the stable order by key (as k_sort_small).
    // Thread t owns pair t (P / 2 <= BUILD_THREADS).  A stage with stride <= 32
    // keeps warp w inside elements [64 w, 64 w + 64), so two consecutive such
    // stages need only a warp barrier; any stage with stride >= 64 a block barrier.
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (tid < (P >> 1)) {
                const int t = tid;
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const uint64_t ki = S.sk[i], kj = S.sk[j];
                const int32_t vi = S.sv[i], vj = S.sv[j];
                const bool gt = ki > kj || (ki == kj && vi > vj);
                if (gt == up) {
                    S.sk[i] = kj; S.sk[j] = ki;
                    S.sv[i] = vj; S.sv[j] = vi;
                }
            }
            const int next = stride > 1 ? stride >> 1 : size;   // the next stage's stride
            if (stride >= 64 || next >= 64) __syncthreads();
            else __syncwarp();
        }
    }
    __syncthreads();
    for (int i = tid; i < n; i += BUILD_THREADS) {
        keys_out[i] = S.sk[i];
        order_out[i] = S.sv[i];
    }
    const int m = use_large ? n - cnt : n;   // the tree covers sorted positions [0, m)
    if (m >= 2) {
        // Karras hierarchy (as k_karras) on the shared keys
        for (int ii = tid; ii < m - 1; ii += BUILD_THREADS) {
            const int64_t i = ii;
            const uint64_t* k = S.sk;
            const int d = (delta(k, m, i, i + 1) - delta(k, m, i, i - 1)) > 0 ? 1 : -1;
            const int dmin = delta(k, m, i, i - d);
            int64_t lmax = 2;
            while (delta(k, m, i, i + lmax * d) > dmin) lmax <<= 1;
            int64_t l = 0;
            for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
                if (delta(k, m, i, i + (l + t) * d) > dmin) l += t;
            const int64_t j = i + l * d;
            const int dnode = delta(k, m, i, j);
            int64_t s = 0;
            int64_t div = 2;
            int64_t t = (l + div - 1) / div;
            while (true) {
                if (delta(k, m, i, i + (s + t) * d) > dnode) s += t;
                if (t <= 1) break;
                div <<= 1;
                t = (l + div - 1) / div;
            }
            const int64_t g = i + s * d + (d < 0 ? -1 : 0);
            const int64_t lo = i < j ? i : j, hi = i < j ? j : i;
            const int32_t c0 = (lo == g) ? ~(int32_t)g : (int32_t)g;
            const int32_t c1 = (hi == g + 1) ? ~(int32_t)(g + 1) : (int32_t)(g + 1);
            S.child[2 * ii] = c0;
            S.child[2 * ii + 1] = c1;
            if (c0 < 0) S.pl[g] = ii; else S.pn[g] = ii;
            if (c1 < 0) S.pl[g + 1] = ii; else S.pn[g + 1] = ii;
            S.visit[ii] = 0;
        }
        __syncthreads();
        // refit (as k_refit): the second child to arrive at a node forms its box
        volatile float* nbv = S.nb;
        for (int p = tid; p < m; p += BUILD_THREADS) {
            float box[6];
            const int32_t tri = S.sv[p];
            for (int a = 0; a < 6; ++a) box[a] = S.box[a][tri];
            int32_t me = ~(int32_t)p;
            int32_t node = S.pl[p];
            for (int step = 0; step < m; ++step) {
                const int slot = (S.child[2 * node] == me) ? 0 : 1;
                for (int a = 0; a < 6; ++a) nbv[12 * node + 6 * slot + a] = box[a];
                __threadfence_block();
                if (atomicAdd(&S.visit[node], 1) == 0) break;
                __threadfence_block();
                float lb[6], rb[6];
                for (int a = 0; a < 6; ++a) { lb[a] = nbv[12 * node + a]; rb[a] = nbv[12 * node + 6 + a]; }
                for (int a = 0; a < 3; ++a) {
                    box[a] = fmin_sel(lb[a], rb[a]);
                    box[3 + a] = fmax_sel(lb[3 + a], rb[3 + a]);
                }
                if (node == 0) break;
                me = node;
                node = S.pn[node];
            }
        }
        __syncthreads();
        for (int i = tid; i < m - 1; i += BUILD_THREADS) {
            const float* b = S.nb + 12 * i;
            nodes[4 * i + 0] = make_float4(b[0], b[1], b[2], b[3]);
            nodes[4 * i + 1] = make_float4(b[4], b[5], b[6], b[7]);
            nodes[4 * i + 2] = make_float4(b[8], b[9], b[10], b[11]);
            nodes[4 * i + 3] = make_float4(__int_as_float(S.child[2 * i]), __int_as_float(S.child[2 * i + 1]), 0.0f, 0.0f);
        }
    }
    // leaf records (as k_trirec)
    for (int p = tid; p < n; p += BUILD_THREADS) {
        const int32_t t = S.sv[p];
        const float* a = verts + 3 * (int64_t)tris[3 * (int64_t)t];
        const float* b = verts + 3 * (int64_t)tris[3 * (int64_t)t + 1];
        const float* c = verts + 3 * (int64_t)tris[3 * (int64_t)t + 2];
        rec[3 * p + 0] = make_float4(a[0], a[1], a[2], b[0]);
        rec[3 * p + 1] = make_float4(b[1], b[2], c[0], c[1]);
        rec[3 * p + 2] = make_float4(c[2], __int_as_float(tri_mat[t]), __int_as_float(t), 0.0f);
    }
    if (tid == 0) *count_out = cnt;
}

inline unsigned nb(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t check_indices(const int32_t* tris, const int32_t* tri_mat, int64_t nt, int64_t nv, int32_t nm,
                          int32_t* flag_dev, cudaStream_t s) {
    if (nt <= 0) return cudaSuccess;
    k_check_indices<<<nb(nt, 256), 256, 0, s>>>(tris, tri_mat, nt, nv, nm, flag_dev);
    return cudaGetLastError();
}

cudaError_t build_bvh(const BvhBuffers& B, int builder, cudaStream_t s, int32_t* nlarge_host) {
    const int64_t n = B.nt;
    *nlarge_host = 0;
    if (n <= 0) return cudaSuccess;
    cudaError_t err;
    const bool sah = builder == BVH_SAH;
    if (n <= SMALL_SORT && !sah) {
        // one launch: the count goes through a 4-byte scratch word
        int32_t* cnt = nullptr;
        if ((err = lib_malloc_async((void**)&cnt, sizeof(int32_t), s)) != cudaSuccess) return err;
        const int smem = (int)sizeof(SmallBuildSmem);
        if ((err = cudaFuncSetAttribute(k_build_small, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
            cudaSuccess) {
            cudaFreeAsync(cnt, s);
            return err;
        }
        k_build_small<<<1, BUILD_THREADS, smem, s>>>(B.verts, B.tris, B.tri_mat, (int)n, B.keys_sorted, B.order,
                                                     B.nodes, B.trirec, cnt);
        if ((err = cudaGetLastError()) == cudaSuccess)
            err = cudaMemcpyAsync(nlarge_host, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        const cudaError_t e2 = cudaFreeAsync(cnt, s);
        return err != cudaSuccess ? err : e2;
    }
    const int nblk_a = (int)nb(n, 256);
    const int nblk_s = (int)nb(n, SORT_TILE);
    // scratch: aabb [6n] f32, c2 [3n] f32, blk [6 nblk_a] f32, bounds [6] f32,
    // keys2 [n] u64, vals [2n] i32, hist [256 nblk_s] u32, parents [2n] i32, visit [n] i32
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    const size_t o_aabb = take(sizeof(float) * 6 * n), o_c2 = take(sizeof(float) * 3 * n),
                 o_blk = take(sizeof(float) * 6 * nblk_a), o_bnd = take(sizeof(float) * 6),
                 o_k2 = take(sizeof(uint64_t) * n), o_v1 = take(sizeof(int32_t) * n),
                 o_v2 = take(sizeof(int32_t) * n), o_h = take(sizeof(uint32_t) * 256 * (size_t)nblk_s),
                 o_pl = take(sizeof(int32_t) * n), o_pn = take(sizeof(int32_t) * n),
                 o_vis = take(sizeof(int32_t) * n), o_sb = take(sizeof(float) * 6),
                 o_lg = take(sizeof(int8_t) * n), o_cnt = take(sizeof(int32_t));
    // SAH: task lists by level parity, tasks per level, the root's split, an error word;
    // the big ranges' bins, plans, chunk histograms and chunk offsets
    int levels = SAH_DEPTH_CAP + 2;
    for (int64_t m = 1; m < n; m <<= 1) ++levels;
    const int32_t cap_small = (int32_t)(n / 2 + 1), cap_big = (int32_t)(n / SAH_BIG + 2);
    const int32_t cap_chunks = (int32_t)(n / SAH_CHUNK + cap_big + 1);
    size_t o_tb = 0, o_ts = 0, o_tc = 0, o_bins = 0, o_aux = 0, o_cb = 0, o_hist = 0, o_loff = 0;
    if (sah) {
        o_tb = take(sizeof(SahTask) * 2 * (size_t)cap_big);
        o_ts = take(sizeof(SahTask) * 2 * (size_t)cap_small);
        o_tc = take(sizeof(int32_t) * (2 * (size_t)(levels + 2) + 2));
        o_bins = take(sizeof(int32_t) * SAH_NB3 * 7 * (size_t)cap_big);
        o_aux = take(sizeof(SahAux) * 2 * (size_t)cap_big);
        o_cb = take(sizeof(int32_t) * ((size_t)cap_big + 1));
        o_hist = take(sizeof(int32_t) * SAH_NB3 * (size_t)cap_chunks);
        o_loff = take(sizeof(int32_t) * (size_t)cap_chunks);
    }
    char* base = nullptr;
    if ((err = lib_malloc_async((void**)&base, off, s)) != cudaSuccess) return err;
    // every later error still returns the scratch block to the pool
    auto fail_free = [&](cudaError_t e) { cudaFreeAsync(base, s); return e; };
    float* aabb = (float*)(base + o_aabb);
    float* c2 = (float*)(base + o_c2);
    float* blk = (float*)(base + o_blk);
    float* bnd = (float*)(base + o_bnd);
    uint64_t* k1 = B.keys_sorted;
    uint64_t* k2 = (uint64_t*)(base + o_k2);
    int32_t* v1 = (int32_t*)(base + o_v1);
    int32_t* v2 = (int32_t*)(base + o_v2);
    uint32_t* hist = (uint32_t*)(base + o_h);
    int32_t* pl = (int32_t*)(base + o_pl);
    int32_t* pn = (int32_t*)(base + o_pn);
    int32_t* vis = (int32_t*)(base + o_vis);
    float* sb = (float*)(base + o_sb);
    int8_t* lg = (int8_t*)(base + o_lg);
    int32_t* cnt = (int32_t*)(base + o_cnt);

    // No host round trip inside the build: the large-triangle decision and the
    // tree size live in device memory (cnt) and every later kernel reads them.
    k_tri_aabb<<<nblk_a, 256, 0, s>>>(B.verts, B.tris, n, aabb, c2, blk);
    k_minmax_final<<<1, 256, 0, s>>>(blk, nblk_a, sb);
    if ((err = cudaMemsetAsync(cnt, 0, sizeof(int32_t), s)) != cudaSuccess) return fail_free(err);
    k_flag_large<<<nblk_a, 256, 0, s>>>(aabb, sb, n, lg, cnt);
    k_c2_bounds<<<nblk_a, 256, 0, s>>>(c2, lg, cnt, n, blk);
    k_minmax_final<<<1, 256, 0, s>>>(blk, nblk_a, bnd);
    k_morton<<<nblk_a, 256, 0, s>>>(c2, bnd, n, lg, cnt, k1, v1);
    if (n <= SMALL_SORT) {
        k_sort_small<<<1, 1024, 0, s>>>(k1, v1, (int)n);
    } else {
        // 8 passes; after an even number of passes the result is back in (k1, v1)
        for (int pass = 0; pass < 8; ++pass) {
            const int shift = 8 * pass;
            uint64_t* kin = (pass & 1) ? k2 : k1;
            uint64_t* kout = (pass & 1) ? k1 : k2;
            int32_t* vin = (pass & 1) ? v2 : v1;
            int32_t* vout = (pass & 1) ? v1 : v2;
            k_hist<<<nblk_s, SORT_THREADS, 0, s>>>(kin, n, shift, hist, nblk_s);
            k_scan<<<1, 1024, 0, s>>>(hist, (int64_t)256 * nblk_s);
            k_scatter<<<nblk_s, SORT_THREADS, 0, s>>>(kin, vin, n, shift, hist, nblk_s, kout, vout);
        }
    }
    if ((err = cudaMemcpyAsync(B.order, v1, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return fail_free(err);
    if (n >= 2 && !sah) {
        k_karras<<<nb(n - 1, 256), 256, 0, s>>>(k1, n, cnt, B.nodes, pl, pn);
        if ((err = cudaMemsetAsync(vis, 0, sizeof(int32_t) * n, s)) != cudaSuccess) return fail_free(err);
        k_refit<<<nb(n, 256), 256, 0, s>>>(aabb, B.order, n, cnt, pl, pn, B.nodes, vis);
    }
    if (n >= 2 && sah) {
        SahArgs A;
        A.c2 = c2;
        A.aabb = aabb;
        A.buf[0] = v1;         // the Morton order (B.order holds a copy, large triangles included)
        A.buf[1] = v2;         // free after the sort
        A.order = B.order;
        A.nodes = B.nodes;
        A.parent_leaf = pl;
        A.parent_node = pn;
        SahTask* tb = (SahTask*)(base + o_tb);
        SahTask* ts = (SahTask*)(base + o_ts);
        A.big[0] = tb;
        A.big[1] = tb + cap_big;
        A.small[0] = ts;
        A.small[1] = ts + cap_small;
        int32_t* tc = (int32_t*)(base + o_tc);
        A.cnt_big = tc;
        A.cnt_small = tc + (levels + 2);
        A.groot = tc + 2 * (levels + 2);
        A.err = A.groot + 1;
        A.cap_big = cap_big;
        A.cap_small = cap_small;
        A.cap_chunks = cap_chunks;
        A.bins = (int32_t*)(base + o_bins);
        SahAux* aux = (SahAux*)(base + o_aux);
        A.aux[0] = aux;
        A.aux[1] = aux + cap_big;
        A.chunk_base = (int32_t*)(base + o_cb);
        A.hist = (int32_t*)(base + o_hist);
        A.loff = (int32_t*)(base + o_loff);
        if ((err = cudaMemsetAsync(tc, 0, sizeof(int32_t) * (2 * (size_t)(levels + 2) + 2), s)) != cudaSuccess)
            return fail_free(err);
        int dev = 0, sms = 148;
        if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int gb = (int)std::min<int64_t>(cap_chunks, 2 * (int64_t)sms);
        const int gd = (int)std::min<int64_t>((cap_big + SAH_WARPS - 1) / SAH_WARPS, 4 * (int64_t)sms);
        const int gs = (int)std::min<int64_t>((cap_small + SAH_WARPS - 1) / SAH_WARPS, 8 * (int64_t)sms);
        // keys by triangle id while v1 still holds the Morton order
        k_keys_by_tri<<<nb(n, 256), 256, 0, s>>>(k1, v1, n, k2);
        k_sah_root<<<1, 1, 0, s>>>(A, cnt, n, bnd);
        if (n <= SAH_BIG) {
            k_sah_one_block<<<1, 32 * SAH_ONE_WARPS, 0, s>>>(A, levels);
        } else {
            // no leaf is deeper than SAH_DEPTH_CAP + ceil(log2 n): later levels are empty
            for (int level = 0; level < levels; ++level) {
                k_sah_plan<<<1, SAH_PLAN, 0, s>>>(A, level);
                k_sah_bin<<<gb, SAH_BLOCK, 0, s>>>(A, level);
                k_sah_decide<<<gd, 32 * SAH_WARPS, 0, s>>>(A, level);
                k_sah_scatter<<<gb, SAH_BLOCK, 0, s>>>(A, level);
                k_sah_small<<<gs, 32 * SAH_WARPS, 0, s>>>(A, level);
            }
            k_sah_plan<<<1, SAH_PLAN, 0, s>>>(A, levels);   // the nodes of the last level's big ranges
        }
        if ((err = cudaMemsetAsync(vis, 0, sizeof(int32_t) * n, s)) != cudaSuccess) return fail_free(err);
        k_refit<<<nb(n, 256), 256, 0, s>>>(aabb, B.order, n, cnt, pl, pn, B.nodes, vis);
        k_keys_gather<<<nb(n, 256), 256, 0, s>>>(k2, B.order, n, k1);
    }
    k_trirec<<<nb(n, 256), 256, 0, s>>>(B.verts, B.tris, B.tri_mat, B.order, n, B.trirec);
    if ((err = cudaGetLastError()) != cudaSuccess) return fail_free(err);
    if ((err = cudaMemcpyAsync(nlarge_host, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return fail_free(err);
    return cudaFreeAsync(base, s);
}

}  // namespace rmsbr
