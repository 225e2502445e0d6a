// Device-side data layouts shared by the kernels of the SBR radio-map library.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rmsbr.h"

namespace rmsbr {

constexpr unsigned FULL_MASK = 0xffffffffu;
constexpr int MAX_BLOCK = 256;        // threads per block of the tracer (at most)
constexpr int STACK_SIZE = 64;        // BVH traversal stack entries per ray
constexpr int32_t NO_CELL = -32768;

// Per-material constants at the trace frequency.  eta = eps_r - j sigma /
// (eps0 omega) for the fields and for the (detached) sampling probabilities;
// k0d = 2 pi d / lambda0 split into two floats (hi + lo) so the slab phase
// keeps FP64 accuracy in its constant.
//
// Diffuse reflection (App. A.10): S, R^2 = (1 - S)(1 + S) and R = sqrt(1 - S^2)
// (Eq. R), sqrt(K_x), sqrt(1 - K_x), the pattern (0 Lambertian, 1 directive,
// 2 backscattering), its lobe exponents and split Lambda.  S = 0, R = R^2 = 1
// when the material (or the call) has no diffuse reflection.
struct MatDev {
    float eta_re, eta_im;
    float seta_re, seta_im;
    float k0d_hi, k0d_lo;
    int32_t slab;
    int32_t pattern;
    float S, R2, Rred;
    float sqk, sq1k;
    int32_t alpha_r, alpha_i;
    float lam;
};

// Per-transmitter constants.
struct TxDev {
    float pos[3];
    float R[9];                  // antenna orientation, row-major
    int32_t pattern, pol;
    float dep_scale;             // (4 pi / (N Delta^2)) (lambda0 / 4 pi)^2
    int32_t ant_mode;            // synthetic array table: 0 one record per element, 1 uniform linear array
    unsigned long long N;        // lattice size
    unsigned long long begin, stride, count;
    unsigned long long work_begin;  // first work item of this transmitter
    unsigned long long seed;
    unsigned long long rec_begin;   // first debug record of this transmitter
    unsigned long long perm;        // visit order: subset index i = (j * perm) mod count (1 = identity)
    unsigned long long perm_m;      // floor((2^64 - 1) / count): Barrett reduction of j * perm mod count
    int32_t n_ant, ant_begin;       // synthetic array elements in the antenna table
};

// One element of a synthetic transmit array: complex precoding weight and
// position in the global frame in units of lambda0 / 2 (d' = 2 d / lambda0,
// so that k.d' is the phase in units of pi) as hi + lo floats.  A uniform
// linear array stores d'_0 and the spacing in two such records, then its
// weights packed as float2 pairs (array.cuh).
struct AntDev {
    float pre, pim;
    float dh[3], dl[3];
};

// Scratch of one trace launch (zeroed before the launch).
struct Scratch {
    unsigned long long next;     // work-queue head
    unsigned long long cnt[6];   // rays, segments, nodes, tris, deposits, escapes
    unsigned long long seg_depth[RM_MAX_DEPTH + 1];
    double pw[RM_MAX_DEPTH + 1], pw2[RM_MAX_DEPTH + 1], esc[RM_MAX_DEPTH + 1];
    double grad[2 * RM_MAX_MATERIALS + 3 * RM_MAX_TX];
    int32_t status;              // bit 0: traversal stack or step budget overflow; bit 1: crossing limit
    int32_t pad;
};

struct TraceArgs {
    const float4* nodes;         // [nt-1][4]
    const float4* tris;          // [nt][3], leaf order: tree leaves, then the large triangles
    int32_t nt;                  // triangles in the tree
    int32_t nlarge;              // large triangles, tested from a list at slots nt .. nt+nlarge-1
    int32_t ntx, nm;
    int32_t L;
    uint32_t flags;
    float x0, y0, zm, cell, inv_cell;
    int32_t nx, ny;
    float inv_eps0_omega;        // 1 / (eps0 omega): d eta / d sigma = -j / (eps0 omega)
    int32_t same_sampling;
    unsigned long long total;    // work items (sum of ray counts)
    unsigned long long qchunk;   // work items a warp takes per queue access (multiple of 32)
    int32_t refill_min;          // idle lanes (1..32) before a warp refills them
    int32_t pad_refill;
    unsigned long long ncell;    // nx * ny
    const MatDev* mats;          // [nm]
    const TxDev* tx;             // [ntx]
    const AntDev* ant;           // synthetic-array elements of all transmitters
    float k0;                    // 2 pi / lambda0
    int32_t rr_depth;            // early termination after this many interactions (0 = off)
    float rr_pmax;               // Russian roulette p_max (0 = off)
    float gain_thr;              // gain threshold (0 = off)
    float lam4pi2;               // (lambda0 / 4 pi)^2
    Scratch* scratch;
    float* maps;                 // [ntx][ny][nx] (forward, FP32 accumulation when maps64 is null)
    double* maps64;              // [ntx][ny][nx] FP64 accumulation buffer (forward), or null
    const float* dLdC;           // [ntx][ny][nx] (adjoint)
    rm_segment_record* record;   // optional
    // optional [L+1][total] leaf slot of every segment's closest hit (-1: escaped), at
    // [depth][work item]: a warp's lanes hold consecutive work items, so its stores and loads
    // coalesce.  The recording forward writes it, the adjoint replays it instead of
    // traversing (a slot outside the scene falls back to the traversal)
    int32_t* hits;
    // optional [total] synthetic-array factor alpha of every work item's ray (transmitters
    // with arrays only), written by k_alpha before the tracer; null: the tracer evaluates
    // alpha at each ray's launch
    const float2* alpha;
    // mesh measurement surface (forward only): its LBVH and leaf records; the
    // maps are then [ntx][surface triangles] and the plane fields are unused
    const float4* snodes;
    const float4* stris;
    int32_t snt, snlarge;
};

// First-order diffraction map (diffraction.cu).  The UTD transition function
// is evaluated through the Faddeeva function w(z) with Weideman's rational
// expansion of FADDEEVA_N terms (coefficients from faddeeva_coefficients).
constexpr int FADDEEVA_N = 16;
struct DiffArgs {
    const float4* nodes;         // LBVH (as for the tracer)
    const float4* tris;
    int32_t nt, nlarge;
    const rm_wedge* wedges;      // [nw] (device copy)
    long long nw;
    const MatDev* mats;          // [nm]
    const TxDev* tx;             // [ntx]
    const AntDev* ant;
    int32_t ntx, nm;
    unsigned long long ns;       // samples per wedge
    unsigned long long total;    // ntx * nw * ns
    float x0, y0, zm, cell, inv_cell;
    int32_t nx, ny, bilinear;
    unsigned long long ncell;
    float k0;                    // 2 pi / lambda0
    float lam4pi2_over_cell2;    // (lambda0 / 4 pi)^2 / Delta^2
    float wz_L;                  // Weideman's L
    float wz_a[FADDEEVA_N];      // a_1 .. a_N
    int32_t npol, stats;
    double* maps64;              // [ntx][ny][nx] (or [ntx][surface triangles])
    rm_segment_record* record;   // optional, [ntx][nw][ns]
    Scratch* scratch;
    // mesh measurement surface (or null for the plane): its LBVH and leaf
    // records; lam4pi2_over_cell2 is then (lambda0 / 4 pi)^2 (cell = 1)
    const float4* snodes;
    const float4* stris;
    int32_t snt, snlarge;
};
cudaError_t launch_diffraction(const DiffArgs& a, int block, cudaStream_t s, int* grid_out, bool mesh = false);
// Weideman's L and a_1..a_N for w(z) = 2 p(Z) / (L - iz)^2 + (1/sqrt(pi)) / (L - iz),
// p(Z) = sum_{n<N} a_{n+1} Z^n, Z = (L + iz)/(L - iz) (host, double).
void faddeeva_coefficients(int N, double* L, double* a);

// Every device and pinned-host allocation of the library goes through these
// wrappers, which count the calls for rm_debug_alloc_count (api.cu).
void note_alloc();
inline cudaError_t lib_malloc(void** p, size_t n) {
    note_alloc();
    return cudaMalloc(p, n);
}
inline cudaError_t lib_malloc_async(void** p, size_t n, cudaStream_t s) {
    note_alloc();
    return cudaMallocAsync(p, n, s);
}
inline cudaError_t lib_host_alloc(void** p, size_t n, unsigned flags) {
    note_alloc();
    return cudaHostAlloc(p, n, flags);
}

// Host-side launchers (trace.cu)
// hits: the plain forward that records every segment's closest hit in a.hits
cudaError_t launch_trace(const TraceArgs& a, int npol, bool debug, bool bilinear, bool adjoint, bool diffuse,
                         int block, int blocks_per_sm, cudaStream_t s, int* grid_out, bool mesh = false,
                         bool hits = false);
int max_blocks_per_sm(int npol, bool debug, bool bilinear, bool adjoint, bool diffuse, int block, bool mesh = false,
                      bool hits = false);
// wR, wT (the coin's weights) of one material at n cosines of incidence (trace.cu)
cudaError_t launch_fresnel_probe(const MatDev& m, const float* cos1, long long n, float* wR, float* wT,
                                 cudaStream_t s);

// BVH build (bvh.cu)
struct BvhBuffers {
    const float* verts;
    const int32_t* tris;
    const int32_t* tri_mat;
    int64_t nt;
    uint64_t* keys_sorted;   // [nt]
    int32_t* order;          // [nt]
    float4* nodes;           // [nt-1][4]
    float4* trirec;          // [nt][3]
};
// at most this many large triangles are kept out of the tree (tested from a list)
constexpr int MAX_LARGE_TRIS = 16;
// tree builders (rm_bvh_build_ex): the Karras LBVH or the binned-SAH tree over the same leaves
constexpr int BVH_LBVH = 1;
constexpr int BVH_SAH = 2;
// Enqueues the build on s; *large_count_host receives the number of large
// triangles (the list is used when it is 1..MAX_LARGE_TRIS) once s reaches it.
cudaError_t build_bvh(const BvhBuffers& b, int builder, cudaStream_t s, int32_t* large_count_host);
cudaError_t check_indices(const int32_t* tris, const int32_t* tri_mat, int64_t nt, int64_t nv, int32_t nm,
                          int32_t* flag_dev, cudaStream_t s);

// loss (loss.cu)
cudaError_t launch_db_mse(const float* maps, const float* target, int64_t n, float floor_lin,
                          double* acc_dev, float* loss, float* dLdC, int64_t* valid, cudaStream_t s);
cudaError_t launch_fill_record(rm_segment_record* rec, unsigned long long n, cudaStream_t s);
// alpha[w] for every work item w of a transmitter with a synthetic array (trace.cu);
// wide = false: the tracer's inline form (debug comparison)
cudaError_t launch_alpha(const TraceArgs& a, float2* alpha, cudaStream_t s, bool wide = true);
cudaError_t launch_map_to_f32(const double* m64, float* m, unsigned long long n, cudaStream_t s);
cudaError_t launch_grad_out(const double* grad, int nm, int ntx, float* d_eps, float* d_sigma, float* d_tx,
                            cudaStream_t s);

}  // namespace rmsbr
