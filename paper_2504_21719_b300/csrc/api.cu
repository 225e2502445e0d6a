// C ABI of the SBR radio-map library (declared in include/rmsbr.h): argument
// validation, scene and plan lifetime, per-call constant tables and launches.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

using namespace rmsbr;

struct rm_scene {
    int device = 0;
    int64_t nv = 0, nt = 0;
    int32_t nm = 0;
    char* mesh_mem = nullptr;    // one allocation: verts, tris, tri_mat
    char* bvh_mem = nullptr;     // one allocation: keys, order, nodes, trirec
    float* verts = nullptr;
    int32_t* tris = nullptr;
    int32_t* tri_mat = nullptr;
    std::vector<rm_material> mats, smats;
    bool has_smats = false;
    bool built = false;
    int32_t builder = 0;         // RM_BVH_LBVH or RM_BVH_SAH once built
    // triangles kept out of the tree (tested from a list).  The build does not
    // wait for its count: the device copies it into a pinned slot and records
    // built_ev; the first call that needs it (resolve_nlarge) waits there.
    mutable int64_t nlarge = 0;
    mutable bool nlarge_pending = false;
    mutable int32_t* nlarge_slot = nullptr;
    mutable cudaEvent_t built_ev = nullptr;
    mutable std::mutex mu;
    uint64_t* keys = nullptr;
    int32_t* order = nullptr;
    float4* nodes = nullptr;
    float4* trirec = nullptr;
};

struct rm_trace_plan {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    char* dev = nullptr;
    Scratch* scratch = nullptr;
    int ntx = 0, L = 0;
    // recorded by the graph around its tracer node: the kernel time of the last launch
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Scene memory comes from the device's stream-ordered pool.  By default the
// pool returns its unused memory to the driver at every synchronisation, so
// the next scene would map fresh pages; keep up to 1 GiB of it cached instead
// (a per-process setting of this device's default pool, set once).
void keep_pool_memory() {
    static thread_local int done_for = -1;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev == done_for) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = 1ull << 30;
        uint64_t cur = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < thr)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done_for = dev;
}

constexpr double PI = 3.14159265358979323846;
constexpr double C0 = 299792458.0;          // m/s
constexpr double EPS0 = 8.8541878128e-12;   // F/m (CODATA 2018)
constexpr int DEFAULT_BLOCK = 128;
constexpr int DEFAULT_REFILL_MIN = 20;  // idle lanes before a warp refills (measured optimum 16..28)
constexpr int MAX_ANT = 4096;   // synthetic-array elements per call

thread_local std::string g_err;

rm_status fail(rm_status s, const std::string& m) {
    g_err = m;
    return s;
}
rm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? RM_ENOMEM : RM_ECUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}
#define RM_CUDA(expr)                                      \
    do {                                                   \
        cudaError_t e_ = (expr);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #expr); \
    } while (0)

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Host-side fault injection (failure detection is tested without a GPU
// fault): an armed kind makes its next `count` checks fail on the host, with
// the status the real failure would return.  Armed by rm_debug_inject or once
// per process by RM_FAULT=<alloc|launch|overflow>[:count].
std::atomic<int> g_fault[4];
std::once_flag g_fault_env;
void arm_from_env() {
    const char* v = std::getenv("RM_FAULT");
    if (!v) return;
    const std::string sv(v);
    const std::string kind = sv.substr(0, sv.find(':'));
    const int count = sv.find(':') == std::string::npos ? 1 : std::atoi(sv.c_str() + sv.find(':') + 1);
    const int k = kind == "alloc" ? RM_FAULT_ALLOC : kind == "launch" ? RM_FAULT_LAUNCH
                : kind == "overflow" ? RM_FAULT_OVERFLOW : 0;
    if (k && count > 0) g_fault[k].store(count);
}
bool injected(int kind) {
    std::call_once(g_fault_env, arm_from_env);
    int c = g_fault[kind].load();
    while (c > 0)
        if (g_fault[kind].compare_exchange_weak(c, c - 1)) return true;
    return false;
}

rm_status check_device(const rm_scene* sc) {
    int dev = -1;
    RM_CUDA(cudaGetDevice(&dev));
    if (dev != sc->device) return fail(RM_ESTATE, "current device differs from the scene's device");
    return RM_OK;
}

// Pinned host slots for the large-triangle count of pending builds: one
// process-wide slab (allocated on first use, kept until exit).
struct PinPool {
    std::mutex m;
    int32_t* slab = nullptr;
    bool tried = false;
    std::vector<int> free;
};
PinPool g_pin;
constexpr int PIN_SLOTS = 4096;

int32_t* pin_slot_acquire() {
    std::lock_guard<std::mutex> g(g_pin.m);
    if (!g_pin.tried) {
        g_pin.tried = true;
        if (lib_host_alloc((void**)&g_pin.slab, sizeof(int32_t) * PIN_SLOTS, cudaHostAllocPortable) == cudaSuccess)
            for (int i = PIN_SLOTS - 1; i >= 0; --i) g_pin.free.push_back(i);
        else
            g_pin.slab = nullptr;
    }
    if (g_pin.free.empty()) return nullptr;
    const int i = g_pin.free.back();
    g_pin.free.pop_back();
    return g_pin.slab + i;
}

void pin_slot_release(int32_t* p) {
    if (!p) return;
    std::lock_guard<std::mutex> g(g_pin.m);
    g_pin.free.push_back((int)(p - g_pin.slab));
}

// The large-triangle count of a scene whose build has not been waited for:
// wait for the build's event, read the slot, release it.  Errors of the
// asynchronous build surface here.
rm_status resolve_nlarge(const rm_scene* sc) {
    std::lock_guard<std::mutex> g(sc->mu);
    if (!sc->nlarge_pending) return RM_OK;
    const cudaError_t e = cudaEventSynchronize(sc->built_ev);
    const int32_t large = *sc->nlarge_slot;
    pin_slot_release(sc->nlarge_slot);
    cudaEventDestroy(sc->built_ev);
    sc->nlarge_slot = nullptr;
    sc->built_ev = nullptr;
    sc->nlarge_pending = false;
    if (e != cudaSuccess) return cuda_fail(e, "rm_bvh_build (asynchronous part)");
    sc->nlarge = (large > 0 && large <= MAX_LARGE_TRIS) ? large : 0;
    return RM_OK;
}

rm_status check_materials(const rm_material* m, int32_t nm) {
    if (nm < 1 || nm > RM_MAX_MATERIALS) return fail(RM_EINVAL, "nm must be in [1, 32]");
    if (!m) return fail(RM_EINVAL, "materials pointer is NULL");
    for (int i = 0; i < nm; ++i) {
        if (!std::isfinite(m[i].eps_r) || !std::isfinite(m[i].sigma) || !std::isfinite(m[i].thickness) ||
            m[i].eps_r <= 0.0f || m[i].sigma < 0.0f)
            return fail(RM_EINVAL, "material " + std::to_string(i) + " has eps_r <= 0, sigma < 0 or a non-finite value");
        if (!(m[i].scattering >= 0.0f && m[i].scattering <= 1.0f))
            return fail(RM_EINVAL, "material " + std::to_string(i) + ": scattering must be in [0, 1]");
        if (m[i].scattering > 0.0f) {
            const rm_material& x = m[i];
            const bool ok = x.xpd_k >= 0.0f && x.xpd_k <= 1.0f && x.pattern >= 0 && x.pattern <= 2 &&
                            (x.pattern == 0 || (x.alpha_r >= 1 && x.alpha_r <= 32)) &&
                            (x.pattern != 2 || (x.alpha_i >= 1 && x.alpha_i <= 32 && x.lobe_lambda >= 0.0f &&
                                                x.lobe_lambda <= 1.0f));
            if (!ok)
                return fail(RM_EINVAL, "material " + std::to_string(i) +
                                           ": xpd_k, lobe_lambda in [0, 1], pattern in {0, 1, 2}, alpha in [1, 32] required");
        }
    }
    return RM_OK;
}

uint64_t tx_count(const rm_tx& t) {
    if (t.ray_count != UINT64_MAX) return t.ray_count;
    if (t.ray_begin >= t.num_rays) return 0;
    return (t.num_rays - t.ray_begin + t.ray_stride - 1) / t.ray_stride;
}

rm_status validate(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p) {
    if (!sc) return fail(RM_EINVAL, "scene is NULL");
    if (!sc->built) return fail(RM_ESTATE, "rm_bvh_build has not been called on this scene");
    if (rm_status r = resolve_nlarge(sc); r != RM_OK) return r;
    if (!tx || !p) return fail(RM_EINVAL, "tx or params is NULL");
    if (ntx < 1 || ntx > RM_MAX_TX) return fail(RM_EINVAL, "ntx must be in [1, 64]");
    if (!(p->freq_hz > 0.0) || !std::isfinite(p->freq_hz)) return fail(RM_EINVAL, "freq_hz must be > 0");
    if (p->max_depth < 0 || p->max_depth > RM_MAX_DEPTH) return fail(RM_EINVAL, "max_depth must be in [0, 15]");
    if (!(p->cell_size > 0.0f) || !std::isfinite(p->cell_size)) return fail(RM_EINVAL, "cell_size must be > 0");
    if (p->nx < 1 || p->ny < 1 || p->nx > 32767 || p->ny > 32767 || (int64_t)p->nx * p->ny > INT32_MAX)
        return fail(RM_EINVAL, "nx, ny must be in [1, 32767] with nx*ny < 2^31");
    if (p->deposit != 0 && p->deposit != 1) return fail(RM_EINVAL, "deposit must be 0 (box) or 1 (bilinear)");
    if (p->block_size != 0 && (p->block_size < 32 || p->block_size > MAX_BLOCK || (p->block_size & 31)))
        return fail(RM_EINVAL, "block_size must be 0 or a multiple of 32 in [32, 256]");
    if (p->blocks_per_sm < 0) return fail(RM_EINVAL, "blocks_per_sm must be >= 0");
    if (p->queue_chunk < 0 || p->queue_chunk > 64) return fail(RM_EINVAL, "queue_chunk must be in [0, 64]");
    if (p->refill_min < 0 || p->refill_min > 32) return fail(RM_EINVAL, "refill_min must be in [0, 32]");
    if (p->rr_depth < 0 || !(p->rr_max_prob >= 0.0f && p->rr_max_prob <= 1.0f) || !(p->gain_threshold >= 0.0f))
        return fail(RM_EINVAL, "rr_depth >= 0, rr_max_prob in [0, 1] and gain_threshold >= 0 are required");
    for (int i = 0; i < 3; ++i)
        if (!std::isfinite(p->map_origin[i])) return fail(RM_EINVAL, "map_origin must be finite");
    for (int t = 0; t < ntx; ++t) {
        const rm_tx& x = tx[t];
        const std::string w = "tx " + std::to_string(t) + ": ";
        if (x.num_rays < 1 || x.num_rays >= (1ULL << 59)) return fail(RM_EINVAL, w + "num_rays must be in [1, 2^59)");
        if (x.ray_stride < 1) return fail(RM_EINVAL, w + "ray_stride must be >= 1");
        if (x.pol < 0 || x.pol > 2) return fail(RM_EINVAL, w + "pol must be 0, 1 or 2");
        if (x.pattern < 0 || x.pattern > 1) return fail(RM_EINVAL, w + "pattern must be 0 or 1");
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(x.pos[i])) return fail(RM_EINVAL, w + "position must be finite");
        if (!std::isfinite(x.yaw) || !std::isfinite(x.pitch) || !std::isfinite(x.roll))
            return fail(RM_EINVAL, w + "orientation must be finite");
        if (x.n_ant < 0 || x.n_ant > MAX_ANT || (x.n_ant > 0 && (!x.ant_pos_host || !x.precoding_host)))
            return fail(RM_EINVAL, w + "n_ant must be in [0, 4096] with element positions and precoding");
        for (int a = 0; a < x.n_ant; ++a)
            for (int c3 = 0; c3 < 3; ++c3)
                if (!std::isfinite(x.ant_pos_host[3 * a + c3]) || (c3 < 2 && !std::isfinite(x.precoding_host[2 * a + c3])))
                    return fail(RM_EINVAL, w + "antenna positions and precoding must be finite");
        const uint64_t c = tx_count(x);
        if (c > 0) {
            if (x.ray_begin >= x.num_rays) return fail(RM_EINVAL, w + "ray_begin >= num_rays");
            if ((c - 1) > (x.num_rays - 1 - x.ray_begin) / x.ray_stride)
                return fail(RM_EINVAL, w + "ray subset exceeds the lattice");
        }
    }
    int64_t nant = 0;
    for (int t = 0; t < ntx; ++t) nant += tx[t].n_ant;
    if (nant > MAX_ANT) return fail(RM_EINVAL, "more than 4096 array elements in one call");
    if (ntx > 1) {
        const int np = tx[0].pol == 2 ? 2 : 1;
        for (int t = 1; t < ntx; ++t)
            if ((tx[t].pol == 2 ? 2 : 1) != np)
                return fail(RM_EINVAL, "all transmitters of one call must be dual-polarised or none");
    }
    return RM_OK;
}

struct Prepared {
    TraceArgs a;
    std::vector<MatDev> mats;
    std::vector<TxDev> tx;
    std::vector<AntDev> ant;
    int npol = 1;
    bool bilinear = false;
    bool diffuse = false;        // a diffuse-capable kernel is needed
    int block = DEFAULT_BLOCK;
    int bps = 0;
    double kernel_ms = 0.0;
    bool mesh = false;          // maps on a mesh measurement surface
};

uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) {
        const uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Visit order of a transmitter's rays.  In a Fibonacci lattice of N points the
// directions n and n + F_k (F_k a Fibonacci number near 1.24 sqrt(N)) are
// nearest neighbours, so visiting i = j F_k mod count gives every warp a tight
// bundle of directions (coherent traversal) without changing which rays are
// traced.  Identity for strided subsets, small counts, or no coprime F_k.
uint64_t visit_step(const rm_tx& t, uint64_t count) {
    if (t.ray_stride != 1 || count < 4096) return 1;
    const double target = 1.24 * std::sqrt((double)t.num_rays);
    std::vector<uint64_t> fib{1, 2};
    while (fib.back() < (1ULL << 40)) fib.push_back(fib[fib.size() - 1] + fib[fib.size() - 2]);
    size_t k = 0;
    for (size_t i = 0; i < fib.size(); ++i)
        if (std::fabs((double)fib[i] - target) < std::fabs((double)fib[k] - target)) k = i;
    const int order[5] = {0, -1, 1, -2, 2};
    for (int d : order) {
        const long long j = (long long)k + d;
        if (j < 1 || j >= (long long)fib.size()) continue;
        const uint64_t F = fib[j];
        if (F >= count || gcd64(F, count) != 1) continue;
        if ((double)F * (double)count >= 9.0e18) continue;  // (j * F) must fit in 64 bits
        return F;
    }
    return 1;
}

void rotation(double a, double b, double g, float* R) {
    // R = Rz(a) Ry(b) Rx(g)  (Eq. rotation)
    const double ca = std::cos(a), sa = std::sin(a), cb = std::cos(b), sb = std::sin(b), cg = std::cos(g),
                 sg = std::sin(g);
    const double M[9] = {ca * cb, ca * sb * sg - sa * cg, ca * sb * cg + sa * sg,
                         sa * cb, sa * sb * sg + ca * cg, sa * sb * cg - ca * sg,
                         -sb,     cb * sg,                cb * cg};
    for (int i = 0; i < 9; ++i) R[i] = (float)M[i];
}
// The synthetic-array table of one transmitter (layout in array.cuh): element
// positions rotated with the antenna (R d), scaled to d' = 2 d / lambda0 and
// split into hi + lo floats, in double.  Elements on one regular line (to
// 1e-8 lambda0) are stored as a uniform linear array: d'_0, the spacing, and
// the weights packed in pairs.
void pack_array(const rm_tx& x, double lam, TxDev& d, std::vector<AntDev>& out) {
    const int n = x.n_ant;
    d.ant_mode = 0;
    if (n <= 0) return;
    const double ca = std::cos(x.yaw), sa = std::sin(x.yaw), cb = std::cos(x.pitch), sb = std::sin(x.pitch),
                 cg = std::cos(x.roll), sg = std::sin(x.roll);
    const double M[9] = {ca * cb, ca * sb * sg - sa * cg, ca * sb * cg + sa * sg,
                         sa * cb, sa * sb * sg + ca * cg, sa * sb * cg - ca * sg,
                         -sb,     cb * sg,                cb * cg};
    std::vector<double> g((size_t)3 * n);
    for (int a = 0; a < n; ++a) {
        const double* l = x.ant_pos_host + 3 * a;
        for (int i = 0; i < 3; ++i) g[3 * a + i] = (M[3 * i] * l[0] + M[3 * i + 1] * l[1] + M[3 * i + 2] * l[2]) * 2.0 / lam;
    }
    auto split = [](const double* v, AntDev& e) {
        for (int i = 0; i < 3; ++i) {
            e.dh[i] = (float)v[i];
            e.dl[i] = (float)(v[i] - (double)e.dh[i]);
        }
    };
    bool ula = n >= 2;
    double step[3] = {0.0, 0.0, 0.0};
    if (ula) {
        for (int i = 0; i < 3; ++i) step[i] = (g[3 * (n - 1) + i] - g[i]) / (n - 1);
        for (int a = 0; a < n && ula; ++a)
            for (int i = 0; i < 3; ++i)
                if (std::fabs(g[3 * a + i] - (g[i] + a * step[i])) > 2e-8) ula = false;
    }
    if (ula) {
        d.ant_mode = 1;
        AntDev h0{}, h1{};
        split(g.data(), h0);
        split(step, h1);
        out.push_back(h0);
        out.push_back(h1);
        for (int a = 0; a < n; a += 4) {
            AntDev w{};
            float* f = reinterpret_cast<float*>(&w);
            for (int j = 0; j < 4 && a + j < n; ++j) {
                f[2 * j] = (float)x.precoding_host[2 * (a + j)];
                f[2 * j + 1] = (float)x.precoding_host[2 * (a + j) + 1];
            }
            out.push_back(w);
        }
        return;
    }
    for (int a = 0; a < n; ++a) {
        AntDev e{};
        e.pre = (float)x.precoding_host[2 * a];
        e.pim = (float)x.precoding_host[2 * a + 1];
        split(&g[3 * a], e);
        out.push_back(e);
    }
}


// Per-material constants at angular frequency omega (k0 = omega / c0): the
// field's eta = eps_r - j sigma / (eps0 omega) from e, the sampling eta from s,
// the slab phase constant k0 d as hi + lo floats and the diffuse parameters.
// Returns whether the material scatters diffusely in this call.
bool fill_matdev(const rm_material& e, const rm_material& s, double omega, double k0, unsigned flags, MatDev* out) {
    MatDev& d = *out;
    d.eta_re = e.eps_r;
    d.eta_im = (float)(-(double)e.sigma / (EPS0 * omega));
    d.seta_re = s.eps_r;
    d.seta_im = (float)(-(double)s.sigma / (EPS0 * omega));
    const double k0d = e.thickness > 0.0f ? k0 * (double)e.thickness : 0.0;
    d.k0d_hi = (float)k0d;
    d.k0d_lo = (float)(k0d - (double)d.k0d_hi);
    d.slab = e.thickness > 0.0f ? 1 : 0;
    const bool dif = (flags & RM_DIFFUSE) && (flags & RM_REFLECT) && e.scattering > 0.0f;
    const double Sd = dif ? (double)e.scattering : 0.0;
    d.S = (float)Sd;
    d.R2 = (float)((1.0 - Sd) * (1.0 + Sd));
    d.Rred = (float)std::sqrt((1.0 - Sd) * (1.0 + Sd));
    d.sqk = dif ? (float)std::sqrt((double)e.xpd_k) : 0.0f;
    d.sq1k = dif ? (float)std::sqrt(1.0 - (double)e.xpd_k) : 1.0f;
    d.pattern = dif ? e.pattern : 0;
    d.alpha_r = dif && e.pattern > 0 ? e.alpha_r : 1;
    d.alpha_i = dif && e.pattern == 2 ? e.alpha_i : 1;
    d.lam = dif && e.pattern == 2 ? e.lobe_lambda : 1.0f;
    return dif;
}

void prepare(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p,
             const rm_material* sampling_override, Prepared* P, const rm_scene* surf = nullptr) {
    const double f = p->freq_hz, omega = 2.0 * PI * f, k0 = omega / C0, lam = C0 / f;
    const std::vector<rm_material>& sm = sc->has_smats ? sc->smats : sc->mats;
    P->mats.resize(sc->nm);
    bool same = !sampling_override && !sc->has_smats;
    for (int m = 0; m < sc->nm; ++m) {
        const rm_material& e = sc->mats[m];
        const rm_material& s = sampling_override ? sampling_override[m] : sm[m];
        if (fill_matdev(e, s, omega, k0, p->flags, &P->mats[m])) P->diffuse = true;
        if (s.eps_r != e.eps_r || s.sigma != e.sigma) same = false;
    }
    P->tx.resize(ntx);
    unsigned long long work = 0, rec = 0;
    const double a = lam / (4.0 * PI);
    for (int t = 0; t < ntx; ++t) {
        TxDev& d = P->tx[t];
        std::memset(&d, 0, sizeof d);
        for (int i = 0; i < 3; ++i) d.pos[i] = tx[t].pos[i];
        rotation(tx[t].yaw, tx[t].pitch, tx[t].roll, d.R);
        d.pattern = tx[t].pattern;
        d.pol = tx[t].pol;
        // planar cells: 4 pi / (N Delta^2) (lambda0 / 4 pi)^2; mesh cells divide by their own area in the kernel
        const double cell2 = surf ? 1.0 : (double)p->cell_size * (double)p->cell_size;
        d.dep_scale = (float)(4.0 * PI / ((double)tx[t].num_rays * cell2) * a * a);
        d.N = tx[t].num_rays;
        d.begin = tx[t].ray_begin;
        d.stride = tx[t].ray_stride;
        d.count = tx_count(tx[t]);
        d.work_begin = work;
        d.seed = tx[t].seed;
        d.rec_begin = rec;
        d.perm = visit_step(tx[t], d.count);
        d.perm_m = d.count > 0 ? ~0ULL / d.count : 0;
        d.n_ant = tx[t].n_ant;
        d.ant_begin = (int32_t)P->ant.size();
        pack_array(tx[t], lam, d, P->ant);
        work += d.count;
        rec += d.count * (unsigned long long)(p->max_depth + 1);
    }
    TraceArgs& A = P->a;
    std::memset(&A, 0, sizeof A);
    A.nodes = sc->nodes;
    A.tris = sc->trirec;
    A.nt = (int32_t)(sc->nt - sc->nlarge);
    A.nlarge = (int32_t)sc->nlarge;
    A.ntx = ntx;
    A.nm = sc->nm;
    A.L = p->max_depth;
    A.flags = p->flags;
    A.x0 = (float)((double)p->map_origin[0] - 0.5 * p->nx * (double)p->cell_size);
    A.y0 = (float)((double)p->map_origin[1] - 0.5 * p->ny * (double)p->cell_size);
    A.zm = p->map_origin[2];
    A.cell = p->cell_size;
    A.inv_cell = (float)(1.0 / (double)p->cell_size);
    A.nx = p->nx;
    A.ny = p->ny;
    A.inv_eps0_omega = (float)(1.0 / (EPS0 * omega));
    A.k0 = (float)k0;
    A.rr_depth = p->rr_depth;
    A.rr_pmax = p->rr_depth > 0 ? p->rr_max_prob : 0.0f;
    A.gain_thr = p->rr_depth > 0 ? p->gain_threshold : 0.0f;
    A.lam4pi2 = (float)(a * a);
    A.same_sampling = same ? 1 : 0;
    A.total = work;
    A.qchunk = 32ULL * (unsigned long long)(p->queue_chunk > 0 ? p->queue_chunk : 1);
    A.refill_min = p->refill_min > 0 ? p->refill_min : DEFAULT_REFILL_MIN;
    A.ncell = (unsigned long long)p->nx * p->ny;
    if (surf) {
        A.snodes = surf->nodes;
        A.stris = surf->trirec;
        A.snt = (int32_t)(surf->nt - surf->nlarge);
        A.snlarge = (int32_t)surf->nlarge;
        A.ncell = (unsigned long long)surf->nt;
    }
    P->mesh = surf != nullptr;
    P->npol = tx[0].pol == 2 ? 2 : 1;
    P->bilinear = p->deposit == 1;
    P->block = p->block_size ? p->block_size : DEFAULT_BLOCK;
    P->bps = p->blocks_per_sm;
}

// device block: [Scratch | MatDev[nm] | TxDev[ntx] | AntDev[n_ant total]]
size_t table_bytes(const Prepared& P, size_t* o_mat, size_t* o_tx) {
    size_t off = (sizeof(Scratch) + 255) & ~size_t(255);
    *o_mat = off;
    off += (P.mats.size() * sizeof(MatDev) + 255) & ~size_t(255);
    *o_tx = off;
    off += P.tx.size() * sizeof(TxDev);
    off = (off + 255) & ~size_t(255);
    off += P.ant.size() * sizeof(AntDev);
    return off;
}
size_t ant_offset(const Prepared& P, size_t o_tx) {
    return (o_tx + P.tx.size() * sizeof(TxDev) + 255) & ~size_t(255);
}

// the same block followed by the FP64 accumulation maps [ntx][ny][nx]
size_t block_bytes_with_maps64(const Prepared& P, size_t* o_mat, size_t* o_tx, size_t* o_m64) {
    const size_t t = table_bytes(P, o_mat, o_tx);
    *o_m64 = (t + 255) & ~size_t(255);
    return *o_m64 + sizeof(double) * P.a.ncell * P.tx.size();
}

void fill_stats(const Scratch& h, const Prepared& P, rm_stats* st) {
    std::memset(st, 0, sizeof *st);
    st->rays = h.cnt[0];
    st->segments = h.cnt[1];
    st->nodes_visited = h.cnt[2];
    st->tris_tested = h.cnt[3];
    st->deposits = h.cnt[4];
    st->escapes = h.cnt[5];
    for (int l = 0; l <= RM_MAX_DEPTH; ++l) {
        st->segments_per_depth[l] = h.seg_depth[l];
        st->power_per_depth[l] = h.pw[l];
        st->power2_per_depth[l] = h.pw2[l];
        st->escaped_power_per_depth[l] = h.esc[l];
    }
    st->status = (h.status & 3) ? RM_EOVERFLOW : RM_OK;
    st->kernel_ms = P.kernel_ms;
}

// Per-thread host resources of run_trace, kept across calls: a pinned staging
// buffer (the table image goes to the device in one copy, the scratch comes
// back in one copy) and two timing events.  Every call synchronises its
// stream before returning, so a staging buffer is never reused while a copy
// from it is pending.
struct ThreadRes {
    char* stage = nullptr;
    size_t cap = 0;
    int ev_device = -1;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    // device block [Scratch | tables | FP64 maps]: kept between calls so that
    // a trace does not map fresh device memory every time
    char* dblock = nullptr;
    size_t dcap = 0;
    int d_device = -1;
    ~ThreadRes() {
        if (stage) cudaFreeHost(stage);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (dblock) cudaFree(dblock);
    }
};
thread_local ThreadRes g_res;

// Per-thread pinned staging of rm_scene_upload_host: the mesh is copied here
// on the host and goes to the device in one asynchronous copy; `done` marks
// the end of that copy so that the next upload does not overwrite the buffer
// before the device has read it.
struct UploadStage {
    char* buf = nullptr;
    size_t cap = 0;
    int device = -1;
    cudaEvent_t done = nullptr;
    bool pending = false;
    ~UploadStage() {
        if (pending && done) cudaEventSynchronize(done);
        if (buf) cudaFreeHost(buf);
        if (done) cudaEventDestroy(done);
    }
};
thread_local UploadStage g_up;

cudaError_t upload_stage(size_t bytes, char** out) {
    cudaError_t e;
    if (g_up.pending) {
        if ((e = cudaEventSynchronize(g_up.done)) != cudaSuccess) return e;
        g_up.pending = false;
    }
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (g_up.device != dev) {
        if (g_up.done) cudaEventDestroy(g_up.done);
        g_up.done = nullptr;
        g_up.device = -1;
        if ((e = cudaEventCreateWithFlags(&g_up.done, cudaEventDisableTiming)) != cudaSuccess) return e;
        g_up.device = dev;
    }
    if (g_up.cap < bytes) {
        if (g_up.buf) cudaFreeHost(g_up.buf);
        g_up.buf = nullptr;
        g_up.cap = 0;
        const size_t want = std::max(bytes, size_t(256) << 10);
        if ((e = lib_host_alloc((void**)&g_up.buf, want, cudaHostAllocPortable)) != cudaSuccess) return e;
        g_up.cap = want;
    }
    *out = g_up.buf;
    return cudaSuccess;
}

cudaError_t device_block(size_t bytes, char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (g_res.dblock && (g_res.d_device != dev || g_res.dcap < bytes)) {
        // the previous call synchronised its stream: nothing uses the block
        int cur = dev;
        if (g_res.d_device != dev) cudaSetDevice(g_res.d_device);
        cudaFree(g_res.dblock);
        if (g_res.d_device != dev) cudaSetDevice(cur);
        g_res.dblock = nullptr;
        g_res.dcap = 0;
    }
    if (!g_res.dblock) {
        const size_t want = (bytes + (size_t(1) << 20) - 1) & ~((size_t(1) << 20) - 1);
        if ((e = lib_malloc((void**)&g_res.dblock, want)) != cudaSuccess) return e;
        g_res.dcap = want;
        g_res.d_device = dev;
    }
    *out = g_res.dblock;
    return cudaSuccess;
}

cudaError_t staging(size_t bytes, char** out) {
    if (g_res.cap < bytes) {
        if (g_res.stage) cudaFreeHost(g_res.stage);
        g_res.stage = nullptr;
        g_res.cap = 0;
        const size_t want = std::max(bytes, size_t(64) << 10);
        cudaError_t e = lib_host_alloc((void**)&g_res.stage, want, cudaHostAllocDefault);
        if (e != cudaSuccess) return e;
        g_res.cap = want;
    }
    *out = g_res.stage;
    return cudaSuccess;
}

cudaError_t timing_events(cudaEvent_t* ev) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (g_res.ev_device != dev) {
        for (cudaEvent_t& x : g_res.ev)
            if (x) {
                cudaEventDestroy(x);
                x = nullptr;
            }
        g_res.ev_device = -1;
        for (cudaEvent_t& x : g_res.ev)
            if ((e = cudaEventCreate(&x)) != cudaSuccess) return e;
        g_res.ev_device = dev;
    }
    ev[0] = g_res.ev[0];
    ev[1] = g_res.ev[1];
    return cudaSuccess;
}

// The table image [Scratch (zero) | MatDev | TxDev | AntDev] in the layout of
// table_bytes, written into host memory at `h`; returns its size.
size_t write_tables(const Prepared& P, size_t o_mat, size_t o_tx, char* h) {
    const size_t o_ant = ant_offset(P, o_tx);
    const size_t end = o_ant + P.ant.size() * sizeof(AntDev);
    std::memset(h, 0, end);
    std::memcpy(h + o_mat, P.mats.data(), P.mats.size() * sizeof(MatDev));
    std::memcpy(h + o_tx, P.tx.data(), P.tx.size() * sizeof(TxDev));
    if (!P.ant.empty()) std::memcpy(h + o_ant, P.ant.data(), P.ant.size() * sizeof(AntDev));
    return end;
}

rm_status run_trace(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p, float* maps,
                    const float* dLdC, float* d_eps, float* d_sig, float* d_tx, const rm_material* smats,
                    rm_stats* stats, rm_segment_record* record, void* stream, bool adjoint,
                    const rm_scene* surf = nullptr, int32_t* hits = nullptr, uint64_t hits_len = 0) {
    rm_status st = validate(sc, tx, ntx, p);
    if (st != RM_OK) return st;
    if ((st = check_device(sc)) != RM_OK) return st;
    if (surf) {
        if (!surf->built) return fail(RM_ESTATE, "rm_bvh_build has not been called on the surface");
        if ((st = resolve_nlarge(surf)) != RM_OK) return st;
        if ((st = check_device(surf)) != RM_OK) return st;
        if (surf->device != sc->device) return fail(RM_EINVAL, "scene and surface live on different devices");
        if (surf->nt < 1) return fail(RM_EINVAL, "the surface has no triangles");
        if (surf->nt > INT32_MAX) return fail(RM_EINVAL, "the surface has too many triangles");
        if (p->deposit != 0) return fail(RM_EINVAL, "mesh surfaces take box cells (deposit = 0)");
    }
    if (!adjoint && !maps) return fail(RM_EINVAL, "maps_dev is NULL");
    if (adjoint && !dLdC) return fail(RM_EINVAL, "dL_dmaps_dev is NULL");
    if (smats && (st = check_materials(smats, sc->nm)) != RM_OK) return st;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RM_CUDA(cudaStreamIsCapturing(S(stream), &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(RM_ESTATE, "stream is capturing; use rm_trace_plan_create for graph launches");

    if (injected(RM_FAULT_LAUNCH))
        return fail(RM_ECUDA, std::string(adjoint ? "rm_radio_map_grad" : "rm_radio_map_trace") +
                                  ": injected launch failure (nothing was enqueued)");
    Prepared P;
    prepare(sc, tx, ntx, p, smats, &P, surf);
    if (hits) {
        unsigned long long need = 0;
        for (const TxDev& t : P.tx) need += t.count * (unsigned long long)(p->max_depth + 1);
        if (hits_len < need) return fail(RM_EINVAL, "hits_len is below the segments' count (rays x (max_depth + 1))");
    }
    // the forward that records its hits runs its own instantiation of the plain tracer (or the debug
    // one, which records them too, when a record or statistics are asked for)
    const bool debug = record != nullptr || (p->flags & RM_STATS);
    const bool record_hits = hits && !adjoint && !debug;
    size_t o_mat, o_tx, o_m64 = 0;
    size_t bytes = adjoint ? table_bytes(P, &o_mat, &o_tx) : block_bytes_with_maps64(P, &o_mat, &o_tx, &o_m64);
    // transmitters with synthetic arrays: alpha of every work item from a pre-pass (8 B per
    // ray, up to 2^31 rays per call; beyond that the tracer evaluates it at each launch)
    bool arrays = false;
    for (const TxDev& t : P.tx) arrays = arrays || t.n_ant > 0;
    const bool pre_alpha = arrays && P.a.total > 0 && P.a.total <= (1ULL << 31);
    const size_t o_alpha = align256(bytes);
    if (pre_alpha) bytes = o_alpha + sizeof(float2) * (size_t)P.a.total;
    cudaEvent_t ev[2];
    RM_CUDA(timing_events(ev));
    char* hst = nullptr;
    RM_CUDA(staging(table_bytes(P, &o_mat, &o_tx), &hst));
    const size_t tab = write_tables(P, o_mat, o_tx, hst);
    bool timed = false;
    char* dev = nullptr;
    RM_CUDA(device_block(bytes, &dev));
    cudaError_t e = cudaSuccess;
    int grid = 0;
    do {
        // zeroed scratch and all constant tables in one copy from pinned memory
        if ((e = cudaMemcpyAsync(dev, hst, tab, cudaMemcpyHostToDevice, S(stream))) != cudaSuccess) break;
        if (!adjoint && (e = cudaMemsetAsync(dev + o_m64, 0, sizeof(double) * P.a.ncell * ntx, S(stream))) != cudaSuccess)
            break;
        unsigned long long nrec = 0;
        for (const TxDev& t : P.tx) nrec += t.count * (unsigned long long)(p->max_depth + 1);
        if (record && (e = launch_fill_record(record, nrec, S(stream))) != cudaSuccess) break;
        P.a.mats = reinterpret_cast<const MatDev*>(dev + o_mat);
        P.a.tx = reinterpret_cast<const TxDev*>(dev + o_tx);
        P.a.ant = reinterpret_cast<const AntDev*>(dev + ant_offset(P, o_tx));
        P.a.scratch = reinterpret_cast<Scratch*>(dev);
        P.a.maps = maps;
        P.a.maps64 = adjoint ? nullptr : reinterpret_cast<double*>(dev + o_m64);
        P.a.dLdC = dLdC;
        P.a.record = record;
        P.a.hits = hits;
        if (pre_alpha) P.a.alpha = reinterpret_cast<const float2*>(dev + o_alpha);
        if (P.a.total > 0) {
            if ((e = cudaEventRecord(ev[0], S(stream))) != cudaSuccess) break;
            if (pre_alpha && (e = launch_alpha(P.a, reinterpret_cast<float2*>(dev + o_alpha), S(stream))) != cudaSuccess)
                break;
            if ((e = launch_trace(P.a, P.npol, debug, P.bilinear, adjoint, P.diffuse, P.block, P.bps, S(stream), &grid,
                                  P.mesh, record_hits)) != cudaSuccess)
                break;
            if ((e = cudaEventRecord(ev[1], S(stream))) != cudaSuccess) break;
            timed = true;
        }
        if (adjoint && (e = launch_grad_out(reinterpret_cast<const Scratch*>(dev)->grad, sc->nm, ntx, d_eps, d_sig,
                                            d_tx, S(stream))) != cudaSuccess) break;
        if (!adjoint && (e = launch_map_to_f32(P.a.maps64, maps, P.a.ncell * ntx, S(stream))) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(hst, dev, sizeof(Scratch), cudaMemcpyDeviceToHost, S(stream))) != cudaSuccess) break;
    } while (false);
    cudaError_t e3 = cudaStreamSynchronize(S(stream));
    Scratch host;
    std::memcpy(&host, hst, sizeof(Scratch));
    float ms = 0.0f;
    if (timed && e == cudaSuccess && e3 == cudaSuccess && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess)
        P.kernel_ms = ms;
    if (e != cudaSuccess) return cuda_fail(e, adjoint ? "rm_radio_map_grad" : "rm_radio_map_trace");
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamSynchronize");
    if (injected(RM_FAULT_OVERFLOW)) host.status |= 1;   // as if the device had set its status word
    if (stats) fill_stats(host, P, stats);
    if (host.status & 1) return fail(RM_EOVERFLOW, "BVH traversal stack overflow; affected rays were dropped");
    return RM_OK;
}

}  // namespace

// Allocation calls made by the library in this process (rm_debug_alloc_count).
static std::atomic<unsigned long long> g_alloc_calls{0};
void rmsbr::note_alloc() { g_alloc_calls.fetch_add(1, std::memory_order_relaxed); }

extern "C" {

const char* rm_last_error(void) { return g_err.c_str(); }

uint64_t rm_debug_alloc_count(void) { return g_alloc_calls.load(std::memory_order_relaxed); }

rm_status rm_debug_inject(int32_t kind, int32_t count) {
    if (kind < RM_FAULT_ALLOC || kind > RM_FAULT_OVERFLOW || count < 0)
        return fail(RM_EINVAL, "kind must be RM_FAULT_ALLOC, RM_FAULT_LAUNCH or RM_FAULT_OVERFLOW, count >= 0");
    std::call_once(g_fault_env, arm_from_env);
    g_fault[kind].store(count);
    return RM_OK;
}

rm_status rm_debug_fresnel_probe(const rm_material* mat, double freq_hz, const float* cos1_dev, int64_t n,
                                 float* wR_dev, float* wT_dev, void* stream) {
    if (!mat) return fail(RM_EINVAL, "mat is NULL");
    if ((n > 0 && (!cos1_dev || !wR_dev || !wT_dev)) || n < 0) return fail(RM_EINVAL, "bad arrays");
    if (!(freq_hz > 0.0) || !std::isfinite(freq_hz)) return fail(RM_EINVAL, "freq_hz must be > 0");
    rm_status st = check_materials(mat, 1);
    if (st != RM_OK) return st;
    const double omega = 2.0 * PI * freq_hz;
    MatDev d;
    std::memset(&d, 0, sizeof d);
    fill_matdev(*mat, *mat, omega, omega / C0, RM_REFLECT | RM_REFRACT, &d);
    RM_CUDA(launch_fresnel_probe(d, cos1_dev, n, wR_dev, wT_dev, S(stream)));
    return RM_OK;
}

rm_status rm_debug_array_factor(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p,
                                float* alpha_prepass_dev, float* alpha_inline_dev, uint64_t len, void* stream) {
    rm_status st = validate(sc, tx, ntx, p);
    if (st != RM_OK) return st;
    if ((st = check_device(sc)) != RM_OK) return st;
    if (!alpha_prepass_dev || !alpha_inline_dev) return fail(RM_EINVAL, "NULL alpha buffer");
    Prepared P;
    prepare(sc, tx, ntx, p, nullptr, &P);
    if (len < P.a.total) return fail(RM_EINVAL, "len is below the number of work items (sum of ray counts)");
    size_t o_mat, o_tx;
    const size_t tab = table_bytes(P, &o_mat, &o_tx);
    char* hst = nullptr;
    RM_CUDA(staging(tab, &hst));
    const size_t used = write_tables(P, o_mat, o_tx, hst);
    char* dev = nullptr;
    RM_CUDA(device_block(tab, &dev));
    P.a.mats = reinterpret_cast<const MatDev*>(dev + o_mat);
    P.a.tx = reinterpret_cast<const TxDev*>(dev + o_tx);
    P.a.ant = reinterpret_cast<const AntDev*>(dev + ant_offset(P, o_tx));
    P.a.scratch = reinterpret_cast<Scratch*>(dev);
    cudaError_t e = cudaMemcpyAsync(dev, hst, used, cudaMemcpyHostToDevice, S(stream));
    if (e == cudaSuccess) e = launch_alpha(P.a, reinterpret_cast<float2*>(alpha_prepass_dev), S(stream), true);
    if (e == cudaSuccess) e = launch_alpha(P.a, reinterpret_cast<float2*>(alpha_inline_dev), S(stream), false);
    const cudaError_t e2 = cudaStreamSynchronize(S(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rm_debug_array_factor");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamSynchronize");
    return RM_OK;
}

const char* rm_version(void) { return "rmsbr 0.1 (sm_103a)"; }

rm_status rm_scene_upload(const float* verts_dev, int64_t nv, const int32_t* tris_dev, int64_t nt,
                          const int32_t* tri_mat_dev, const rm_material* mats_host, int32_t nm, void* stream,
                          rm_scene** out) {
    if (!out) return fail(RM_EINVAL, "out is NULL");
    if (nv < 0 || nt < 0) return fail(RM_EINVAL, "nv and nt must be >= 0");
    if (nt > (int64_t)INT32_MAX / 4) return fail(RM_EINVAL, "nt too large");
    if (nt > 0 && (!verts_dev || !tris_dev || !tri_mat_dev || nv < 1))
        return fail(RM_EINVAL, "mesh pointers are NULL for a non-empty mesh");
    rm_status st = check_materials(mats_host, nm);
    if (st != RM_OK) return st;
    if (injected(RM_FAULT_ALLOC)) return fail(RM_ENOMEM, "rm_scene_upload: injected allocation failure");
    rm_scene* sc = new rm_scene();
    RM_CUDA(cudaGetDevice(&sc->device));
    sc->nv = nv;
    sc->nt = nt;
    sc->nm = nm;
    sc->mats.assign(mats_host, mats_host + nm);
    auto cleanup = [&](rm_status s) { rm_scene_free(sc); return s; };
    cudaError_t e;
    if (nt > 0) {
        const size_t o_t = align256(sizeof(float) * 3 * nv), o_m = o_t + align256(sizeof(int32_t) * 3 * nt),
                     o_f = o_m + align256(sizeof(int32_t) * nt);
        keep_pool_memory();
        if ((e = lib_malloc_async((void**)&sc->mesh_mem, o_f + sizeof(int32_t), S(stream))) != cudaSuccess)
            return cleanup(cuda_fail(e, "cudaMallocAsync"));
        sc->verts = reinterpret_cast<float*>(sc->mesh_mem);
        sc->tris = reinterpret_cast<int32_t*>(sc->mesh_mem + o_t);
        sc->tri_mat = reinterpret_cast<int32_t*>(sc->mesh_mem + o_m);
        int32_t* flag = reinterpret_cast<int32_t*>(sc->mesh_mem + o_f);
        int32_t hflag = 0;
        do {
            if ((e = cudaMemcpyAsync(sc->verts, verts_dev, sizeof(float) * 3 * nv, cudaMemcpyDeviceToDevice, S(stream))) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(sc->tris, tris_dev, sizeof(int32_t) * 3 * nt, cudaMemcpyDeviceToDevice, S(stream))) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(sc->tri_mat, tri_mat_dev, sizeof(int32_t) * nt, cudaMemcpyDeviceToDevice, S(stream))) != cudaSuccess) break;
            if ((e = cudaMemsetAsync(flag, 0, sizeof(int32_t), S(stream))) != cudaSuccess) break;
            if ((e = check_indices(sc->tris, sc->tri_mat, nt, nv, nm, flag, S(stream))) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(&hflag, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, S(stream))) != cudaSuccess) break;
        } while (false);
        cudaError_t es = cudaStreamSynchronize(S(stream));
        if (e != cudaSuccess) return cleanup(cuda_fail(e, "rm_scene_upload"));
        if (es != cudaSuccess) return cleanup(cuda_fail(es, "cudaStreamSynchronize"));
        if (hflag) return cleanup(fail(RM_EINVAL, "a vertex or material index is out of range"));
    }
    *out = sc;
    return RM_OK;
}

rm_status rm_scene_upload_host(const float* verts_host, int64_t nv, const int32_t* tris_host, int64_t nt,
                               const int32_t* tri_mat_host, const rm_material* mats_host, int32_t nm, void* stream,
                               rm_scene** out) {
    if (!out) return fail(RM_EINVAL, "out is NULL");
    if (nv < 0 || nt < 0) return fail(RM_EINVAL, "nv and nt must be >= 0");
    if (nt > (int64_t)INT32_MAX / 4) return fail(RM_EINVAL, "nt too large");
    if (nt > 0 && (!verts_host || !tris_host || !tri_mat_host || nv < 1))
        return fail(RM_EINVAL, "mesh pointers are NULL for a non-empty mesh");
    rm_status st = check_materials(mats_host, nm);
    if (st != RM_OK) return st;
    // index ranges, on the host: no device round trip
    for (int64_t i = 0; i < 3 * nt; ++i)
        if (tris_host[i] < 0 || (int64_t)tris_host[i] >= nv)
            return fail(RM_EINVAL, "a vertex or material index is out of range");
    for (int64_t i = 0; i < nt; ++i)
        if (tri_mat_host[i] < 0 || tri_mat_host[i] >= nm)
            return fail(RM_EINVAL, "a vertex or material index is out of range");
    if (injected(RM_FAULT_ALLOC)) return fail(RM_ENOMEM, "rm_scene_upload_host: injected allocation failure");
    rm_scene* sc = new rm_scene();
    RM_CUDA(cudaGetDevice(&sc->device));
    sc->nv = nv;
    sc->nt = nt;
    sc->nm = nm;
    sc->mats.assign(mats_host, mats_host + nm);
    auto cleanup = [&](rm_status s) { rm_scene_free(sc); return s; };
    if (nt > 0) {
        const size_t o_t = align256(sizeof(float) * 3 * nv), o_m = o_t + align256(sizeof(int32_t) * 3 * nt),
                     o_f = o_m + align256(sizeof(int32_t) * nt);
        keep_pool_memory();
        cudaError_t e;
        if ((e = lib_malloc_async((void**)&sc->mesh_mem, o_f + sizeof(int32_t), S(stream))) != cudaSuccess)
            return cleanup(cuda_fail(e, "cudaMallocAsync"));
        sc->verts = reinterpret_cast<float*>(sc->mesh_mem);
        sc->tris = reinterpret_cast<int32_t*>(sc->mesh_mem + o_t);
        sc->tri_mat = reinterpret_cast<int32_t*>(sc->mesh_mem + o_m);
        char* h = nullptr;
        if ((e = upload_stage(o_f, &h)) != cudaSuccess) return cleanup(cuda_fail(e, "pinned staging"));
        std::memcpy(h, verts_host, sizeof(float) * 3 * nv);
        std::memcpy(h + o_t, tris_host, sizeof(int32_t) * 3 * nt);
        std::memcpy(h + o_m, tri_mat_host, sizeof(int32_t) * nt);
        if ((e = cudaMemcpyAsync(sc->mesh_mem, h, o_f, cudaMemcpyHostToDevice, S(stream))) != cudaSuccess)
            return cleanup(cuda_fail(e, "cudaMemcpyAsync"));
        if ((e = cudaEventRecord(g_up.done, S(stream))) != cudaSuccess) {
            cudaStreamSynchronize(S(stream));
            return cleanup(cuda_fail(e, "cudaEventRecord"));
        }
        g_up.pending = true;
    }
    *out = sc;
    return RM_OK;
}

rm_status rm_scene_set_materials(rm_scene* sc, const rm_material* mats_host, int32_t nm,
                                 const rm_material* sampling_host_or_null) {
    if (!sc) return fail(RM_EINVAL, "scene is NULL");
    if (nm != sc->nm) return fail(RM_EINVAL, "nm must equal the scene's material count");
    rm_status st = check_materials(mats_host, nm);
    if (st != RM_OK) return st;
    if (sampling_host_or_null && (st = check_materials(sampling_host_or_null, nm)) != RM_OK) return st;
    sc->mats.assign(mats_host, mats_host + nm);
    sc->has_smats = sampling_host_or_null != nullptr;
    if (sc->has_smats) sc->smats.assign(sampling_host_or_null, sampling_host_or_null + nm);
    else sc->smats.clear();
    return RM_OK;
}

rm_status rm_bvh_build(rm_scene* sc, void* stream) { return rm_bvh_build_ex(sc, RM_BVH_AUTO, stream); }

rm_status rm_bvh_build_ex(rm_scene* sc, int32_t builder, void* stream) {
    if (!sc) return fail(RM_EINVAL, "scene is NULL");
    if (builder != RM_BVH_AUTO && builder != RM_BVH_LBVH && builder != RM_BVH_SAH)
        return fail(RM_EINVAL, "builder must be RM_BVH_AUTO, RM_BVH_LBVH or RM_BVH_SAH");
    rm_status st = check_device(sc);
    if (st != RM_OK) return st;
    if (sc->built) return fail(RM_ESTATE, "the BVH of this scene is already built");
    if (builder == RM_BVH_AUTO) builder = sc->nt > RM_BVH_AUTO_SAH_MIN ? RM_BVH_SAH : RM_BVH_LBVH;
    if (injected(RM_FAULT_ALLOC)) return fail(RM_ENOMEM, "rm_bvh_build: injected allocation failure");
    const int64_t n = sc->nt;
    if (n > 0) {
        const size_t o_o = align256(sizeof(uint64_t) * n), o_n = o_o + align256(sizeof(int32_t) * n),
                     o_r = o_n + align256(sizeof(float4) * 4 * (n > 1 ? n - 1 : 1));
        keep_pool_memory();
        if (sc->bvh_mem) {  // left by a build that failed: reuse nothing of it
            RM_CUDA(cudaStreamSynchronize(S(stream)));
            cudaFree(sc->bvh_mem);
            sc->bvh_mem = nullptr;
        }
        RM_CUDA(lib_malloc_async((void**)&sc->bvh_mem, o_r + sizeof(float4) * 3 * n, S(stream)));
        sc->keys = reinterpret_cast<uint64_t*>(sc->bvh_mem);
        sc->order = reinterpret_cast<int32_t*>(sc->bvh_mem + o_o);
        sc->nodes = reinterpret_cast<float4*>(sc->bvh_mem + o_n);
        sc->trirec = reinterpret_cast<float4*>(sc->bvh_mem + o_r);
        BvhBuffers B{sc->verts, sc->tris, sc->tri_mat, n, sc->keys, sc->order, sc->nodes, sc->trirec};
        // the large-triangle count goes to a pinned slot; the host does not wait for it here
        int32_t* slot = pin_slot_acquire();
        cudaEvent_t ev = nullptr;
        if (slot && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            pin_slot_release(slot);
            slot = nullptr;
            ev = nullptr;
        }
        if (!slot) {  // no pinned slot: wait for the count
            int32_t large = 0;
            RM_CUDA(build_bvh(B, builder == RM_BVH_SAH ? BVH_SAH : BVH_LBVH, S(stream), &large));
            RM_CUDA(cudaStreamSynchronize(S(stream)));
            sc->nlarge = (large > 0 && large <= MAX_LARGE_TRIS) ? large : 0;
        } else {
            cudaError_t e = build_bvh(B, builder == RM_BVH_SAH ? BVH_SAH : BVH_LBVH, S(stream), slot);
            if (e == cudaSuccess) e = cudaEventRecord(ev, S(stream));
            if (e != cudaSuccess) {
                cudaStreamSynchronize(S(stream));
                pin_slot_release(slot);
                cudaEventDestroy(ev);
                return cuda_fail(e, "rm_bvh_build");
            }
            std::lock_guard<std::mutex> g(sc->mu);
            sc->nlarge_slot = slot;
            sc->built_ev = ev;
            sc->nlarge_pending = true;
        }
    }
    sc->built = true;
    sc->builder = builder;
    return RM_OK;
}

rm_status rm_bvh_export(const rm_scene* sc, uint64_t* keys_host, int32_t* order_host, int32_t* child_host,
                        float* child_aabb_host) {
    if (!sc) return fail(RM_EINVAL, "scene is NULL");
    if (!sc->built) return fail(RM_ESTATE, "rm_bvh_build has not been called on this scene");
    rm_status st = check_device(sc);
    if (st != RM_OK) return st;
    if ((st = resolve_nlarge(sc)) != RM_OK) return st;
    const int64_t n = sc->nt;
    if (n <= 0) return RM_OK;
    if (keys_host) RM_CUDA(cudaMemcpy(keys_host, sc->keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost));
    if (order_host) RM_CUDA(cudaMemcpy(order_host, sc->order, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    const int64_t ns = n - sc->nlarge;
    if (ns > 1 && (child_host || child_aabb_host)) {
        std::vector<float4> nodes((size_t)4 * (ns - 1));
        RM_CUDA(cudaMemcpy(nodes.data(), sc->nodes, sizeof(float4) * 4 * (ns - 1), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < ns - 1; ++i) {
            const float* f = reinterpret_cast<const float*>(&nodes[4 * i]);
            if (child_host) {
                std::memcpy(&child_host[2 * i], &f[12], sizeof(int32_t));
                std::memcpy(&child_host[2 * i + 1], &f[13], sizeof(int32_t));
            }
            if (child_aabb_host) std::memcpy(&child_aabb_host[12 * i], f, 12 * sizeof(float));
        }
    }
    return RM_OK;
}

rm_status rm_radio_map_trace(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p,
                             float* maps_dev, rm_stats* stats, rm_segment_record* record, void* stream) {
    return run_trace(sc, tx, ntx, p, maps_dev, nullptr, nullptr, nullptr, nullptr, nullptr, stats, record, stream,
                     false);
}

rm_status rm_radio_map_trace_mesh(const rm_scene* sc, const rm_scene* surface, const rm_tx* tx, int32_t ntx,
                                  const rm_trace_params* p, float* maps_dev, rm_stats* stats,
                                  rm_segment_record* record, void* stream) {
    if (!surface) return fail(RM_EINVAL, "surface is NULL");
    return run_trace(sc, tx, ntx, p, maps_dev, nullptr, nullptr, nullptr, nullptr, nullptr, stats, record, stream,
                     false, surface);
}

rm_status rm_radio_map_grad(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p,
                            const float* dL_dmaps_dev, float* d_eps_dev, float* d_sigma_dev, float* d_txpos_dev,
                            const rm_material* sampling_host_or_null, rm_stats* stats, rm_segment_record* record,
                            void* stream) {
    return run_trace(sc, tx, ntx, p, nullptr, dL_dmaps_dev, d_eps_dev, d_sigma_dev, d_txpos_dev,
                     sampling_host_or_null, stats, record, stream, true);
}

rm_status rm_radio_map_trace_hits(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p,
                                  float* maps_dev, int32_t* hits_dev, uint64_t hits_len, rm_stats* stats,
                                  void* stream) {
    if (!hits_dev) return fail(RM_EINVAL, "hits_dev is NULL");
    return run_trace(sc, tx, ntx, p, maps_dev, nullptr, nullptr, nullptr, nullptr, nullptr, stats, nullptr, stream,
                     false, nullptr, hits_dev, hits_len);
}

rm_status rm_radio_map_grad_hits(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p,
                                 const float* dL_dmaps_dev, const int32_t* hits_dev, uint64_t hits_len,
                                 float* d_eps_dev, float* d_sigma_dev, float* d_txpos_dev,
                                 const rm_material* sampling_host_or_null, rm_stats* stats,
                                 rm_segment_record* record, void* stream) {
    if (!hits_dev) return fail(RM_EINVAL, "hits_dev is NULL");
    // the adjoint only reads the buffer
    return run_trace(sc, tx, ntx, p, nullptr, dL_dmaps_dev, d_eps_dev, d_sigma_dev, d_txpos_dev,
                     sampling_host_or_null, stats, record, stream, true, nullptr, const_cast<int32_t*>(hits_dev),
                     hits_len);
}

rm_status rm_radio_map_grad_mesh(const rm_scene* sc, const rm_scene* surface, const rm_tx* tx, int32_t ntx,
                                 const rm_trace_params* p, const float* dL_dmaps_dev, float* d_eps_dev,
                                 float* d_sigma_dev, float* d_txpos_dev, const rm_material* sampling_host_or_null,
                                 rm_stats* stats, rm_segment_record* record, void* stream) {
    if (!surface) return fail(RM_EINVAL, "surface is NULL");
    return run_trace(sc, tx, ntx, p, nullptr, dL_dmaps_dev, d_eps_dev, d_sigma_dev, d_txpos_dev,
                     sampling_host_or_null, stats, record, stream, true, surface);
}

rm_status rm_radio_map_trace_mesh_hits(const rm_scene* sc, const rm_scene* surface, const rm_tx* tx, int32_t ntx,
                                       const rm_trace_params* p, float* maps_dev, int32_t* hits_dev,
                                       uint64_t hits_len, rm_stats* stats, void* stream) {
    if (!surface) return fail(RM_EINVAL, "surface is NULL");
    if (!hits_dev) return fail(RM_EINVAL, "hits_dev is NULL");
    return run_trace(sc, tx, ntx, p, maps_dev, nullptr, nullptr, nullptr, nullptr, nullptr, stats, nullptr, stream,
                     false, surface, hits_dev, hits_len);
}

rm_status rm_radio_map_grad_mesh_hits(const rm_scene* sc, const rm_scene* surface, const rm_tx* tx, int32_t ntx,
                                      const rm_trace_params* p, const float* dL_dmaps_dev, const int32_t* hits_dev,
                                      uint64_t hits_len, float* d_eps_dev, float* d_sigma_dev, float* d_txpos_dev,
                                      const rm_material* sampling_host_or_null, rm_stats* stats,
                                      rm_segment_record* record, void* stream) {
    if (!surface) return fail(RM_EINVAL, "surface is NULL");
    if (!hits_dev) return fail(RM_EINVAL, "hits_dev is NULL");
    // the adjoint only reads the buffer
    return run_trace(sc, tx, ntx, p, nullptr, dL_dmaps_dev, d_eps_dev, d_sigma_dev, d_txpos_dev,
                     sampling_host_or_null, stats, record, stream, true, surface, const_cast<int32_t*>(hits_dev),
                     hits_len);
}

rm_status rm_db_mse_loss(const float* maps_dev, const float* target_dev, int64_t ncells, float floor_linear,
                         float* loss_dev, float* dL_dmaps_dev, int64_t* valid_dev, void* stream) {
    if (!maps_dev || !target_dev || !dL_dmaps_dev) return fail(RM_EINVAL, "NULL buffer");
    if (ncells < 1) return fail(RM_EINVAL, "ncells must be >= 1");
    if (!(floor_linear >= 0.0f)) return fail(RM_EINVAL, "floor_linear must be >= 0");
    double* acc = nullptr;
    RM_CUDA(lib_malloc_async((void**)&acc, 2 * sizeof(double), S(stream)));
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), S(stream));
    if (e == cudaSuccess)
        e = launch_db_mse(maps_dev, target_dev, ncells, floor_linear, acc, loss_dev, dL_dmaps_dev, valid_dev, S(stream));
    cudaError_t e2 = cudaFreeAsync(acc, S(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rm_db_mse_loss");
    return RM_OK;
}

rm_status rm_trace_plan_create(const rm_scene* sc, const rm_tx* tx, int32_t ntx, const rm_trace_params* p,
                               float* maps_dev, void* stream, rm_trace_plan** out) {
    if (!out) return fail(RM_EINVAL, "out is NULL");
    rm_status st = validate(sc, tx, ntx, p);
    if (st != RM_OK) return st;
    if ((st = check_device(sc)) != RM_OK) return st;
    if (!maps_dev) return fail(RM_EINVAL, "maps_dev is NULL");
    if (p->flags & RM_STATS) return fail(RM_EINVAL, "RM_STATS is not available in a plan");
    Prepared P;
    prepare(sc, tx, ntx, p, nullptr, &P);
    size_t o_mat, o_tx, o_m64;
    const size_t bytes = block_bytes_with_maps64(P, &o_mat, &o_tx, &o_m64);
    rm_trace_plan* pl = new rm_trace_plan();
    pl->ntx = ntx;
    pl->L = p->max_depth;
    auto cleanup = [&](rm_status s) { rm_trace_plan_free(pl); return s; };
    cudaError_t e;
    if ((e = cudaStreamSynchronize(S(stream))) != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamSynchronize"));
    if ((e = lib_malloc((void**)&pl->dev, bytes)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaMalloc"));
    if ((e = cudaMemcpy(pl->dev + o_mat, P.mats.data(), P.mats.size() * sizeof(MatDev), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMemcpy"));
    if ((e = cudaMemcpy(pl->dev + o_tx, P.tx.data(), P.tx.size() * sizeof(TxDev), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMemcpy"));
    if (!P.ant.empty() && (e = cudaMemcpy(pl->dev + ant_offset(P, o_tx), P.ant.data(), P.ant.size() * sizeof(AntDev),
                                          cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaMemcpy"));
    pl->scratch = reinterpret_cast<Scratch*>(pl->dev);
    P.a.mats = reinterpret_cast<const MatDev*>(pl->dev + o_mat);
    P.a.tx = reinterpret_cast<const TxDev*>(pl->dev + o_tx);
    P.a.ant = reinterpret_cast<const AntDev*>(pl->dev + ant_offset(P, o_tx));
    P.a.scratch = pl->scratch;
    P.a.maps = maps_dev;
    P.a.maps64 = reinterpret_cast<double*>(pl->dev + o_m64);
    if ((e = cudaEventCreate(&pl->ev0)) != cudaSuccess || (e = cudaEventCreate(&pl->ev1)) != cudaSuccess)
        return cleanup(cuda_fail(e, "cudaEventCreate"));
    cudaStream_t cap;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return cleanup(cuda_fail(e, "cudaStreamCreate"));
    cudaError_t ec = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ec == cudaSuccess) {
        cudaError_t ek = cudaMemsetAsync(pl->dev, 0, sizeof(Scratch), cap);
        if (ek == cudaSuccess) ek = cudaMemsetAsync(P.a.maps64, 0, sizeof(double) * P.a.ncell * ntx, cap);
        if (ek == cudaSuccess) ek = cudaEventRecordWithFlags(pl->ev0, cap, cudaEventRecordExternal);
        int grid = 0;
        if (ek == cudaSuccess && P.a.total > 0)
            ek = launch_trace(P.a, P.npol, false, P.bilinear, false, P.diffuse, P.block, P.bps, cap, &grid);
        if (ek == cudaSuccess) ek = cudaEventRecordWithFlags(pl->ev1, cap, cudaEventRecordExternal);
        if (ek == cudaSuccess) ek = launch_map_to_f32(P.a.maps64, maps_dev, P.a.ncell * ntx, cap);
        ec = cudaStreamEndCapture(cap, &pl->graph);
        if (ek != cudaSuccess) ec = ek;
    }
    if (ec == cudaSuccess) ec = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    cudaStreamDestroy(cap);
    if (ec != cudaSuccess) return cleanup(cuda_fail(ec, "graph capture"));
    *out = pl;
    return RM_OK;
}

rm_status rm_trace_plan_launch(rm_trace_plan* pl, void* stream) {
    if (!pl || !pl->exec) return fail(RM_EINVAL, "plan is NULL");
    RM_CUDA(cudaGraphLaunch(pl->exec, S(stream)));
    return RM_OK;
}

rm_status rm_trace_plan_stats(rm_trace_plan* pl, void* stream, rm_stats* out) {
    if (!pl || !out) return fail(RM_EINVAL, "NULL argument");
    Scratch h;
    RM_CUDA(cudaMemcpyAsync(&h, pl->scratch, sizeof(Scratch), cudaMemcpyDeviceToHost, S(stream)));
    RM_CUDA(cudaStreamSynchronize(S(stream)));
    Prepared P;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, pl->ev0, pl->ev1) == cudaSuccess) P.kernel_ms = ms;
    fill_stats(h, P, out);
    if (h.status & 1) return fail(RM_EOVERFLOW, "BVH traversal stack overflow; affected rays were dropped");
    return RM_OK;
}

void rm_trace_plan_free(rm_trace_plan* pl) {
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->dev) cudaFree(pl->dev);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    delete pl;
}

rm_status rm_scene_wedges(const rm_scene* sc, rm_wedge* out, int64_t cap, int64_t* count) {
    if (!sc || !count) return fail(RM_EINVAL, "scene or count is NULL");
    if (cap < 0 || (cap > 0 && !out)) return fail(RM_EINVAL, "cap must be >= 0 with an output array");
    rm_status st = check_device(sc);
    if (st != RM_OK) return st;
    *count = 0;
    if (sc->nt == 0) return RM_OK;
    std::vector<float> v(3 * sc->nv);
    std::vector<int32_t> t(3 * sc->nt), m(sc->nt);
    RM_CUDA(cudaMemcpy(v.data(), sc->verts, sizeof(float) * v.size(), cudaMemcpyDeviceToHost));
    RM_CUDA(cudaMemcpy(t.data(), sc->tris, sizeof(int32_t) * t.size(), cudaMemcpyDeviceToHost));
    RM_CUDA(cudaMemcpy(m.data(), sc->tri_mat, sizeof(int32_t) * m.size(), cudaMemcpyDeviceToHost));
    // edges keyed by their vertex indices (low, high) -> the triangles that own them
    std::vector<std::pair<uint64_t, int32_t>> edges;
    edges.reserve(3 * sc->nt);
    for (int64_t i = 0; i < sc->nt; ++i)
        for (int k = 0; k < 3; ++k) {
            const uint32_t a = (uint32_t)t[3 * i + k], b = (uint32_t)t[3 * i + (k + 1) % 3];
            edges.push_back({((uint64_t)std::min(a, b) << 32) | std::max(a, b), (int32_t)i});
        }
    std::sort(edges.begin(), edges.end());
    auto vert = [&](uint32_t id, double* p) {
        for (int c = 0; c < 3; ++c) p[c] = v[3 * (size_t)id + c];
    };
    auto normal = [&](int32_t tri, double* n) {
        double a[3], b[3], c[3];
        vert(t[3 * tri], a);
        vert(t[3 * tri + 1], b);
        vert(t[3 * tri + 2], c);
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        n[0] = e1[1] * e2[2] - e1[2] * e2[1];
        n[1] = e1[2] * e2[0] - e1[0] * e2[2];
        n[2] = e1[0] * e2[1] - e1[1] * e2[0];
        const double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(l > 0.0)) return false;
        for (int q = 0; q < 3; ++q) n[q] /= l;
        return true;
    };
    std::vector<rm_wedge> W;
    for (size_t i = 0; i < edges.size();) {
        size_t j = i;
        while (j < edges.size() && edges[j].first == edges[i].first) ++j;
        if (j - i == 2) {
            const int32_t A = std::min(edges[i].second, edges[i + 1].second);
            const int32_t B = std::max(edges[i].second, edges[i + 1].second);
            const uint32_t ia = (uint32_t)(edges[i].first >> 32), ib = (uint32_t)(edges[i].first & 0xffffffffu);
            double na[3], nb[3];
            if (A != B && normal(A, na) && normal(B, nb)) {
                const double c[3] = {na[1] * nb[2] - na[2] * nb[1], na[2] * nb[0] - na[0] * nb[2],
                                     na[0] * nb[1] - na[1] * nb[0]};
                const double sn = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
                int32_t third = -1;
                for (int k = 0; k < 3; ++k)
                    if ((uint32_t)t[3 * B + k] != ia && (uint32_t)t[3 * B + k] != ib) third = t[3 * B + k];
                double p[3], q[3], r[3];
                vert(ia, p);
                vert(ib, q);
                bool convex = false;
                if (third >= 0) {
                    vert((uint32_t)third, r);
                    convex = (r[0] - p[0]) * na[0] + (r[1] - p[1]) * na[1] + (r[2] - p[2]) * na[2] < 0.0;
                }
                if (sn >= 1e-9 && convex) {
                    rm_wedge w;
                    double e[3];
                    for (int k = 0; k < 3; ++k) e[k] = c[k] / sn;
                    const double dp = p[0] * e[0] + p[1] * e[1] + p[2] * e[2], dq = q[0] * e[0] + q[1] * e[1] + q[2] * e[2];
                    const double* o = dp <= dq ? p : q;
                    for (int k = 0; k < 3; ++k) {
                        w.origin[k] = (float)o[k];
                        w.edge[k] = (float)e[k];
                        w.n0[k] = (float)na[k];
                        w.nn[k] = (float)nb[k];
                    }
                    w.length = (float)std::sqrt((q[0] - p[0]) * (q[0] - p[0]) + (q[1] - p[1]) * (q[1] - p[1]) +
                                                (q[2] - p[2]) * (q[2] - p[2]));
                    const double cn = std::max(-1.0, std::min(1.0, na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2]));
                    w.n = (float)(1.0 + std::acos(cn) / PI);
                    w.tri0 = A;
                    w.trin = B;
                    w.mat0 = m[A];
                    w.matn = m[B];
                    W.push_back(w);
                }
            }
        }
        i = j;
    }
    std::sort(W.begin(), W.end(), [](const rm_wedge& a, const rm_wedge& b) {
        return a.tri0 != b.tri0 ? a.tri0 < b.tri0 : a.trin < b.trin;
    });
    *count = (int64_t)W.size();
    if (out && cap > 0) std::memcpy(out, W.data(), sizeof(rm_wedge) * (size_t)std::min<int64_t>(cap, *count));
    return RM_OK;
}

}  // extern "C"

namespace {
rm_status run_diffraction(const rm_scene* sc, const rm_scene* surf, const rm_wedge* wedges, int64_t nw,
                          const rm_tx* tx, int32_t ntx, const rm_trace_params* p, int64_t ns, float* maps,
                          rm_stats* stats, rm_segment_record* record, void* stream) {
    rm_status st = validate(sc, tx, ntx, p);
    if (st != RM_OK) return st;
    if ((st = check_device(sc)) != RM_OK) return st;
    if (surf) {
        if (!surf->built) return fail(RM_ESTATE, "rm_bvh_build has not been called on the surface");
        if ((st = resolve_nlarge(surf)) != RM_OK) return st;
        if ((st = check_device(surf)) != RM_OK) return st;
        if (surf->device != sc->device) return fail(RM_EINVAL, "scene and surface live on different devices");
        if (surf->nt < 1 || surf->nt > INT32_MAX) return fail(RM_EINVAL, "the surface needs 1 .. 2^31-1 triangles");
        if (p->deposit != 0) return fail(RM_EINVAL, "mesh surfaces take box cells (deposit = 0)");
    }
    if (!maps) return fail(RM_EINVAL, "maps_dev is NULL");
    if (nw < 0 || (nw > 0 && !wedges)) return fail(RM_EINVAL, "nw must be >= 0 with a wedge array");
    if (ns < 1) return fail(RM_EINVAL, "samples_per_wedge must be >= 1");
    if ((double)nw * (double)ns * (double)ntx >= 1099511627776.0)
        return fail(RM_EINVAL, "nw * samples_per_wedge * ntx must stay below 2^40");
    for (int64_t i = 0; i < nw; ++i) {
        const rm_wedge& w = wedges[i];
        if (!(w.length > 0.0f) || !(w.n > 1.0f && w.n <= 2.0f) || w.mat0 < 0 || w.mat0 >= sc->nm || w.matn < 0 ||
            w.matn >= sc->nm || !std::isfinite(w.origin[0]) || !std::isfinite(w.origin[1]) ||
            !std::isfinite(w.origin[2]))
            return fail(RM_EINVAL, "wedge " + std::to_string(i) + ": length > 0, 1 < n <= 2 and valid materials required");
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RM_CUDA(cudaStreamIsCapturing(S(stream), &cs));
    if (cs != cudaStreamCaptureStatusNone) return fail(RM_ESTATE, "stream is capturing");
    Prepared P;
    prepare(sc, tx, ntx, p, nullptr, &P);
    size_t o_mat, o_tx;
    const size_t tab = table_bytes(P, &o_mat, &o_tx);
    const size_t o_w = (tab + 255) & ~size_t(255);
    const size_t o_m64 = (o_w + sizeof(rm_wedge) * (size_t)std::max<int64_t>(nw, 1) + 255) & ~size_t(255);
    const unsigned long long ncell = surf ? (unsigned long long)surf->nt : (unsigned long long)p->nx * p->ny;
    const size_t bytes = o_m64 + sizeof(double) * ncell * ntx;
    cudaEvent_t ev[2];
    RM_CUDA(timing_events(ev));
    char* hst = nullptr;
    RM_CUDA(staging(o_w + sizeof(rm_wedge) * (size_t)std::max<int64_t>(nw, 1), &hst));
    const size_t tab_used = write_tables(P, o_mat, o_tx, hst);
    if (nw > 0) std::memcpy(hst + o_w, wedges, sizeof(rm_wedge) * (size_t)nw);
    char* dev = nullptr;
    RM_CUDA(device_block(bytes, &dev));
    DiffArgs A;
    std::memset(&A, 0, sizeof A);
    A.nodes = sc->nodes;
    A.tris = sc->trirec;
    A.nt = (int32_t)(sc->nt - sc->nlarge);
    A.nlarge = (int32_t)sc->nlarge;
    A.wedges = reinterpret_cast<const rm_wedge*>(dev + o_w);
    A.nw = nw;
    A.mats = reinterpret_cast<const MatDev*>(dev + o_mat);
    A.tx = reinterpret_cast<const TxDev*>(dev + o_tx);
    A.ant = reinterpret_cast<const AntDev*>(dev + ant_offset(P, o_tx));
    A.ntx = ntx;
    A.nm = sc->nm;
    A.ns = (unsigned long long)ns;
    A.total = (unsigned long long)nw * (unsigned long long)ns * (unsigned long long)ntx;
    A.x0 = P.a.x0;
    A.y0 = P.a.y0;
    A.zm = P.a.zm;
    A.cell = P.a.cell;
    A.inv_cell = P.a.inv_cell;
    A.nx = p->nx;
    A.ny = p->ny;
    A.bilinear = p->deposit == 1;
    A.ncell = ncell;
    A.k0 = P.a.k0;
    const double lam4pi = C0 / p->freq_hz / (4.0 * PI);
    // a mesh cell divides by its own area in the kernel
    const double cell2 = surf ? 1.0 : (double)p->cell_size * (double)p->cell_size;
    A.lam4pi2_over_cell2 = (float)(lam4pi * lam4pi / cell2);
    if (surf) {
        A.snodes = surf->nodes;
        A.stris = surf->trirec;
        A.snt = (int32_t)(surf->nt - surf->nlarge);
        A.snlarge = (int32_t)surf->nlarge;
    }
    double L, a[FADDEEVA_N];
    faddeeva_coefficients(FADDEEVA_N, &L, a);
    A.wz_L = (float)L;
    for (int k = 0; k < FADDEEVA_N; ++k) A.wz_a[k] = (float)a[k];
    A.npol = P.npol;
    A.stats = (p->flags & RM_STATS) ? 1 : 0;
    A.maps64 = reinterpret_cast<double*>(dev + o_m64);
    A.record = record;
    A.scratch = reinterpret_cast<Scratch*>(dev);
    cudaError_t e = cudaSuccess;
    bool timed = false;
    int grid = 0;
    do {
        if ((e = cudaMemcpyAsync(dev, hst, tab_used, cudaMemcpyHostToDevice, S(stream))) != cudaSuccess) break;
        if (nw > 0 && (e = cudaMemcpyAsync(dev + o_w, hst + o_w, sizeof(rm_wedge) * (size_t)nw, cudaMemcpyHostToDevice,
                                           S(stream))) != cudaSuccess)
            break;
        if ((e = cudaMemsetAsync(dev + o_m64, 0, sizeof(double) * ncell * ntx, S(stream))) != cudaSuccess) break;
        if (A.total > 0) {
            if ((e = cudaEventRecord(ev[0], S(stream))) != cudaSuccess) break;
            if ((e = launch_diffraction(A, p->block_size ? p->block_size : 256, S(stream), &grid, surf != nullptr)) !=
                cudaSuccess)
                break;
            if ((e = cudaEventRecord(ev[1], S(stream))) != cudaSuccess) break;
            timed = true;
        }
        if ((e = launch_map_to_f32(A.maps64, maps, ncell * ntx, S(stream))) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(hst, dev, sizeof(Scratch), cudaMemcpyDeviceToHost, S(stream))) != cudaSuccess) break;
    } while (false);
    cudaError_t e3 = cudaStreamSynchronize(S(stream));
    Scratch host;
    std::memcpy(&host, hst, sizeof(Scratch));
    float ms = 0.0f;
    if (timed && e == cudaSuccess && e3 == cudaSuccess && cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess)
        P.kernel_ms = ms;
    if (e != cudaSuccess) return cuda_fail(e, "rm_diffraction_map");
    if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamSynchronize");
    if (stats) fill_stats(host, P, stats);
    if (host.status & 1) return fail(RM_EOVERFLOW, "BVH traversal stack overflow in a visibility query");
    if (host.status & 2)
        return fail(RM_EOVERFLOW, "a diffracted ray crossed the measurement surface more than 8 times; "
                                  "its crossings beyond the 8th were dropped");
    return RM_OK;
}
}  // namespace

extern "C" {

rm_status rm_diffraction_map(const rm_scene* sc, const rm_wedge* wedges, int64_t nw, const rm_tx* tx, int32_t ntx,
                             const rm_trace_params* p, int64_t ns, float* maps, rm_stats* stats,
                             rm_segment_record* record, void* stream) {
    return run_diffraction(sc, nullptr, wedges, nw, tx, ntx, p, ns, maps, stats, record, stream);
}

rm_status rm_diffraction_map_mesh(const rm_scene* sc, const rm_scene* surface, const rm_wedge* wedges, int64_t nw,
                                  const rm_tx* tx, int32_t ntx, const rm_trace_params* p, int64_t ns, float* maps,
                                  rm_stats* stats, rm_segment_record* record, void* stream) {
    if (!surface) return fail(RM_EINVAL, "surface is NULL");
    return run_diffraction(sc, surface, wedges, nw, tx, ntx, p, ns, maps, stats, record, stream);
}

rm_status rm_scene_info(const rm_scene* sc, int64_t* nt, int64_t* nnodes, int32_t* nm, int32_t* built) {
    if (!sc) return fail(RM_EINVAL, "scene is NULL");
    if (nt) *nt = sc->nt;
    if (sc->built) {
        rm_status st = resolve_nlarge(sc);
        if (st != RM_OK) return st;
    }
    const int64_t ns = sc->nt - sc->nlarge;
    if (nnodes) *nnodes = ns > 1 ? ns - 1 : 0;
    if (nm) *nm = sc->nm;
    if (built) *built = sc->built ? sc->builder : 0;
    return RM_OK;
}

void rm_scene_free(rm_scene* sc) {
    if (!sc) return;
    // pool memory: wait for the device first, so that no kernel still reads it
    if (sc->mesh_mem || sc->bvh_mem) cudaDeviceSynchronize();
    if (sc->nlarge_pending) {
        pin_slot_release(sc->nlarge_slot);
        cudaEventDestroy(sc->built_ev);
    }
    cudaFree(sc->mesh_mem);
    cudaFree(sc->bvh_mem);
    delete sc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free variant of rm_radio_map_trace.
//
// The tracer's per-call scratch (work counter, counters, status word and the
// material / transmitter tables) lives here in one file-scope device array
// instead of a cudaMallocAsync block.  The array holds the largest call the
// ABI allows (RM_MAX_MATERIALS materials, RM_MAX_TX transmitters); every
// device that loads the library keeps it until the process exits.  Host code
// never passes the array's name to a kernel: in host code that name is only a
// stand-in, so its device address is looked up with cudaGetSymbolAddress,
// once per device, with that device current, and cached.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 16384;
constexpr int NOALLOC_MAX_DEVICES = 64;
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mutex;
char* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

rm_status noalloc_scratch(int dev, char** out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(RM_EINVAL, "device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        g_noalloc_addr[dev] = static_cast<char*>(p);
    }
    *out = g_noalloc_addr[dev];
    return RM_OK;
}

}  // namespace

extern "C" rm_status rm_radio_map_trace_noalloc(const rm_scene* sc, const rm_tx* tx, int32_t ntx,
                                                const rm_trace_params* p, float* maps_dev, rm_stats* stats,
                                                void* stream) {
    rm_status st = validate(sc, tx, ntx, p);
    if (st != RM_OK) return st;
    if ((st = check_device(sc)) != RM_OK) return st;
    if (!maps_dev) return fail(RM_EINVAL, "maps_dev is NULL");
    // the call reads its counters back and waits for them: a stream in capture
    // mode would fail there and invalidate the caller's capture, so it is
    // refused before anything is enqueued
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    RM_CUDA(cudaStreamIsCapturing(S(stream), &cs));
    if (cs != cudaStreamCaptureStatusNone)
        return fail(RM_ESTATE, "rm_radio_map_trace_noalloc synchronises its stream, which is capturing");
    Prepared P;
    prepare(sc, tx, ntx, p, nullptr, &P);
    size_t o_mat, o_tx;
    const size_t bytes = table_bytes(P, &o_mat, &o_tx);
    if (bytes > NOALLOC_SCRATCH_BYTES)
        return fail(RM_EINVAL, "call needs " + std::to_string(bytes) + " bytes of scratch; the static scratch of "
                               "rm_radio_map_trace_noalloc holds " + std::to_string(NOALLOC_SCRATCH_BYTES));
    char* dev = nullptr;
    if ((st = noalloc_scratch(sc->device, &dev)) != RM_OK) return st;
    const bool debug = (p->flags & RM_STATS) != 0;
    Scratch host;
    cudaError_t e = cudaSuccess;
    int grid = 0;
    do {
        // the array keeps the previous call's contents: clear the counters and status
        if ((e = cudaMemsetAsync(dev, 0, sizeof(Scratch), S(stream))) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(dev + o_mat, P.mats.data(), P.mats.size() * sizeof(MatDev),
                                 cudaMemcpyHostToDevice, S(stream))) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(dev + o_tx, P.tx.data(), P.tx.size() * sizeof(TxDev), cudaMemcpyHostToDevice,
                                 S(stream))) != cudaSuccess) break;
        if (!P.ant.empty() && (e = cudaMemcpyAsync(dev + ant_offset(P, o_tx), P.ant.data(), P.ant.size() * sizeof(AntDev),
                                                   cudaMemcpyHostToDevice, S(stream))) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(maps_dev, 0, sizeof(float) * P.a.ncell * ntx, S(stream))) != cudaSuccess) break;
        P.a.mats = reinterpret_cast<const MatDev*>(dev + o_mat);
        P.a.tx = reinterpret_cast<const TxDev*>(dev + o_tx);
        P.a.ant = reinterpret_cast<const AntDev*>(dev + ant_offset(P, o_tx));
        P.a.scratch = reinterpret_cast<Scratch*>(dev);
        P.a.maps = maps_dev;
        if (P.a.total > 0 &&
            (e = launch_trace(P.a, P.npol, debug, P.bilinear, false, P.diffuse, P.block, P.bps, S(stream), &grid)) != cudaSuccess)
            break;
        if ((e = cudaMemcpyAsync(&host, dev, sizeof(Scratch), cudaMemcpyDeviceToHost, S(stream))) != cudaSuccess) break;
    } while (false);
    const cudaError_t es = cudaStreamSynchronize(S(stream));
    if (e != cudaSuccess) return cuda_fail(e, "rm_radio_map_trace_noalloc");
    if (es != cudaSuccess) return cuda_fail(es, "cudaStreamSynchronize");
    if (stats) fill_stats(host, P, stats);
    if (host.status & 1) return fail(RM_EOVERFLOW, "BVH traversal stack overflow; affected rays were dropped");
    return RM_OK;
}

