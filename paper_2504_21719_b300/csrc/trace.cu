// Persistent SBR tracer (forward radio map and its adjoint) for sm_103a.
//
// One launch handles every transmitter of a call.  A global work counter
// hands out work items w in [0, total); item w is ray i of transmitter t
// (w = work_begin[t] + i), lattice direction n = begin + i * stride.  Each
// thread owns one ray slot kept entirely in registers; whenever lanes of a
// warp are free the warp refills them with ONE atomic on the counter
// (warp-level compaction between bounces: a warp never idles while work is
// left).  Per loop iteration every active lane traces one segment:
//   1. closest hit through the LBVH (stack traversal, nearer child first,
//      robust slab test, watertight ray-triangle test of Woop, Benthin &
//      Wald, JCGT 2013);
//   2. deposit at the plane crossing (Eq. radio-map-solver-ci-all-2-estimator),
//      one FP64 atomic reduction per deposit into the map accumulator;
//   3. if l < L and the ray hit: Fresnel / slab coefficients (App. A.7),
//      sampling of specular reflection, diffuse reflection or refraction with
//      q(R), q(S), q(T) (Eq. path-solver-used-dist-event, q(D) = 0), field
//      update with the TE/TM basis (specular) or Eq. scattered_field
//      (diffuse, App. A.10), new direction and origin.  The diffuse code is
//      compiled only into the DIFF instantiations.
// The adjoint instantiation re-traces the identical rays and, instead of
// writing the map, accumulates d(sum_i g_i C_i)/d(theta) by forward-mode
// tangents of the field with respect to each material met on the path.
//
// This file is compiled with -fmad=false: every operation that steers a
// discrete choice is rounded the same way in the forward and the adjoint
// instantiations, so both take the same hits, decisions and cells.  Division
// and square root are the approximate (few-ulp) forms, except the slab test's
// reciprocals.
#include <algorithm>
#include <cfloat>

#include "common.cuh"
#include "array.cuh"
#include "vec.cuh"

namespace rmsbr {
namespace {

// ------------------------------------------------------------------ RNG
// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
// uniform in [0, 1) on a 2^-24 grid: exact in FP32
__device__ __forceinline__ float rng_u(unsigned long long seed, unsigned long long n, int l) {
    const unsigned long long h = splitmix64(seed ^ splitmix64((n << 4) | (unsigned long long)(l & 15)));
    return (float)(unsigned)(h >> 40) * 0x1p-24f;
}
// the Russian-roulette variate of the same interaction: a second stream
constexpr unsigned long long RR_STREAM = 0xD6E8FEB86659FD93ULL;

// ------------------------------------------------------------------ Fresnel
struct Coef {
    cf rp, rl, tp, tl;  // r_perp, r_par, t_perp, t_par
};
// Incidence from vacuum (Eq. fresnel_vac); for a slab, the single-layer
// coefficients of Eqs. fresnel_slab / q_fresnel_slab with r' the
// half-space r of the same polarisation.  A half-space has t = 0.
__device__ __forceinline__ Coef fresnel(cf eta, float cos1, float k0d_hi, float k0d_lo, bool slab, cf* s_out) {
    const float sin2 = (1.0f - cos1) * (1.0f + cos1);
    const cf s = csqrt_p(C(eta.r - sin2, eta.i));
    const cf c = C(cos1);
    const cf ec = eta * cos1;
    Coef o;
    o.rp = cdiv(c - s, c + s);
    o.rl = cdiv(ec - s, ec + s);
    if (s_out) *s_out = s;
    if (!slab) {
        o.tp = C(0.0f);
        o.tl = C(0.0f);
        return o;
    }
    const cf q = C(k0d_hi * s.r + k0d_lo * s.r, k0d_hi * s.i + k0d_lo * s.i);
    const cf e1 = cexp_mj(q);
    const cf e2 = e1 * e1;
    const cf one = C(1.0f);
    const cf rp2 = o.rp * o.rp, rl2 = o.rl * o.rl;
    const cf dp = one - rp2 * e2, dl = one - rl2 * e2;
    const cf rp = cdiv(o.rp * (one - e2), dp);
    const cf rl = cdiv(o.rl * (one - e2), dl);
    o.tp = cdiv((one - rp2) * e1, dp);
    o.tl = cdiv((one - rl2) * e1, dl);
    o.rp = rp;
    o.rl = rl;
    return o;
}

// d/d eta of the chosen pair of coefficients (hand-derived; the oracle checks
// them through its dual numbers).  Half-space: r_perp = (c - s)/(c + s),
// r_par = (eta c - s)/(eta c + s), s = sqrt(eta - sin^2), ds/deta = 1/(2s).
// Slab: r = r'(1 - x)/(1 - r'^2 x), t = (1 - r'^2) y / (1 - r'^2 x),
// y = exp(-j k0d s), x = y^2.
__device__ __forceinline__ void fresnel_deta(cf eta, float cos1, float k0d, bool slab, int dec, cf* dperp,
                                             cf* dpar) {
    const float sin2 = (1.0f - cos1) * (1.0f + cos1);
    const cf s = csqrt_p(C(eta.r - sin2, eta.i));
    const cf c = C(cos1);
    const cf ec = eta * cos1;
    const cf one = C(1.0f);
    const cf cps = c + s, ecs = ec + s;
    const cf rp = cdiv(c - s, cps), rl = cdiv(ec - s, ecs);
    // d r_perp / d eta = -c / (s (c + s)^2);  d r_par / d eta = c (2 s^2 - eta) / (s (eta c + s)^2)
    const cf drp = cdiv(C(-cos1), s * cps * cps);
    const cf drl = cdiv((s * s * 2.0f - eta) * cos1, s * ecs * ecs);
    if (!slab) {
        *dperp = drp;
        *dpar = drl;
        return;
    }
    const cf y = cexp_mj(s * k0d);
    const cf x = y * y;
    const cf dq = cdiv(C(k0d * 0.5f), s);          // dq/deta = k0d / (2 s)
    const cf dy = y * C(0.0f, -1.0f) * dq;          // dy/deta = -j y dq
    const cf dx = y * dy * 2.0f;
    cf out[2];
    for (int p = 0; p < 2; ++p) {
        const cf r1 = p == 0 ? rp : rl;
        const cf dr1 = p == 0 ? drp : drl;
        const cf r2 = r1 * r1;
        const cf D = one - r2 * x;
        const cf D2 = D * D;
        if (dec == 0) {
            // dr/dr' = (1 - x)(1 + r'^2 x) / D^2 ; dr/dx = r'(r'^2 - 1) / D^2
            const cf a = cdiv((one - x) * (one + r2 * x), D2);
            const cf b = cdiv(r1 * (r2 - one), D2);
            out[p] = a * dr1 + b * dx;
        } else {
            // dt/dr' = -2 r' y (1 - x) / D^2 ; dt/dy = (1 - r'^2)(1 + r'^2 x) / D^2
            const cf a = cdiv(r1 * y * (one - x) * (-2.0f), D2);
            const cf b = cdiv((one - r2) * (one + r2 * x), D2);
            out[p] = a * dr1 + b * dy;
        }
    }
    *dperp = out[0];
    *dpar = out[1];
}

// ------------------------------------------------------------------ diffuse reflection
// App. A.10.  Four more RNG streams give the variates of a diffuse event:
// u1, u2 the direction, u3, u4 the random phases chi_1, chi_2 = 2 pi u.
constexpr unsigned long long DIFF_STREAM0 = 0x2545F4914F6CDD1DULL, DIFF_STREAM1 = 0x9E6C63D0676A9A99ULL,
                             DIFF_STREAM2 = 0x7F4A7C159E3779B9ULL, DIFF_STREAM3 = 0xC2B2AE3D27D4EB4FULL;

// theta_hat(k), phi_hat(k) (Eq. spherical_vecs) from the Cartesian
// components: with rho = |(k_x, k_y)|, cos phi = k_x / rho, sin phi = k_y / rho,
// theta_hat = (k_z cos phi, k_z sin phi, -rho), phi_hat = (-sin phi, cos phi, 0);
// at the poles phi = 0.
__device__ __forceinline__ void sph_basis(f3 k, f3& th, f3& ph) {
    const float rho = sqrtf(k.x * k.x + k.y * k.y);
    float c = 1.0f, s = 0.0f;
    if (rho > 0.0f) {
        c = k.x / rho;
        s = k.y / rho;
    }
    th = {k.z * c, k.z * s, -rho};
    ph = {-s, c, 0.0f};
}

// Uniform direction on the hemisphere around the unit normal n: cos theta_s =
// 1 - u1, phi_s = 2 pi u2 in the tangent frame of m = n (or -n when
// n_z < -1/2): t1 = (1 - m_x^2 a, -m_x m_y a, -m_x), t2 = (-m_x m_y a,
// 1 - m_y^2 a, -m_y), a = 1 / (1 + m_z)  (Frisvad, JGT 2012).
__device__ __forceinline__ f3 diffuse_dir(f3 n, float u1, float u2) {
    const f3 m = n.z >= -0.5f ? n : n * -1.0f;
    const float a = 1.0f / (1.0f + m.z), b = -m.x * m.y * a;
    const f3 t1{1.0f - m.x * m.x * a, b, -m.x}, t2{b, 1.0f - m.y * m.y * a, -m.y};
    const float cs = 1.0f - u1, sn = sqrtf(u1 * (2.0f - u1));
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    const float a1 = sn * cp, a2 = sn * sp;
    return {t1.x * a1 + t2.x * a2 + n.x * cs, t1.y * a1 + t2.y * a2 + n.y * cs, t1.z * a1 + t2.z * a2 + n.z * cs};
}

// F_alpha(theta_i) = 2^-alpha sum_k C(alpha, k) I_k (Eq. directive_model) in one
// pass: C(alpha, k) and the partial sums of C(2w, w) (sin^2 theta_i / 4)^w
// that the odd I_k share are both updated by their term ratios.
__device__ __noinline__ float f_alpha(int alpha, float cos_i) {
    const float x = 0.25f * (1.0f - cos_i) * (1.0f + cos_i);
    float binom = 1.0f, inner = 0.0f, term = 1.0f, F = 0.0f;
    for (int k = 0; k <= alpha; ++k) {
        float ik = 1.0f;
        if (k & 1) {
            const float w = (float)(k >> 1);
            inner += term;
            term *= x * (2.0f * w + 1.0f) * (2.0f * w + 2.0f) / ((w + 1.0f) * (w + 1.0f));
            ik = cos_i * inner;
        }
        F += binom * ik / (float)(k + 1);
        binom = binom * (float)(alpha - k) / (float)(k + 1);
    }
    return F * 6.283185307179586f * exp2f(-(float)alpha);
}
__device__ __forceinline__ float powi(float x, int a) {
    float r = 1.0f;
#pragma unroll 1
    for (int i = 0; i < a; ++i) r *= x;
    return r;
}
// Scattering pattern f_s(k_i, k_s, n) (Eqs. lambertian_model,
// directive_model, backscattering_model); n on the incident side,
// cos_i = -k_i.n, cos_s = k_s.n.
__device__ float scat_pattern(const MatDev& M, f3 k, f3 ks, f3 n, float cos_i, float cos_s) {
    if (M.pattern == 0) return cos_s * 0.31830988618379067f;
    const float kn = 2.0f * dot(k, n);
    const f3 kr{k.x - kn * n.x, k.y - kn * n.y, k.z - kn * n.z};
    const float lr = powi(0.5f * (1.0f + dot(kr, ks)), M.alpha_r);
    const float fr = f_alpha(M.alpha_r, cos_i);
    if (M.pattern == 1) return lr / fr;
    const float li = powi(0.5f * (1.0f - dot(k, ks)), M.alpha_i);
    return (M.lam * lr + (1.0f - M.lam) * li) / (M.lam * fr + (1.0f - M.lam) * f_alpha(M.alpha_i, cos_i));
}

// Constants of one diffuse event: TE/TM basis of the incidence, spherical
// bases of k_i and k_s, the unreduced reflection coefficients, the random
// phases and c0 = S sqrt(2 pi f_s) (the estimator's weight 2 pi r^2 / |n.k_i|
// per diffuse point cancels the tube length and cos theta_i of Eq.
// scattered_field).
struct Diffuse {
    f3 ep, epi, thi, phi, ths, phs;
    cf rp, rl, ph1, ph2;
    float c0, sqk, sq1k;
};
// Scattered field of one polarisation column (Eq. scattered_field):
// E_s = c0 Gamma [(sqrt(1-K) E_th - sqrt(K) E_ph) e^{j chi_1} theta_hat(k_s)
//               + (sqrt(K) E_th + sqrt(1-K) E_ph) e^{j chi_2} phi_hat(k_s)],
// Gamma^2 = (|r_perp E_perp|^2 + |r_par E_par|^2) / |E|^2.
__device__ __forceinline__ void diffuse_field(const Diffuse& D, const cf* E, cf* Eo) {
    const cf a = edot(D.ep, E), b = edot(D.epi, E);
    const float g2 = cabs2(D.rp * a) + cabs2(D.rl * b);
    const float e2 = cabs2(E[0]) + cabs2(E[1]) + cabs2(E[2]);
    const float c = (e2 > 0.0f && g2 > 0.0f) ? D.c0 * sqrtf(g2 / e2) : 0.0f;
    const cf et = edot(D.thi, E), ef = edot(D.phi, E);
    const cf as = (et * D.sq1k - ef * D.sqk) * D.ph1 * c;
    const cf bs = (et * D.sqk + ef * D.sq1k) * D.ph2 * c;
    Eo[0] = as * D.ths.x + bs * D.phs.x;
    Eo[1] = as * D.ths.y + bs * D.phs.y;
    Eo[2] = as * D.ths.z + bs * D.phs.z;
}
// Its derivative along one real parameter direction: T = dE of the incident
// field, deta = d eta (0 unless the parameter belongs to this material),
// drp, drl = d r / d eta.  Gamma depends on |.| of complex numbers, so the
// map is not holomorphic in eta: permittivity and conductivity directions
// are carried separately through a diffuse event.
__device__ __forceinline__ void diffuse_tangent(const Diffuse& D, const cf* E, const cf* T, cf deta, cf drp,
                                                cf drl, cf* To) {
    const cf a = edot(D.ep, E), b = edot(D.epi, E);
    const cf A = D.rp * a, B = D.rl * b;
    const float g2 = cabs2(A) + cabs2(B);
    const float e2 = cabs2(E[0]) + cabs2(E[1]) + cabs2(E[2]);
    if (!(e2 > 0.0f && g2 > 0.0f && D.c0 > 0.0f)) {
        for (int j = 0; j < 3; ++j) To[j] = C(0.0f);
        return;
    }
    const float c = D.c0 * sqrtf(g2 / e2);
    const cf da = edot(D.ep, T), db = edot(D.epi, T);
    const cf dA = drp * deta * a + D.rp * da;
    const cf dB = drl * deta * b + D.rl * db;
    const float dg2 = 2.0f * (cjmul(A, dA).r + cjmul(B, dB).r);
    const float de2 = 2.0f * (cjmul(E[0], T[0]).r + cjmul(E[1], T[1]).r + cjmul(E[2], T[2]).r);
    const float dc = c * (0.5f * dg2 / g2 - 0.5f * de2 / e2);
    const cf et = edot(D.thi, E), ef = edot(D.phi, E), det = edot(D.thi, T), def = edot(D.phi, T);
    const cf as = (et * D.sq1k - ef * D.sqk) * D.ph1, bs = (et * D.sqk + ef * D.sq1k) * D.ph2;
    const cf das = (det * D.sq1k - def * D.sqk) * D.ph1, dbs = (det * D.sqk + def * D.sq1k) * D.ph2;
    const cf ao = as * dc + das * c, bo = bs * dc + dbs * c;
    To[0] = ao * D.ths.x + bo * D.phs.x;
    To[1] = ao * D.ths.y + bo * D.phs.y;
    To[2] = ao * D.ths.z + bo * D.phs.z;
}

// Direction, pattern value, bases and random phases of one diffuse event.
__device__ __forceinline__ void diffuse_setup_body(const MatDev& M, f3 k, f3 nrm, float cos1, cf rp, cf rl, f3 ep,
                                                   f3 epi, unsigned long long seed, unsigned long long n, int depth,
                                                   Diffuse* D, f3* ko_out) {
    const f3 ko = diffuse_dir(nrm, rng_u(seed ^ DIFF_STREAM0, n, depth), rng_u(seed ^ DIFF_STREAM1, n, depth));
    const float fs = scat_pattern(M, k, ko, nrm, cos1, dot(ko, nrm));
    D->ep = ep;
    D->epi = epi;
    sph_basis(k, D->thi, D->phi);
    sph_basis(ko, D->ths, D->phs);
    D->rp = rp;
    D->rl = rl;
    float s1, k1, s2, k2;
    sincospif(2.0f * rng_u(seed ^ DIFF_STREAM2, n, depth), &s1, &k1);
    sincospif(2.0f * rng_u(seed ^ DIFF_STREAM3, n, depth), &s2, &k2);
    D->ph1 = C(k1, s1);
    D->ph2 = C(k2, s2);
    D->c0 = fs > 0.0f ? M.S * sqrtf(6.283185307179586f * fs) : 0.0f;
    D->sqk = M.sqk;
    D->sq1k = M.sq1k;
    *ko_out = ko;
}
// out of line, for the adjoint (which differentiates through D)
__device__ __noinline__ void diffuse_setup(const MatDev& M, f3 k, f3 nrm, float cos1, cf rp, cf rl, f3 ep, f3 epi,
                                           unsigned long long seed, unsigned long long n, int depth, Diffuse* D,
                                           f3* ko_out) {
    diffuse_setup_body(M, k, nrm, cos1, rp, rl, ep, epi, seed, n, depth, D, ko_out);
}
// the forward's whole diffuse event out of line: D stays in this function's
// registers and only the field goes through memory
template <int NPOL>
__device__ __noinline__ void diffuse_event(const MatDev& M, f3 k, f3 nrm, float cos1, cf rp, cf rl, f3 ep, f3 epi,
                                           unsigned long long seed, unsigned long long n, int depth, cf (*E)[3],
                                           f3* ko_out) {
    Diffuse D;
    diffuse_setup_body(M, k, nrm, cos1, rp, rl, ep, epi, seed, n, depth, &D, ko_out);
    for (int p = 0; p < NPOL; ++p) {
        cf eo[3];
        diffuse_field(D, E[p], eo);
        for (int a = 0; a < 3; ++a) E[p][a] = eo[a];
    }
}

// ------------------------------------------------------------------ traversal
struct Ray {
    float ox, oy, oz, kx, ky, kz;
};

__device__ __forceinline__ bool box_hit(float lx, float ly, float lz, float hx, float hy, float hz, const Ray& r,
                                        float ix, float iy, float iz, float tmax, float& tnear) {
    const float t0x = (lx - r.ox) * ix, t1x = (hx - r.ox) * ix;
    const float t0y = (ly - r.oy) * iy, t1y = (hy - r.oy) * iy;
    const float t0z = (lz - r.oz) * iz, t1z = (hz - r.oz) * iz;
    const float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), 0.0f));
    float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), tmax));
    // robust slab test: widen the far distance by 1 + 2 gamma_3 (Ize, JCGT 2013)
    tf = tf * 1.0000004f;
    tnear = tn;
    return tn <= tf;
}

struct Hit {
    int slot;   // leaf position, -1 = none
    int prim;   // original triangle index
    float t;
};

// Closest hit along the ray, excluding leaf `exclude`.  Equal distances go to
// the smaller original triangle index; distances within 8 ulps (relative
// TIE_REL) count as equal, so coplanar triangles resolve by index.  COUNT:
// node visits and triangle tests are counted (the debug and statistics
// instantiations only; the two increments cost the plain tracer 1-2 %).
constexpr float TIE_REL = 4.8e-7f;
template <bool ONE_SITE, bool COUNT>
__device__ __forceinline__ Hit closest_hit(const float4* __restrict__ nodes, const float4* __restrict__ tris, int nt,
                                           int nlarge, const Ray& r, int exclude, unsigned& c_nodes,
                                           unsigned& c_tris, bool& overflow) {
    Hit h{-1, 0x7fffffff, INFINITY};
    if (nt <= 0 && nlarge <= 0) return h;
    const float ooeps = 0x1p-80f;
    // correctly rounded reciprocals (this file builds with approximate division;
    // the robust slab test's error bound counts one rounding here)
    const float ix = __frcp_rn(fabsf(r.kx) > ooeps ? r.kx : copysignf(ooeps, r.kx));
    const float iy = __frcp_rn(fabsf(r.ky) > ooeps ? r.ky : copysignf(ooeps, r.ky));
    const float iz = __frcp_rn(fabsf(r.kz) > ooeps ? r.kz : copysignf(ooeps, r.kz));
    // watertight test set-up: kz = dominant axis, (kx, ky) keep the winding
    const float ax = fabsf(r.kx), ay = fabsf(r.ky), az = fabsf(r.kz);
    int kzi = (ay > ax) ? 1 : 0;
    if (az > fmaxf(ax, ay)) kzi = 2;
    int kxi = kzi == 2 ? 0 : kzi + 1;
    int kyi = kxi == 2 ? 0 : kxi + 1;
    const f3 k{r.kx, r.ky, r.kz};
    const float dz = sel(k, kzi);
    if (dz < 0.0f) {
        const int t = kxi;
        kxi = kyi;
        kyi = t;
    }
    const float Sx = sel(k, kxi) / dz, Sy = sel(k, kyi) / dz, Sz = 1.0f / dz;
    const f3 o{r.ox, r.oy, r.oz};
    const float opx = sel(o, kxi), opy = sel(o, kyi), opz = sel(o, kzi);

    // ray-triangle test of leaf `slot` (watertight; Woop, Benthin & Wald 2013)
    auto test_leaf = [&](int slot) {
        if (slot == exclude) return;
        if (COUNT) ++c_tris;
        const float4* tp = tris + 3 * (size_t)slot;
        const float4 r0 = __ldg(tp), r1 = __ldg(tp + 1), r2 = __ldg(tp + 2);
        const f3 va{r0.x, r0.y, r0.z}, vb{r0.w, r1.x, r1.y}, vc{r1.z, r1.w, r2.x};
        const float Akx = sel(va, kxi) - opx, Aky = sel(va, kyi) - opy, Akz = sel(va, kzi) - opz;
        const float Bkx = sel(vb, kxi) - opx, Bky = sel(vb, kyi) - opy, Bkz = sel(vb, kzi) - opz;
        const float Ckx = sel(vc, kxi) - opx, Cky = sel(vc, kyi) - opy, Ckz = sel(vc, kzi) - opz;
        const float Ax = Akx - Sx * Akz, Ay = Aky - Sy * Akz;
        const float Bx = Bkx - Sx * Bkz, By = Bky - Sy * Bkz;
        const float Cx = Ckx - Sx * Ckz, Cy = Cky - Sy * Ckz;
        float U = Cx * By - Cy * Bx;
        float V = Ax * Cy - Ay * Cx;
        float W = Bx * Ay - By * Ax;
        if (U == 0.0f || V == 0.0f || W == 0.0f) {
            U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
            V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
            W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
        }
        const bool neg = (U < 0.0f || V < 0.0f || W < 0.0f);
        const bool pos = (U > 0.0f || V > 0.0f || W > 0.0f);
        float det = U + V + W;
        if ((neg && pos) || det == 0.0f) return;
        float T = U * (Sz * Akz) + V * (Sz * Bkz) + W * (Sz * Ckz);
        if (det < 0.0f) {
            T = -T;
            det = -det;
        }
        const float thi = h.t * (1.0f + TIE_REL);
        if (!(T > 0.0f) || T > thi * det) return;
        const float t = T / det;
        const int prim = __float_as_int(r2.z);
        if (t < h.t * (1.0f - TIE_REL) || (t <= thi && prim < h.prim)) {
            h.t = t;
            h.slot = slot;
            h.prim = prim;
        }
    };
    if (ONE_SITE) {
        // One loop serves the large triangles (tested first: their hit distance
        // then prunes the traversal), a one-triangle tree, and the stack traversal
        // over internal nodes, whose hit leaf children are tested in their
        // parent's step.  Every triangle test goes through the single call site at
        // the bottom of the loop, which keeps the kernel's code small (the diffuse,
        // adjoint and mesh-surface instantiations, whose longer shading or second
        // walk otherwise crowds the instruction cache, use this form).
        const int npre = nlarge + (nt == 1 ? 1 : 0);
        int stack[STACK_SIZE];
        int sp = 0;
        int cur = 0;
        int j = 0;
        bool trav = nt > 1;
        // a valid tree has nt - 1 internal nodes, each visited at most once
        int budget = 2 * nt + 8;   // nt <= INT32_MAX / 4 (checked at upload): no overflow
        while (true) {
            int la = -1, lb = -1;
            if (j < npre) {
                la = j < nlarge ? nt + j : 0;
                ++j;
            } else if (trav) {
                if (--budget < 0) {
                    overflow = true;
                    break;
                }
                if (COUNT) ++c_nodes;
                const float4* nd = nodes + 4 * (size_t)cur;
                const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
                float tn0, tn1;
                const float tmax = h.t * (1.0f + TIE_REL);
                bool h0 = box_hit(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, r, ix, iy, iz, tmax, tn0);
                bool h1 = box_hit(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, r, ix, iy, iz, tmax, tn1);
                const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
                if (h0 && c0 < 0) {
                    la = ~c0;
                    h0 = false;
                }
                if (h1 && c1 < 0) {
                    lb = ~c1;
                    h1 = false;
                }
                if (h0 && h1) {
                    const bool first0 = tn0 <= tn1;
                    if (sp < STACK_SIZE) stack[sp++] = first0 ? c1 : c0;
                    else overflow = true;
                    cur = first0 ? c0 : c1;
                } else if (h0) {
                    cur = c0;
                } else if (h1) {
                    cur = c1;
                } else if (sp == 0) {
                    trav = false;
                } else {
                    cur = stack[--sp];
                }
            } else {
                break;
            }
    #pragma unroll 1
            for (int q = 0; q < 2; ++q) {
                const int lf = q ? lb : la;
                if (lf >= 0) test_leaf(lf);
            }
        }
    } else {
        // large triangles first: their hit distance then prunes the traversal
        for (int j = 0; j < nlarge; ++j) test_leaf(nt + j);
        if (nt <= 0) return h;
        if (nt == 1) {
            test_leaf(0);
            return h;
        }

        // Stack traversal over internal nodes; a hit leaf child is tested inside
        // its parent's step, so leaves never take a loop iteration of their own.
        int stack[STACK_SIZE];
        int sp = 0;
        int cur = 0;
        // a valid tree has nt - 1 internal nodes, each visited at most once
        int budget = 2 * nt + 8;   // nt <= INT32_MAX / 4 (checked at upload): no overflow
        while (true) {
            if (--budget < 0) {
                overflow = true;
                break;
            }
            if (COUNT) ++c_nodes;
            const float4* nd = nodes + 4 * (size_t)cur;
            const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
            float tn0, tn1;
            const float tmax = h.t * (1.0f + TIE_REL);
            bool h0 = box_hit(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, r, ix, iy, iz, tmax, tn0);
            bool h1 = box_hit(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, r, ix, iy, iz, tmax, tn1);
            const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
            if (h0 && c0 < 0) {
                test_leaf(~c0);
                h0 = false;
            }
            if (h1 && c1 < 0) {
                test_leaf(~c1);
                h1 = false;
            }
            if (h0 && h1) {
                const bool first0 = tn0 <= tn1;
                if (sp < STACK_SIZE) stack[sp++] = first0 ? c1 : c0;
                else overflow = true;
                cur = first0 ? c0 : c1;
            } else if (h0) {
                cur = c0;
            } else if (h1) {
                cur = c1;
            } else {
                if (sp == 0) break;
                cur = stack[--sp];
            }
        }
    }
    return h;
}

// The hit of one given leaf (the adjoint's replay of the forward's recorded
// closest hit): closest_hit's watertight set-up and leaf test, expression for
// expression and in the same translation unit, so that t equals the
// forward's bit for bit.  Returns false if the test rejects the leaf (the
// caller then traverses).
__device__ __forceinline__ bool recorded_hit(const float4* __restrict__ tris, const Ray& r, int slot, Hit& h) {
    const float ax = fabsf(r.kx), ay = fabsf(r.ky), az = fabsf(r.kz);
    int kzi = (ay > ax) ? 1 : 0;
    if (az > fmaxf(ax, ay)) kzi = 2;
    int kxi = kzi == 2 ? 0 : kzi + 1;
    int kyi = kxi == 2 ? 0 : kxi + 1;
    const f3 k{r.kx, r.ky, r.kz};
    const float dz = sel(k, kzi);
    if (dz < 0.0f) {
        const int t = kxi;
        kxi = kyi;
        kyi = t;
    }
    const float Sx = sel(k, kxi) / dz, Sy = sel(k, kyi) / dz, Sz = 1.0f / dz;
    const f3 o{r.ox, r.oy, r.oz};
    const float opx = sel(o, kxi), opy = sel(o, kyi), opz = sel(o, kzi);
    const float4* tp = tris + 3 * (size_t)slot;
    const float4 r0 = __ldg(tp), r1 = __ldg(tp + 1), r2 = __ldg(tp + 2);
    const f3 va{r0.x, r0.y, r0.z}, vb{r0.w, r1.x, r1.y}, vc{r1.z, r1.w, r2.x};
    const float Akx = sel(va, kxi) - opx, Aky = sel(va, kyi) - opy, Akz = sel(va, kzi) - opz;
    const float Bkx = sel(vb, kxi) - opx, Bky = sel(vb, kyi) - opy, Bkz = sel(vb, kzi) - opz;
    const float Ckx = sel(vc, kxi) - opx, Cky = sel(vc, kyi) - opy, Ckz = sel(vc, kzi) - opz;
    const float Ax = Akx - Sx * Akz, Ay = Aky - Sy * Akz;
    const float Bx = Bkx - Sx * Bkz, By = Bky - Sy * Bkz;
    const float Cx = Ckx - Sx * Ckz, Cy = Cky - Sy * Ckz;
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    const bool neg = (U < 0.0f || V < 0.0f || W < 0.0f);
    const bool pos = (U > 0.0f || V > 0.0f || W > 0.0f);
    float det = U + V + W;
    if ((neg && pos) || det == 0.0f) return false;
    float T = U * (Sz * Akz) + V * (Sz * Bkz) + W * (Sz * Ckz);
    if (det < 0.0f) {
        T = -T;
        det = -det;
    }
    if (!(T > 0.0f)) return false;
    h.t = T / det;
    h.slot = slot;
    h.prim = __float_as_int(r2.z);
    return true;
}

// ------------------------------------------------------------------ mesh measurement surface
// Crossings of the open segment (1e-9, tmax) with a mesh measurement surface
// (Sec. 4, practical notes): every crossed triangle is a cell and receives
// v0 / (A |n . k|), the planar estimator (Eq. radio-map-solver-ci-all-2-
// estimator) with the triangle's own area and normal; v0 = 4 pi / N
// (lambda0 / 4 pi)^2 |E|^2 / Pr.  With det = e1 . (k x e2) = -(e1 x e2) . k,
// A |n . k| = |det| / 2.  Edges count on both sides (u, v >= 0, u + v <= 1).
// Returns the number of crossings; *overflow is set if the traversal stack or
// its step budget runs out.  GATHER (the adjoint): instead of depositing,
// *g_out receives sum_i dLdC_i 2 / |det_i| over the crossings, so that
// sum_i dLdC_i dC_i = v0-derivative times dep_scale / Pr times that sum.
template <bool GATHER>
__device__ __noinline__ unsigned surface_crossings(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                                   int nt, int nlarge, float ox, float oy, float oz, float kx,
                                                   float ky, float kz, float tmax, float v0,
                                                   double* __restrict__ map, const float* __restrict__ dldc,
                                                   float* g_out, bool* overflow) {
    unsigned cnt = 0;
    float gsum = 0.0f;
    const f3 o{ox, oy, oz}, k{kx, ky, kz};
    auto leaf = [&](int slot) {
        const float4* tp = tris + 3 * (size_t)slot;
        const float4 r0 = __ldg(tp), r1 = __ldg(tp + 1), r2 = __ldg(tp + 2);
        const f3 a{r0.x, r0.y, r0.z}, b{r0.w, r1.x, r1.y}, c{r1.z, r1.w, r2.x};
        const f3 e1 = b - a, e2 = c - a;
        const f3 pv = cross(k, e2);
        const float det = dot(e1, pv);
        if (det == 0.0f) return;
        const float inv = 1.0f / det;
        const f3 tv = o - a;
        const float u = dot(tv, pv) * inv;
        if (u < 0.0f || u > 1.0f) return;
        const f3 q = cross(tv, e1);
        const float v = dot(k, q) * inv;
        if (v < 0.0f || u + v > 1.0f) return;
        const float t = dot(e2, q) * inv;
        if (!(t > 1e-9f && t < tmax)) return;
        if (GATHER) gsum += __ldg(dldc + __float_as_int(r2.z)) * (2.0f / fabsf(det));
        else atomicAdd(map + __float_as_int(r2.z), (double)(2.0f * v0 / fabsf(det)));
        ++cnt;
    };
#pragma unroll 1
    for (int j = 0; j < nlarge; ++j) leaf(nt + j);
    if (nt == 1) leaf(0);
    if (nt < 2) {
        if (GATHER) *g_out = gsum;
        return cnt;
    }
    const float ooeps = 0x1p-80f;
    const float ix = __frcp_rn(fabsf(kx) > ooeps ? kx : copysignf(ooeps, kx));
    const float iy = __frcp_rn(fabsf(ky) > ooeps ? ky : copysignf(ooeps, ky));
    const float iz = __frcp_rn(fabsf(kz) > ooeps ? kz : copysignf(ooeps, kz));
    auto box = [&](float lx, float ly, float lz, float hx, float hy, float hz) {
        const float t0x = (lx - ox) * ix, t1x = (hx - ox) * ix;
        const float t0y = (ly - oy) * iy, t1y = (hy - oy) * iy;
        const float t0z = (lz - oz) * iz, t1z = (hz - oz) * iz;
        const float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), 0.0f));
        const float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), tmax)) * 1.0000004f;
        return tn <= tf;
    };
    int stack[STACK_SIZE];
    int sp = 0, cur = 0;
    int budget = 2 * nt + 8;   // nt <= INT32_MAX / 4 (checked at upload): no overflow
    while (true) {
        if (--budget < 0) {
            *overflow = true;
            if (GATHER) *g_out = gsum;
            return cnt;
        }
        const float4* nd = nodes + 4 * (size_t)cur;
        const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        bool h0 = box(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
        bool h1 = box(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
        const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        if (h0 && c0 < 0) {
            leaf(~c0);
            h0 = false;
        }
        if (h1 && c1 < 0) {
            leaf(~c1);
            h1 = false;
        }
        if (h0 && h1) {
            if (sp < STACK_SIZE) stack[sp++] = c1;
            else *overflow = true;
            cur = c0;
        } else if (h0) {
            cur = c0;
        } else if (h1) {
            cur = c1;
        } else {
            if (sp == 0) {
                if (GATHER) *g_out = gsum;
                return cnt;
            }
            cur = stack[--sp];
        }
    }
}

// ------------------------------------------------------------------ work items
// Transmitter of work item w (the transmitters' work_begin ascending).
__device__ __forceinline__ int work_tx(const TxDev* tx, int ntx, unsigned long long w) {
    int lo = 0, hi = ntx - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tx[mid].work_begin <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Lattice index n of work item w of transmitter T (and its position isub in
// T's subset).  Neighbouring work items visit neighbouring lattice directions:
// i = j * F mod count with F a Fibonacci number (lattice neighbour step).
__device__ __forceinline__ unsigned long long work_lattice(const TxDev& T, unsigned long long w,
                                                          unsigned long long& isub) {
    isub = w - T.work_begin;
    if (T.perm > 1ULL) {
        // (isub * perm) mod count by Barrett reduction (isub, perm < count,
        // product < 2^63): the estimate q is at most 2 below the quotient
        const unsigned long long xp = isub * T.perm;
        const unsigned long long q = __umul64hi(xp, T.perm_m);
        unsigned long long rr = xp - q * T.count;
        if (rr >= T.count) rr -= T.count;
        if (rr >= T.count) rr -= T.count;
        isub = rr;
    }
    return T.begin + isub * T.stride;
}

// The synthetic-array factor of every work item's ray before the tracer runs
// (transmitters with arrays only): the tracer's own arithmetic (four unrolled
// Horner chains instead of two rolled ones, the same bits), evaluated here by
// full warps at the occupancy of a small kernel instead of inside the
// tracer's ray launch, where its chains run beside the tracer's divergent loop.
// (WIDE = false: the tracer's inline two-chain form, for the debug comparison
// of the two forms.)
template <bool WIDE>
__global__ void __launch_bounds__(256) k_alpha(const TraceArgs A, float2* __restrict__ alpha) {
    __shared__ TxDev s_tx[RM_MAX_TX];
    {
        const int ntw = A.ntx * (int)(sizeof(TxDev) / 4);
        for (int i = threadIdx.x; i < ntw; i += blockDim.x)
            reinterpret_cast<int*>(s_tx)[i] = reinterpret_cast<const int*>(A.tx)[i];
    }
    __syncthreads();
    for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w < A.total;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const TxDev& T = s_tx[work_tx(s_tx, A.ntx, w)];
        if (T.n_ant <= 0) continue;
        unsigned long long isub;
        const unsigned long long n = work_lattice(T, w, isub);
        float are, aim;
        if (WIDE) array_factor_lattice_wide(T, A.ant, n, are, aim);
        else array_factor_lattice(T, A.ant, n, are, aim);
        alpha[w] = make_float2(are, aim);
    }
}

// ------------------------------------------------------------------ kernel
constexpr int NGRAD = 2 * RM_MAX_MATERIALS + 3 * RM_MAX_TX;
constexpr int MAXSLOT = RM_MAX_DEPTH;

// Register budget: 64 registers (four 256-thread blocks per SM) for every
// instantiation; the extra resident warps hide more latency (much of it
// instruction fetch) than the spills cost, for the adjoint as well (its
// tangents live in local memory anyway).
// HITS: the plain forward that also writes every segment's closest-hit leaf
// to A.hits (the debug instantiations write it too when A.hits is set).
template <bool ADJ, int NPOL, bool DEBUG, bool BILIN, bool DIFF, bool MESH, bool HITS = false>
__global__ void __launch_bounds__(MAX_BLOCK, 4) k_trace(const TraceArgs A) {
    __shared__ MatDev s_mat[RM_MAX_MATERIALS];
    __shared__ TxDev s_tx[RM_MAX_TX];
    __shared__ float s_grad[ADJ ? NGRAD : 1];
    __shared__ unsigned long long s_cnt[6];
    __shared__ unsigned long long s_segd[DEBUG ? RM_MAX_DEPTH + 1 : 1];
    __shared__ double s_pw[DEBUG ? 3 * (RM_MAX_DEPTH + 1) : 1];

    const int tid = threadIdx.x, lane = tid & 31;
    {
        const int nmw = A.nm * (int)(sizeof(MatDev) / 4), ntw = A.ntx * (int)(sizeof(TxDev) / 4);
        for (int i = tid; i < nmw; i += blockDim.x) reinterpret_cast<int*>(s_mat)[i] = reinterpret_cast<const int*>(A.mats)[i];
        for (int i = tid; i < ntw; i += blockDim.x) reinterpret_cast<int*>(s_tx)[i] = reinterpret_cast<const int*>(A.tx)[i];
        if (ADJ)
            for (int i = tid; i < NGRAD; i += blockDim.x) s_grad[i] = 0.0f;
        if (tid < 6) s_cnt[tid] = 0;
        if (DEBUG) {
            for (int i = tid; i < RM_MAX_DEPTH + 1; i += blockDim.x) s_segd[i] = 0;
            for (int i = tid; i < 3 * (RM_MAX_DEPTH + 1); i += blockDim.x) s_pw[i] = 0.0;
        }
    }
    __syncthreads();

    const unsigned lt = (1u << lane) - 1u;
    const bool stats = DEBUG && (A.flags & RM_STATS);
    // ray state
    bool active = false, exhausted = false;
    // warp-local work queue [qb, qe) (warp-uniform), refilled A.qchunk items at a time
    unsigned long long qb = 0, qe = 0;
    Ray r{0, 0, 0, 0, 0, 1};
    cf E[NPOL][3];
    float inv_pr = 1.0f;
    float plen = 0.0f;  // unfolded tube length to the current origin
    int depth = 0, prev = -1, txi = 0;
    unsigned long long n = 0, isub = 0;
    unsigned long long witem = 0;   // the ray's work item: its column of the recorded hits
    // adjoint state: tangents dE/d eta per material met on the path
    cf Tg[ADJ ? MAXSLOT : 1][NPOL][3];
    cf Ts[(ADJ && DIFF) ? MAXSLOT : 1][NPOL][3];  // dE / d(sigma / (eps0 omega)) once diffuse events occur
    int Tm[ADJ ? MAXSLOT : 1];
    int nslot = 0;
    float J[(ADJ && BILIN) ? 9 : 1];  // d origin / d tx position, column-major
    unsigned c_rays = 0, c_seg = 0, c_nodes = 0, c_tris = 0, c_dep = 0, c_esc = 0;
    bool overflow = false;

    while (true) {
        // ---------------- refill free lanes (one atomic per warp) ----------------
        // (refills wait for A.refill_min idle lanes so that new rays, lattice
        // neighbours, enter a warp in coherent groups; an all-idle warp always refills)
        const unsigned need = __ballot_sync(FULL_MASK, !active);
        if (need && !(exhausted && qb >= qe) && __popc(need) >= A.refill_min) {
            const unsigned long long nneed = (unsigned long long)__popc(need);
            const unsigned long long rem = qe - qb;
            unsigned long long b = 0;
            const bool fetch = rem < nneed && !exhausted;
            // queue chunk of one warp (the default): take exactly the items the free lanes need
            const unsigned long long take = A.qchunk > 32ULL ? A.qchunk : nneed;
            if (fetch) {
                if (lane == 0) b = atomicAdd(&A.scratch->next, take);
                b = __shfl_sync(FULL_MASK, b, 0);
                if (b + take >= A.total) exhausted = true;
            }
            // lane rank r takes the r-th item of (rest of the local queue, then the new chunk)
            const unsigned long long rk = (unsigned long long)__popc(need & lt);
            const bool got_chunk = fetch && b < A.total;
            const unsigned long long ce = got_chunk ? min(b + take, A.total) : b;
            {
                if (!active) {
                    unsigned long long w = ~0ULL;
                    if (rk < rem) w = qb + rk;
                    else if (got_chunk && b + (rk - rem) < ce) w = b + (rk - rem);
                    if (w < A.total) {
                        txi = work_tx(s_tx, A.ntx, w);
                        const TxDev& T = s_tx[txi];
                        witem = w;
                        n = work_lattice(T, w, isub);
                        // Fibonacci lattice (Sec. 3.1.1): cos theta = 1 - 2n/(N-1),
                        // sin theta = 2 sqrt(n (N-1-n)) / (N-1), phi = 2 pi frac(n (phi_g - 1))
                        float ct, st, sp, cp;
                        if (T.N <= 1ULL) {
                            ct = 0.0f; st = 1.0f; sp = 0.0f; cp = -1.0f;
                        } else {
                            const unsigned long long Nm1 = T.N - 1ULL;
                            const float inv = 1.0f / (float)Nm1;
                            ct = (float)((long long)Nm1 - 2LL * (long long)n) * inv;
                            st = 2.0f * sqrtf((float)n * (float)(Nm1 - n)) * inv;
                            const unsigned long long f = n * 0x9E3779B97F4A7C16ULL;  // nearest integer to 2^64 (phi_g - 1)
                            const float x = (float)(int)(unsigned)(f >> 32) * 0x1p-31f;  // phi / pi in [-1, 1)
                            sincospif(x, &sp, &cp);
                        }
                        r.kx = st * cp; r.ky = st * sp; r.kz = ct;
                        r.ox = T.pos[0]; r.oy = T.pos[1]; r.oz = T.pos[2];
                        // antenna field R (C_theta theta' + C_phi phi') in the local angles (App. A.1)
                        const float lx = T.R[0] * r.kx + T.R[3] * r.ky + T.R[6] * r.kz;
                        const float ly = T.R[1] * r.kx + T.R[4] * r.ky + T.R[7] * r.kz;
                        const float lz = T.R[2] * r.kx + T.R[5] * r.ky + T.R[8] * r.kz;
                        const float sxy = sqrtf(lx * lx + ly * ly);
                        float cph = 1.0f, sph = 0.0f;
                        if (sxy > 0.0f) { cph = lx / sxy; sph = ly / sxy; }
                        const float g = (T.pattern == 1) ? 1.2247448713915890f * sxy : 1.0f;
                        const f3 th_l{lz * cph, lz * sph, -sxy}, ph_l{-sph, cph, 0.0f};
                        // synthetic array (Sec. 4.4): alpha = sum_k u_P,k exp(j k0 k.d_k) at the
                        // lattice direction rebuilt in double-float (array.cuh)
                        float are = 1.0f, aim = 0.0f;
                        if (T.n_ant > 0) {
                            if (A.alpha) {
                                const float2 al = A.alpha[w];
                                are = al.x;
                                aim = al.y;
                            } else {
                                array_factor_lattice(T, A.ant, n, are, aim);
                            }
                        }
                        for (int p = 0; p < NPOL; ++p) {
                            const int pol = (NPOL == 2) ? p : T.pol;
                            const f3 e = pol == 0 ? th_l : ph_l;
                            const float ex = g * (T.R[0] * e.x + T.R[1] * e.y + T.R[2] * e.z);
                            const float ey = g * (T.R[3] * e.x + T.R[4] * e.y + T.R[5] * e.z);
                            const float ez = g * (T.R[6] * e.x + T.R[7] * e.y + T.R[8] * e.z);
                            E[p][0] = C(ex * are, ex * aim);
                            E[p][1] = C(ey * are, ey * aim);
                            E[p][2] = C(ez * are, ez * aim);
                        }
                        inv_pr = 1.0f;
                        plen = 0.0f;
                        depth = 0;
                        prev = -1;
                        active = true;
                        ++c_rays;
                        if (ADJ) {
                            nslot = 0;
                            if (BILIN) {
                                for (int j = 0; j < 9; ++j) J[j] = (j % 4 == 0) ? 1.0f : 0.0f;
                            }
                        }
                    }
                }
            }
            // advance the warp-local queue (identical on every lane)
            if (rem >= nneed) {
                qb += nneed;
            } else if (got_chunk) {
                const unsigned long long used = nneed - rem;
                qb = min(b + used, ce);
                qe = ce;
            } else {
                qb = qe;
            }
        }
        if (__ballot_sync(FULL_MASK, active) == 0) break;

        // ---------------- closest hit ----------------
        Hit h{-1, 0x7fffffff, INFINITY};
        if (active) {
            bool replayed = false;
            if (ADJ && A.hits) {
                // the forward's closest hit of this segment (-1: escaped), tested alone
                const int s = A.hits[(unsigned long long)depth * A.total + witem];
                if (s == -1) replayed = true;
                else if (s >= 0 && s < A.nt + A.nlarge) replayed = recorded_hit(A.tris, r, s, h);
            }
            // the diffuse, adjoint and mesh-surface forms traverse through one triangle-test call site
            // (their longer code otherwise crowds the instruction cache)
            if (!replayed)
                h = closest_hit<DIFF || ADJ || MESH, DEBUG>(A.nodes, A.tris, A.nt, A.nlarge, r, prev, c_nodes,
                                                            c_tris, overflow);
            if ((DEBUG || HITS) && !ADJ && A.hits)
                A.hits[(unsigned long long)depth * A.total + witem] = h.slot;
            ++c_seg;
            if (h.slot < 0) ++c_esc;
        }
        float e2 = 0.0f;
        if (active)
            for (int p = 0; p < NPOL; ++p) e2 += cabs2(E[p][0]) + cabs2(E[p][1]) + cabs2(E[p][2]);
        if (DEBUG && active) atomicAdd(&s_segd[depth], 1ULL);
        if (stats && active) {
            const float pw = e2 * inv_pr;
            atomicAdd(&s_pw[depth], (double)pw);
            atomicAdd(&s_pw[RM_MAX_DEPTH + 1 + depth], (double)pw * (double)pw);
            if (h.slot < 0) atomicAdd(&s_pw[2 * (RM_MAX_DEPTH + 1) + depth], (double)pw);
        }

        // ---------------- plane crossing ----------------
        bool dep = false;
        int ix = NO_CELL, iy = NO_CELL;
        float fx = 0.0f, fy = 0.0f;
        if (!MESH && active && r.kz != 0.0f && (depth > 0 || (A.flags & RM_LOS))) {
            const float tc = (A.zm - r.oz) / r.kz;
            if (tc > 1e-9f && tc < h.t) {
                const float cx = r.ox + tc * r.kx, cy = r.oy + tc * r.ky;
                float ux = (cx - A.x0) * A.inv_cell, uy = (cy - A.y0) * A.inv_cell;
                if (BILIN) {
                    ux -= 0.5f;
                    uy -= 0.5f;
                    if (ux >= -1.0f && ux < (float)A.nx && uy >= -1.0f && uy < (float)A.ny) {
                        const float flx = floorf(ux), fly = floorf(uy);
                        ix = (int)flx; iy = (int)fly;
                        fx = ux - flx; fy = uy - fly;
                        dep = true;
                    }
                } else if (ux >= 0.0f && ux < (float)A.nx && uy >= 0.0f && uy < (float)A.ny) {
                    ix = (int)ux; iy = (int)uy;
                    dep = true;
                }
            }
        }
        rm_segment_record* rec = nullptr;
        if (DEBUG && active && A.record) {
            rec = A.record + s_tx[txi].rec_begin + isub * (unsigned long long)(A.L + 1) + depth;
            rec->prim = h.slot >= 0 ? h.prim : -1;
            rec->ix = ix;
            rec->iy = iy;
            rec->decision = -1;
        }
        const float value = dep ? s_tx[txi].dep_scale * e2 * inv_pr / fabsf(r.kz) : 0.0f;
        if (dep) ++c_dep;
        const unsigned long long mbase = (unsigned long long)txi * A.ncell;
        float tg0 = 0.0f, tg1 = 0.0f, tg2 = 0.0f;   // adjoint: this deposit's TX-position gradient

        if (MESH && !ADJ) {
            // mesh measurement surface: every triangle the segment crosses
            if (active && (depth > 0 || (A.flags & RM_LOS)))
                c_dep += surface_crossings<false>(A.snodes, A.stris, A.snt, A.snlarge, r.ox, r.oy, r.oz, r.kx, r.ky,
                                                  r.kz, h.t, s_tx[txi].dep_scale * e2 * inv_pr, A.maps64 + mbase,
                                                  nullptr, nullptr, &overflow);
        } else if (!ADJ) {
            // one FP64 reduction per deposit (per stencil corner): a cell may
            // receive ~1e5 deposits, which FP32 accumulation would round to
            // ~1e-2.  Lanes that hit the same cell go to the L2 atomic units
            // unmerged; merging them in the warp first (match + shared-memory
            // sum) measured 4-6 % slower.
            if (dep) {
                const int ncorner = BILIN ? 4 : 1;
                for (int cn = 0; cn < ncorner; ++cn) {
                    float v = value;
                    int cxi = ix, cyi = iy;
                    if (BILIN) {
                        const int a = cn & 1, b = cn >> 1;
                        cxi += a; cyi += b;
                        v *= (a ? fx : 1.0f - fx) * (b ? fy : 1.0f - fy);
                        if (cxi < 0 || cxi >= A.nx || cyi < 0 || cyi >= A.ny) continue;
                    }
                    const unsigned long long key = mbase + (unsigned long long)cyi * A.nx + cxi;
                    if (A.maps64) atomicAdd(A.maps64 + key, (double)v);
                    else atomicAdd(A.maps + key, v);
                }
            }
        } else if (MESH ? (active && (depth > 0 || (A.flags & RM_LOS))) : dep) {
            // adjoint: gather g = dL/dC at the deposit (and its spatial derivative)
            float G = 0.0f, Gx = 0.0f, Gy = 0.0f;
            float sc = s_tx[txi].dep_scale * inv_pr;
            if (MESH) {
                // every crossed triangle: G = sum_i dLdC_i / (A_i |n_i . k|)
                c_dep += surface_crossings<true>(A.snodes, A.stris, A.snt, A.snlarge, r.ox, r.oy, r.oz, r.kx, r.ky,
                                                 r.kz, h.t, 0.0f, nullptr, A.dLdC + mbase, &G, &overflow);
            } else if (BILIN) {
#pragma unroll 1
                for (int cn = 0; cn < 4; ++cn) {
                    const int a = cn & 1, b = cn >> 1;
                    const int cxi = ix + a, cyi = iy + b;
                    if (cxi < 0 || cxi >= A.nx || cyi < 0 || cyi >= A.ny) continue;
                    const float g = __ldg(A.dLdC + mbase + (unsigned long long)cyi * A.nx + cxi);
                    const float wx = a ? fx : 1.0f - fx, wy = b ? fy : 1.0f - fy;
                    G += g * wx * wy;
                    Gx += g * (a ? 1.0f : -1.0f) * wy;
                    Gy += g * wx * (b ? 1.0f : -1.0f);
                }
                Gx *= A.inv_cell;
                Gy *= A.inv_cell;
            } else {
                G = __ldg(A.dLdC + mbase + (unsigned long long)iy * A.nx + ix);
            }
            if (!MESH) sc /= fabsf(r.kz);
            if (G != 0.0f) {
#pragma unroll 1
                for (int s = 0; s < nslot; ++s) {
                    cf z = C(0.0f);
                    for (int p = 0; p < NPOL; ++p)
                        for (int a = 0; a < 3; ++a) z = z + cjmul(E[p][a], Tg[s][p][a]);
                    // d|E|^2/d eps_r = 2 Re(E^H T); d|E|^2/d sigma = 2 Re(E^H T (-j/(eps0 w))) = 2 Im(E^H T)/(eps0 w)
                    // (with diffuse events the sigma direction has its own tangent Ts = dE/d(sigma/(eps0 w)))
                    float zs = z.i;
                    if (DIFF) {
                        cf w = C(0.0f);
                        for (int p = 0; p < NPOL; ++p)
                            for (int a = 0; a < 3; ++a) w = w + cjmul(E[p][a], Ts[s][p][a]);
                        zs = w.r;
                    }
                    atomicAdd(&s_grad[Tm[s]], 2.0f * sc * G * z.r);
                    atomicAdd(&s_grad[RM_MAX_MATERIALS + Tm[s]], 2.0f * sc * G * zs * A.inv_eps0_omega);
                }
            }
            if (BILIN && (Gx != 0.0f || Gy != 0.0f)) {
                // crossing x_c = o + t_c k with t_c = (z_M - o_z)/k_z: dx_c/do = I - k e_z^T / k_z
                const float ax = r.kx / r.kz, ay = r.ky / r.kz;
                const float v = sc * e2;
                float tg[3];
                for (int c = 0; c < 3; ++c) {
                    const float dx = J[3 * c + 0] - ax * J[3 * c + 2];
                    const float dy = J[3 * c + 1] - ay * J[3 * c + 2];
                    tg[c] = v * (Gx * dx + Gy * dy);
                }
                tg0 = tg[0];
                tg1 = tg[1];
                tg2 = tg[2];
            }
        }

        if (ADJ && BILIN) {
            // TX-position gradient: one warp sum per transmitter and step instead
            // of one shared atomic per deposit on the same three words (the lanes
            // of a warp nearly always trace the same transmitter)
            const bool c = tg0 != 0.0f || tg1 != 0.0f || tg2 != 0.0f;
            const unsigned cm = __ballot_sync(FULL_MASK, c);
            if (cm) {
                const int t0 = __shfl_sync(FULL_MASK, txi, __ffs(cm) - 1);
                if (__all_sync(FULL_MASK, !c || txi == t0)) {
                    for (int o = 16; o > 0; o >>= 1) {
                        tg0 += __shfl_xor_sync(FULL_MASK, tg0, o);
                        tg1 += __shfl_xor_sync(FULL_MASK, tg1, o);
                        tg2 += __shfl_xor_sync(FULL_MASK, tg2, o);
                    }
                    if (lane == 0) {
                        atomicAdd(&s_grad[2 * RM_MAX_MATERIALS + 3 * t0 + 0], tg0);
                        atomicAdd(&s_grad[2 * RM_MAX_MATERIALS + 3 * t0 + 1], tg1);
                        atomicAdd(&s_grad[2 * RM_MAX_MATERIALS + 3 * t0 + 2], tg2);
                    }
                } else if (c) {
                    atomicAdd(&s_grad[2 * RM_MAX_MATERIALS + 3 * txi + 0], tg0);
                    atomicAdd(&s_grad[2 * RM_MAX_MATERIALS + 3 * txi + 1], tg1);
                    atomicAdd(&s_grad[2 * RM_MAX_MATERIALS + 3 * txi + 2], tg2);
                }
            }
        }

        // ---------------- termination / interaction ----------------
        if (active) {
            if (h.slot < 0 || depth >= A.L) {
                active = false;
            } else {
                const float4* tp = A.tris + 3 * (size_t)h.slot;
                const float4 q0 = __ldg(tp), q1 = __ldg(tp + 1), q2 = __ldg(tp + 2);
                const f3 va{q0.x, q0.y, q0.z}, vb{q0.w, q1.x, q1.y}, vc{q1.z, q1.w, q2.x};
                const int mat = __float_as_int(q2.y);
                f3 nrm = normalize(cross(vb - va, vc - va));
                const f3 k{r.kx, r.ky, r.kz};
                if (dot(k, nrm) > 0.0f) nrm = nrm * -1.0f;  // oriented towards the incident side
                const float cos1 = fminf(1.0f, fmaxf(0.0f, -dot(k, nrm)));
                const MatDev M = s_mat[mat];
                const cf eta = C(M.eta_re, M.eta_im);
                const Coef co = fresnel(eta, cos1, M.k0d_hi, M.k0d_lo, M.slab != 0, nullptr);
                float wR, wT;
                if (A.same_sampling) {
                    wR = cabs2(co.rp) + cabs2(co.rl);
                    wT = cabs2(co.tp) + cabs2(co.tl);
                } else {
                    const Coef cs = fresnel(C(M.seta_re, M.seta_im), cos1, M.k0d_hi, M.k0d_lo, M.slab != 0, nullptr);
                    wR = cabs2(cs.rp) + cabs2(cs.rl);
                    wT = cabs2(cs.tp) + cabs2(cs.tl);
                }
                if (!(A.flags & RM_REFLECT)) wR = 0.0f;
                if (!(A.flags & RM_REFRACT)) wT = 0.0f;
                const float wsum = wR + wT;
                if (!(wsum > 0.0f)) {
                    active = false;
                } else {
                    // coin (Eq. path-solver-used-dist-event, q(D) = 0): u < q(R) = R^2 wR / wsum
                    // -> R; u < wR / wsum -> S (diffuse, share S^2); else T
                    const float c2 = wR / wsum;
                    const float c1 = DIFF ? M.R2 * c2 : c2;
                    const float u = rng_u(s_tx[txi].seed, n, depth);
                    const int dec = (u < c1) ? 0 : ((DIFF && u < c2) ? 2 : 1);
                    // (debug) the threshold q(R) the coin compared u with, in units of 2^-22
                    if (rec) rec->decision = dec | ((A.flags & RM_RECORD_COIN) ? __float2int_rn(c1 * 0x1p22f) << 8 : 0);
                    if (DIFF)
                        inv_pr = inv_pr * (wsum / (dec == 0 ? M.R2 * wR : (dec == 2 ? M.S * M.S * wR : wT)));
                    else
                        inv_pr = inv_pr * (wsum / (dec == 0 ? wR : wT));
                    // TE/TM basis (Eqs. fresnel_in_vectors, fresnel_out_vectors)
                    f3 ep = cross(k, nrm);
                    const float len = sqrtf(dot(ep, ep));
                    if (len > 1e-6f) {
                        ep = ep * (1.0f / len);
                    } else {
                        const f3 axv = fabsf(k.x) < 0.5f ? f3{1.0f, 0.0f, 0.0f} : f3{0.0f, 1.0f, 0.0f};
                        ep = normalize(cross(k, axv));
                    }
                    const f3 epi = cross(ep, k);
                    f3 ko, epo;
                    cf cpe, cpa;
                    Diffuse D;
                    if (DIFF && dec == 2) {
                        // diffuse reflection: a new tube in a uniform direction of the
                        // incident-side hemisphere (App. A.10); set up out of line to keep
                        // the loop body small
                        if (ADJ)
                            diffuse_setup(M, k, nrm, cos1, co.rp, co.rl, ep, epi, s_tx[txi].seed, n, depth, &D, &ko);
                        else
                            diffuse_event<NPOL>(M, k, nrm, cos1, co.rp, co.rl, ep, epi, s_tx[txi].seed, n, depth, E, &ko);
                        epo = epi;
                        cpe = cpa = C(0.0f);
                    } else if (dec == 0) {
                        ko = normalize(k - nrm * (2.0f * dot(k, nrm)));
                        epo = normalize(cross(ep, ko));
                        cpe = DIFF ? co.rp * M.Rred : co.rp;
                        cpa = DIFF ? co.rl * M.Rred : co.rl;
                    } else {
                        ko = k;  // thin slab: no deflection (Sec. 2.3)
                        epo = epi;
                        cpe = co.tp; cpa = co.tl;
                    }
                    if (ADJ) {
                        // slot of this interaction's material (new slots start at zero)
                        int sm = 0;
                        while (sm < nslot && Tm[sm] != mat) ++sm;
                        if (sm == nslot) {
                            if (nslot < MAXSLOT) {
                                Tm[sm] = mat;
                                for (int p = 0; p < NPOL; ++p)
                                    for (int a = 0; a < 3; ++a) {
                                        Tg[sm][p][a] = C(0.0f);
                                        if (DIFF) Ts[sm][p][a] = C(0.0f);
                                    }
                                ++nslot;
                            } else {
                                sm = -1;
                                overflow = true;
                            }
                        }
                        if (DIFF && dec == 2) {
                            // tangents through the (non-holomorphic) diffuse map, eps and
                            // sigma directions separately; d eta = 1 resp. -j on this material
                            cf drp, drl;
                            fresnel_deta(eta, cos1, M.k0d_hi + M.k0d_lo, M.slab != 0, 0, &drp, &drl);
#pragma unroll 1
                            for (int s = 0; s < nslot; ++s) {
                                const bool own = s == sm;
                                for (int p = 0; p < NPOL; ++p) {
                                    cf t[3];
                                    diffuse_tangent(D, E[p], Tg[s][p], own ? C(1.0f) : C(0.0f), drp, drl, t);
                                    for (int a = 0; a < 3; ++a) Tg[s][p][a] = t[a];
                                    diffuse_tangent(D, E[p], Ts[s][p], own ? C(0.0f, -1.0f) : C(0.0f), drp, drl, t);
                                    for (int a = 0; a < 3; ++a) Ts[s][p][a] = t[a];
                                }
                            }
                        } else {
                            // existing tangents see the same interaction matrix
#pragma unroll 1
                            for (int s = 0; s < nslot; ++s)
                                for (int p = 0; p < NPOL; ++p) {
                                    const cf a = edot(ep, Tg[s][p]), b = edot(epi, Tg[s][p]);
                                    const cf ca = cpe * a, cb = cpa * b;
                                    Tg[s][p][0] = ca * ep.x + cb * epo.x;
                                    Tg[s][p][1] = ca * ep.y + cb * epo.y;
                                    Tg[s][p][2] = ca * ep.z + cb * epo.z;
                                    if (DIFF) {
                                        const cf as = edot(ep, Ts[s][p]), bs = edot(epi, Ts[s][p]);
                                        const cf cas = cpe * as, cbs = cpa * bs;
                                        Ts[s][p][0] = cas * ep.x + cbs * epo.x;
                                        Ts[s][p][1] = cas * ep.y + cbs * epo.y;
                                        Ts[s][p][2] = cas * ep.z + cbs * epo.z;
                                    }
                                }
                            // plus d(interaction matrix)/d eta applied to the field
                            cf dpe, dpa;
                            fresnel_deta(eta, cos1, M.k0d_hi + M.k0d_lo, M.slab != 0, dec, &dpe, &dpa);
                            if (DIFF && dec == 0) {
                                dpe = dpe * M.Rred;
                                dpa = dpa * M.Rred;
                            }
                            if (sm >= 0)
                                for (int p = 0; p < NPOL; ++p) {
                                    const cf a = edot(ep, E[p]), b = edot(epi, E[p]);
                                    const cf ca = dpe * a, cb = dpa * b;
                                    const cf v[3] = {ca * ep.x + cb * epo.x, ca * ep.y + cb * epo.y, ca * ep.z + cb * epo.z};
                                    for (int a2 = 0; a2 < 3; ++a2) {
                                        Tg[sm][p][a2] = Tg[sm][p][a2] + v[a2];
                                        if (DIFF) Ts[sm][p][a2] = Ts[sm][p][a2] + v[a2] * C(0.0f, -1.0f);
                                    }
                                }
                        }
                        if (BILIN) {
                            // hit point on the plane of the triangle: dp/do = I - k n^T / (n . k)
                            const float inv_nk = 1.0f / dot(nrm, k);
                            for (int c = 0; c < 3; ++c) {
                                const float nj = (nrm.x * J[3 * c] + nrm.y * J[3 * c + 1] + nrm.z * J[3 * c + 2]) * inv_nk;
                                J[3 * c + 0] -= k.x * nj;
                                J[3 * c + 1] -= k.y * nj;
                                J[3 * c + 2] -= k.z * nj;
                            }
                        }
                    }
                    if (DIFF && dec == 2) {
                        // (the forward updated E in diffuse_event)
                        if (ADJ) {
                            for (int p = 0; p < NPOL; ++p) {
                                cf eo[3];
                                diffuse_field(D, E[p], eo);
                                for (int a = 0; a < 3; ++a) E[p][a] = eo[a];
                            }
                        }
                    } else {
                        for (int p = 0; p < NPOL; ++p) {
                            const cf a = edot(ep, E[p]), b = edot(epi, E[p]);
                            const cf ca = cpe * a, cb = cpa * b;
                            E[p][0] = ca * ep.x + cb * epo.x;
                            E[p][1] = ca * ep.y + cb * epo.y;
                            E[p][2] = ca * ep.z + cb * epo.z;
                        }
                    }
                    // new origin: hit point pushed 2^-16 max(1, |p|_inf) off the surface
                    // (incident side for R and S, far side for T)
                    const float px = r.ox + h.t * r.kx, py = r.oy + h.t * r.ky, pz = r.oz + h.t * r.kz;
                    const float pm = fmaxf(fabsf(px), fmaxf(fabsf(py), fabsf(pz)));
                    const float delta = fmaxf(1.0f, pm) * 0x1p-16f;
                    const float sgn = dec == 1 ? -delta : delta;
                    r.ox = px + sgn * nrm.x;
                    r.oy = py + sgn * nrm.y;
                    r.oz = pz + sgn * nrm.z;
                    r.kx = ko.x; r.ky = ko.y; r.kz = ko.z;
                    prev = h.slot;
                    plen += h.t;
                    if (DIFF && dec == 2) plen = 0.0f;  // a diffuse reflection starts a new tube
                    ++depth;
                    // early termination once the path has rr_depth interactions (Sec. 4.5):
                    // threshold on (lambda0/4pi)^2 w|E|^2 / r^2, then Russian roulette with
                    // p = min(w|E|^2, p_max) (Eq. radio-map-solver-rr-prob), survivors x 1/p
                    if (A.rr_depth > 0 && depth >= A.rr_depth && (A.gain_thr > 0.0f || A.rr_pmax > 0.0f)) {
                        float w2 = 0.0f;
                        for (int p = 0; p < NPOL; ++p) w2 += cabs2(E[p][0]) + cabs2(E[p][1]) + cabs2(E[p][2]);
                        w2 *= inv_pr;
                        int kill = 0;
                        // (a tube a diffuse reflection has just spawned, plen = 0, is not thresholded)
                        if (A.gain_thr > 0.0f && plen > 0.0f && A.lam4pi2 * w2 / (plen * plen) < A.gain_thr) kill = 8;
                        if (!kill && A.rr_pmax > 0.0f) {
                            const float prr = fminf(w2, A.rr_pmax);
                            const float urr = rng_u(s_tx[txi].seed ^ RR_STREAM, n, depth - 1);
                            if (urr < prr) inv_pr = inv_pr / prr;
                            else kill = 4;
                        }
                        if (kill) {
                            active = false;
                            if (rec) rec->decision |= kill;
                        }
                    }
                }
            }
        }
    }

    // ---------------- flush counters ----------------
    if (overflow) atomicOr(&A.scratch->status, 1);
    unsigned v[6] = {c_rays, c_seg, c_nodes, c_tris, c_dep, c_esc};
    for (int j = 0; j < 6; ++j) {
        unsigned s = __reduce_add_sync(FULL_MASK, v[j]);
        if (lane == 0 && s) atomicAdd(&s_cnt[j], (unsigned long long)s);
    }
    __syncthreads();
    if (tid < 6 && s_cnt[tid]) atomicAdd(&A.scratch->cnt[tid], s_cnt[tid]);
    if (DEBUG)
        for (int i = tid; i < RM_MAX_DEPTH + 1; i += blockDim.x)
            if (s_segd[i]) atomicAdd(&A.scratch->seg_depth[i], s_segd[i]);
    if (DEBUG && stats) {
        for (int i = tid; i < RM_MAX_DEPTH + 1; i += blockDim.x) {
            atomicAdd(&A.scratch->pw[i], s_pw[i]);
            atomicAdd(&A.scratch->pw2[i], s_pw[RM_MAX_DEPTH + 1 + i]);
            atomicAdd(&A.scratch->esc[i], s_pw[2 * (RM_MAX_DEPTH + 1) + i]);
        }
    }
    if (ADJ)
        for (int i = tid; i < NGRAD; i += blockDim.x)
            if (s_grad[i] != 0.0f) atomicAdd(&A.scratch->grad[i], (double)s_grad[i]);
}

template <bool ADJ, int NPOL, bool DEBUG, bool BILIN, bool DIFF, bool MESH = false, bool HITS = false>
const void* kernel_ptr() {
    return reinterpret_cast<const void*>(&k_trace<ADJ, NPOL, DEBUG, BILIN, DIFF, MESH, HITS>);
}

template <bool ADJ, int NPOL, bool DEBUG, bool BILIN>
const void* select_diff(bool diffuse) {
    return diffuse ? kernel_ptr<ADJ, NPOL, DEBUG, BILIN, true>() : kernel_ptr<ADJ, NPOL, DEBUG, BILIN, false>();
}

const void* select_kernel(int npol, bool debug, bool bilinear, bool adjoint, bool diffuse, bool mesh, bool hits) {
    if (hits && !adjoint && !debug) {
        // the plain forward recording its closest hits (mesh surfaces: box cells only)
        if (mesh) {
            if (bilinear) return nullptr;
#define RM_SELHM(P) \
    if (npol == P) \
        return diffuse ? kernel_ptr<false, P, false, false, true, true, true>() \
                       : kernel_ptr<false, P, false, false, false, true, true>();
            RM_SELHM(1) RM_SELHM(2)
#undef RM_SELHM
            return nullptr;
        }
#define RM_SELH(P, B) \
    if (npol == P && bilinear == B) \
        return diffuse ? kernel_ptr<false, P, false, B, true, false, true>() \
                       : kernel_ptr<false, P, false, B, false, false, true>();
        RM_SELH(1, false) RM_SELH(1, true) RM_SELH(2, false) RM_SELH(2, true)
#undef RM_SELH
        return nullptr;
    }
    if (mesh) {
        // mesh surfaces: box cells only
        if (bilinear) return nullptr;
#define RM_SELM(A, P, D) \
    if (adjoint == A && npol == P && debug == D) \
        return diffuse ? kernel_ptr<A, P, D, false, true, true>() : kernel_ptr<A, P, D, false, false, true>();
        RM_SELM(false, 1, false) RM_SELM(false, 1, true) RM_SELM(false, 2, false) RM_SELM(false, 2, true)
        RM_SELM(true, 1, false) RM_SELM(true, 1, true) RM_SELM(true, 2, false) RM_SELM(true, 2, true)
#undef RM_SELM
        return nullptr;
    }
#define RM_SEL(A, P, D, B) \
    if (adjoint == A && npol == P && debug == D && bilinear == B) return select_diff<A, P, D, B>(diffuse);
    RM_SEL(false, 1, false, false) RM_SEL(false, 1, false, true) RM_SEL(false, 1, true, false)
    RM_SEL(false, 1, true, true) RM_SEL(false, 2, false, false) RM_SEL(false, 2, false, true)
    RM_SEL(false, 2, true, false) RM_SEL(false, 2, true, true) RM_SEL(true, 1, false, false)
    RM_SEL(true, 1, false, true) RM_SEL(true, 1, true, false) RM_SEL(true, 1, true, true)
    RM_SEL(true, 2, false, false) RM_SEL(true, 2, false, true) RM_SEL(true, 2, true, false)
    RM_SEL(true, 2, true, true)
#undef RM_SEL
    return nullptr;
}

// The sampling weights of one material at given cosines of incidence, from
// the tracer's own fresnel() (same translation unit, same rounding): wR =
// |r_perp|^2 + |r_par|^2 and wT = |t_perp|^2 + |t_par|^2, whose ratio the
// coin of every interaction compares with its variate.
__global__ void k_fresnel_probe(const MatDev M, const float* __restrict__ cos1, long long n, float* wR,
                                float* wT) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Coef co = fresnel(C(M.eta_re, M.eta_im), cos1[i], M.k0d_hi, M.k0d_lo, M.slab != 0, nullptr);
        wR[i] = cabs2(co.rp) + cabs2(co.rl);
        wT[i] = cabs2(co.tp) + cabs2(co.tl);
    }
}

}  // namespace

cudaError_t launch_fresnel_probe(const MatDev& m, const float* cos1, long long n, float* wR, float* wT,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 148LL * 8);
    k_fresnel_probe<<<(unsigned)blocks, 256, 0, s>>>(m, cos1, n, wR, wT);
    return cudaGetLastError();
}

cudaError_t launch_alpha(const TraceArgs& a, float2* alpha, cudaStream_t s, bool wide) {
    if (a.total == 0) return cudaSuccess;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t err;
    const void* k = wide ? reinterpret_cast<const void*>(&k_alpha<true>) : reinterpret_cast<const void*>(&k_alpha<false>);
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, 0)) != cudaSuccess) return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const unsigned long long need = (a.total + 255) / 256, cap = (unsigned long long)occ * sms;
    void* args[] = {const_cast<TraceArgs*>(&a), &alpha};
    return cudaLaunchKernel(k, dim3((unsigned)(need < cap ? need : cap)), dim3(256), args, 0, s);
}

int max_blocks_per_sm(int npol, bool debug, bool bilinear, bool adjoint, bool diffuse, int block, bool mesh,
                      bool hits) {
    const void* k = select_kernel(npol, debug, bilinear, adjoint, diffuse, mesh, hits);
    int nb = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, 0) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_trace(const TraceArgs& a, int npol, bool debug, bool bilinear, bool adjoint, bool diffuse,
                         int block, int blocks_per_sm, cudaStream_t s, int* grid_out, bool mesh, bool hits) {
    const void* k = select_kernel(npol, debug, bilinear, adjoint, diffuse, mesh, hits);
    if (!k) return cudaErrorInvalidValue;
    if (block <= 0 || block > MAX_BLOCK || (block & 31)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t err;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, 0)) != cudaSuccess) return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int bps = (blocks_per_sm > 0 && blocks_per_sm < occ) ? blocks_per_sm : occ;
    const int grid = bps * sms;
    if (grid_out) *grid_out = grid;
    void* args[] = {const_cast<TraceArgs*>(&a)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, 0, s);
}

}  // namespace rmsbr
