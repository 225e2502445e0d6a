// First-order diffraction radio map on sm_103a (Sec. 4, "Computation of
// Radio Map due to Diffraction"; UTD of App. A.8; weighting factor of the
// appendix on diffraction radio maps).
//
// One thread per sample (x, phi) of a wedge, in a grid-stride loop over
// (transmitter, wedge, sample); consecutive threads take neighbouring lattice
// samples of one wedge.  Per sample:
//   1. diffraction point v = o + x e and Keller-cone direction k_s;
//   2. crossing of the measurement plane and its cell;
//   3. two any-hit visibility queries through the LBVH (source -> v and
//      v -> plane, the wedge's own faces excluded);
//   4. the UTD field (Eq. diffracted-field) of the antenna field in the
//      direction of v, for one or two polarisation columns;
//   5. the weighting factor |dt/dx x dt/dphi|, derived by hand;
//   6. an FP64 atomic deposit.
// This file is compiled with -fmad=false like the tracer.
#include <cmath>

#include "common.cuh"
#include "array.cuh"
#include "vec.cuh"

namespace rmsbr {
namespace {

constexpr float PI_F = 3.14159265358979323846f;

// ------------------------------------------------------------------ UTD transition function
// w(z), Im z >= 0, by Weideman's rational expansion in Z = (L + iz)/(L - iz)
// (SIAM J. Numer. Anal. 31, 1994).
__device__ __forceinline__ cf faddeeva(cf z, const DiffArgs& A) {
    const cf iz = C(-z.i, z.r);
    const cf lp = C(A.wz_L + iz.r, iz.i), lm = C(A.wz_L - iz.r, -iz.i);
    const cf Z = cdiv(lp, lm);
    cf p = C(A.wz_a[FADDEEVA_N - 1]);
    for (int k = FADDEEVA_N - 2; k >= 0; --k) p = p * Z + C(A.wz_a[k]);
    const cf il = cdiv(C(1.0f), lm);
    return p * il * il * 2.0f + il * 0.56418958354775628f;
}
// F(x) = 2 j sqrt(x) e^{jx} int_{sqrt x}^inf e^{-j t^2} dt = sqrt(pi x) e^{j pi/4} w(sqrt(x/2)(-1 + j))
__device__ __forceinline__ cf utd_F(float x, const DiffArgs& A) {
    if (!(x > 0.0f)) return C(0.0f);
    const float r = sqrtf(0.5f * x);
    const cf w = faddeeva(C(-r, r), A);
    const float m = sqrtf(PI_F * x) * 0.70710678118654752f;
    return w * C(m, m);
}

// ------------------------------------------------------------------ any-hit visibility
// Is the open segment o + t d, t in (tmin, tmax), blocked by a triangle other
// than the original triangles ex0, ex1?  Moeller-Trumbore per triangle,
// stack traversal without ordering, early exit on the first blocker.  The
// plane kernel inlines it at its one call site; the mesh kernel calls it
// (inlined at its two sites it spills).
__device__ __forceinline__ bool tri_blocks(const float4* __restrict__ tris, int slot, f3 o, f3 d, float tmin,
                                           float tmax, int ex0, int ex1, unsigned& c_tris) {
    const float4* tp = tris + 3 * (size_t)slot;
    const float4 r2 = __ldg(tp + 2);
    const int prim = __float_as_int(r2.z);
    if (prim == ex0 || prim == ex1) return false;
    ++c_tris;
    const float4 r0 = __ldg(tp), r1 = __ldg(tp + 1);
    const f3 a{r0.x, r0.y, r0.z}, b{r0.w, r1.x, r1.y}, c{r1.z, r1.w, r2.x};
    const f3 e1 = b - a, e2 = c - a;
    const f3 p = cross(d, e2);
    const float det = dot(e1, p);
    if (det == 0.0f) return false;
    const float inv = 1.0f / det;
    const f3 tv = o - a;
    const float u = dot(tv, p) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    const f3 q = cross(tv, e1);
    const float v = dot(d, q) * inv;
    if (v < 0.0f || u + v > 1.0f) return false;
    const float t = dot(e2, q) * inv;
    return t > tmin && t < tmax;
}

__device__ __forceinline__ bool segment_blocked_inl(const DiffArgs& A, f3 o, f3 d, float tmin, float tmax, int ex0,
                                                   int ex1, unsigned& c_nodes, unsigned& c_tris, bool& overflow) {
    for (int j = 0; j < A.nlarge; ++j)
        if (tri_blocks(A.tris, A.nt + j, o, d, tmin, tmax, ex0, ex1, c_tris)) return true;
    if (A.nt <= 0) return false;
    if (A.nt == 1) return tri_blocks(A.tris, 0, o, d, tmin, tmax, ex0, ex1, c_tris);
    const float ooeps = 0x1p-80f;
    // correctly rounded reciprocals: the slab test's widening assumes one rounding
    const float ix = __frcp_rn(fabsf(d.x) > ooeps ? d.x : copysignf(ooeps, d.x));
    const float iy = __frcp_rn(fabsf(d.y) > ooeps ? d.y : copysignf(ooeps, d.y));
    const float iz = __frcp_rn(fabsf(d.z) > ooeps ? d.z : copysignf(ooeps, d.z));
    auto box = [&](float lx, float ly, float lz, float hx, float hy, float hz) {
        const float t0x = (lx - o.x) * ix, t1x = (hx - o.x) * ix;
        const float t0y = (ly - o.y) * iy, t1y = (hy - o.y) * iy;
        const float t0z = (lz - o.z) * iz, t1z = (hz - o.z) * iz;
        const float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), tmin));
        const float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), tmax)) * 1.0000004f;
        return tn <= tf;
    };
    int stack[STACK_SIZE];
    int sp = 0, cur = 0;
    int budget = 2 * A.nt + 8;   // nt <= INT32_MAX / 4 (checked at upload): no overflow
    while (true) {
        if (--budget < 0) {
            overflow = true;
            return false;
        }
        ++c_nodes;
        const float4* nd = A.nodes + 4 * (size_t)cur;
        const float4 n0 = __ldg(nd), n1 = __ldg(nd + 1), n2 = __ldg(nd + 2), n3 = __ldg(nd + 3);
        bool h0 = box(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
        bool h1 = box(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
        const int c0 = __float_as_int(n3.x), c1 = __float_as_int(n3.y);
        if (h0 && c0 < 0) {
            if (tri_blocks(A.tris, ~c0, o, d, tmin, tmax, ex0, ex1, c_tris)) return true;
            h0 = false;
        }
        if (h1 && c1 < 0) {
            if (tri_blocks(A.tris, ~c1, o, d, tmin, tmax, ex0, ex1, c_tris)) return true;
            h1 = false;
        }
        if (h0 && h1) {
            if (sp < STACK_SIZE) stack[sp++] = c1;
            else overflow = true;
            cur = c0;
        } else if (h0) {
            cur = c0;
        } else if (h1) {
            cur = c1;
        } else {
            if (sp == 0) return false;
            cur = stack[--sp];
        }
    }
}

__device__ __noinline__ bool segment_blocked(const DiffArgs& A, f3 o, f3 d, float tmin, float tmax, int ex0, int ex1,
                                             unsigned& c_nodes, unsigned& c_tris, bool& overflow) {
    return segment_blocked_inl(A, o, d, tmin, tmax, ex0, ex1, c_nodes, c_tris, overflow);
}

// ------------------------------------------------------------------ antenna field
// R (C_theta theta' + C_phi phi') in direction k (App. A.1) times the
// synthetic-array factor alpha = sum_k u_P,k exp(j k0 k.d_k) (Sec. 4.4).
__device__ void antenna_field(const TxDev& T, const AntDev* __restrict__ ant, f3 k, int pol, cf* E) {
    const float lx = T.R[0] * k.x + T.R[3] * k.y + T.R[6] * k.z;
    const float ly = T.R[1] * k.x + T.R[4] * k.y + T.R[7] * k.z;
    const float lz = T.R[2] * k.x + T.R[5] * k.y + T.R[8] * k.z;
    const float sxy = sqrtf(lx * lx + ly * ly);
    float cph = 1.0f, sph = 0.0f;
    if (sxy > 0.0f) {
        cph = lx / sxy;
        sph = ly / sxy;
    }
    const float g = (T.pattern == 1) ? 1.2247448713915890f * sxy : 1.0f;
    const f3 e = pol == 0 ? f3{lz * cph, lz * sph, -sxy} : f3{-sph, cph, 0.0f};
    float are = 1.0f, aim = 0.0f;
    if (T.n_ant > 0) array_factor_dir(T, ant, k.x, k.y, k.z, are, aim);
    const float ex = g * (T.R[0] * e.x + T.R[1] * e.y + T.R[2] * e.z);
    const float ey = g * (T.R[3] * e.x + T.R[4] * e.y + T.R[5] * e.z);
    const float ez = g * (T.R[6] * e.x + T.R[7] * e.y + T.R[8] * e.z);
    E[0] = C(ex * are, ex * aim);
    E[1] = C(ey * are, ey * aim);
    E[2] = C(ez * are, ez * aim);
}

// ------------------------------------------------------------------ UTD field
struct Mat2 {
    cf m[2][2];
};
__device__ __forceinline__ f3 unit3(f3 a) { return a * (1.0f / sqrtf(dot(a, a))); }

// Face matrix W(phi_SB, beta_SB, e_r,perp, e_r,par) diag(r_perp, r_par)
// W(e_i,perp, e_i,par, phi', beta0') with the half-space coefficients of
// Eq. fresnel_vac at cos theta = |n . s'|.
__device__ Mat2 face_matrix(f3 nf, cf eta, f3 si, f3 e, f3 phi_i, f3 beta_i) {
    const float cr = fminf(1.0f, fabsf(dot(nf, si)));
    const float sin2 = (1.0f - cr) * (1.0f + cr);
    const cf s = csqrt_p(C(eta.r - sin2, eta.i));
    const cf c = C(cr);
    const cf ec = eta * cr;
    const cf rp = cdiv(c - s, c + s), rl = cdiv(ec - s, ec + s);
    const f3 sSB = si - nf * (2.0f * dot(si, nf));
    f3 eip = cross(si, nf);
    const float len = sqrtf(dot(eip, eip));
    if (len > 1e-6f) {
        eip = eip * (1.0f / len);
    } else {
        const f3 ax = fabsf(si.x) < 0.5f ? f3{1.0f, 0.0f, 0.0f} : f3{0.0f, 1.0f, 0.0f};
        eip = unit3(cross(si, ax));
    }
    const f3 eil = cross(eip, si);
    const f3 erl = cross(eip, sSB);
    const f3 phSB = unit3(cross(sSB, e)) * -1.0f;
    const f3 beSB = cross(phSB, sSB);
    const float wo[2][2] = {{dot(phSB, eip), dot(phSB, erl)}, {dot(beSB, eip), dot(beSB, erl)}};
    const float wi[2][2] = {{dot(eip, phi_i), dot(eip, beta_i)}, {dot(eil, phi_i), dot(eil, beta_i)}};
    Mat2 M;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) M.m[a][b] = rp * (wo[a][0] * wi[0][b]) + rl * (wo[a][1] * wi[1][b]);
    return M;
}

// One term pre cot((pi + pm beta)/(2n)) F(k L a^pm(beta)), a^pm(beta) = 2 cos^2((2 n pi N - beta)/2),
// N = round((beta + pm pi)/(2 n pi)).  With u = pi + pm beta, K = round(u / (2 n pi)) and
// d = u - 2 n pi K (so N = pm K): cot(u / 2n) = cot(d / 2n) and, exactly,
// a^pm = 2 cos^2(pm (pi - d) / 2) = 2 sin^2(d / 2).  Both factors take the same d
// (the distance to the nearest shadow boundary, reduced with a two-part 2 n pi),
// so near a boundary, where the cotangent grows like 1/d and F like d, their
// product keeps FP32 accuracy.  0 at an exact shadow boundary.
__device__ __forceinline__ cf utd_term(float beta, float pm, float n, float kL, cf pre, const DiffArgs& A) {
    const float u = PI_F + pm * beta;
    const float twon_pi = 2.0f * n * PI_F;
    const float K = roundf(u / twon_pi);
    // 2 n pi = hi + lo with hi on 12 significant bits, so that K * hi is exact for |K| < 2^12
    const float hi = __uint_as_float(__float_as_uint(twon_pi) & 0xfffff000u);
    const float lo = (float)(2.0 * (double)n * 3.14159265358979323846 - (double)hi);
    const float d = (u - K * hi) - K * lo;
    float sd, cd;
    sincosf(d / (2.0f * n), &sd, &cd);
    if (sd == 0.0f) return C(0.0f);
    const float sh = sinf(0.5f * d);
    return pre * (cd / sd) * utd_F(kL * 2.0f * sh * sh, A);
}

// |E_d|^2 of one sample at observation distance sobs (Eq. diffracted-field,
// summed over the antenna's field columns): the UTD coefficients D_1..D_4
// through one rolled call site, the face matrices R_0 and (when the n-face is
// lit) R_n through another.
__device__ __forceinline__ float diffracted_power(const DiffArgs& A, const TxDev& T, f3 s, f3 v, f3 e, f3 n0, f3 nn,
                                                  f3 t0, int m0, int mn, float nw_, float phi, float sb, f3 si,
                                                  float dn, float sobs) {
    const f3 sr = s - v;
    const f3 srt = sr - e * dot(sr, e);
    float phip = atan2f(dot(srt, n0), dot(srt, t0));
    if (phip < 0.0f) phip += 2.0f * PI_F;
    const float L = sobs * dn / (sobs + dn) * sb * sb;
    const float kL = A.k0 * L;
    const float pm = 1.0f / (2.0f * nw_ * sqrtf(2.0f * PI_F * A.k0) * sb);
    const cf pre = C(-0.70710678118654752f * pm, 0.70710678118654752f * pm);  // -e^{-j pi/4} pm
    // D_1..D_4 through one rolled call site (beta = phi -+ phi', pm = +-1)
    cf Dq[4];
#pragma unroll 1
    for (int q = 0; q < 4; ++q)
        Dq[q] = utd_term(q < 2 ? phi - phip : phi + phip, (q & 1) ? -1.0f : 1.0f, nw_, kL, pre, A);
    const f3 phi_i = unit3(cross(si, e));
    const f3 beta_i = cross(phi_i, si);
    // R_0 and (when the n-face is lit) R_n through one call site
    const bool n_lit = (nw_ - 1.0f) * PI_F <= phip;
    Mat2 Rf[2];
#pragma unroll 1
    for (int q = 0; q < (n_lit ? 2 : 1); ++q) {
        const MatDev& Mq = A.mats[q ? mn : m0];
        Rf[q] = face_matrix(q ? nn : n0, C(Mq.eta_re, Mq.eta_im), si, e, phi_i, beta_i);
    }
    const Mat2& R0 = Rf[0];
    Mat2 Rn;
    if (n_lit) {
        Rn = Rf[1];
    } else {
        Rn.m[0][0] = Rn.m[1][1] = C(-1.0f);
        Rn.m[0][1] = Rn.m[1][0] = C(0.0f);
    }
    const cf a0 = Dq[3] - Dq[0], an = Dq[2] - Dq[1];
    float pw = 0.0f;
    for (int p = 0; p < A.npol; ++p) {
        cf E[3];
        antenna_field(T, A.ant, si, A.npol == 2 ? p : T.pol, E);
        const cf ein[2] = {edot(phi_i, E), edot(beta_i, E)};
        for (int r = 0; r < 2; ++r) {
            cf acc = C(0.0f);
            for (int c = 0; c < 2; ++c) acc = acc + (a0 * R0.m[r][c] + an * Rn.m[r][c]) * ein[c];
            pw += cabs2(acc);
        }
    }
    // (the minus sign of Eq. diffracted-field does not change |E_d|^2)
    return pw;
}

// Crossings t > 1e-9 of the ray v + t k with a mesh measurement surface, up to
// MAX_CROSS of them (more set *xlimit; a traversal overflow sets *overflow):
// distance, triangle, and the unnormalised normal (b - a) x (c - a), whose
// length is twice the area.
constexpr int MAX_CROSS = 8;
struct Crossing {
    float t;
    int tri;
    f3 nrm;
};
__device__ __noinline__ int surface_hits(const float4* __restrict__ nodes, const float4* __restrict__ tris, int nt,
                                         int nlarge, f3 o, f3 k, Crossing* out, bool* overflow, bool* xlimit) {
    int nh = 0;
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
        const float uu = dot(tv, pv) * inv;
        if (uu < 0.0f || uu > 1.0f) return;
        const f3 q = cross(tv, e1);
        const float vv = dot(k, q) * inv;
        if (vv < 0.0f || uu + vv > 1.0f) return;
        const float t = dot(e2, q) * inv;
        if (!(t > 1e-9f)) return;
        if (nh < MAX_CROSS) out[nh++] = Crossing{t, __float_as_int(r2.z), cross(e1, e2)};
        else *xlimit = true;
    };
#pragma unroll 1
    for (int j = 0; j < nlarge; ++j) leaf(nt + j);
    if (nt == 1) leaf(0);
    if (nt < 2) return nh;
    const float ooeps = 0x1p-80f;
    const float ix = __frcp_rn(fabsf(k.x) > ooeps ? k.x : copysignf(ooeps, k.x));
    const float iy = __frcp_rn(fabsf(k.y) > ooeps ? k.y : copysignf(ooeps, k.y));
    const float iz = __frcp_rn(fabsf(k.z) > ooeps ? k.z : copysignf(ooeps, k.z));
    auto box = [&](float lx, float ly, float lz, float hx, float hy, float hz) {
        const float t0x = (lx - o.x) * ix, t1x = (hx - o.x) * ix;
        const float t0y = (ly - o.y) * iy, t1y = (hy - o.y) * iy;
        const float t0z = (lz - o.z) * iz, t1z = (hz - o.z) * iz;
        const float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), 0.0f));
        const float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fmaxf(t0z, t1z)) * 1.0000004f;
        return tn <= tf;
    };
    int stack[STACK_SIZE];
    int sp = 0, cur = 0;
    int budget = 2 * nt + 8;   // nt <= INT32_MAX / 4 (checked at upload): no overflow
    while (true) {
        if (--budget < 0) {
            *overflow = true;
            return nh;
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
            if (sp == 0) return nh;
            cur = stack[--sp];
        }
    }
}

// ------------------------------------------------------------------ sample geometry
// Sample w of the (transmitter, wedge, sample) sequence: the wedge turned so
// that the source lies in front of its 0-face (the UTD assumes phi' <= pi;
// otherwise the faces swap, and a source behind both faces gives code -2),
// the lattice sample x = L (i + 1/2)/N, phi = n pi frac(i (phi_g - 1)) (24-bit
// fixed point), the diffraction point v, the Keller-cone direction ks and
// the crossing of the measurement plane with its cell.
struct DSample {
    int txi, m0, mn, tri0, trin;
    int code;            // -2: source behind both faces; -1: lit
    f3 s, o, e, n0, nn, t0, v, d, u, ks;
    float wlen, wn, u2, sp, cp, dn, cb, sb;
    bool dep;            // the diffracted ray crosses the plane inside the map
    float tc, fx, fy;
    int cxi, cyi;
};

__device__ __forceinline__ void diff_sample(const DiffArgs& A, unsigned long long w, DSample& G) {
    const unsigned long long per_tx = (unsigned long long)A.nw * A.ns;
    G.txi = (int)(w / per_tx);
    const unsigned long long rem = w - (unsigned long long)G.txi * per_tx;
    const long long wi = (long long)(rem / A.ns);
    const unsigned long long i = rem - (unsigned long long)wi * A.ns;
    const TxDev& T = A.tx[G.txi];
    const rm_wedge W = A.wedges[wi];
    G.s = f3{T.pos[0], T.pos[1], T.pos[2]};
    G.o = f3{W.origin[0], W.origin[1], W.origin[2]};
    G.e = f3{W.edge[0], W.edge[1], W.edge[2]};
    G.n0 = f3{W.n0[0], W.n0[1], W.n0[2]};
    G.nn = f3{W.nn[0], W.nn[1], W.nn[2]};
    G.m0 = W.mat0;
    G.mn = W.matn;
    G.tri0 = W.tri0;
    G.trin = W.trin;
    G.wlen = W.length;
    G.wn = W.n;
    if (dot(G.s - G.o, G.n0) < 0.0f) {
        G.o = G.o + G.e * W.length;
        G.e = G.e * -1.0f;
        const f3 t = G.n0;
        G.n0 = G.nn;
        G.nn = t;
        const int tm = G.m0;
        G.m0 = G.mn;
        G.mn = tm;
    }
    G.code = -2;
    G.dep = false;
    G.cxi = G.cyi = NO_CELL;
    G.tc = G.fx = G.fy = 0.0f;
    if (!(dot(G.s - G.o, G.n0) >= 0.0f)) return;
    G.code = -1;
    G.t0 = cross(G.n0, G.e);
    const float u1 = A.ns < (1ULL << 24) ? ((float)i + 0.5f) / (float)A.ns : (float)(((double)i + 0.5) / (double)A.ns);
    const unsigned long long fr = i * 0x9E3779B97F4A7C16ULL;
    G.u2 = (float)(unsigned)(fr >> 40) * 0x1p-24f;
    const float x = u1 * W.length;
    sincospif(G.u2 * W.n, &G.sp, &G.cp);
    G.v = G.o + G.e * x;
    G.d = G.v - G.s;
    G.dn = sqrtf(dot(G.d, G.d));
    const f3 so = G.s - G.o;
    const f3 perp = so - G.e * dot(so, G.e);
    const float rho = sqrtf(dot(perp, perp));
    G.cb = dot(G.d, G.e) / G.dn;
    G.sb = rho / G.dn;
    G.u = f3{G.cp * G.t0.x + G.sp * G.n0.x, G.cp * G.t0.y + G.sp * G.n0.y, G.cp * G.t0.z + G.sp * G.n0.z};
    G.ks = G.u * G.sb + G.e * G.cb;
    {
        // plane crossing and cell (as the tracer's deposit)
        const float tc = (A.zm - G.v.z) / G.ks.z;
        if (G.ks.z != 0.0f && tc > 1e-9f) {
            const float px = G.v.x + tc * G.ks.x, py = G.v.y + tc * G.ks.y;
            float ux = (px - A.x0) * A.inv_cell, uy = (py - A.y0) * A.inv_cell;
            if (A.bilinear) {
                ux -= 0.5f;
                uy -= 0.5f;
                if (ux >= -1.0f && ux < (float)A.nx && uy >= -1.0f && uy < (float)A.ny) {
                    const float flx = floorf(ux), fly = floorf(uy);
                    G.cxi = (int)flx;
                    G.cyi = (int)fly;
                    G.fx = ux - flx;
                    G.fy = uy - fly;
                    G.dep = true;
                }
            } else if (ux >= 0.0f && ux < (float)A.nx && uy >= 0.0f && uy < (float)A.ny) {
                G.cxi = (int)ux;
                G.cyi = (int)uy;
                G.dep = true;
            }
            G.tc = tc;
        }
    }
}

__device__ __forceinline__ void put_record(const DiffArgs& A, unsigned long long w, int code, int ix, int iy) {
    if (!A.record) return;
    rm_segment_record* rec = A.record + w;
    rec->prim = code;
    rec->ix = code == -2 ? NO_CELL : ix;
    rec->iy = code == -2 ? NO_CELL : iy;
    rec->decision = 0;
}

// The two visibility queries of a sample that reaches the plane (source -> v,
// v -> plane, the wedge's own faces excluded) through one rolled call site:
// 0 visible, bit 0 incident segment blocked, bit 1 diffracted segment blocked.
__device__ __forceinline__ int plane_visibility(const DiffArgs& A, const DSample& G, unsigned& c_nodes,
                                                unsigned& c_tris, bool& overflow) {
    const float vm = fmaxf(fabsf(G.v.x), fmaxf(fabsf(G.v.y), fabsf(G.v.z)));
    const float eps = fmaxf(1.0f, vm) * 0x1p-16f;
    const f3 si = G.d * (1.0f / G.dn);
    int code = 0;
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {
        const bool blk = segment_blocked_inl(A, q ? G.v : G.s, q ? G.ks : si, eps, q ? G.tc : G.dn - eps, G.tri0,
                                             G.trin, c_nodes, c_tris, overflow);
        if (blk) code |= 1 << q;
    }
    return code;
}

// The deposit of a visible sample: weighting factor |dt/dx x dt/dphi|
// (hand-derived), UTD field (Eq. diffracted-field) and FP64 atomics.
__device__ __forceinline__ void plane_deposit(const DiffArgs& A, const DSample& G) {
    // with a = (v - s).e, d cb/dx = sb^2/dn, d sb/dx = -sb cb/dn, so
    // dk/dx = (sb/dn)(sb e - cb u), dk/dphi = sb (-sin phi t0 + cos phi n0),
    // dtc/dq = -(dv_z/dq + tc dk_z/dq)/k_z, dt/dq = dv/dq + dtc/dq k + tc dk/dq.
    const float sb = G.sb, cb = G.cb, tc = G.tc;
    const f3 e = G.e, ks = G.ks;
    const f3 dkx = (e * sb - G.u * cb) * (sb / G.dn);
    const f3 dkp{sb * (G.cp * G.n0.x - G.sp * G.t0.x), sb * (G.cp * G.n0.y - G.sp * G.t0.y),
                 sb * (G.cp * G.n0.z - G.sp * G.t0.z)};
    const float dtcx = -(e.z + tc * dkx.z) / ks.z;
    const float dtcp = -(tc * dkp.z) / ks.z;
    const float txx = e.x + dtcx * ks.x + tc * dkx.x, txy = e.y + dtcx * ks.y + tc * dkx.y;
    const float tpx = dtcp * ks.x + tc * dkp.x, tpy = dtcp * ks.y + tc * dkp.y;
    const float J = fabsf(txx * tpy - txy * tpx);
    // UTD: angles from the 0-face, phi of the sample
    const float phi = G.u2 * G.wn * PI_F;
    const float sobs = tc;
    const f3 si = G.d * (1.0f / G.dn);
    const float pw = diffracted_power(A, A.tx[G.txi], G.s, G.v, e, G.n0, G.nn, G.t0, G.m0, G.mn, G.wn, phi, sb, si,
                                      G.dn, sobs);
    const float spread = 1.0f / (G.dn * sobs * (G.dn + sobs));
    const float value = A.lam4pi2_over_cell2 * (G.wlen * G.wn * PI_F / (float)A.ns) * J * pw * spread;
    const unsigned long long mb = (unsigned long long)G.txi * A.ncell;
    if (A.bilinear) {
        for (int cn = 0; cn < 4; ++cn) {
            const int a = cn & 1, b = cn >> 1;
            const int xx = G.cxi + a, yy = G.cyi + b;
            if (xx < 0 || xx >= A.nx || yy < 0 || yy >= A.ny) continue;
            const float wgt = (a ? G.fx : 1.0f - G.fx) * (b ? G.fy : 1.0f - G.fy);
            atomicAdd(A.maps64 + mb + (unsigned long long)yy * A.nx + xx, (double)(value * wgt));
        }
    } else {
        atomicAdd(A.maps64 + mb + (unsigned long long)G.cyi * A.nx + G.cxi, (double)value);
    }
}

__device__ __forceinline__ void flush_counters(const DiffArgs& A, unsigned long long* s_cnt, const unsigned (&v)[6],
                                               bool overflow, bool xlimit) {
    if (overflow) atomicOr(&A.scratch->status, 1);
    if (xlimit) atomicOr(&A.scratch->status, 2);
    for (int j = 0; j < 6; ++j) {
        const unsigned sum = __reduce_add_sync(0xffffffffu, v[j]);
        if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&s_cnt[j], (unsigned long long)sum);
    }
    __syncthreads();
    if (threadIdx.x < 6 && s_cnt[threadIdx.x]) atomicAdd(&A.scratch->cnt[threadIdx.x], s_cnt[threadIdx.x]);
}

// ------------------------------------------------------------------ kernel: measurement plane
// Most samples end early (their diffracted ray leaves upwards or outside the
// map, or the source is behind both faces), so one sample per thread would
// run the visibility queries and the UTD field with a few lanes of a warp.
// Instead each warp works in three stages with two queues of sample indices
// in shared memory: it classifies 32 samples at a time and queues those that
// reach the map; once 32 are queued it runs their visibility queries together
// and queues the visible ones; once 32 of those are queued it evaluates their
// field and deposits them.  Every stage recomputes the sample's geometry from
// its index (the same arithmetic, so the same cell).  Warps take their
// samples 128 at a time from a queue head in the scratch block; the queue
// lengths and the head are warp-uniform, and every pass of the loop either
// consumes queued samples or takes new ones, so the loop ends after
// O(samples / 32) passes.
constexpr int DQ_CAP = 64;                     // per warp and stage; never holds more than 63
constexpr unsigned long long DQ_CHUNK = 128;   // samples per queue-head access

__global__ void __launch_bounds__(256) k_diffraction_plane(const DiffArgs A) {
    __shared__ unsigned long long s_cnt[6];
    __shared__ unsigned long long s_q[2][256 / 32][DQ_CAP];
    if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long* qa = s_q[0][wid];   // samples that reach the map
    unsigned long long* qb = s_q[1][wid];   // ... and are visible from the source and the plane
    unsigned c_rays = 0, c_seg = 0, c_nodes = 0, c_tris = 0, c_dep = 0;
    bool overflow = false;
    int na = 0, nb = 0;
    bool done = false;
    unsigned long long base = 0, end = 0;
    while (true) {
        if (nb >= 32 || (done && na == 0 && nb > 0)) {
            // stage 3: field and deposit of up to 32 visible samples
            const int take = nb < 32 ? nb : 32;
            if (lane < take) {
                const unsigned long long w = qb[nb - take + lane];
                DSample G;
                diff_sample(A, w, G);
                plane_deposit(A, G);
                ++c_dep;
                put_record(A, w, 0, G.cxi, G.cyi);
            }
            __syncwarp();
            nb -= take;
        } else if (na >= 32 || (done && na > 0)) {
            // stage 2: visibility queries of up to 32 samples that reach the map
            const int take = na < 32 ? na : 32;
            unsigned long long w = 0;
            bool vis = false;
            if (lane < take) {
                w = qa[na - take + lane];
                DSample G;
                diff_sample(A, w, G);
                ++c_seg;
                const int code = plane_visibility(A, G, c_nodes, c_tris, overflow);
                if (code == 0) vis = true;
                else put_record(A, w, code, G.cxi, G.cyi);
            }
            __syncwarp();
            na -= take;
            const unsigned m = __ballot_sync(0xffffffffu, vis);
            if (vis) qb[nb + __popc(m & lt)] = w;
            nb += __popc(m);
            __syncwarp();
        } else if (!done) {
            // stage 1: take and classify the next 32 samples
            if (base >= end) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(&A.scratch->next, DQ_CHUNK);
                b = __shfl_sync(0xffffffffu, b, 0);
                if (b >= A.total) {
                    done = true;
                    continue;
                }
                base = b;
                end = b + DQ_CHUNK < A.total ? b + DQ_CHUNK : A.total;
            }
            const unsigned long long w = base + lane;
            bool dep = false;
            if (w < end) {
                ++c_rays;
                DSample G;
                diff_sample(A, w, G);
                dep = G.dep;
                if (!dep) put_record(A, w, G.code, NO_CELL, NO_CELL);
            }
            base += 32;
            const unsigned m = __ballot_sync(0xffffffffu, dep);
            if (dep) qa[na + __popc(m & lt)] = w;
            na += __popc(m);
            __syncwarp();
        } else {
            break;
        }
    }
    const unsigned v[6] = {c_rays, c_seg, c_nodes, c_tris, c_dep, 0u};
    flush_counters(A, s_cnt, v, overflow, false);
}

// ------------------------------------------------------------------ kernel: mesh measurement surface
// One thread per sample in a grid-stride loop over (transmitter, wedge,
// sample): the incident segment once, then every crossing of the diffracted
// ray with the surface, each with its own visibility, weighting factor on the
// triangle's plane, UTD field at its distance and 1/A.
__global__ void __launch_bounds__(256) k_diffraction_mesh(const DiffArgs A) {
    __shared__ unsigned long long s_cnt[6];
    if (threadIdx.x < 6) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    unsigned c_rays = 0, c_seg = 0, c_nodes = 0, c_tris = 0, c_dep = 0;
    bool overflow = false, xlimit = false;
    const unsigned long long per_tx = (unsigned long long)A.nw * A.ns;
    for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w < A.total;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const int txi = (int)(w / per_tx);
        const unsigned long long rem = w - (unsigned long long)txi * per_tx;
        const long long wi = (long long)(rem / A.ns);
        const unsigned long long i = rem - (unsigned long long)wi * A.ns;
        ++c_rays;
        const TxDev& T = A.tx[txi];
        const rm_wedge W = A.wedges[wi];
        const f3 s{T.pos[0], T.pos[1], T.pos[2]};
        // orientation: the source in front of the 0-face (phi' <= pi), else the faces swap
        f3 o{W.origin[0], W.origin[1], W.origin[2]}, e{W.edge[0], W.edge[1], W.edge[2]};
        f3 n0{W.n0[0], W.n0[1], W.n0[2]}, nn{W.nn[0], W.nn[1], W.nn[2]};
        int m0 = W.mat0, mn = W.matn;
        if (dot(s - o, n0) < 0.0f) {
            o = o + e * W.length;
            e = e * -1.0f;
            const f3 t = n0;
            n0 = nn;
            nn = t;
            const int tm = m0;
            m0 = mn;
            mn = tm;
        }
        int code = -2, nh = NO_CELL;
        if (dot(s - o, n0) >= 0.0f) {
            const f3 t0 = cross(n0, e);
            // sample i: x = L (i + 1/2)/N, phi = n pi frac(i (phi_g - 1)) (24-bit fixed point)
            const float u1 = A.ns < (1ULL << 24) ? ((float)i + 0.5f) / (float)A.ns
                                                 : (float)(((double)i + 0.5) / (double)A.ns);
            const unsigned long long fr = i * 0x9E3779B97F4A7C16ULL;
            const float u2 = (float)(unsigned)(fr >> 40) * 0x1p-24f;
            const float x = u1 * W.length;
            float sp, cp;
            sincospif(u2 * W.n, &sp, &cp);
            const f3 v = o + e * x;
            const f3 d = v - s;
            const float dn = sqrtf(dot(d, d));
            const f3 so = s - o;
            const f3 perp = so - e * dot(so, e);
            const float rho = sqrtf(dot(perp, perp));
            const float cb = dot(d, e) / dn, sb = rho / dn;
            const f3 u{cp * t0.x + sp * n0.x, cp * t0.y + sp * n0.y, cp * t0.z + sp * n0.z};
            const f3 ks = u * sb + e * cb;
            ++c_seg;
            const float vm = fmaxf(fabsf(v.x), fmaxf(fabsf(v.y), fabsf(v.z)));
            const float eps = fmaxf(1.0f, vm) * 0x1p-16f;
            const f3 si = d * (1.0f / dn);
            code = segment_blocked(A, s, si, eps, dn - eps, W.tri0, W.trin, c_nodes, c_tris, overflow) ? 1 : 0;
            nh = 0;
            if (code == 0) {
                Crossing hits[MAX_CROSS];
                nh = surface_hits(A.snodes, A.stris, A.snt, A.snlarge, v, ks, hits, &overflow, &xlimit);
                const float nw_ = W.n;
                const float phi = u2 * nw_ * PI_F;
                const f3 dkx = (e * sb - u * cb) * (sb / dn);
                const f3 dkp{sb * (cp * n0.x - sp * t0.x), sb * (cp * n0.y - sp * t0.y), sb * (cp * n0.z - sp * t0.z)};
                const unsigned long long mb = (unsigned long long)txi * A.ncell;
#pragma unroll 1
                for (int c = 0; c < nh; ++c) {
                    const float tc = hits[c].t;
                    if (segment_blocked(A, v, ks, eps, tc, W.tri0, W.trin, c_nodes, c_tris, overflow)) continue;
                    // weighting factor on the plane n.(t - a) = 0: dtc/dq = -(n.dv/dq + tc n.dk/dq) / (n.k)
                    const f3 nc = hits[c].nrm;
                    const float nk = dot(nc, ks);
                    if (nk == 0.0f) continue;
                    const float dtcx = -(dot(nc, e) + tc * dot(nc, dkx)) / nk;
                    const float dtcp = -(tc * dot(nc, dkp)) / nk;
                    const f3 tx = e + ks * dtcx + dkx * tc;
                    const f3 tp = ks * dtcp + dkp * tc;
                    const f3 cr = cross(tx, tp);
                    const float J = sqrtf(dot(cr, cr));
                    const float pw = diffracted_power(A, T, s, v, e, n0, nn, t0, m0, mn, nw_, phi, sb, si, dn, tc);
                    const float spread = 1.0f / (dn * tc * (dn + tc));
                    const float inv_area = 2.0f / sqrtf(dot(nc, nc));
                    const float value =
                        A.lam4pi2_over_cell2 * (W.length * nw_ * PI_F / (float)A.ns) * J * pw * spread * inv_area;
                    atomicAdd(A.maps64 + mb + (unsigned long long)hits[c].tri, (double)value);
                    ++c_dep;
                }
            }
        }
        // records {bits: 1 incident blocked, -2 source behind both faces; crossings found; 0; 0}
        put_record(A, w, code, nh, 0);
    }
    const unsigned v[6] = {c_rays, c_seg, c_nodes, c_tris, c_dep, 0u};
    flush_counters(A, s_cnt, v, overflow, xlimit);
}

}  // namespace

cudaError_t launch_diffraction(const DiffArgs& a, int block, cudaStream_t s, int* grid_out, bool mesh) {
    if (block <= 0 || block > 256 || (block & 31)) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t err;
    const void* k = mesh ? reinterpret_cast<const void*>(&k_diffraction_mesh)
                         : reinterpret_cast<const void*>(&k_diffraction_plane);
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, block, 0)) != cudaSuccess)
        return err;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const unsigned long long need = (a.total + block - 1) / block;
    const unsigned long long cap = (unsigned long long)occ * sms;
    const int grid = (int)(need < cap ? (need > 0 ? need : 1) : cap);
    if (grid_out) *grid_out = grid;
    void* args[] = {const_cast<DiffArgs*>(&a)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, 0, s);
}

void faddeeva_coefficients(int N, double* L_out, double* a) {
    // a_n: Fourier coefficients of f(theta) = (L^2 + t^2) exp(-t^2), t = L tan(theta/2),
    // on (-pi, pi), by the midpoint rule (spectrally accurate for this smooth periodic f)
    const double L = std::sqrt(N / std::sqrt(2.0));
    const int M = 4096;
    for (int n = 1; n <= N; ++n) {
        double acc = 0.0;
        for (int k = 0; k < M; ++k) {
            const double th = -M_PI + (k + 0.5) * 2.0 * M_PI / M;
            const double t = L * std::tan(0.5 * th);
            acc += std::exp(-t * t) * (L * L + t * t) * std::cos(n * th);
        }
        a[n - 1] = acc / M;
    }
    *L_out = L;
}

}  // namespace rmsbr
