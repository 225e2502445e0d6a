// FP64 CPU oracle for the SBR radio-map method of the Sionna RT technical
// report (arXiv 2504.21719).  TEST INFRASTRUCTURE ONLY: it is loaded by the
// test-suite, the smoke check and the benchmark's CPU-baseline leg, never by
// the product path.  It shares no code, header or constant table with the
// CUDA library; the only common input is the seeded scene data.
//
// What it computes (each function names the passage it follows):
//   * spherical Fibonacci lattice (Sec. 3.1.1);
//   * transmitter field from antenna pattern and orientation (App. A.1,
//     Eqs. rotation / theta_phi_prime / F_prime_2_F, antenna pattern Eq. C);
//   * closest hit by brute force over every triangle (Moller-Trumbore, FP64);
//   * Fresnel coefficients for incidence from vacuum (Eq. fresnel_vac) and the
//     single-layer slab (Eqs. fresnel_slab, q_fresnel_slab), complex
//     permittivity (Eq. eta);
//   * interaction-type sampling q(R), q(T) (Eq. path-solver-used-dist-event
//     with S = 0 and q(D) = 0), field update with the TE/TM basis
//     (Eqs. fresnel_in_vectors, fresnel_out_vectors, reflected_refracted_vectors);
//   * the radio-map Monte-Carlo estimator (Eq. radio-map-solver-ci-all-2-estimator
//     with n_S = 0) where the squared tube length cancels against the 1/r
//     spreading of the path gain (Eq. radio-map-solver-path-gain, Alg. 2);
//   * a branch-all enumeration (every reflection AND refraction branch, no
//     sampling) that gives the estimator's exact expectation on tiny scenes;
//   * forward-mode dual numbers for the gradient with frozen discrete choices;
//   * a reference LBVH (Morton codes + stable sort + top-down binary radix
//     tree) and a reference binned-SAH tree over the same leaves, which the
//     GPU's two builders must equal bit for bit;
//   * diffuse reflection (App. A.10: S / R split of the sampling, the
//     scattered field with cross-polarisation, Lambertian / directive /
//     backscattering patterns);
//   * early termination by Russian roulette and gain thresholding (Sec. 4);
//   * synthetic transmit arrays with precoding (Sec. 4);
//   * the first-order diffraction map (Sec. 4, UTD of App. A.8, the weighting
//     factor by dual numbers) with the Fresnel transition function by a
//     Gauss-Legendre integral;
//   * radio maps on a mesh measurement surface (Sec. 4, practical notes) by
//     brute force over the surface's triangles.
//
// Readings of points the paper leaves open are stated where they are used.
//
// Parity status: every function here is pinned by a CPU test to a closed
// form, an identity, a library routine or brute force (tests/test_oracle_*.py);
// none is "parity unpinned".

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <map>
#include <type_traits>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double C0 = 299792458.0;          // speed of light in vacuum, m/s
constexpr double EPS0 = 8.8541878128e-12;   // vacuum permittivity, F/m (CODATA 2018)

// ---------------------------------------------------------------------------
// dual numbers (value + NT tangents) for the frozen-choice gradient
// ---------------------------------------------------------------------------
constexpr int NT = 19;  // 8 permittivities + 8 conductivities + 3 TX coordinates

struct D {
    double v;
    double g[NT];
    D() : v(0) { std::memset(g, 0, sizeof g); }
    D(double x) : v(x) { std::memset(g, 0, sizeof g); }  // NOLINT: implicit by design
};
inline D operator+(const D& a, const D& b) { D r(a.v + b.v); for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] + b.g[i]; return r; }
inline D operator-(const D& a, const D& b) { D r(a.v - b.v); for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] - b.g[i]; return r; }
inline D operator-(const D& a) { D r(-a.v); for (int i = 0; i < NT; ++i) r.g[i] = -a.g[i]; return r; }
inline D operator*(const D& a, const D& b) { D r(a.v * b.v); for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * b.v + a.v * b.g[i]; return r; }
inline D operator/(const D& a, const D& b) {
    D r(a.v / b.v);
    const double ib = 1.0 / b.v;
    for (int i = 0; i < NT; ++i) r.g[i] = (a.g[i] - r.v * b.g[i]) * ib;
    return r;
}
inline D operator+(const D& a, double b) { D r = a; r.v += b; return r; }
inline D operator+(double b, const D& a) { return a + b; }
inline D operator-(const D& a, double b) { D r = a; r.v -= b; return r; }
inline D operator-(double b, const D& a) { return (-a) + b; }
inline D operator*(const D& a, double b) { D r(a.v * b); for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * b; return r; }
inline D operator*(double b, const D& a) { return a * b; }
inline D operator/(const D& a, double b) { return a * (1.0 / b); }
inline D operator/(double a, const D& b) { return D(a) / b; }
inline D& operator+=(D& a, const D& b) { a = a + b; return a; }

inline double val(double x) { return x; }
inline double val(const D& x) { return x.v; }
inline double r_sqrt(double x) { return std::sqrt(x); }
inline D r_sqrt(const D& a) {
    D r(std::sqrt(a.v));
    const double k = (r.v > 0) ? 0.5 / r.v : 0.0;
    for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * k;
    return r;
}
inline double r_sin(double x) { return std::sin(x); }
inline double r_cos(double x) { return std::cos(x); }
inline double r_exp(double x) { return std::exp(x); }
inline D r_sin(const D& a) { D r(std::sin(a.v)); const double c = std::cos(a.v); for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * c; return r; }
inline D r_cos(const D& a) { D r(std::cos(a.v)); const double s = -std::sin(a.v); for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * s; return r; }
inline D r_exp(const D& a) { D r(std::exp(a.v)); for (int i = 0; i < NT; ++i) r.g[i] = a.g[i] * r.v; return r; }
template <class R> inline R r_abs(const R& a) { return val(a) < 0 ? R(-a) : a; }

// ---------------------------------------------------------------------------
// complex numbers over a real type R (std::complex is unspecified for D)
// ---------------------------------------------------------------------------
template <class R>
struct Cx {
    R re, im;
    Cx() : re(0.0), im(0.0) {}
    Cx(const R& a) : re(a), im(0.0) {}  // NOLINT
    Cx(const R& a, const R& b) : re(a), im(b) {}
};
template <class R> inline Cx<R> operator+(const Cx<R>& a, const Cx<R>& b) { return {a.re + b.re, a.im + b.im}; }
template <class R> inline Cx<R> operator-(const Cx<R>& a, const Cx<R>& b) { return {a.re - b.re, a.im - b.im}; }
template <class R> inline Cx<R> operator*(const Cx<R>& a, const Cx<R>& b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class R> inline Cx<R> operator*(const Cx<R>& a, const R& s) { return {a.re * s, a.im * s}; }
template <class R> inline Cx<R> operator/(const Cx<R>& a, const Cx<R>& b) {
    R d = b.re * b.re + b.im * b.im;
    return {(a.re * b.re + a.im * b.im) / d, (a.im * b.re - a.re * b.im) / d};
}
template <class R> inline R abs2(const Cx<R>& a) { return a.re * a.re + a.im * a.im; }

// Principal square root, written from the definition
//   sqrt(z) = sqrt((|z|+x)/2) + j sgn(y) sqrt((|z|-x)/2),
// evaluated in the cancellation-free arrangement of Kahan, "Branch cuts for
// complex elementary functions" (1987): the larger of the two parts comes from
// a square root, the smaller one from y / (2 * larger).
template <class R>
Cx<R> csqrt(const Cx<R>& z) {
    const double xv = val(z.re), yv = val(z.im);
    if (xv == 0.0 && yv == 0.0) return Cx<R>(R(0.0), R(0.0));
    // |z| scaled by a constant so that the squares neither underflow nor overflow
    const double sc = std::max(std::fabs(xv), std::fabs(yv));
    R xs = z.re / sc, ys = z.im / sc;
    R m = r_sqrt(xs * xs + ys * ys) * sc;
    if (xv >= 0.0) {
        R a = r_sqrt((m + z.re) * 0.5);
        return Cx<R>(a, z.im / (a * 2.0));
    }
    R b = r_sqrt((m - z.re) * 0.5);
    R a = r_abs(z.im) / (b * 2.0);
    return Cx<R>(a, std::signbit(yv) ? R(-b) : b);
}
// exp(-j w) for complex w = a + j b:  exp(b) (cos a - j sin a)
template <class R>
Cx<R> cexp_mj(const Cx<R>& w) {
    R e = r_exp(w.im);
    return Cx<R>(e * r_cos(w.re), -(e * r_sin(w.re)));
}

// ---------------------------------------------------------------------------
// small vectors
// ---------------------------------------------------------------------------
template <class R>
struct V3 {
    R x, y, z;
};
template <class R> inline V3<R> operator+(const V3<R>& a, const V3<R>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R> inline V3<R> operator-(const V3<R>& a, const V3<R>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class R, class S> inline V3<R> scl(const V3<R>& a, const S& s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(const V3<double>& a, const V3<double>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3<double> cross(const V3<double>& a, const V3<double>& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(const V3<double>& a) { return std::sqrt(dot(a, a)); }
inline V3<double> unit(const V3<double>& a) { return scl(a, 1.0 / norm(a)); }
template <class R> inline V3<R> lift(const V3<double>& a) { return {R(a.x), R(a.y), R(a.z)}; }
template <class R> inline V3<double> vval(const V3<R>& a) { return {val(a.x), val(a.y), val(a.z)}; }
// position + t * direction with a real-typed t
template <class R> inline V3<R> axpy(const V3<R>& o, const R& t, const V3<double>& k) {
    return {o.x + t * k.x, o.y + t * k.y, o.z + t * k.z};
}

// complex 3-vector (a field phasor in global Cartesian coordinates)
template <class R>
struct CV3 {
    Cx<R> x, y, z;
};
template <class R> inline Cx<R> cdot(const V3<double>& e, const CV3<R>& f) {
    // e^T f with e real
    return f.x * R(e.x) + f.y * R(e.y) + f.z * R(e.z);
}
template <class R> inline CV3<R> outer(const V3<double>& e, const Cx<R>& a) {
    return {a * R(e.x), a * R(e.y), a * R(e.z)};
}
template <class R> inline CV3<R> operator+(const CV3<R>& a, const CV3<R>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class R> inline R cnorm2(const CV3<R>& f) { return abs2(f.x) + abs2(f.y) + abs2(f.z); }

// ---------------------------------------------------------------------------
// counter-based random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014)
// ---------------------------------------------------------------------------
inline uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
// Reading: the paper does not fix its random-number generator.  The uniform
// variate for the interaction at the end of segment l of lattice ray n is the
// top 24 bits of splitmix64(seed ^ splitmix64(n * 16 + l)), scaled by 2^-24;
// it is exactly representable in FP32 and FP64.
inline double rng_u(uint64_t seed, uint64_t n, int l) {
    uint64_t h = splitmix64(seed ^ splitmix64((n << 4) | (uint64_t)(l & 15)));
    return (double)(h >> 40) * (1.0 / 16777216.0);
}
// The Russian-roulette variate of the same interaction comes from a second
// stream: the seed xor-ed with a fixed odd constant.
constexpr uint64_t RR_STREAM = 0xD6E8FEB86659FD93ULL;
inline double rng_rr(uint64_t seed, uint64_t n, int l) { return rng_u(seed ^ RR_STREAM, n, l); }
// The four variates of a diffuse reflection (two for the direction, two for
// the random phases) come from four more streams.
constexpr uint64_t DIFF_STREAM[4] = {0x2545F4914F6CDD1DULL, 0x9E6C63D0676A9A99ULL, 0x7F4A7C159E3779B9ULL,
                                     0xC2B2AE3D27D4EB4FULL};
inline double rng_diff(uint64_t seed, uint64_t n, int l, int j) { return rng_u(seed ^ DIFF_STREAM[j], n, l); }

// ---------------------------------------------------------------------------
// Spherical Fibonacci lattice (Sec. 3.1.1)
// ---------------------------------------------------------------------------
// cos(theta_n) = 1 - 2n/(N-1); phi_n = 2 pi frac(n / phi_g).  Since
// 1/phi_g = phi_g - 1, frac(n / phi_g) = frac(n (phi_g - 1)), evaluated as the
// 64-bit fixed-point product n * round(2^64 (phi_g - 1)) mod 2^64 so that the
// fractional part carries no cancellation for large n.  N = 1 gives
// theta = pi/2, phi = pi.
constexpr uint64_t WEYL_GOLDEN = 0x9E3779B97F4A7C16ULL;  // nearest integer to 2^64 * (phi_g - 1)

V3<double> fibonacci_dir(int64_t n, int64_t N) {
    double ct, st, phi;
    if (N == 1) {
        ct = 0.0; st = 1.0; phi = PI;
    } else {
        ct = 1.0 - 2.0 * (double)n / (double)(N - 1);
        st = std::sqrt((1.0 - ct) * (1.0 + ct));
        uint64_t f = (uint64_t)n * WEYL_GOLDEN;
        phi = 2.0 * PI * ((double)f * 0x1.0p-64);
    }
    return {st * std::cos(phi), st * std::sin(phi), ct};
}

// ---------------------------------------------------------------------------
// Transmitter field (App. A.1 and the antenna pattern, Eq. C)
// ---------------------------------------------------------------------------
struct Rot { double m[3][3]; };
// R(alpha, beta, gamma) = Rz(alpha) Ry(beta) Rx(gamma)   (Eq. rotation)
Rot rotation(double a, double b, double g) {
    double Rz[3][3] = {{std::cos(a), -std::sin(a), 0}, {std::sin(a), std::cos(a), 0}, {0, 0, 1}};
    double Ry[3][3] = {{std::cos(b), 0, std::sin(b)}, {0, 1, 0}, {-std::sin(b), 0, std::cos(b)}};
    double Rx[3][3] = {{1, 0, 0}, {0, std::cos(g), -std::sin(g)}, {0, std::sin(g), std::cos(g)}};
    double T[3][3] = {};
    Rot R = {};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) T[i][j] += Ry[i][k] * Rx[k][j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) R.m[i][j] += Rz[i][k] * T[k][j];
    return R;
}
inline V3<double> mul(const Rot& R, const V3<double>& v) {
    return {R.m[0][0] * v.x + R.m[0][1] * v.y + R.m[0][2] * v.z,
            R.m[1][0] * v.x + R.m[1][1] * v.y + R.m[1][2] * v.z,
            R.m[2][0] * v.x + R.m[2][1] * v.y + R.m[2][2] * v.z};
}
inline V3<double> mulT(const Rot& R, const V3<double>& v) {
    return {R.m[0][0] * v.x + R.m[1][0] * v.y + R.m[2][0] * v.z,
            R.m[0][1] * v.x + R.m[1][1] * v.y + R.m[2][1] * v.z,
            R.m[0][2] * v.x + R.m[1][2] * v.y + R.m[2][2] * v.z};
}
// spherical unit vectors theta_hat, phi_hat at (theta, phi)  (Eq. spherical_vecs)
inline V3<double> theta_hat(double th, double ph) {
    return {std::cos(th) * std::cos(ph), std::cos(th) * std::sin(ph), -std::sin(th)};
}
inline V3<double> phi_hat(double ph) { return {-std::sin(ph), std::cos(ph), 0.0}; }

// Antenna pattern C = (C_theta, C_phi) in the antenna's local frame.
//   pattern 0: isotropic, |C|^2 = 1 for the chosen polarisation;
//   pattern 1: short dipole along the local z axis, C_theta = sqrt(3/2) sin(theta').
// Both satisfy the normalisation integral of G = |C|^2 over the sphere = 4 pi.
// Polarisation 0 puts the pattern on theta' (vertical), 1 on phi' (horizontal).
// Returns the global-frame field vector R (C_theta theta_hat' + C_phi phi_hat')
// for the departure direction k (global frame), i.e. the first column of the
// transfer cascade applied to the pattern.
V3<double> tx_field(const V3<double>& k, const Rot& R, int pattern, int pol) {
    V3<double> kl = mulT(R, k);  // direction in the antenna frame (Eq. theta_phi_prime)
    double zc = std::max(-1.0, std::min(1.0, kl.z));
    double th = std::acos(zc);
    // Reading at the poles: atan2(0, 0) = 0.
    double ph = std::atan2(kl.y, kl.x);
    double g = 1.0;
    if (pattern == 1) g = std::sqrt(1.5) * std::sin(th);
    V3<double> e_local = (pol == 0) ? theta_hat(th, ph) : phi_hat(ph);
    return scl(mul(R, e_local), g);
}

// ---------------------------------------------------------------------------
// Fresnel / slab coefficients (App. A.7 and A.7.1)
// ---------------------------------------------------------------------------
template <class R>
struct Coefs {
    Cx<R> r_perp, r_par, t_perp, t_par;
};
// Complex relative permittivity, Eq. eta:  eta = eps_r - j sigma / (eps0 omega)
template <class R>
inline Cx<R> permittivity(const R& eps_r, const R& sigma, double omega) {
    return Cx<R>(eps_r, -(sigma / (EPS0 * omega)));
}
// Incidence from vacuum on a half-space (Eq. fresnel_vac), or on a slab of
// electrical thickness k0d = 2 pi d / lambda0 (Eqs. fresnel_slab,
// q_fresnel_slab) when k0d > 0.  Reading: thickness <= 0 means a half-space,
// whose transmitted wave never leaves the material: t = 0.
template <class R>
Coefs<R> fresnel(const Cx<R>& eta, double cos1, const R& k0d, bool slab) {
    const double sin2 = (1.0 - cos1) * (1.0 + cos1);
    Cx<R> s = csqrt(eta - Cx<R>(R(sin2)));
    Cx<R> c{R(cos1)};
    Cx<R> ec = eta * R(cos1);
    Coefs<R> o;
    Cx<R> rp = (c - s) / (c + s);
    Cx<R> rl = (ec - s) / (ec + s);
    if (!slab) {
        o.r_perp = rp;
        o.r_par = rl;
        o.t_perp = Cx<R>(R(0.0));
        o.t_par = Cx<R>(R(0.0));
        return o;
    }
    Cx<R> q = s * k0d;
    Cx<R> e1 = cexp_mj(q);                      // exp(-j q)
    Cx<R> e2 = e1 * e1;                         // exp(-j 2q)
    Cx<R> one(R(1.0));
    Cx<R> rp2 = rp * rp, rl2 = rl * rl;
    o.r_perp = rp * (one - e2) / (one - rp2 * e2);
    o.r_par = rl * (one - e2) / (one - rl2 * e2);
    o.t_perp = (one - rp2) * e1 / (one - rp2 * e2);
    o.t_par = (one - rl2) * e1 / (one - rl2 * e2);
    return o;
}
// The vacuum-incidence transmission coefficients of Eq. fresnel_vac (used by
// the pins only; the slab model above replaces them on the path).
template <class R>
void fresnel_vac_t(const Cx<R>& eta, double cos1, Cx<R>* t_perp, Cx<R>* t_par) {
    const double sin2 = (1.0 - cos1) * (1.0 + cos1);
    Cx<R> s = csqrt(eta - Cx<R>(R(sin2)));
    Cx<R> c{R(cos1)};
    Cx<R> ec = eta * R(cos1);
    *t_perp = (c * R(2.0)) / (c + s);
    *t_par = (csqrt(eta) * R(2.0 * cos1)) / (ec + s);
}

// ---------------------------------------------------------------------------
// scene
// ---------------------------------------------------------------------------
struct Tri {
    V3<double> a, b, c, e1, e2, n;  // n = unit((b - a) x (c - a))
    double area2;                    // |(b - a) x (c - a)|
    double len[3];                   // |c-b|, |a-c|, |b-a| (edge opposite a, b, c)
    int mat;
};

struct Scene {
    std::vector<Tri> tris;
    std::vector<double> eps, sigma, thick;
    // diffuse reflection (App. A.10): scattering coefficient S, cross-polarisation
    // share K_x, pattern (0 Lambertian, 1 directive, 2 backscattering), alpha_R,
    // alpha_I, Lambda
    std::vector<double> scS, scK, scLam;
    std::vector<int> scPat, scAR, scAI;
};

Scene make_scene(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                 const int32_t* tri_mat, const float* mats, int nm, const float* scat = nullptr) {
    (void)nv;
    Scene s;
    s.tris.resize(nt);
    for (int64_t i = 0; i < nt; ++i) {
        Tri& t = s.tris[i];
        auto V = [&](int j) {
            const float* p = verts + 3 * (int64_t)tris[3 * i + j];
            return V3<double>{p[0], p[1], p[2]};
        };
        t.a = V(0); t.b = V(1); t.c = V(2);
        t.e1 = t.b - t.a;
        t.e2 = t.c - t.a;
        V3<double> cr = cross(t.e1, t.e2);
        t.area2 = norm(cr);
        t.n = t.area2 > 0 ? scl(cr, 1.0 / t.area2) : V3<double>{0, 0, 1};
        t.len[0] = norm(t.c - t.b);
        t.len[1] = norm(t.a - t.c);
        t.len[2] = norm(t.b - t.a);
        t.mat = tri_mat[i];
    }
    for (int m = 0; m < nm; ++m) {
        s.eps.push_back(mats[3 * m]);
        s.sigma.push_back(mats[3 * m + 1]);
        s.thick.push_back(mats[3 * m + 2]);
        const float* sc = scat ? scat + 6 * m : nullptr;
        s.scS.push_back(sc ? sc[0] : 0.0);
        s.scK.push_back(sc ? sc[1] : 0.0);
        s.scPat.push_back(sc ? (int)sc[2] : 0);
        s.scAR.push_back(sc ? (int)sc[3] : 1);
        s.scAI.push_back(sc ? (int)sc[4] : 1);
        s.scLam.push_back(sc ? sc[5] : 1.0);
    }
    return s;
}

// Moller-Trumbore in FP64, edges inclusive (a hit on a shared edge counts for
// both triangles).  Returns t > 0 or +inf.
inline double hit_mt(const Tri& T, const V3<double>& o, const V3<double>& k) {
    V3<double> p = cross(k, T.e2);
    double det = dot(T.e1, p);
    if (det == 0.0) return INFINITY;
    double inv = 1.0 / det;
    V3<double> tv = o - T.a;
    double u = dot(tv, p) * inv;
    if (u < 0.0 || u > 1.0) return INFINITY;
    V3<double> q = cross(tv, T.e1);
    double v = dot(k, q) * inv;
    if (v < 0.0 || u + v > 1.0) return INFINITY;
    double t = dot(T.e2, q) * inv;
    return t > 0.0 ? t : INFINITY;
}

// Reading (paper silent): the closest hit excludes the primitive the ray just
// left; equal distances go to the smaller triangle index.  Distances that
// agree to a relative 1e-12 count as equal, so coplanar triangles (a box
// floor lying on the ground plane) are resolved by index, not by rounding.
inline void closest_hit(const Scene& S, const V3<double>& o, const V3<double>& k, int exclude,
                        int* prim, double* t) {
    int best = -1;
    double tb = INFINITY;
    const int nt = (int)S.tris.size();
    for (int i = 0; i < nt; ++i) {  // ascending index: a later triangle must be clearly closer
        if (i == exclude) continue;
        double ti = hit_mt(S.tris[i], o, k);
        if (ti < tb * (1.0 - 1e-12)) { tb = ti; best = i; }
    }
    *prim = best;
    *t = tb;
}

// Intersection with the plane of a given triangle, plus the signed distance
// (m) of the hit point to the triangle (positive inside, negative outside):
// min over edges of barycentric * (2 area / edge length).
inline bool plane_hit(const Tri& T, const V3<double>& o, const V3<double>& k, double* t, double* margin) {
    double den = dot(T.n, k);
    if (den == 0.0 || T.area2 == 0.0) return false;
    *t = dot(T.n, T.a - o) / den;
    V3<double> p = o + scl(k, *t);
    // barycentrics via sub-triangle areas (signed along n)
    double wa = dot(cross(T.b - p, T.c - p), T.n) / T.area2;
    double wb = dot(cross(T.c - p, T.a - p), T.n) / T.area2;
    double wc = 1.0 - wa - wb;
    double da = wa * T.area2 / T.len[0];
    double db = wb * T.area2 / T.len[1];
    double dc = wc * T.area2 / T.len[2];
    *margin = std::min(da, std::min(db, dc));
    return true;
}

// ---------------------------------------------------------------------------
// public structs (mirrored by the ctypes wrapper)
// ---------------------------------------------------------------------------
struct or_tx {
    double pos[3];
    double yaw, pitch, roll;
    int32_t pol, pattern;
    int64_t num_rays, ray_begin, ray_count, ray_stride;
    uint64_t seed;
    int64_t n_ant;             // synthetic array (Sec. 4.4): 0 = single antenna
    const double* ant_pos;     // [n_ant][3] element positions in the antenna frame (m)
    const double* precoding;   // [n_ant][2] complex precoding weights
};
struct or_params {
    double freq_hz;
    int32_t max_depth, flags;
    double map_origin[3];
    double cell_size;
    int32_t nx, ny, deposit, pad;
    int32_t rr_depth, pad2;    // early termination after this many interactions (Sec. 4.5); 0 = off
    double rr_max_prob;        // p_rr,max; 0 = no Russian roulette
    double gain_threshold;     // linear gain below which a path stops; 0 = off
};
enum { F_REFLECT = 1, F_REFRACT = 2, F_LOS = 4, F_DIFFUSE = 16 };
struct or_report {
    int64_t segments, deposits, adopted_hit, adopted_cell, adopted_decision, failures;
    int64_t adopted_hit_tie;  // adopted hits whose distance equals the FP64 closest hit within tol
    int64_t fail_ray;
    int32_t fail_depth, fail_kind;  // 1 hit, 2 deposit cell, 3 decision, 4 segment
    double fail_info[4];
    // Records that carry the GPU's coin probability q(R) (bits 8.. of the
    // decision, units of 2^-22): how many were checked, the largest
    // |q_gpu - q(R)| and its largest ratio to the replay's decision window,
    // and how many fell outside that window.
    int64_t coin_checked, coin_outside;
    double coin_max_dev, coin_max_ratio;
};
constexpr int32_t NO_CELL = -32768;
enum { MODE_PLAIN = 0, MODE_REPLAY = 1, MODE_FROZEN = 2 };

// per-segment record, shared layout with the GPU's debug record:
// {prim (-2 no segment, -1 miss), ix, iy (NO_CELL = no deposit), decision (0 R, 1 T, -1 none)}
struct Rec {
    int32_t prim, ix, iy, dec;
};

struct MapGeom {
    double x0, y0, z, cell, K;  // K = 4 pi / (N Delta^2) * (lambda0 / 4 pi)^2
    int nx, ny, bilinear;
};

// ---------------------------------------------------------------------------
// deposit (Eq. radio-map-solver-ci-all-2-estimator, n_S = 0)
// ---------------------------------------------------------------------------
// For a segment with origin o and direction k that ends at t_h (inf = escaped):
// t_c = (z_M - o_z) / k_z; if 1e-9 < t_c < t_h the crossing (x, y) adds
//   K * |E|^2 / (|k_z| * Pr)
// to its cell (box), or splits it over the four nearest cell centres with
// tent weights (bilinear).  Rays parallel to the plane (k_z = 0) never
// deposit.  The plane does not stop the ray.
template <class R>
struct Crossing {
    bool valid;
    double tc_v;      // value of t_c
    R x, y;           // crossing point
    int ix, iy;       // box: cell; bilinear: lower-left cell of the 2x2 stencil
    double ux, uy;    // (x - x0)/Delta (box) or (x - x0)/Delta - 0.5 (bilinear)
};
template <class R>
Crossing<R> crossing(const MapGeom& g, const V3<R>& o, const V3<double>& k, double t_h) {
    Crossing<R> c;
    c.valid = false;
    if (k.z == 0.0) return c;
    R tc = (R(g.z) - o.z) / k.z;
    c.tc_v = val(tc);
    if (!(c.tc_v > 1e-9 && c.tc_v < t_h)) return c;
    c.x = o.x + tc * k.x;
    c.y = o.y + tc * k.y;
    double sh = g.bilinear ? 0.5 : 0.0;
    c.ux = (val(c.x) - g.x0) / g.cell - sh;
    c.uy = (val(c.y) - g.y0) / g.cell - sh;
    c.ix = (int)std::floor(c.ux);
    c.iy = (int)std::floor(c.uy);
    if (g.bilinear) {
        if (c.ix < -1 || c.ix > g.nx - 1 || c.iy < -1 || c.iy > g.ny - 1) return c;
    } else {
        if (c.ix < 0 || c.ix >= g.nx || c.iy < 0 || c.iy >= g.ny) return c;
    }
    c.valid = true;
    return c;
}

// A deposit sink accumulates either a map (double) or a gradient functional.
struct DepList {
    std::vector<int32_t> cell;
    std::vector<double> val;
};

template <class R>
struct Sink;
template <>
struct Sink<double> {
    DepList* list;
    DepList* mass = nullptr;   // unweighted deposit value per stencil cell (bilinear error bound)
    DepList* cmass = nullptr;  // the same, times the crossing's conditioning factor
    DepList* slack = nullptr;  // mesh surfaces: values of crossings within tol of a cell's boundary
    DepList* amass = nullptr;  // values times the ray's array-factor conditioning (synthetic arrays)
    double acond = 0.0;        // that factor for the ray being traced
    bool want_acond() const { return amass != nullptr; }
    void set_acond(double c) { acond = c; }
    void add(int cell, const double& v) { list->cell.push_back(cell); list->val.push_back(v); }
    void add_slack(int cell, double v) {
        if (slack) { slack->cell.push_back(cell); slack->val.push_back(v); }
    }
    void add_mass(int cell, const double& v, double cond) {
        if (mass) { mass->cell.push_back(cell); mass->val.push_back(v); }
        if (cmass) { cmass->cell.push_back(cell); cmass->val.push_back(v * cond); }
        if (amass && acond > 0.0) { amass->cell.push_back(cell); amass->val.push_back(v * acond); }
    }
};
template <>
struct Sink<D> {
    const double* gmap;  // dL/dC per cell
    double acc[NT];
    void add(int cell, const D& v) {
        const double w = gmap[cell];
        for (int i = 0; i < NT; ++i) acc[i] += w * v.g[i];
    }
    void add_mass(int, const D&, double) {}
    void add_slack(int, double) {}
    bool want_acond() const { return false; }
    void set_acond(double) {}
};

// cond: first-order conditioning of the crossing point x_c = o + t_c k against
// perturbations of the origin and direction (test bookkeeping only, see
// trace_ray); it does not enter the map.
template <class R, class SinkT>
void deposit(const MapGeom& g, const Crossing<R>& c, int ix, int iy, const R& value, SinkT& sink,
             double cond = 1.0) {
    if (!g.bilinear) {
        if (ix >= 0 && ix < g.nx && iy >= 0 && iy < g.ny) {
            sink.add(iy * g.nx + ix, value);
            sink.add_mass(iy * g.nx + ix, value, cond);
        }
        return;
    }
    // tent weights relative to the (possibly adopted) lower-left index
    double sh = 0.5;
    R fx = (c.x - g.x0) / g.cell - (sh + ix);
    R fy = (c.y - g.y0) / g.cell - (sh + iy);
    R wx[2] = {R(1.0) - fx, fx};
    R wy[2] = {R(1.0) - fy, fy};
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
            int cx = ix + a, cy = iy + b;
            if (cx < 0 || cx >= g.nx || cy < 0 || cy >= g.ny) continue;
            sink.add(cy * g.nx + cx, value * (wx[a] * wy[b]));
            sink.add_mass(cy * g.nx + cx, value, cond);
        }
}

// ---------------------------------------------------------------------------
// diffuse reflection (App. A.10)
// ---------------------------------------------------------------------------
inline double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}
// F_alpha(theta_i) of Eq. directive_model: the integral of ((1 + k_r.k_s)/2)^alpha
// over the hemisphere of k_s, in the closed form printed with the model.
double f_alpha(int alpha, double cos_i) {
    const double sin2 = (1.0 - cos_i) * (1.0 + cos_i);
    double F = 0.0;
    for (int k = 0; k <= alpha; ++k) {
        double Ik = 2.0 * PI / (k + 1);
        if (k % 2 == 1) {
            double s = 0.0;
            for (int w = 0; w <= (k - 1) / 2; ++w) s += binom(2 * w, w) * std::pow(sin2, w) / std::pow(2.0, 2 * w);
            Ik *= cos_i * s;
        }
        F += binom(alpha, k) * Ik;
    }
    return F / std::pow(2.0, alpha);
}
// Scattering pattern f_s(k_i, k_s, n): Lambertian (0, Eq. lambertian_model),
// directive (1, Eq. directive_model) or backscattering (2, Eq.
// backscattering_model).  n is the unit normal on the incident side.
double scat_pattern(int pattern, int aR, int aI, double lam, const V3<double>& ki, const V3<double>& ks,
                    const V3<double>& n) {
    if (pattern == 0) return dot(n, ks) / PI;
    const double cos_i = -dot(ki, n);
    const V3<double> kr = ki - scl(n, 2.0 * dot(ki, n));  // specular direction
    const double lobe_r = std::pow((1.0 + dot(kr, ks)) / 2.0, aR);
    if (pattern == 1) return lobe_r / f_alpha(aR, cos_i);
    const double lobe_i = std::pow((1.0 - dot(ki, ks)) / 2.0, aI);
    return (lam * lobe_r + (1.0 - lam) * lobe_i) / (lam * f_alpha(aR, cos_i) + (1.0 - lam) * f_alpha(aI, cos_i));
}
// Direction of the ray tube a diffuse reflection spawns: uniform on the
// hemisphere around n (solid angle 2 pi, Sec. 4 estimator).  Reading (the
// paper fixes no parametrisation): cos theta_s = 1 - u1, phi_s = 2 pi u2 in
// the tangent frame (t1, t2) of m = n (or m = -n when n_z < -1/2), with
// t1 = (1 - m_x^2 a, -m_x m_y a, -m_x), t2 = (-m_x m_y a, 1 - m_y^2 a, -m_y),
// a = 1 / (1 + m_z)  (Frisvad, JGT 2012).
V3<double> diffuse_dir(const V3<double>& n, double u1, double u2) {
    const V3<double> m = n.z >= -0.5 ? n : scl(n, -1.0);
    const double a = 1.0 / (1.0 + m.z), b = -m.x * m.y * a;
    const V3<double> t1{1.0 - m.x * m.x * a, b, -m.x}, t2{b, 1.0 - m.y * m.y * a, -m.y};
    const double cs = 1.0 - u1, sn = std::sqrt(u1 * (2.0 - u1)), ph = 2.0 * PI * u2;
    return scl(t1, sn * std::cos(ph)) + scl(t2, sn * std::sin(ph)) + scl(n, cs);
}
// theta_hat(k), phi_hat(k) of a direction (Eq. spherical_vecs); poles: phi = 0.
inline void sph_basis(const V3<double>& k, V3<double>* th, V3<double>* ph) {
    const double t = std::acos(std::max(-1.0, std::min(1.0, k.z)));
    const double p = std::atan2(k.y, k.x);
    *th = theta_hat(t, p);
    *ph = phi_hat(p);
}
bool scat_valid(const Scene& S) {
    for (size_t m = 0; m < S.scS.size(); ++m) {
        if (!(S.scS[m] >= 0.0 && S.scS[m] <= 1.0) || !(S.scK[m] >= 0.0 && S.scK[m] <= 1.0)) return false;
        if (S.scPat[m] < 0 || S.scPat[m] > 2 || S.scAR[m] < 1 || S.scAR[m] > 32 || S.scAI[m] < 1 ||
            S.scAI[m] > 32 || !(S.scLam[m] >= 0.0 && S.scLam[m] <= 1.0))
            return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// the SBR loop for one lattice ray
// ---------------------------------------------------------------------------
struct TxC {
    Rot R;
    int pattern, pol;
    int64_t N;
    uint64_t seed;
    // synthetic array: element positions in the global frame (R d) and precoding
    std::vector<V3<double>> ant;
    std::vector<std::complex<double>> prec;
};

// Array factor of a synthetic transmit array for departure direction k
// (Sec. 4.4 with the array response vector of Eq. path-solver-array-response-vector):
//   alpha = sum_k u_P,k exp(j (2 pi / lambda0) k^T d_k).
// The non-coherent map sees |alpha|^2 times the single-antenna power.
std::complex<double> array_factor(const TxC& T, const V3<double>& k, double k0) {
    if (T.ant.empty()) return {1.0, 0.0};
    std::complex<double> a(0.0, 0.0);
    for (size_t i = 0; i < T.ant.size(); ++i) {
        const double ph = k0 * dot(k, T.ant[i]);
        a += T.prec[i] * std::complex<double>(std::cos(ph), std::sin(ph));
    }
    return a;
}

// Array-factor conditioning (test bookkeeping only; it does not enter the map).
// A deposit's value is |alpha|^2 times the single-antenna value; an FP32
// evaluation of alpha that carries the direction and each element's phase in
// double-float (hi + lo) arithmetic keeps, per element:
//   - a direction error below 2^-40 per component, i.e. a phase error below
//     k0 2^-40 |d_i|_1;
//   - the rounding of the reduced phase (a few units of 2^-24 pi) and of the
//     sine and cosine (2^-22);
//   - when elements on a regular line are summed by a Horner recurrence in
//     blocks of B = 16, the powers z^m (m < B) of z = exp(j k0 k.delta):
//     m (2^-24 pi + 2^-23 + 4 * 2^-24) of phase and modulus;
// and the sums over N elements add (B + N / B + 2) 2^-24 sum_i |w_i|.  With
//   delta = sum_i |w_i| eps_i + (B + N / B + 2) 2^-24 sum_i |w_i|,
//   eps_i = 15 (2^-24 pi + 2^-23 + 2^-22) + 8 pi 2^-24 + 2^-22 + k0 2^-40 |d_i|_1,
// |alpha|^2 moves by at most 2 |alpha| delta + delta^2; the factor returned is
// that over |alpha|^2 (0 for a single antenna).
double array_cond(const TxC& T, const V3<double>& k, double k0, const std::complex<double>& a) {
    (void)k;
    if (T.ant.empty()) return 0.0;
    const double u = 0x1p-24, B = 16.0;
    const double eps0 = 15.0 * (u * PI + 2.0 * u + 4.0 * u) + 8.0 * PI * u + 4.0 * u;
    double sw = 0.0, ew = 0.0;
    for (size_t i = 0; i < T.ant.size(); ++i) {
        const V3<double>& d = T.ant[i];
        const double aw = std::abs(T.prec[i]);
        sw += aw;
        ew += aw * (eps0 + k0 * 0x1p-40 * (std::fabs(d.x) + std::fabs(d.y) + std::fabs(d.z)));
    }
    const double n = (double)T.ant.size();
    const double delta = ew + (B + n / B + 2.0) * u * sw;
    const double a2 = std::norm(a);
    return (2.0 * std::sqrt(a2) * delta + delta * delta) / std::max(a2, 1e-300);
}

TxC make_txc(const or_tx& t) {
    TxC T;
    T.R = rotation(t.yaw, t.pitch, t.roll);
    T.pattern = t.pattern;
    T.pol = t.pol;
    T.N = t.num_rays;
    T.seed = t.seed;
    for (int64_t i = 0; i < t.n_ant; ++i) {
        T.ant.push_back(mul(T.R, V3<double>{t.ant_pos[3 * i], t.ant_pos[3 * i + 1], t.ant_pos[3 * i + 2]}));
        T.prec.emplace_back(t.precoding[2 * i], t.precoding[2 * i + 1]);
    }
    return T;
}

// ---------------------------------------------------------------------------
// mesh-based measurement surface (Sec. 4, practical notes): every triangle of
// a separate mesh is one cell.  The estimator is the planar one with the
// cell's own area A_i and unit normal n_i in the change of variables
// dA = r^2 / |n_i . k| d omega: a crossing of triangle i adds
//   4 pi / (N A_i) (lambda0 / 4 pi)^2 |E|^2 / (|n_i . k| Pr)
// to cell i, for every crossing of the open segment (1e-9, t_h).  The surface
// does not stop or deflect rays.  A crossing exactly on an edge shared by two
// triangles counts for both (a set of measure zero).
// ---------------------------------------------------------------------------
struct MeshSurface {
    std::vector<V3<double>> a, e1, e2;  // vertex a, edges b - a, c - a
    std::vector<double> inv_area, max_edge;
    int64_t n = 0;
};
MeshSurface make_surface(const float* verts, const int32_t* tris, int64_t nt) {
    MeshSurface M;
    M.n = nt;
    for (int64_t i = 0; i < nt; ++i) {
        auto v = [&](int j) {
            const float* q = verts + 3 * (int64_t)tris[3 * i + j];
            return V3<double>{q[0], q[1], q[2]};
        };
        V3<double> a = v(0), b = v(1), c = v(2);
        V3<double> e1 = b - a, e2 = c - a;
        V3<double> cr = cross(e1, e2);
        double area = 0.5 * std::sqrt(dot(cr, cr));
        M.a.push_back(a);
        M.e1.push_back(e1);
        M.e2.push_back(e2);
        M.inv_area.push_back(area > 0.0 ? 1.0 / area : 0.0);
        double le = std::max(std::sqrt(dot(e1, e1)), std::max(std::sqrt(dot(e2, e2)), std::sqrt(dot(c - b, c - b))));
        M.max_edge.push_back(le);
    }
    return M;
}

struct Ctx {
    const Scene* S;
    const MeshSurface* meas = nullptr;  // mesh measurement surface, or null for the plane
    double Kmesh = 0.0;                 // 4 pi / N (lambda0 / 4 pi)^2
    MapGeom g;
    double omega, k0;  // angular frequency, vacuum wavenumber
    int L, flags;
    int mode;
    // early termination (Sec. 4.5)
    int rr_depth = 0;
    double rr_pmax = 0.0, gain_thr = 0.0, lam4pi2 = 0.0;
    // sampling materials (detached q): eps, sigma
    const double* s_eps;
    const double* s_sig;
};

// Tolerance (m) for certifying a discrete near-tie in replay-check mode.
// FP32 carries a unit roundoff of 6e-8; positions accumulate O(10) roundings
// per bounce relative to the coordinate magnitude and the distance travelled,
// so 1e-5 * (1 m + |p|_inf + path length) is a >10x margin.
inline double tie_tol(const V3<double>& p, double path) {
    double pm = std::max(std::fabs(p.x), std::max(std::fabs(p.y), std::fabs(p.z)));
    return 1e-5 * (1.0 + pm + path);
}

struct ReplayState {
    or_report rep;
    void fail(int64_t ray, int depth, int kind, double a, double b, double c, double d) {
        if (rep.failures == 0) {
            rep.fail_ray = ray;
            rep.fail_depth = depth;
            rep.fail_kind = kind;
            rep.fail_info[0] = a; rep.fail_info[1] = b; rep.fail_info[2] = c; rep.fail_info[3] = d;
        }
        rep.failures++;
    }
};

// Is the GPU's choice of closest primitive (pg; -1 = miss) consistent with
// FP64 up to a perturbation of size tol?  pg must be a near-hit no farther
// than every robust hit (margin >= +tol) by more than tol.
bool certify_hit(const Scene& S, const V3<double>& o, const V3<double>& k, int exclude, int pg,
                 double path, double* tg) {
    double tgv = INFINITY;
    if (pg >= 0) {
        if (pg == exclude || pg >= (int)S.tris.size()) return false;
        double t, m;
        if (!plane_hit(S.tris[pg], o, k, &t, &m)) return false;
        V3<double> p = o + scl(k, t);
        double tol = tie_tol(p, path + std::max(t, 0.0));
        if (!(t > -tol) || m < -tol) return false;
        tgv = t;
    }
    for (int i = 0; i < (int)S.tris.size(); ++i) {
        if (i == exclude || i == pg) continue;
        double t, m;
        if (!plane_hit(S.tris[i], o, k, &t, &m)) continue;
        if (!(t > 0.0)) continue;
        V3<double> p = o + scl(k, t);
        double tol = tie_tol(p, path + t);
        if (m >= tol && t < tgv - tol) return false;  // a robust hit clearly in front
    }
    *tg = tgv;
    return true;
}

// Field of the ray tube a diffuse reflection spawns in direction ks (Eq.
// scattered_field), for an incident field E travelling along k: the theta/phi
// components of E (basis of k) are mixed by the cross-polarisation matrix
// with random phases chi_1, chi_2, mapped onto the theta/phi basis of ks and
// scaled by S Gamma sqrt(2 pi f_s), with
//   Gamma^2 = (|r_perp E_perp|^2 + |r_par E_par|^2) / |E|^2
// from the unreduced reflection coefficients of cf (e_perp, e_par,i: ep, epi).
// The sqrt(2 pi f_s) collects the sqrt(f_s cos theta_i dA) of the model and the
// weight 2 pi r^2 / |n.k_i| the estimator gives a diffuse point (Sec. 4): the
// tube length and cos theta_i cancel.
template <class R>
CV3<R> diffuse_field(const V3<double>& k, const V3<double>& ks, const V3<double>& ep, const V3<double>& epi,
                     const Coefs<R>& cf, double Sd, double Kx, double fs, double chi1, double chi2,
                     const CV3<R>& E) {
    CV3<R> out;
    const Cx<R> a = cdot(ep, E), b = cdot(epi, E);
    const R g2 = abs2(cf.r_perp * a) + abs2(cf.r_par * b);
    const R e2 = cnorm2(E);
    if (!(val(e2) > 0.0 && val(g2) > 0.0 && fs > 0.0)) return out;
    const R c = r_sqrt(g2 / e2) * (Sd * std::sqrt(2.0 * PI * fs));
    const double sK = std::sqrt(Kx), cK = std::sqrt(1.0 - Kx);
    const Cx<R> ph1(R(std::cos(chi1)), R(std::sin(chi1))), ph2(R(std::cos(chi2)), R(std::sin(chi2)));
    V3<double> thi, phi_i, ths, phs;
    sph_basis(k, &thi, &phi_i);
    sph_basis(ks, &ths, &phs);
    const Cx<R> Et = cdot(thi, E), Ef = cdot(phi_i, E);
    const Cx<R> As = (Et * R(cK) - Ef * R(sK)) * ph1 * c;
    const Cx<R> Bs = (Et * R(sK) + Ef * R(cK)) * ph2 * c;
    return outer(ths, As) + outer(phs, Bs);
}

template <class R, class SinkT>
void trace_ray(const Ctx& C, const TxC& tx, const V3<R>& txpos, const Cx<R>* eta, const R* k0d,
               int64_t n, int64_t i_sub, Rec* rec_io, SinkT& sink, ReplayState* rs,
               double* pw, double* pw2, double* esc) {
    const Scene& S = *C.S;
    const int L = C.L;
    const int npol = (tx.pol == 2) ? 2 : 1;
    V3<double> k = fibonacci_dir(n, tx.N);
    CV3<R> E[2];
    const std::complex<double> alpha = array_factor(tx, k, C.k0);
    if (sink.want_acond()) sink.set_acond(array_cond(tx, k, C.k0, alpha));
    for (int p = 0; p < npol; ++p) {
        int pol = (tx.pol == 2) ? p : tx.pol;
        V3<double> f = tx_field(k, tx.R, tx.pattern, pol);
        E[p] = {Cx<R>(R(f.x * alpha.real()), R(f.x * alpha.imag())), Cx<R>(R(f.y * alpha.real()), R(f.y * alpha.imag())),
                Cx<R>(R(f.z * alpha.real()), R(f.z * alpha.imag()))};
    }
    V3<R> o = txpos;
    double inv_pr = 1.0;  // 1 / Pr(chi): detached from the parameters
    double path = 0.0;    // unfolded length (only used for tie tolerances)
    double tube = 0.0;    // length of the current ray tube (since the source or the last diffuse point)
    int prev = -1;
    int l = 0;
    for (; l <= L; ++l) {
        V3<double> ov = vval(o);
        Rec* rec = rec_io ? rec_io + (size_t)i_sub * (L + 1) + l : nullptr;
        // ---- closest hit -------------------------------------------------
        int prim;
        double th;
        if (C.mode == MODE_FROZEN) {
            prim = rec->prim;
            th = INFINITY;
            if (prim >= 0) {
                double m;
                plane_hit(S.tris[prim], ov, k, &th, &m);
            }
        } else {
            closest_hit(S, ov, k, prev, &prim, &th);
            if (C.mode == MODE_REPLAY) {
                rs->rep.segments++;
                if (rec->prim == -2) { rs->fail(i_sub, l, 4, prim, 0, 0, 0); return; }
                if (rec->prim != prim) {
                    double tg;
                    if (certify_hit(S, ov, k, prev, rec->prim, path, &tg)) {
                        rs->rep.adopted_hit++;
                        if (prim >= 0 && std::isfinite(tg) &&
                            std::fabs(tg - th) <= tie_tol(ov + scl(k, th), path + th))
                            rs->rep.adopted_hit_tie++;
                        prim = rec->prim;
                        th = tg;
                    } else {
                        rs->fail(i_sub, l, 1, prim, rec->prim, th, path);
                        return;
                    }
                }
            }
        }
        // exact (typed) hit distance along the frozen primitive's plane
        R t_h(INFINITY);
        if (prim >= 0) {
            const Tri& T = S.tris[prim];
            R num = R(dot(T.n, T.a)) - (o.x * T.n.x + o.y * T.n.y + o.z * T.n.z);
            t_h = num / dot(T.n, k);
        }
        double w2 = 0.0;
        for (int p = 0; p < npol; ++p) w2 += val(cnorm2(E[p]));
        const double pwr = w2 * inv_pr;
        if (pw) { pw[l] += pwr; pw2[l] += pwr * pwr; if (prim < 0) esc[l] += pwr; }
        // ---- deposit -------------------------------------------------------
        bool los_ok = (l > 0) || (C.flags & F_LOS);
        {
            if (C.meas) {
                // mesh measurement surface: every crossed triangle of the open
                // segment (1e-9, t_h); crossings within tol of a triangle's
                // boundary or of the window ends also go to the slack of that
                // triangle (FP32 may put them on the other side)
                if (los_ok) {
                    const MeshSurface& M = *C.meas;
                    R e2r(0.0);
                    for (int p = 0; p < npol; ++p) e2r = e2r + cnorm2(E[p]);
                    const double e2v = val(e2r);
                    const double th_v = prim >= 0 ? val(t_h) : INFINITY;
                    for (int64_t j = 0; j < M.n; ++j) {
                        if (M.inv_area[j] == 0.0) continue;
                        // Moeller-Trumbore in FP64
                        V3<double> pv = cross(k, M.e2[j]);
                        double det = dot(M.e1[j], pv);
                        if (det == 0.0) continue;
                        V3<double> tv = ov - M.a[j];
                        double u = dot(tv, pv) / det;
                        V3<double> qv = cross(tv, M.e1[j]);
                        double v = dot(k, qv) / det;
                        double t = dot(M.e2[j], qv) / det;
                        double w = 1.0 - u - v;
                        V3<double> pc = ov + scl(k, t);
                        double tol = tie_tol(pc, path + std::max(t, 0.0));
                        // barycentric slack: tol over the triangle's smallest altitude
                        double tb = tol * M.max_edge[j] * 0.5 * M.inv_area[j];
                        bool inside = u >= 0.0 && v >= 0.0 && w >= 0.0;
                        bool in_win = t > 1e-9 && t < th_v;
                        bool near_edge = std::min(u, std::min(v, w)) >= -tb && std::min(u, std::min(v, w)) <= tb;
                        bool near_win = std::fabs(t - 1e-9) <= tol || (std::isfinite(th_v) && std::fabs(t - th_v) <= tol);
                        double nk = std::fabs(det) * 0.5 * M.inv_area[j];  // |n_i . k| = |det| / |e1 x e2|
                        if (nk == 0.0) continue;
                        const double scale = C.Kmesh * M.inv_area[j] * inv_pr / nk;
                        const double value = e2v * scale;
                        if (inside && in_win) {
                            sink.add((int)j, e2r * scale);
                            if (rs) rs->rep.deposits++;
                        }
                        if ((near_edge && (in_win || near_win)) || ((inside || near_edge) && near_win))
                            sink.add_slack((int)j, value);
                    }
                }
                if (rec && C.mode == MODE_PLAIN) { rec->prim = prim; rec->ix = NO_CELL; rec->iy = NO_CELL; rec->dec = -1; }
                goto after_deposit;
            }
        }
        {
        Crossing<R> cr = crossing(C.g, o, k, prim >= 0 ? val(t_h) : INFINITY);
        int dix = NO_CELL, diy = NO_CELL;
        if (cr.valid && los_ok) { dix = cr.ix; diy = cr.iy; }
        if (C.mode == MODE_FROZEN) {
            dix = rec->ix; diy = rec->iy;
            if (dix != NO_CELL && !cr.valid) {
                // recompute the crossing point without the validity window
                R tc = (R(C.g.z) - o.z) / k.z;
                cr.x = o.x + tc * k.x;
                cr.y = o.y + tc * k.y;
            }
        } else if (C.mode == MODE_REPLAY) {
            if (rec->ix != dix || rec->iy != diy) {
                // certify: the crossing sits within tol of a cell boundary, the
                // map edge, the segment end or the minimum distance
                double tc = (k.z != 0.0) ? (C.g.z - ov.z) / k.z : INFINITY;
                V3<double> pc = ov + scl(k, std::isfinite(tc) ? tc : 0.0);
                double tol = tie_tol(pc, path + std::max(0.0, std::isfinite(tc) ? tc : 0.0));
                double sh = C.g.bilinear ? 0.5 : 0.0;
                double ux = (pc.x - C.g.x0) / C.g.cell - sh, uy = (pc.y - C.g.y0) / C.g.cell - sh;
                double bx = tol / C.g.cell;
                auto near_int = [&](double u) { return std::fabs(u - std::nearbyint(u)) <= bx; };
                bool ok = false;
                bool gpu_dep = rec->ix != NO_CELL, or_dep = dix != NO_CELL;
                double th_v = prim >= 0 ? val(t_h) : INFINITY;
                if (gpu_dep && or_dep) {
                    ok = std::abs(rec->ix - dix) <= 1 && std::abs(rec->iy - diy) <= 1 &&
                         (rec->ix == dix || near_int(ux)) && (rec->iy == diy || near_int(uy));
                } else if (los_ok && std::isfinite(tc)) {
                    // existence differs: the window ends or the map edge decide
                    bool near_end = std::fabs(tc - th_v) <= tol || std::fabs(tc) <= tol;
                    bool near_edge = near_int(ux) || near_int(uy);
                    ok = near_end || near_edge;
                    if (gpu_dep) {
                        int ex = (int)std::floor(ux), ey = (int)std::floor(uy);
                        ok = ok && std::abs(rec->ix - ex) <= 1 && std::abs(rec->iy - ey) <= 1;
                    }
                }
                if (!ok) { rs->fail(i_sub, l, 2, dix, diy, rec->ix, rec->iy); return; }
                rs->rep.adopted_cell++;
                dix = rec->ix; diy = rec->iy;
                if (gpu_dep && !cr.valid) {
                    R tcr = (R(C.g.z) - o.z) / k.z;
                    cr.x = o.x + tcr * k.x;
                    cr.y = o.y + tcr * k.y;
                }
            }
        }
        if (rec && C.mode == MODE_PLAIN) { rec->prim = prim; rec->ix = dix; rec->iy = diy; rec->dec = -1; }
        if (dix != NO_CELL) {
            R e2(0.0);
            for (int p = 0; p < npol; ++p) e2 = e2 + cnorm2(E[p]);
            R value = e2 * (C.g.K * inv_pr / std::fabs(k.z));
            // A perturbation (d o, d k) of the segment moves x_c by at most
            //   (|d o| + t_c |d k|) (1 + (|k_x| + |k_y|) / |k_z|);
            // with |d o| ~ eps (1 + |o|_inf + path) and |d k| ~ eps this is
            // eps * cond with the cond below.
            const double tcv = (C.g.z - ov.z) / k.z;
            const double om = std::max(std::fabs(ov.x), std::max(std::fabs(ov.y), std::fabs(ov.z)));
            const double cond = (1.0 + om + path + std::fabs(tcv)) * (1.0 + (std::fabs(k.x) + std::fabs(k.y)) / std::fabs(k.z));
            deposit(C.g, cr, dix, diy, value, sink, cond);
            if (rs) rs->rep.deposits++;
        }
        }
    after_deposit:
        // ---- termination ---------------------------------------------------
        if (prim < 0 || l == L) break;
        // ---- shading (Sec. 3.1.2 sampling, App. A.7 field update) ---------
        const Tri& T = S.tris[prim];
        const int m = T.mat;
        // normal oriented towards the incident side (n . k < 0)
        V3<double> nn = dot(T.n, k) < 0.0 ? T.n : scl(T.n, -1.0);
        double cos1 = -dot(k, nn);
        cos1 = std::min(1.0, std::max(0.0, cos1));
        bool slab = S.thick[m] > 0.0;
        Coefs<R> cf = fresnel(eta[m], cos1, k0d[m], slab);
        // Diffuse reflection (App. A.10) takes the share S^2 of the reflected
        // power; the specular coefficients are reduced by R = sqrt(1 - S^2)
        // (Eq. R).  Sampling (Eq. path-solver-used-dist-event, q(D) = 0):
        // q(R) = R^2 wR / (wR + wT), q(S) = S^2 wR / (wR + wT), q(T) = wT / (wR + wT)
        // with wR, wT the squared magnitudes of the unreduced coefficients.
        // The coin: u < q(R) -> R, else u < wR / (wR + wT) -> S, else T.
        const double Sd = ((C.flags & F_DIFFUSE) && (C.flags & F_REFLECT)) ? S.scS[m] : 0.0;
        const double R2 = (1.0 - Sd) * (1.0 + Sd);
        const double Rred = std::sqrt(R2);
        double c1, c2, qR, qS, qT;
        const Cx<double> es = permittivity(C.s_eps[m], C.s_sig[m], C.omega);
        const double kd = C.k0 * S.thick[m];
        {
            Coefs<double> cs = fresnel(es, cos1, kd, slab);
            double wR = (C.flags & F_REFLECT) ? abs2(cs.r_perp) + abs2(cs.r_par) : 0.0;
            double wT = (C.flags & F_REFRACT) ? abs2(cs.t_perp) + abs2(cs.t_par) : 0.0;
            if (!(wR + wT > 0.0)) {
                if (rec && C.mode == MODE_PLAIN) rec->dec = -1;
                if (C.mode == MODE_REPLAY && rec->dec != -1) rs->fail(i_sub, l, 3, -1, rec->dec, 0, 0);
                break;
            }
            c2 = wR / (wR + wT);
            c1 = R2 * c2;
            qR = c1;
            qS = Sd * Sd * c2;
            qT = wT / (wR + wT);
        }
        double u = rng_u(tx.seed, (uint64_t)n, l);
        int dec = (u < c1) ? 0 : (u < c2 ? 2 : 1);
        // The replay's decision window: 1e-5, plus for a slab the change of the
        // interval bounds when the slab phase (2 pi d / lambda0) s (App. A.7)
        // moves by 2^-20 of itself: an FP32 phase of ~300 rad, from an FP32 s
        // and incidence angle, is good to a few units of 2^-24
        auto window = [&]() {
            double tol = 1e-5;
            if (slab)
                for (double f : {1.0 - 0x1p-20, 1.0 + 0x1p-20}) {
                    const Coefs<double> cp = fresnel(es, cos1, kd * f, slab);
                    const double wR = (C.flags & F_REFLECT) ? abs2(cp.r_perp) + abs2(cp.r_par) : 0.0;
                    const double wT = (C.flags & F_REFRACT) ? abs2(cp.t_perp) + abs2(cp.t_par) : 0.0;
                    if (!(wR + wT > 0.0)) continue;
                    const double c2p = wR / (wR + wT), c1p = R2 * c2p;
                    tol = std::max(tol, 1e-5 + std::max(std::fabs(c1p - c1), std::fabs(c2p - c2)));
                }
            return tol;
        };
        if (C.mode == MODE_REPLAY && rec->dec >= 256) {
            // the GPU recorded the q(R) its coin used: it must lie in the window
            const double qg = (double)(rec->dec >> 8) * 0x1p-22;
            const double dev = std::fabs(qg - c1), w = window();
            rs->rep.coin_checked++;
            rs->rep.coin_max_dev = std::max(rs->rep.coin_max_dev, dev);
            rs->rep.coin_max_ratio = std::max(rs->rep.coin_max_ratio, dev / w);
            if (dev > w) rs->rep.coin_outside++;
        }
        if (C.mode == MODE_FROZEN) {
            dec = rec->dec & 3;
        } else if (C.mode == MODE_REPLAY) {
            if ((rec->dec & 3) != dec) {
                // adopt the GPU's choice g if u lies within the window of g's
                // interval [lo, hi) of positive probability
                const int g = rec->dec & 3;
                const double lo = g == 0 ? 0.0 : (g == 2 ? c1 : c2);
                const double hi = g == 0 ? c1 : (g == 2 ? c2 : 1.0);
                const double tol = window();
                if (rec->dec >= 0 && g != 3 && hi > lo && u > lo - tol && u < hi + tol) {
                    rs->rep.adopted_decision++;
                    dec = g;
                } else {
                    rs->fail(i_sub, l, 3, dec, rec->dec, u, dec == 0 || g == 0 ? c1 : c2);
                    return;
                }
            }
        } else if (rec) {
            rec->dec = dec;
        }
        // TE/TM basis: e_perp = k x n / |k x n|, e_par,i = e_perp x k.
        // At normal incidence any transverse basis is valid (the field update
        // is then independent of the choice); take e_perp from the axis least
        // aligned with k.
        V3<double> kxn = cross(k, nn);
        double kxn_n = norm(kxn);
        V3<double> ep;
        if (kxn_n > 1e-12) {
            ep = scl(kxn, 1.0 / kxn_n);
        } else {
            V3<double> ax = std::fabs(k.x) < 0.5 ? V3<double>{1, 0, 0} : V3<double>{0, 1, 0};
            ep = unit(cross(k, ax));
        }
        V3<double> epi = cross(ep, k);
        V3<double> k_out;
        if (dec == 2) {
            // Diffuse reflection: a new ray tube in a uniformly sampled direction
            // of the incident-side hemisphere.  Its field follows Eq.
            // scattered_field with Gamma^2 = (|r_perp E_perp|^2 + |r_par E_par|^2) / |E|^2
            // (unreduced r), the cross-polarisation split K_x and the random
            // phases chi_1, chi_2 = 2 pi u.  The estimator (Sec. 4, weight
            // 2 pi r^2 / |n.k_i| per diffuse point) cancels the tube length and
            // cos theta_i against Eq. scattered_field's 1/r and
            // sqrt(cos theta_i dA), which leaves the factor sqrt(2 pi f_s).
            k_out = diffuse_dir(nn, rng_diff(tx.seed, (uint64_t)n, l, 0), rng_diff(tx.seed, (uint64_t)n, l, 1));
            const double fs = scat_pattern(S.scPat[m], S.scAR[m], S.scAI[m], S.scLam[m], k, k_out, nn);
            const double x1 = 2.0 * PI * rng_diff(tx.seed, (uint64_t)n, l, 2);
            const double x2 = 2.0 * PI * rng_diff(tx.seed, (uint64_t)n, l, 3);
            for (int p = 0; p < npol; ++p) E[p] = diffuse_field(k, k_out, ep, epi, cf, Sd, S.scK[m], fs, x1, x2, E[p]);
            inv_pr /= qS;
        } else {
            V3<double> epo;
            Cx<R> cperp, cpar;
            if (dec == 0) {
                k_out = k - scl(nn, 2.0 * dot(k, nn));
                epo = unit(cross(ep, k_out));
                cperp = cf.r_perp * R(Rred);
                cpar = cf.r_par * R(Rred);
                inv_pr /= qR;
            } else {
                k_out = k;  // thin slab: no deflection (Sec. 2.3)
                epo = epi;
                cperp = cf.t_perp;
                cpar = cf.t_par;
                inv_pr /= qT;
            }
            for (int p = 0; p < npol; ++p) {
                Cx<R> a = cdot(ep, E[p]);
                Cx<R> b = cdot(epi, E[p]);
                E[p] = outer(ep, cperp * a) + outer(epo, cpar * b);
            }
        }
        // new origin: hit point pushed off the surface along the outgoing side.
        // Reading (paper silent): offset 2^-16 * max(1, |p|_inf) metres.
        V3<R> ph = axpy(o, t_h, k);
        V3<double> phv = vval(ph);
        const R* big = &ph.x;
        if (std::fabs(phv.y) > std::fabs(val(*big))) big = &ph.y;
        if (std::fabs(phv.z) > std::fabs(val(*big))) big = &ph.z;
        R delta = std::fabs(val(*big)) > 1.0 ? r_abs(*big) * 0x1.0p-16 : R(0x1.0p-16);
        V3<double> nout = (dec == 1) ? scl(nn, -1.0) : nn;
        o = {ph.x + delta * nout.x, ph.y + delta * nout.y, ph.z + delta * nout.z};
        path += val(t_h);
        tube = (dec == 2) ? 0.0 : tube + val(t_h);  // a diffuse reflection starts a new tube
        k = k_out;
        prev = prim;
        // ---- early termination after rr_depth interactions (Sec. 4.5) ----
        // Reading: the gain of a sample is w |E|^2 with w = 1 / Pr(chi) (the
        // tube-length-normalised gain of the paper); gain thresholding stops a
        // path when (lambda0 / 4 pi)^2 w |E|^2 / r^2 < threshold at its tube
        // length r > 0 (a tube a diffuse reflection has just spawned has r = 0
        // and is not thresholded); Russian roulette (Eq. radio-map-solver-rr-prob) keeps it
        // with p = min(w |E|^2, p_max) and reweights the power of survivors by
        // 1 / p (the field by 1 / sqrt(p)); p is detached like q.
        if (C.rr_depth > 0 && l + 1 >= C.rr_depth && (C.gain_thr > 0.0 || C.rr_pmax > 0.0)) {
            double w2v = 0.0;
            for (int p = 0; p < npol; ++p) w2v += val(cnorm2(E[p]));
            w2v *= inv_pr;
            int kill = 0;
            if (C.gain_thr > 0.0 && tube > 0.0) {
                const double gain = C.lam4pi2 * w2v / (tube * tube);
                kill = gain < C.gain_thr ? 8 : 0;
                if (C.mode == MODE_FROZEN) {
                    kill = rec->dec & 8;
                } else if (C.mode == MODE_REPLAY && (rec->dec & 8) != kill) {
                    if (std::fabs(gain - C.gain_thr) <= 1e-5 * C.gain_thr) {
                        rs->rep.adopted_decision++;
                        kill = rec->dec & 8;
                    } else {
                        rs->fail(i_sub, l, 3, kill, rec->dec, gain, C.gain_thr);
                        return;
                    }
                }
            }
            if (!kill && C.rr_pmax > 0.0) {
                const double prr = std::min(w2v, C.rr_pmax);
                const double urr = rng_rr(tx.seed, (uint64_t)n, l);
                kill = (urr < prr) ? 0 : 4;
                if (C.mode == MODE_FROZEN) {
                    kill = rec->dec & 4;
                } else if (C.mode == MODE_REPLAY && (rec->dec & 4) != kill) {
                    if (std::fabs(urr - prr) <= 1e-5) {
                        rs->rep.adopted_decision++;
                        kill = rec->dec & 4;
                    } else {
                        rs->fail(i_sub, l, 3, kill, rec->dec, urr, prr);
                        return;
                    }
                }
                if (!kill) inv_pr /= prr;
            }
            if (rec && C.mode == MODE_PLAIN) rec->dec |= kill;
            if (kill) break;
        }
    }
    // remaining record slots: no segment
    if (rec_io && C.mode == MODE_PLAIN)
        for (int j = l + 1; j <= L; ++j) rec_io[(size_t)i_sub * (L + 1) + j] = Rec{-2, NO_CELL, NO_CELL, -1};
    if (C.mode == MODE_REPLAY)
        for (int j = l + 1; j <= L; ++j)
            if (rec_io[(size_t)i_sub * (L + 1) + j].prim != -2) { rs->fail(i_sub, j, 4, -2, rec_io[(size_t)i_sub * (L + 1) + j].prim, 0, 0); return; }
}

void set_early_termination(Ctx& C, const or_params& P) {
    C.rr_depth = P.rr_depth;
    C.rr_pmax = P.rr_max_prob;
    C.gain_thr = P.gain_threshold;
    const double a = C0 / P.freq_hz / (4.0 * PI);
    C.lam4pi2 = a * a;
}

MapGeom make_geom(const or_params& P, int64_t N) {
    MapGeom g;
    g.cell = P.cell_size;
    g.nx = P.nx;
    g.ny = P.ny;
    g.x0 = P.map_origin[0] - 0.5 * P.nx * P.cell_size;
    g.y0 = P.map_origin[1] - 0.5 * P.ny * P.cell_size;
    g.z = P.map_origin[2];
    g.bilinear = P.deposit == 1;
    double lam = C0 / P.freq_hz;
    double a = lam / (4.0 * PI);
    g.K = 4.0 * PI / ((double)N * P.cell_size * P.cell_size) * a * a;
    return g;
}

inline int64_t subset_count(const or_tx& t) {
    if (t.ray_count >= 0) return t.ray_count;
    return (t.num_rays - t.ray_begin + t.ray_stride - 1) / t.ray_stride;
}

}  // namespace

// ===========================================================================
// C entry points (loaded with ctypes by the tests)
// ===========================================================================
extern "C" {

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

double or_rng_u(uint64_t seed, uint64_t n, int l) { return rng_u(seed, n, l); }
double or_rng_diff(uint64_t seed, uint64_t n, int l, int j) { return rng_diff(seed, n, l, j & 3); }

// Diffuse-reflection pieces, for the pins.
double or_f_alpha(int alpha, double cos_i) { return f_alpha(alpha, cos_i); }
void or_scat_pattern(int pattern, int aR, int aI, double lam, const double* ki, const double* n,
                     const double* ks, int64_t count, double* out) {
    const V3<double> a{ki[0], ki[1], ki[2]}, nn{n[0], n[1], n[2]};
    for (int64_t i = 0; i < count; ++i)
        out[i] = scat_pattern(pattern, aR, aI, lam, a, {ks[3 * i], ks[3 * i + 1], ks[3 * i + 2]}, nn);
}
void or_diffuse_dir(const double* n, const double* u, int64_t count, double* out) {
    const V3<double> nn{n[0], n[1], n[2]};
    for (int64_t i = 0; i < count; ++i) {
        V3<double> d = diffuse_dir(nn, u[2 * i], u[2 * i + 1]);
        out[3 * i] = d.x; out[3 * i + 1] = d.y; out[3 * i + 2] = d.z;
    }
}
uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

void or_fibonacci(int64_t N, int64_t begin, int64_t count, int64_t stride, double* out) {
    for (int64_t i = 0; i < count; ++i) {
        V3<double> k = fibonacci_dir(begin + i * stride, N);
        out[3 * i] = k.x; out[3 * i + 1] = k.y; out[3 * i + 2] = k.z;
    }
}

void or_tx_field(const double* dirs, int64_t n, double yaw, double pitch, double roll,
                 int pattern, int pol, double* out) {
    Rot R = rotation(yaw, pitch, roll);
    for (int64_t i = 0; i < n; ++i) {
        V3<double> f = tx_field({dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2]}, R, pattern, pol);
        out[3 * i] = f.x; out[3 * i + 1] = f.y; out[3 * i + 2] = f.z;
    }
}

void or_rotation(double yaw, double pitch, double roll, double* out9) {
    Rot R = rotation(yaw, pitch, roll);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out9[3 * i + j] = R.m[i][j];
}

void or_csqrt(double re, double im, double* out) {
    Cx<double> z = csqrt(Cx<double>(re, im));
    out[0] = z.re; out[1] = z.im;
}

// out[8] = r_perp, r_par, t_perp, t_par (re, im).  k0d <= 0: half-space.
void or_fresnel(double eps_r, double sigma, double omega, double cos1, double k0d, double* out) {
    Cx<double> eta = permittivity(eps_r, sigma, omega);
    Coefs<double> c = fresnel(eta, cos1, k0d, k0d > 0.0);
    Cx<double> v[4] = {c.r_perp, c.r_par, c.t_perp, c.t_par};
    for (int i = 0; i < 4; ++i) { out[2 * i] = v[i].re; out[2 * i + 1] = v[i].im; }
}

void or_fresnel_vac_t(double eps_r, double sigma, double omega, double cos1, double* out) {
    Cx<double> eta = permittivity(eps_r, sigma, omega);
    Cx<double> a, b;
    fresnel_vac_t(eta, cos1, &a, &b);
    out[0] = a.re; out[1] = a.im; out[2] = b.re; out[3] = b.im;
}

// Field update at one interface, for the pins: incident direction k, surface
// normal n (any sign), incident field E (complex, 6 doubles), decision (0 R,
// 1 T).  Writes the outgoing direction (3) and field (6).
void or_interact(const double* k3, const double* n3, const double* E6, double eps_r, double sigma,
                 double omega, double k0d, int dec, double* kout, double* Eout) {
    V3<double> k{k3[0], k3[1], k3[2]}, n{n3[0], n3[1], n3[2]};
    n = unit(n);
    V3<double> nn = dot(n, k) < 0.0 ? n : scl(n, -1.0);
    double cos1 = std::min(1.0, std::max(0.0, -dot(k, nn)));
    Coefs<double> cf = fresnel(permittivity(eps_r, sigma, omega), cos1, k0d, k0d > 0.0);
    V3<double> kxn = cross(k, nn);
    double kn = norm(kxn);
    V3<double> ep;
    if (kn > 1e-12) ep = scl(kxn, 1.0 / kn);
    else {
        V3<double> ax = std::fabs(k.x) < 0.5 ? V3<double>{1, 0, 0} : V3<double>{0, 1, 0};
        ep = unit(cross(k, ax));
    }
    V3<double> epi = cross(ep, k);
    V3<double> ko = dec == 0 ? k - scl(nn, 2.0 * dot(k, nn)) : k;
    V3<double> epo = dec == 0 ? unit(cross(ep, ko)) : epi;
    CV3<double> E{Cx<double>(E6[0], E6[1]), Cx<double>(E6[2], E6[3]), Cx<double>(E6[4], E6[5])};
    Cx<double> a = cdot(ep, E), b = cdot(epi, E);
    CV3<double> Eo = dec == 0 ? outer(ep, cf.r_perp * a) + outer(epo, cf.r_par * b)
                              : outer(ep, cf.t_perp * a) + outer(epo, cf.t_par * b);
    kout[0] = ko.x; kout[1] = ko.y; kout[2] = ko.z;
    Eout[0] = Eo.x.re; Eout[1] = Eo.x.im; Eout[2] = Eo.y.re; Eout[3] = Eo.y.im;
    Eout[4] = Eo.z.re; Eout[5] = Eo.z.im;
}

// A diffuse reflection at one interface, for the pins: incident direction k,
// normal n (any sign), field E (6 doubles), material (eps_r, sigma, k0d),
// scattering parameters and the four variates u4 (direction, phases).
// Writes the scattered direction (3) and field (6).
void or_diffuse_interact(const double* k3, const double* n3, const double* E6, double eps_r, double sigma,
                         double omega, double k0d, double Sd, double Kx, int pattern, int aR, int aI, double lam,
                         const double* u4, double* kout, double* Eout) {
    V3<double> k{k3[0], k3[1], k3[2]}, n{n3[0], n3[1], n3[2]};
    n = unit(n);
    V3<double> nn = dot(n, k) < 0.0 ? n : scl(n, -1.0);
    double cos1 = std::min(1.0, std::max(0.0, -dot(k, nn)));
    Coefs<double> cf = fresnel(permittivity(eps_r, sigma, omega), cos1, k0d, k0d > 0.0);
    V3<double> kxn = cross(k, nn);
    double kn = norm(kxn);
    V3<double> ep;
    if (kn > 1e-12) ep = scl(kxn, 1.0 / kn);
    else {
        V3<double> ax = std::fabs(k.x) < 0.5 ? V3<double>{1, 0, 0} : V3<double>{0, 1, 0};
        ep = unit(cross(k, ax));
    }
    V3<double> epi = cross(ep, k);
    V3<double> ks = diffuse_dir(nn, u4[0], u4[1]);
    double fs = scat_pattern(pattern, aR, aI, lam, k, ks, nn);
    CV3<double> E{Cx<double>(E6[0], E6[1]), Cx<double>(E6[2], E6[3]), Cx<double>(E6[4], E6[5])};
    CV3<double> Eo = diffuse_field(k, ks, ep, epi, cf, Sd, Kx, fs, 2.0 * PI * u4[2], 2.0 * PI * u4[3], E);
    kout[0] = ks.x; kout[1] = ks.y; kout[2] = ks.z;
    Eout[0] = Eo.x.re; Eout[1] = Eo.x.im; Eout[2] = Eo.y.re; Eout[3] = Eo.y.im;
    Eout[4] = Eo.z.re; Eout[5] = Eo.z.im;
}

// Closest hit of a batch of rays (brute force), for the pins.
void or_closest_hit(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                    const double* o, const double* k, int64_t nrays, const int32_t* exclude,
                    int32_t* prim_out, double* t_out) {
    std::vector<int32_t> mat(nt, 0);
    float dummy[3] = {1, 0, 0};
    Scene S = make_scene(verts, nv, tris, nt, mat.data(), dummy, 1);
    for (int64_t i = 0; i < nrays; ++i) {
        int p;
        double t;
        closest_hit(S, {o[3 * i], o[3 * i + 1], o[3 * i + 2]}, {k[3 * i], k[3 * i + 1], k[3 * i + 2]},
                    exclude ? exclude[i] : -1, &p, &t);
        prim_out[i] = p;
        t_out[i] = t;
    }
}

// Radio map of one transmitter.
//   mode 0 plain:  RNG decisions; writes rec (if non-null) and the map;
//   mode 1 replay: follows the given record, certifying every differing
//                  discrete choice as an FP64 near-tie (report.failures = 0
//                  when all differences are certified);
//   mode 2 frozen: takes hits, cells and decisions from rec.
// sampling_mats (nm x 2: eps, sigma) or null = the scene's own materials;
// eval_mats likewise overrides the materials the fields are evaluated with.
// map_out [ny][nx] is overwritten.  stats (or null): per depth 0..L
// [power, power^2, escaped power] sums of w |E|^2 (without the 4 pi / N factor).
// mass_out (or null) [3][ny][nx]: per cell, the sum of the unweighted values
// of the deposits whose stencil covers it, the same sum with every value
// multiplied by its crossing's conditioning factor, and with every value
// multiplied by its ray's array-factor conditioning (test error bounds).
int or_radio_map(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                 const int32_t* tri_mat, const float* mats, int nm, const float* scat, const or_tx* tx,
                 const or_params* P, int mode, int32_t* rec, const double* sampling_mats,
                 const double* eval_mats, double* map_out, double* stats, or_report* report,
                 double* mass_out) {
    if (P->max_depth < 0 || P->max_depth > 15) return 1;
    Scene S = make_scene(verts, nv, tris, nt, tri_mat, mats, nm, scat);
    if (!scat_valid(S)) return 2;
    if (eval_mats)
        for (int m = 0; m < nm; ++m) { S.eps[m] = eval_mats[2 * m]; S.sigma[m] = eval_mats[2 * m + 1]; }
    std::vector<double> seps(S.eps), ssig(S.sigma);
    if (sampling_mats)
        for (int m = 0; m < nm; ++m) { seps[m] = sampling_mats[2 * m]; ssig[m] = sampling_mats[2 * m + 1]; }
    Ctx C;
    C.S = &S;
    C.g = make_geom(*P, tx->num_rays);
    C.omega = 2.0 * PI * P->freq_hz;
    C.k0 = C.omega / C0;
    C.L = P->max_depth;
    C.flags = P->flags;
    C.mode = mode;
    C.s_eps = seps.data();
    C.s_sig = ssig.data();
    set_early_termination(C, *P);
    TxC T = make_txc(*tx);
    std::vector<Cx<double>> eta(nm);
    std::vector<double> k0d(nm);
    for (int m = 0; m < nm; ++m) {
        eta[m] = permittivity(S.eps[m], S.sigma[m], C.omega);
        k0d[m] = C.k0 * S.thick[m];
    }
    V3<double> pos{tx->pos[0], tx->pos[1], tx->pos[2]};
    const int64_t cnt = subset_count(*tx);
    const int L = P->max_depth;
    const int64_t CH = 2048;  // fixed chunking: the summation order is independent of threads
    const int64_t nch = (cnt + CH - 1) / CH;
    std::vector<DepList> lists(nch), masses(mass_out ? nch : 0), cmasses(mass_out ? nch : 0),
        amasses(mass_out ? nch : 0);
    const int nthr = or_num_threads();
    std::vector<double> st((size_t)nthr * 3 * (L + 1), 0.0);
    std::vector<ReplayState> rss(nch);
    for (auto& r : rss) std::memset(&r.rep, 0, sizeof r.rep);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < nch; ++c) {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        double* sp = stats ? st.data() + (size_t)tid * 3 * (L + 1) : nullptr;
        Sink<double> sink{&lists[c], mass_out ? &masses[c] : nullptr, mass_out ? &cmasses[c] : nullptr};
        sink.amass = mass_out ? &amasses[c] : nullptr;
        int64_t e = std::min(cnt, (c + 1) * CH);
        for (int64_t i = c * CH; i < e; ++i) {
            int64_t n = tx->ray_begin + i * tx->ray_stride;
            trace_ray<double>(C, T, pos, eta.data(), k0d.data(), n, i, (Rec*)rec, sink,
                              mode == MODE_REPLAY ? &rss[c] : nullptr, sp, sp ? sp + (L + 1) : nullptr,
                              sp ? sp + 2 * (L + 1) : nullptr);
        }
    }
    std::memset(map_out, 0, sizeof(double) * (size_t)P->nx * P->ny);
    for (int64_t c = 0; c < nch; ++c)
        for (size_t j = 0; j < lists[c].cell.size(); ++j) map_out[lists[c].cell[j]] += lists[c].val[j];
    if (mass_out) {
        const size_t nc = (size_t)P->nx * P->ny;
        std::memset(mass_out, 0, sizeof(double) * 3 * nc);
        for (int64_t c = 0; c < nch; ++c) {
            for (size_t j = 0; j < masses[c].cell.size(); ++j) mass_out[masses[c].cell[j]] += masses[c].val[j];
            for (size_t j = 0; j < cmasses[c].cell.size(); ++j) mass_out[nc + cmasses[c].cell[j]] += cmasses[c].val[j];
            for (size_t j = 0; j < amasses[c].cell.size(); ++j)
                mass_out[2 * nc + amasses[c].cell[j]] += amasses[c].val[j];
        }
    }
    if (stats) {
        std::memset(stats, 0, sizeof(double) * 3 * (L + 1));
        for (int t = 0; t < nthr; ++t)
            for (int j = 0; j < 3 * (L + 1); ++j) stats[j] += st[(size_t)t * 3 * (L + 1) + j];
    }
    if (report) {
        std::memset(report, 0, sizeof *report);
        bool have_fail = false;
        for (int64_t c = 0; c < nch; ++c) {
            const or_report& r = rss[c].rep;
            report->segments += r.segments;
            report->deposits += r.deposits;
            report->adopted_hit += r.adopted_hit;
            report->adopted_cell += r.adopted_cell;
            report->adopted_decision += r.adopted_decision;
            report->adopted_hit_tie += r.adopted_hit_tie;
            report->failures += r.failures;
            report->coin_checked += r.coin_checked;
            report->coin_outside += r.coin_outside;
            report->coin_max_dev = std::max(report->coin_max_dev, r.coin_max_dev);
            report->coin_max_ratio = std::max(report->coin_max_ratio, r.coin_max_ratio);
            if (r.failures && !have_fail) {
                have_fail = true;
                report->fail_ray = r.fail_ray;
                report->fail_depth = r.fail_depth;
                report->fail_kind = r.fail_kind;
                std::memcpy(report->fail_info, r.fail_info, sizeof r.fail_info);
            }
        }
    }
    return 0;
}

// Radio map on a mesh measurement surface (one cell per surface triangle) of
// one transmitter, mode 0 plain or 1 replay (the map parameters of P other
// than frequency, depth, flags and early termination are unused).  map_out
// [n_surf] is overwritten; slack_out [n_surf] (or null) receives per cell the
// sum of the values of the crossings that lie within tol of its boundary or of
// a window end, whose cell FP32 arithmetic may decide otherwise.
int or_radio_map_mesh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tri_mat,
                      const float* mats, int nm, const float* scat, const or_tx* tx, const or_params* P,
                      const float* surf_verts, const int32_t* surf_tris, int64_t n_surf, int mode, int32_t* rec,
                      double* map_out, double* slack_out, or_report* report) {
    if (P->max_depth < 0 || P->max_depth > 15) return 1;
    if (mode != MODE_PLAIN && mode != MODE_REPLAY) return 3;
    Scene S = make_scene(verts, nv, tris, nt, tri_mat, mats, nm, scat);
    if (!scat_valid(S)) return 2;
    MeshSurface M = make_surface(surf_verts, surf_tris, n_surf);
    Ctx C;
    C.S = &S;
    C.meas = &M;
    C.g = make_geom(*P, tx->num_rays);
    C.omega = 2.0 * PI * P->freq_hz;
    C.k0 = C.omega / C0;
    const double a = C0 / P->freq_hz / (4.0 * PI);
    C.Kmesh = 4.0 * PI / (double)tx->num_rays * a * a;
    C.L = P->max_depth;
    C.flags = P->flags;
    C.mode = mode;
    std::vector<double> seps(S.eps), ssig(S.sigma);
    C.s_eps = seps.data();
    C.s_sig = ssig.data();
    set_early_termination(C, *P);
    TxC T = make_txc(*tx);
    std::vector<Cx<double>> eta(nm);
    std::vector<double> k0d(nm);
    for (int m = 0; m < nm; ++m) {
        eta[m] = permittivity(S.eps[m], S.sigma[m], C.omega);
        k0d[m] = C.k0 * S.thick[m];
    }
    V3<double> pos{tx->pos[0], tx->pos[1], tx->pos[2]};
    const int64_t cnt = subset_count(*tx);
    const int64_t CH = 2048;
    const int64_t nch = (cnt + CH - 1) / CH;
    std::vector<DepList> lists(nch), slacks(nch);
    std::vector<ReplayState> rss(nch);
    for (auto& r : rss) std::memset(&r.rep, 0, sizeof r.rep);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < nch; ++c) {
        Sink<double> sink{&lists[c]};
        sink.slack = slack_out ? &slacks[c] : nullptr;
        int64_t e = std::min(cnt, (c + 1) * CH);
        for (int64_t i = c * CH; i < e; ++i) {
            int64_t n = tx->ray_begin + i * tx->ray_stride;
            trace_ray<double>(C, T, pos, eta.data(), k0d.data(), n, i, (Rec*)rec, sink,
                              mode == MODE_REPLAY ? &rss[c] : nullptr, nullptr, nullptr, nullptr);
        }
    }
    std::memset(map_out, 0, sizeof(double) * (size_t)n_surf);
    for (int64_t c = 0; c < nch; ++c)
        for (size_t j = 0; j < lists[c].cell.size(); ++j) map_out[lists[c].cell[j]] += lists[c].val[j];
    if (slack_out) {
        std::memset(slack_out, 0, sizeof(double) * (size_t)n_surf);
        for (int64_t c = 0; c < nch; ++c)
            for (size_t j = 0; j < slacks[c].cell.size(); ++j) slack_out[slacks[c].cell[j]] += slacks[c].val[j];
    }
    if (report) {
        std::memset(report, 0, sizeof *report);
        bool have_fail = false;
        for (int64_t c = 0; c < nch; ++c) {
            const or_report& r = rss[c].rep;
            report->segments += r.segments;
            report->deposits += r.deposits;
            report->adopted_hit += r.adopted_hit;
            report->adopted_cell += r.adopted_cell;
            report->adopted_decision += r.adopted_decision;
            report->adopted_hit_tie += r.adopted_hit_tie;
            report->failures += r.failures;
            report->coin_checked += r.coin_checked;
            report->coin_outside += r.coin_outside;
            report->coin_max_dev = std::max(report->coin_max_dev, r.coin_max_dev);
            report->coin_max_ratio = std::max(report->coin_max_ratio, r.coin_max_ratio);
            if (r.failures && !have_fail) {
                have_fail = true;
                report->fail_ray = r.fail_ray;
                report->fail_depth = r.fail_depth;
                report->fail_kind = r.fail_kind;
                std::memcpy(report->fail_info, r.fail_info, sizeof r.fail_info);
            }
        }
    }
    return 0;
}

// Gradient of  sum_i dLdC[i] * C_i  with respect to (eps_r[m], sigma[m] for
// m < nm, tx position), with hits, cells and decisions frozen to rec (from a
// plain run) and the sampling probabilities detached.  Forward-mode dual
// numbers; nm <= 8.  grad_out: [nm] d/deps, [nm] d/dsigma, [3] d/dtx.
static int grad_impl(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tri_mat,
                     const float* mats, int nm, const float* scat, const or_tx* tx, const or_params* P,
                     const int32_t* rec, const double* dLdC, double* grad_out, const MeshSurface* meas) {
    if (nm > 8) return 1;
    Scene S = make_scene(verts, nv, tris, nt, tri_mat, mats, nm, scat);
    if (!scat_valid(S)) return 2;
    Ctx C;
    C.S = &S;
    C.meas = meas;
    if (meas) {
        const double a = C0 / P->freq_hz / (4.0 * PI);
        C.Kmesh = 4.0 * PI / (double)tx->num_rays * a * a;
    }
    C.g = make_geom(*P, tx->num_rays);
    C.omega = 2.0 * PI * P->freq_hz;
    C.k0 = C.omega / C0;
    C.L = P->max_depth;
    C.flags = P->flags;
    C.mode = MODE_FROZEN;
    C.s_eps = S.eps.data();
    C.s_sig = S.sigma.data();
    set_early_termination(C, *P);
    TxC T = make_txc(*tx);
    std::vector<Cx<D>> eta(nm);
    std::vector<D> k0d(nm);
    for (int m = 0; m < nm; ++m) {
        D e(S.eps[m]);
        e.g[m] = 1.0;
        D s(S.sigma[m]);
        s.g[8 + m] = 1.0;
        eta[m] = permittivity(e, s, C.omega);
        k0d[m] = D(C.k0 * S.thick[m]);
    }
    V3<D> pos{D(tx->pos[0]), D(tx->pos[1]), D(tx->pos[2])};
    pos.x.g[16] = 1.0;
    pos.y.g[17] = 1.0;
    pos.z.g[18] = 1.0;
    const int64_t cnt = subset_count(*tx);
    const int nthr = or_num_threads();
    std::vector<double> acc((size_t)nthr * NT, 0.0);
#pragma omp parallel
    {
#ifdef _OPENMP
        int tid = omp_get_thread_num();
#else
        int tid = 0;
#endif
        Sink<D> sink;
        sink.gmap = dLdC;
        std::memset(sink.acc, 0, sizeof sink.acc);
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < cnt; ++i) {
            int64_t n = tx->ray_begin + i * tx->ray_stride;
            trace_ray<D>(C, T, pos, eta.data(), k0d.data(), n, i, (Rec*)rec, sink, nullptr, nullptr,
                         nullptr, nullptr);
        }
        for (int j = 0; j < NT; ++j) acc[(size_t)tid * NT + j] = sink.acc[j];
    }
    double g[NT] = {};
    for (int t = 0; t < nthr; ++t)
        for (int j = 0; j < NT; ++j) g[j] += acc[(size_t)t * NT + j];
    for (int m = 0; m < nm; ++m) { grad_out[m] = g[m]; grad_out[nm + m] = g[8 + m]; }
    for (int j = 0; j < 3; ++j) grad_out[2 * nm + j] = g[16 + j];
    return 0;
}

int or_grad(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tri_mat,
            const float* mats, int nm, const float* scat, const or_tx* tx, const or_params* P,
            const int32_t* rec, const double* dLdC, double* grad_out) {
    return grad_impl(verts, nv, tris, nt, tri_mat, mats, nm, scat, tx, P, rec, dLdC, grad_out, nullptr);
}

// The same gradient for a map on a mesh measurement surface: dLdC [n_surf];
// crossings are recomputed along the frozen path (they do not depend on the
// materials; the cells are boxes, so the TX-position gradient is zero).
int or_grad_mesh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tri_mat,
                 const float* mats, int nm, const float* scat, const or_tx* tx, const or_params* P,
                 const float* surf_verts, const int32_t* surf_tris, int64_t n_surf, const int32_t* rec,
                 const double* dLdC, double* grad_out) {
    MeshSurface M = make_surface(surf_verts, surf_tris, n_surf);
    return grad_impl(verts, nv, tris, nt, tri_mat, mats, nm, scat, tx, P, rec, dLdC, grad_out, &M);
}

// ---------------------------------------------------------------------------
// Branch-all enumeration: both R and T are followed at every interaction with
// their full fields (no sampling, no 1/Pr), which is the exact expectation of
// the Monte-Carlo estimator over the interaction-type choices (Sec. 3.1.2 and
// the importance-sampling primer, App. E: E[|a|^2 / q] = sum over branches).
// power_out[l]: sum over all branches alive at segment l of |E|^2; escaped_out[l]:
// the part of it whose segment hits nothing.  (Multiply by 4 pi / N for
// power x solid angle.)
// ---------------------------------------------------------------------------
namespace {
struct BranchCtx {
    const Ctx* C;
    const Scene* S;
    const Cx<double>* eta;
    const double* k0d;
    int npol;
    DepList* list;
    double* pw;
    double* esc;
};
void branch(const BranchCtx& B, V3<double> o, V3<double> k, CV3<double>* E, int prev, int l) {
    const Ctx& C = *B.C;
    const Scene& S = *B.S;
    int prim;
    double th;
    closest_hit(S, o, k, prev, &prim, &th);
    double w2 = 0.0;
    for (int p = 0; p < B.npol; ++p) w2 += cnorm2(E[p]);
    B.pw[l] += w2;
    if (prim < 0) B.esc[l] += w2;
    bool los_ok = (l > 0) || (C.flags & F_LOS);
    Crossing<double> cr = crossing(C.g, o, k, prim >= 0 ? th : INFINITY);
    if (cr.valid && los_ok) {
        Sink<double> sink{B.list};
        deposit(C.g, cr, cr.ix, cr.iy, w2 * (C.g.K / std::fabs(k.z)), sink);
    }
    if (prim < 0 || l == C.L) return;
    const Tri& T = S.tris[prim];
    const int m = T.mat;
    V3<double> nn = dot(T.n, k) < 0.0 ? T.n : scl(T.n, -1.0);
    double cos1 = std::min(1.0, std::max(0.0, -dot(k, nn)));
    bool slab = S.thick[m] > 0.0;
    Coefs<double> cf = fresnel(B.eta[m], cos1, B.k0d[m], slab);
    V3<double> kxn = cross(k, nn);
    double kn = norm(kxn);
    V3<double> ep;
    if (kn > 1e-12) ep = scl(kxn, 1.0 / kn);
    else {
        V3<double> ax = std::fabs(k.x) < 0.5 ? V3<double>{1, 0, 0} : V3<double>{0, 1, 0};
        ep = unit(cross(k, ax));
    }
    V3<double> epi = cross(ep, k);
    V3<double> ph = o + scl(k, th);
    double pm = std::max(std::fabs(ph.x), std::max(std::fabs(ph.y), std::fabs(ph.z)));
    double delta = std::ldexp(std::max(1.0, pm), -16);
    double wR = (C.flags & F_REFLECT) ? abs2(cf.r_perp) + abs2(cf.r_par) : 0.0;
    double wT = (C.flags & F_REFRACT) ? abs2(cf.t_perp) + abs2(cf.t_par) : 0.0;
    for (int dec = 0; dec < 2; ++dec) {
        if ((dec == 0 ? wR : wT) <= 0.0) continue;
        V3<double> ko = dec == 0 ? k - scl(nn, 2.0 * dot(k, nn)) : k;
        V3<double> epo = dec == 0 ? unit(cross(ep, ko)) : epi;
        Cx<double> cp = dec == 0 ? cf.r_perp : cf.t_perp;
        Cx<double> cl = dec == 0 ? cf.r_par : cf.t_par;
        CV3<double> En[2];
        for (int p = 0; p < B.npol; ++p) {
            Cx<double> a = cdot(ep, E[p]), b = cdot(epi, E[p]);
            En[p] = outer(ep, cp * a) + outer(epo, cl * b);
        }
        V3<double> nout = dec == 0 ? nn : scl(nn, -1.0);
        branch(B, ph + scl(nout, delta), ko, En, prim, l + 1);
    }
}
}  // namespace

int or_branch_all(const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                  const int32_t* tri_mat, const float* mats, int nm, const or_tx* tx,
                  const or_params* P, double* map_out, double* power_out, double* escaped_out) {
    if (P->max_depth < 0 || P->max_depth > 12) return 1;
    // diffuse directions are continuous: they cannot be enumerated
    if (P->flags & F_DIFFUSE) return 3;
    Scene S = make_scene(verts, nv, tris, nt, tri_mat, mats, nm);
    Ctx C;
    C.S = &S;
    C.g = make_geom(*P, tx->num_rays);
    C.omega = 2.0 * PI * P->freq_hz;
    C.k0 = C.omega / C0;
    C.L = P->max_depth;
    C.flags = P->flags;
    C.mode = MODE_PLAIN;
    std::vector<Cx<double>> eta(nm);
    std::vector<double> k0d(nm);
    for (int m = 0; m < nm; ++m) {
        eta[m] = permittivity(S.eps[m], S.sigma[m], C.omega);
        k0d[m] = C.k0 * S.thick[m];
    }
    TxC T = make_txc(*tx);
    const Rot& R = T.R;
    const int npol = tx->pol == 2 ? 2 : 1;
    const int64_t cnt = subset_count(*tx);
    const int L = P->max_depth;
    const int64_t CH = 256;
    const int64_t nch = (cnt + CH - 1) / CH;
    std::vector<DepList> lists(nch);
    std::vector<double> pw((size_t)nch * (L + 1), 0.0), es((size_t)nch * (L + 1), 0.0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < nch; ++c) {
        BranchCtx B{&C, &S, eta.data(), k0d.data(), npol, &lists[c], pw.data() + c * (L + 1),
                    es.data() + c * (L + 1)};
        int64_t e = std::min(cnt, (c + 1) * CH);
        for (int64_t i = c * CH; i < e; ++i) {
            int64_t n = tx->ray_begin + i * tx->ray_stride;
            V3<double> k = fibonacci_dir(n, tx->num_rays);
            const std::complex<double> al = array_factor(T, k, C.k0);
            CV3<double> E[2];
            for (int p = 0; p < npol; ++p) {
                V3<double> f = tx_field(k, R, tx->pattern, tx->pol == 2 ? p : tx->pol);
                E[p] = {Cx<double>(f.x * al.real(), f.x * al.imag()), Cx<double>(f.y * al.real(), f.y * al.imag()),
                        Cx<double>(f.z * al.real(), f.z * al.imag())};
            }
            branch(B, {tx->pos[0], tx->pos[1], tx->pos[2]}, k, E, -1, 0);
        }
    }
    std::memset(map_out, 0, sizeof(double) * (size_t)P->nx * P->ny);
    for (int64_t c = 0; c < nch; ++c)
        for (size_t j = 0; j < lists[c].cell.size(); ++j) map_out[lists[c].cell[j]] += lists[c].val[j];
    for (int j = 0; j <= L; ++j) {
        power_out[j] = 0;
        escaped_out[j] = 0;
        for (int64_t c = 0; c < nch; ++c) { power_out[j] += pw[c * (L + 1) + j]; escaped_out[j] += es[c * (L + 1) + j]; }
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Reference LBVH.  Not in the paper (it relies on Mitsuba's acceleration
// structure); the tree here is the binary radix tree of Karras (HPG 2012) over
// the sorted Morton codes, built TOP-DOWN by splitting each range at its
// highest differing key bit -- a different algorithm from the GPU's
// per-node parallel construction that must give the identical tree.
//
// Morton codes, in FP32 with round-to-nearest and no fused operations (this
// file is compiled with -ffp-contract=off):
//   lo, hi   = per-triangle AABB (exact min / max of the FP32 vertices);
//   c2       = lo + hi                    (doubled centroid);
//   cmin/cmax= min / max of c2 over all triangles;
//   e        = max_a (cmax_a - cmin_a)     (one scale for the three axes, so
//              that the Morton order splits space isotropically: a flat city
//              does not spend a third of its top splits on height);
//   scale    = 2097151 / e                 (0 if e is 0);
//   q_a      = min(trunc((c2_a - cmin_a) * scale), 2097151);
//   key      = interleave(qx, qy, qz): bit i of qx -> bit 3i+2, qy -> 3i+1, qz -> 3i.
// Keys are sorted stably (ties keep triangle order); equal keys are told
// apart by their sorted position: delta(i, j) = clz64(k_i ^ k_j) if the keys
// differ, else 64 + clz32(i ^ j).  Internal node of range [a, b] with split g:
// left = leaf g if a == g else internal g; right = leaf g+1 if b == g+1 else
// internal g+1; the root is internal node 0.  Leaves are encoded as ~pos.
// ---------------------------------------------------------------------------
namespace {
inline uint64_t spread3(uint32_t v) {
    uint64_t r = 0;
    for (int i = 0; i < 21; ++i) r |= (uint64_t)((v >> i) & 1u) << (3 * i);
    return r;
}
inline int clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }
inline int clz32(uint32_t x) { return x ? __builtin_clz(x) : 32; }
}  // namespace

// Large triangles (the ground of a city) would inflate every box on their
// path to the root; they are kept out of the tree and tested from a short
// list instead.  A triangle is large when its largest AABB extent is at
// least a quarter of the scene AABB's largest extent (FP32: extents are
// hi - lo, the threshold 0.25f * scene extent), unless more than 16 are, in
// which case none is.  Large triangles get the key 2^64 - 1 (after every
// Morton code) and take no part in the Morton bounds.
constexpr int MAX_LARGE = 16;

void or_morton(const float* verts, const int32_t* tris, int64_t nt, uint64_t* keys_out,
               float* aabb_out /* [nt][6] lo, hi */, int64_t* nlarge_out) {
    std::vector<float> c2(3 * nt), box(6 * nt);
    float slo[3] = {INFINITY, INFINITY, INFINITY}, shi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nt; ++i) {
        for (int a = 0; a < 3; ++a) {
            float v0 = verts[3 * tris[3 * i] + a], v1 = verts[3 * tris[3 * i + 1] + a],
                  v2 = verts[3 * tris[3 * i + 2] + a];
            float lo = std::min(v0, std::min(v1, v2));
            float hi = std::max(v0, std::max(v1, v2));
            box[6 * i + a] = lo;
            box[6 * i + 3 + a] = hi;
            volatile float s = lo + hi;
            c2[3 * i + a] = s;
            slo[a] = std::min(slo[a], lo);
            shi[a] = std::max(shi[a], hi);
        }
    }
    if (aabb_out) std::memcpy(aabb_out, box.data(), sizeof(float) * 6 * nt);
    auto extent = [](const float* lo, const float* hi) {
        volatile float ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
        return std::max(std::max((float)ex, (float)ey), (float)ez);
    };
    const float es = nt > 0 ? extent(slo, shi) : 0.0f;
    volatile float thr = 0.25f * es;
    std::vector<char> large(nt, 0);
    int64_t nl = 0;
    for (int64_t i = 0; i < nt; ++i) {
        large[i] = extent(&box[6 * i], &box[6 * i + 3]) >= (float)thr;
        nl += large[i];
    }
    if (nl > MAX_LARGE) {
        std::fill(large.begin(), large.end(), 0);
        nl = 0;
    }
    if (nlarge_out) *nlarge_out = nl;
    float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nt; ++i)
        if (!large[i])
            for (int a = 0; a < 3; ++a) {
                cmin[a] = std::min(cmin[a], c2[3 * i + a]);
                cmax[a] = std::max(cmax[a], c2[3 * i + a]);
            }
    float e = -INFINITY;
    for (int a = 0; a < 3; ++a) {
        volatile float ea = cmax[a] - cmin[a];
        e = std::max(e, (float)ea);
    }
    const float scale = (e > 0.0f) ? (float)(2097151.0f / e) : 0.0f;
    for (int64_t i = 0; i < nt; ++i) {
        if (large[i]) {
            keys_out[i] = ~0ULL;
            continue;
        }
        uint32_t q[3];
        for (int a = 0; a < 3; ++a) {
            volatile float d = c2[3 * i + a] - cmin[a];
            volatile float f = (float)d * scale;
            uint32_t u = (uint32_t)(float)f;
            q[a] = u > 2097151u ? 2097151u : u;
        }
        keys_out[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    }
}

// Outputs: sorted keys [nt] (the large triangles last, key 2^64 - 1), sorted
// triangle ids [nt], the number of large triangles, and for each internal
// node i < ns-1 of the tree over the ns = nt - nlarge others: child[2]
// (>= 0 internal, < 0 = ~leaf position) and the two child AABBs [2][6]
// (lo xyz, hi xyz).
int or_lbvh(const float* verts, const int32_t* tris, int64_t nt_all, uint64_t* keys_sorted,
            int32_t* order, int32_t* child, float* child_aabb, int64_t* nlarge_out) {
    if (nlarge_out) *nlarge_out = 0;
    if (nt_all <= 0) return 0;
    std::vector<uint64_t> keys(nt_all);
    std::vector<float> box(6 * nt_all);
    int64_t nl = 0;
    or_morton(verts, tris, nt_all, keys.data(), box.data(), &nl);
    if (nlarge_out) *nlarge_out = nl;
    std::vector<int32_t> idx(nt_all);
    for (int64_t i = 0; i < nt_all; ++i) idx[i] = (int32_t)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return keys[a] < keys[b]; });
    for (int64_t i = 0; i < nt_all; ++i) { order[i] = idx[i]; keys_sorted[i] = keys[idx[i]]; }
    const int64_t nt = nt_all - nl;  // the tree covers sorted positions [0, nt)
    if (nt <= 1) return 0;
    auto delta = [&](int64_t i, int64_t j) -> int {
        if (keys_sorted[i] != keys_sorted[j]) return clz64(keys_sorted[i] ^ keys_sorted[j]);
        return 64 + clz32((uint32_t)i ^ (uint32_t)j);
    };
    std::vector<float> nodebox(6 * (nt - 1));
    // explicit stack of ranges (top-down); AABBs are filled bottom-up afterwards
    struct Rg { int64_t a, b, id; };
    std::vector<Rg> st{{0, nt - 1, 0}};
    std::vector<Rg> all;
    while (!st.empty()) {
        Rg r = st.back();
        st.pop_back();
        all.push_back(r);
        int cp = delta(r.a, r.b);
        int64_t g = r.a;
        while (g + 1 <= r.b - 1 && delta(r.a, g + 1) > cp) ++g;
        int32_t L = (r.a == g) ? ~(int32_t)g : (int32_t)g;
        int32_t R = (r.b == g + 1) ? ~(int32_t)(g + 1) : (int32_t)(g + 1);
        child[2 * r.id] = L;
        child[2 * r.id + 1] = R;
        if (L >= 0) st.push_back({r.a, g, L});
        if (R >= 0) st.push_back({g + 1, r.b, R});
    }
    // AABBs: a node's box is the exact union of its leaves' boxes; process
    // ranges from the smallest up so children are done before parents.
    std::sort(all.begin(), all.end(), [](const Rg& x, const Rg& y) { return (x.b - x.a) < (y.b - y.a); });
    auto cbox = [&](int32_t c, float* out) {
        const float* src = c < 0 ? &box[6 * (size_t)idx[~c]] : &nodebox[6 * (size_t)c];
        std::memcpy(out, src, 6 * sizeof(float));
    };
    for (const Rg& r : all) {
        float lb[6], rb[6];
        cbox(child[2 * r.id], lb);
        cbox(child[2 * r.id + 1], rb);
        std::memcpy(&child_aabb[12 * (size_t)r.id], lb, sizeof lb);
        std::memcpy(&child_aabb[12 * (size_t)r.id + 6], rb, sizeof rb);
        float* nb = &nodebox[6 * (size_t)r.id];
        for (int a = 0; a < 3; ++a) {
            nb[a] = std::min(lb[a], rb[a]);
            nb[3 + a] = std::max(lb[3 + a], rb[3 + a]);
        }
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Reference binned-SAH BVH.  Not in the paper either; a second tree over the
// same leaves (one triangle per leaf, the same large-triangle list) whose
// splits minimise the surface-area heuristic (MacDonald & Booth 1990) over 32
// centroid bins per axis (Wald, "On fast construction of SAH-based bounding
// volume hierarchies", 2007).  Written recursively over ranges of positions,
// one node at a time, independently of the GPU's level-by-level build.
//
// Start: the LBVH's stable Morton order; the tree covers positions [0, ns).
// A range [lo, hi) of at least 2 positions at depth d (the root [0, ns) at
// d = 0) is split as follows (FP32 with round-to-nearest, no fused
// operations, left to right):
//   c2         = lo + hi of each triangle's AABB (the Morton code's centroid);
//   cl_a, ch_a = min / max of c2_a over the range;
//   axis a is binned when d < 32, e_a = ch_a - cl_a > 0 and k_a = 32 / e_a is
//   finite;  bin_a(t) = min(31, trunc((c2_a(t) - cl_a) * k_a));
//   each bin holds the count and the union of its triangles' AABBs; split b
//   in 1..31 puts bins < b left (L) and bins >= b right (R); with
//   s = 2^-E where max_a e_a = f 2^E, f in [0.5, 1) (an exact power of two,
//   so that the areas neither overflow nor round differently at any scale),
//   H(B) = dx dy + dy dz + dz dx, dx = (hi_x - lo_x) s,
//   cost(a, b) = H(L) nL + H(R) nR, skipped when a side is empty; the first
//   minimum in the order a = 0, 1, 2, b = 1..31 wins (strict <);
//   the range is partitioned stably (bin_a < b first) and mid = lo + nL;
//   with no binned axis: mid = lo + (hi - lo) / 2 and the order is kept.
// (An axis with e_a > 0 puts the smallest c2 in bin 0 and the largest in bin
// 31, so a binned axis always has a candidate.)  Depth 32 onwards splits at
// the middle, so no leaf is deeper than 32 + ceil(log2 ns).
// Children: [lo, mid) and [mid, hi); a child of one position p is the leaf
// ~p.  Numbering: the node split at mid has g = mid - 1, which no other node
// of the tree has (g is in [0, ns - 2]); the root is internal node 0, the
// node with g = 0 takes the root's g, every other node is numbered g.
// Outputs as or_lbvh, except that keys_out[p] is the Morton key of the
// triangle at position p (the keys are no longer sorted inside the tree).
// ---------------------------------------------------------------------------
int or_sah_bvh(const float* verts, const int32_t* tris, int64_t nt_all, uint64_t* keys_out, int32_t* order,
               int32_t* child, float* child_aabb, int64_t* nlarge_out) {
    if (nlarge_out) *nlarge_out = 0;
    if (nt_all <= 0) return 0;
    std::vector<uint64_t> keys(nt_all);
    std::vector<float> box(6 * nt_all);
    int64_t nl = 0;
    or_morton(verts, tris, nt_all, keys.data(), box.data(), &nl);
    if (nlarge_out) *nlarge_out = nl;
    std::vector<int32_t> idx(nt_all);
    for (int64_t i = 0; i < nt_all; ++i) idx[i] = (int32_t)i;
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return keys[a] < keys[b]; });
    const int64_t ns = nt_all - nl;
    constexpr int NB = 32, DEPTH_CAP = 32;
    std::vector<float> c2(3 * nt_all);
    for (int64_t t = 0; t < nt_all; ++t)
        for (int a = 0; a < 3; ++a) c2[3 * t + a] = box[6 * t + a] + box[6 * t + 3 + a];
    auto half_area = [](const float* b, float sc) {
        const float dx = (b[3] - b[0]) * sc, dy = (b[4] - b[1]) * sc, dz = (b[5] - b[2]) * sc;
        return dx * dy + dy * dz + dz * dx;
    };
    auto unite = [](float* acc, const float* b) {
        for (int a = 0; a < 3; ++a) {
            acc[a] = std::min(acc[a], b[a]);
            acc[3 + a] = std::max(acc[3 + a], b[3 + a]);
        }
    };
    const float empty[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    struct Task { int64_t lo, hi; int depth; int64_t parent; int side; };
    struct Done { int64_t id, lo, hi; };
    std::vector<Task> st;
    std::vector<Done> all;
    if (ns >= 2) st.push_back({0, ns, 0, -1, 0});
    int64_t g_root = -1;
    while (!st.empty()) {
        const Task tk = st.back();
        st.pop_back();
        float cl[3] = {INFINITY, INFINITY, INFINITY}, ch[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int64_t p = tk.lo; p < tk.hi; ++p)
            for (int a = 0; a < 3; ++a) {
                cl[a] = std::min(cl[a], c2[3 * (size_t)idx[p] + a]);
                ch[a] = std::max(ch[a], c2[3 * (size_t)idx[p] + a]);
            }
        int best_a = -1, best_b = -1;
        float best = INFINITY;
        float k[3] = {0.0f, 0.0f, 0.0f};
        int e_exp = 0;
        std::frexp(std::max(std::max(ch[0] - cl[0], ch[1] - cl[1]), ch[2] - cl[2]), &e_exp);
        const float sc = std::ldexp(1.0f, -e_exp);
        auto bin_of = [&](int32_t t, int a) {
            const float d = c2[3 * (size_t)t + a] - cl[a];
            const float f = d * k[a];
            const int b = (int)f;
            return b < NB - 1 ? b : NB - 1;
        };
        for (int a = 0; a < 3 && tk.depth < DEPTH_CAP; ++a) {
            const float e = ch[a] - cl[a];
            if (!(e > 0.0f)) continue;
            k[a] = (float)NB / e;
            if (!std::isfinite(k[a])) continue;
            int64_t cnt[NB] = {0};
            float bb[NB][6];
            for (int b = 0; b < NB; ++b) std::memcpy(bb[b], empty, sizeof empty);
            for (int64_t p = tk.lo; p < tk.hi; ++p) {
                const int b = bin_of(idx[p], a);
                ++cnt[b];
                unite(bb[b], &box[6 * (size_t)idx[p]]);
            }
            // H and count of every right side R_b = bins b..31
            float h_right[NB];
            int64_t n_right[NB];
            float acc[6];
            std::memcpy(acc, empty, sizeof acc);
            int64_t n = 0;
            for (int b = NB - 1; b >= 1; --b) {
                unite(acc, bb[b]);
                n += cnt[b];
                h_right[b] = half_area(acc, sc);
                n_right[b] = n;
            }
            std::memcpy(acc, empty, sizeof acc);
            n = 0;
            for (int b = 1; b < NB; ++b) {
                unite(acc, bb[b - 1]);
                n += cnt[b - 1];
                if (n == 0 || n_right[b] == 0) continue;
                const float c = half_area(acc, sc) * (float)n + h_right[b] * (float)n_right[b];
                if (c < best) {
                    best = c;
                    best_a = a;
                    best_b = b;
                }
            }
        }
        int64_t mid;
        if (best_a < 0) {
            mid = tk.lo + (tk.hi - tk.lo) / 2;
        } else {
            const auto it = std::stable_partition(idx.begin() + tk.lo, idx.begin() + tk.hi,
                                                  [&](int32_t t) { return bin_of(t, best_a) < best_b; });
            mid = it - idx.begin();
        }
        const int64_t g = mid - 1;
        if (tk.parent < 0) g_root = g;
        const int64_t id = (tk.parent < 0) ? 0 : (g == 0 ? g_root : g);
        if (tk.parent >= 0) child[2 * tk.parent + tk.side] = (int32_t)id;
        all.push_back({id, tk.lo, tk.hi});
        if (mid - tk.lo == 1) child[2 * id] = ~(int32_t)tk.lo;
        else st.push_back({tk.lo, mid, tk.depth + 1, id, 0});
        if (tk.hi - mid == 1) child[2 * id + 1] = ~(int32_t)mid;
        else st.push_back({mid, tk.hi, tk.depth + 1, id, 1});
    }
    for (int64_t p = 0; p < nt_all; ++p) {
        order[p] = idx[p];
        keys_out[p] = keys[idx[p]];
    }
    // boxes bottom-up: smaller ranges first, so children are done before parents
    std::vector<float> nodebox(6 * (size_t)std::max<int64_t>(ns - 1, 1));
    std::sort(all.begin(), all.end(), [](const Done& x, const Done& y) { return (x.hi - x.lo) < (y.hi - y.lo); });
    for (const Done& d : all) {
        float* nb = &nodebox[6 * (size_t)d.id];
        std::memcpy(nb, empty, sizeof empty);
        for (int s = 0; s < 2; ++s) {
            const int32_t c = child[2 * d.id + s];
            const float* src = c < 0 ? &box[6 * (size_t)idx[~c]] : &nodebox[6 * (size_t)c];
            std::memcpy(&child_aabb[12 * (size_t)d.id + 6 * s], src, 6 * sizeof(float));
            unite(nb, src);
        }
    }
    return 0;
}

}  // extern "C"

// ===========================================================================
// First-order diffraction radio map (Sec. 4, "Computation of Radio Map due to
// Diffraction"; UTD of App. A.8; weighting factor of the appendix on
// diffraction radio maps).  Test infrastructure like the rest of this file.
// ===========================================================================
namespace {

// 64-point Gauss-Legendre rule on [-1, 1]; nodes by Newton's method on P_64.
struct GLRule {
    std::vector<double> x, w;
};
const GLRule& gl64() {
    static const GLRule rule = [] {
        GLRule r;
        const int n = 64;
        r.x.resize(n);
        r.w.resize(n);
        auto legendre = [n](double z, double* dp) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            *dp = n * (z * p1 - p0) / (z * z - 1.0);
            return p1;
        };
        for (int i = 0; i < n / 2; ++i) {
            double z = std::cos(PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
            for (int it = 0; it < 100; ++it) {
                const double dz = legendre(z, &dp) / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) break;
            }
            legendre(z, &dp);
            r.x[i] = -z;
            r.x[n - 1 - i] = z;
            r.w[i] = r.w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
        }
        return r;
    }();
    return rule;
}

// UTD transition function F(x) = 2 j sqrt(x) e^{jx} int_{sqrt x}^inf e^{-j t^2} dt
// (App. A.8), from its defining integral.  The path of integration is turned
// by -pi/4 about t = sqrt(x) (Cauchy: e^{-j t^2} decays in the sector swept),
// t = sqrt(x) + e^{-j pi/4} u, which gives
//   F(x) = 2 j e^{-j pi/4} sqrt(x) int_0^inf exp(-u^2 - b (1 + j) u) du,  b = sqrt(2x),
// a smooth integrand below e^-40 beyond T = (sqrt(b^2 + 160) - b) / 2; the
// integral over [0, T] is taken with the 64-point Gauss-Legendre rule.
std::complex<double> utd_F(double x) {
    if (!(x > 0.0)) return {0.0, 0.0};
    const double b = std::sqrt(2.0 * x);
    const double T = 0.5 * (std::sqrt(b * b + 160.0) - b);
    const GLRule& g = gl64();
    std::complex<double> I(0.0, 0.0);
    for (size_t i = 0; i < g.x.size(); ++i) {
        const double u = 0.5 * T * (g.x[i] + 1.0);
        const double m = 0.5 * T * g.w[i] * std::exp(-u * u - b * u);
        I += m * std::complex<double>(std::cos(b * u), -std::sin(b * u));
    }
    const std::complex<double> j(0.0, 1.0);
    return 2.0 * j * std::exp(std::complex<double>(0.0, -PI / 4.0)) * std::sqrt(x) * I;
}

struct Wedge {
    V3<double> o, e;      // edge origin and unit edge vector, e = n0 x nn / |n0 x nn|
    V3<double> n0, nn;    // outward normals of the 0-face and the n-face
    V3<double> t0;        // t0 = n0 x e, tangent to the 0-face
    double len, n;        // edge length, exterior angle n pi
    int tri0, trin, mat0, matn;
};

// Wedges of a mesh.  Reading (the paper keeps wedges "near the source"
// found during SBR): every edge shared by exactly two triangles whose
// outward normals, from the winding, meet at a convex corner (the far
// vertex of the second triangle lies behind the first one's plane) and are
// not parallel; visibility from the source is then decided per sample.
// The triangle of lower index is the 0-face; wedges are ordered by
// (tri0, trin).
std::vector<Wedge> find_wedges(const Scene& S, const float* verts, const int32_t* tris, int64_t nt) {
    std::map<std::pair<int, int>, std::vector<int>> edges;
    for (int64_t i = 0; i < nt; ++i)
        for (int k = 0; k < 3; ++k) {
            const int a = tris[3 * i + k], b = tris[3 * i + (k + 1) % 3];
            edges[{std::min(a, b), std::max(a, b)}].push_back((int)i);
        }
    auto vert = [&](int id) { return V3<double>{verts[3 * id], verts[3 * id + 1], verts[3 * id + 2]}; };
    std::vector<Wedge> out;
    for (const auto& kv : edges) {
        if (kv.second.size() != 2) continue;
        const int A = std::min(kv.second[0], kv.second[1]), B = std::max(kv.second[0], kv.second[1]);
        const Tri& TA = S.tris[A];
        const Tri& TB = S.tris[B];
        if (TA.area2 == 0.0 || TB.area2 == 0.0) continue;
        const V3<double> c = cross(TA.n, TB.n);
        const double sn = norm(c);
        if (sn < 1e-9) continue;
        int third = -1;
        for (int k = 0; k < 3; ++k) {
            const int id = tris[3 * B + k];
            if (id != kv.first.first && id != kv.first.second) third = id;
        }
        const V3<double> p = vert(kv.first.first), q = vert(kv.first.second);
        if (third < 0 || !(dot(vert(third) - p, TA.n) < 0.0)) continue;
        Wedge W;
        W.e = scl(c, 1.0 / sn);
        W.n0 = TA.n;
        W.nn = TB.n;
        W.t0 = cross(W.n0, W.e);
        W.n = 1.0 + std::acos(std::max(-1.0, std::min(1.0, dot(TA.n, TB.n)))) / PI;
        W.o = dot(p, W.e) <= dot(q, W.e) ? p : q;
        W.len = norm(q - p);
        W.tri0 = A;
        W.trin = B;
        W.mat0 = TA.mat;
        W.matn = TB.mat;
        out.push_back(W);
    }
    std::sort(out.begin(), out.end(),
              [](const Wedge& a, const Wedge& b) { return a.tri0 != b.tri0 ? a.tri0 < b.tri0 : a.trin < b.trin; });
    return out;
}

// The UTD requires phi' <= pi (the source in front of the 0-face).  Reading:
// otherwise the faces swap roles (e -> -e, t0 from the new 0-face); the
// exterior angle is unchanged.  Whether phi' <= pi depends only on which side
// of the 0-face's plane the source lies.
Wedge oriented(const Wedge& W, const V3<double>& s) {
    if (dot(s - W.o, W.n0) >= 0.0) return W;
    Wedge R = W;
    std::swap(R.n0, R.nn);
    std::swap(R.mat0, R.matn);
    std::swap(R.tri0, R.trin);
    R.e = scl(W.e, -1.0);
    R.o = W.o + scl(W.e, W.len);
    R.t0 = cross(R.n0, R.e);
    return R;
}

// Diffraction point v(x) = o + x e and Keller-cone direction
//   k_s = sin b0' cos phi t0 + sin b0' sin phi n0 + cos b0' e,
// cos b0' = (v - s).e / |v - s|, sin b0' = |s - s_E| / |v - s| (s_E the
// projection of s onto the edge line): Eq. radio-map-solver-ci-D-reparametrization
// and the weighting-factor appendix.  Typed so that dual numbers carry
// d/dx and d/dphi.
template <class R>
void keller(const Wedge& W, const V3<double>& s, const R& x, const R& phi, V3<R>* v, V3<R>* ks) {
    *v = {R(W.o.x) + x * W.e.x, R(W.o.y) + x * W.e.y, R(W.o.z) + x * W.e.z};
    const V3<R> d{v->x - s.x, v->y - s.y, v->z - s.z};
    const R dn = r_sqrt(d.x * d.x + d.y * d.y + d.z * d.z);
    const V3<double> so = s - W.o;
    const double rho = norm(so - scl(W.e, dot(so, W.e)));
    const R cb = (d.x * W.e.x + d.y * W.e.y + d.z * W.e.z) / dn;
    const R sb = R(rho) / dn;
    const R cp = r_cos(phi), sp = r_sin(phi);
    *ks = {sb * cp * W.t0.x + sb * sp * W.n0.x + cb * W.e.x, sb * cp * W.t0.y + sb * sp * W.n0.y + cb * W.e.y,
           sb * cp * W.t0.z + sb * sp * W.n0.z + cb * W.e.z};
}

// Diffracted field (Eq. diffracted-field, with D_1..D_4 and the face
// matrices R_0, R_n of the same appendix) for a 3-D incident field E (the
// antenna field at unit distance): returns (E_d,phi, E_d,beta0) including the
// spreading factor sqrt(1 / (s' s (s' + s))), without the phase
// e^{-jk(s'+s)} (the map is non-coherent).  W must be oriented (phi' <= pi).
// r_perp, r_par of a face are the half-space coefficients of Eq.
// fresnel_vac at cos theta_r = |n . s'|.  Reading: a term whose cotangent
// argument is exactly a multiple of pi (an exact shadow boundary, measure
// zero) takes the mean of its one-sided limits, 0.
void utd_field(const Wedge& W, const Cx<double>& eta0, const Cx<double>& etan, double k0, const V3<double>& s,
               const V3<double>& v, const V3<double>& sd, double sobs, const CV3<double>& E,
               std::complex<double> out[2]) {
    typedef std::complex<double> cd;
    const V3<double> sp_v = v - s;
    const double sprime = norm(sp_v);
    const V3<double> si = scl(sp_v, 1.0 / sprime);  // s' hat
    const V3<double>& e = W.e;
    const double sinb = norm(cross(sd, e));
    const V3<double> phi_i = unit(cross(si, e));
    const V3<double> beta_i = cross(phi_i, si);
    auto proj = [&](const V3<double>& a) { return unit(a - scl(e, dot(a, e))); };
    auto sgn = [](double z) { return z >= 0.0 ? 1.0 : -1.0; };
    auto acl = [](double z) { return std::acos(std::max(-1.0, std::min(1.0, z))); };
    const V3<double> sit = proj(si), sdt = proj(sd);
    const double phip = PI - (PI - acl(-dot(sit, W.t0))) * sgn(-dot(sit, W.n0));
    const double phid = PI - (PI - acl(dot(sdt, W.t0))) * sgn(dot(sdt, W.n0));
    const double n = W.n;
    const double L = sobs * sprime / (sobs + sprime) * sinb * sinb;
    const cd pre = -std::exp(cd(0.0, -PI / 4.0)) / (2.0 * n * std::sqrt(2.0 * PI * k0) * sinb);
    auto a_pm = [&](double beta, double pm) {
        const double N = std::round((beta + pm * PI) / (2.0 * n * PI));
        const double c = std::cos((2.0 * n * PI * N - beta) / 2.0);
        return 2.0 * c * c;
    };
    auto D = [&](double beta, double pm) {
        const double arg = (PI + pm * beta) / (2.0 * n);
        const double sa = std::sin(arg);
        if (sa == 0.0) return cd(0.0, 0.0);
        return pre * (std::cos(arg) / sa) * utd_F(k0 * L * a_pm(beta, pm));
    };
    const cd D1 = D(phid - phip, +1.0), D2 = D(phid - phip, -1.0);
    const cd D3 = D(phid + phip, +1.0), D4 = D(phid + phip, -1.0);
    // face matrix W(phi_SB, beta_SB, e_r,perp, e_r,par) diag(r_perp, r_par) W(e_i,perp, e_i,par, phi', beta0')
    auto face = [&](const V3<double>& nf, const Cx<double>& eta, cd M[2][2]) {
        const double cr = std::fabs(dot(nf, si));
        const Coefs<double> c = fresnel(eta, cr, 0.0, false);
        const cd rp(c.r_perp.re, c.r_perp.im), rl(c.r_par.re, c.r_par.im);
        const V3<double> sSB = si - scl(nf, 2.0 * dot(si, nf));
        V3<double> x = cross(si, nf);
        V3<double> eip;
        if (norm(x) > 1e-12) {
            eip = unit(x);
        } else {
            V3<double> ax = std::fabs(si.x) < 0.5 ? V3<double>{1, 0, 0} : V3<double>{0, 1, 0};
            eip = unit(cross(si, ax));
        }
        const V3<double> eil = cross(eip, si);
        const V3<double> erl = cross(eip, sSB);
        const V3<double> phSB = scl(unit(cross(sSB, e)), -1.0);
        const V3<double> beSB = cross(phSB, sSB);
        const double Wo[2][2] = {{dot(phSB, eip), dot(phSB, erl)}, {dot(beSB, eip), dot(beSB, erl)}};
        const double Wi[2][2] = {{dot(eip, phi_i), dot(eip, beta_i)}, {dot(eil, phi_i), dot(eil, beta_i)}};
        const cd rr[2] = {rp, rl};
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                cd m(0.0, 0.0);
                for (int q = 0; q < 2; ++q) m += Wo[a][q] * rr[q] * Wi[q][b];
                M[a][b] = m;
            }
    };
    cd R0[2][2], Rn[2][2];
    face(W.n0, eta0, R0);
    if ((n - 1.0) * PI <= phip) {
        face(W.nn, etan, Rn);
    } else {
        Rn[0][0] = Rn[1][1] = -1.0;
        Rn[0][1] = Rn[1][0] = 0.0;
    }
    const cd ein[2] = {cd(E.x.re, E.x.im) * phi_i.x + cd(E.y.re, E.y.im) * phi_i.y + cd(E.z.re, E.z.im) * phi_i.z,
                       cd(E.x.re, E.x.im) * beta_i.x + cd(E.y.re, E.y.im) * beta_i.y + cd(E.z.re, E.z.im) * beta_i.z};
    const double spread = 1.0 / std::sqrt(sprime * sobs * (sprime + sobs));
    for (int a = 0; a < 2; ++a) {
        cd acc(0.0, 0.0);
        for (int b = 0; b < 2; ++b) acc += ((-D1 + D4) * R0[a][b] + (-D2 + D3) * Rn[a][b]) * ein[b];
        out[a] = -acc * spread;
    }
}

// Is the open segment o + t d, t in (t0, t1), blocked by a triangle other
// than ex0, ex1?
bool blocked(const Scene& S, const V3<double>& o, const V3<double>& d, double t0, double t1, int ex0, int ex1) {
    for (int i = 0; i < (int)S.tris.size(); ++i) {
        if (i == ex0 || i == ex1) continue;
        const double t = hit_mt(S.tris[i], o, d);
        if (t > t0 && t < t1) return true;
    }
    return false;
}
// Could an FP32 computation decide the other way?  A triangle whose plane
// hit lies within tol of the segment's open interval and within tol of the
// triangle's boundary, or a hit within tol of an end.
bool blocked_near_tie(const Scene& S, const V3<double>& o, const V3<double>& d, double t0, double t1, int ex0,
                      int ex1, double tol) {
    for (int i = 0; i < (int)S.tris.size(); ++i) {
        if (i == ex0 || i == ex1) continue;
        double t, m;
        if (!plane_hit(S.tris[i], o, d, &t, &m)) continue;
        if (!(t > t0 - tol && t < t1 + tol)) continue;
        if (std::fabs(m) <= tol) return true;
        if (m > 0.0 && (std::fabs(t - t0) <= tol || std::fabs(t - t1) <= tol)) return true;
    }
    return false;
}

// Sample i of N on a wedge: (u1, u2) = ((i + 1/2) / N, frac(i (phi_g - 1))),
// the second coordinate from the 64-bit fixed-point product of the
// Fibonacci lattice, truncated to 24 bits; x = u1 L_E, phi = u2 n pi.
// Reading: the paper draws x and phi uniformly; this rank-1 lattice is the
// quasi-Monte-Carlo counterpart, like the Fibonacci directions of SBR.
inline void wedge_sample(int64_t i, int64_t N, double* u1, double* u2) {
    *u1 = ((double)i + 0.5) / (double)N;
    const uint64_t f = (uint64_t)i * 0x9E3779B97F4A7C16ULL;
    *u2 = (double)(f >> 40) * 0x1.0p-24;
}

}  // namespace

extern "C" {

// Wedges of a mesh (see find_wedges).  out (or null): [cap][16] doubles
// o(3) e(3) n0(3) nn(3) len n tri0 trin; returns the number of wedges.
int64_t or_wedges(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tri_mat,
                  double* out, int64_t cap) {
    std::vector<int32_t> mat(tri_mat, tri_mat + nt);
    int nm = 1;
    for (int32_t m : mat) nm = std::max(nm, m + 1);
    std::vector<float> mats(3 * nm, 1.0f);
    Scene S = make_scene(verts, nv, tris, nt, mat.data(), mats.data(), nm);
    std::vector<Wedge> W = find_wedges(S, verts, tris, nt);
    for (int64_t i = 0; i < (int64_t)W.size() && i < cap && out; ++i) {
        double* o = out + 16 * i;
        const Wedge& w = W[i];
        const double v[16] = {w.o.x, w.o.y, w.o.z, w.e.x, w.e.y, w.e.z, w.n0.x, w.n0.y, w.n0.z,
                              w.nn.x, w.nn.y, w.nn.z, w.len, w.n, (double)w.tri0, (double)w.trin};
        std::memcpy(o, v, sizeof v);
    }
    return (int64_t)W.size();
}

// F(x) for the pins: out[2] = (re, im).
void or_utd_F(double x, double* out) {
    const std::complex<double> f = utd_F(x);
    out[0] = f.real();
    out[1] = f.imag();
}

// Diffracted field of one incident field for the pins: wedge w16 as written by
// or_wedges (oriented here), source s, diffraction point v, diffracted
// direction sd, observation distance sobs, incident field E6, face
// materials (eps, sigma) x 2 at angular frequency omega.  out[4] = E_d,phi
// and E_d,beta0 (re, im).
void or_utd_field(const double* w16, const double* s, const double* v, const double* sd, double sobs,
                  const double* E6, const double* mats4, double omega, double* out) {
    Wedge W;
    W.o = {w16[0], w16[1], w16[2]};
    W.e = {w16[3], w16[4], w16[5]};
    W.n0 = {w16[6], w16[7], w16[8]};
    W.nn = {w16[9], w16[10], w16[11]};
    W.len = w16[12];
    W.n = w16[13];
    W.t0 = cross(W.n0, W.e);
    W.tri0 = W.trin = -1;
    W.mat0 = 0;
    W.matn = 1;
    const V3<double> S{s[0], s[1], s[2]};
    Wedge R = oriented(W, S);
    const Cx<double> e0 = permittivity(mats4[2 * R.mat0], mats4[2 * R.mat0 + 1], omega);
    const Cx<double> en = permittivity(mats4[2 * R.matn], mats4[2 * R.matn + 1], omega);
    const CV3<double> E{Cx<double>(E6[0], E6[1]), Cx<double>(E6[2], E6[3]), Cx<double>(E6[4], E6[5])};
    std::complex<double> o[2];
    utd_field(R, e0, en, omega / C0, S, {v[0], v[1], v[2]}, {sd[0], sd[1], sd[2]}, sobs, E, o);
    out[0] = o[0].real(); out[1] = o[0].imag(); out[2] = o[1].real(); out[3] = o[1].imag();
}

// Measurement point t(x, phi) on the plane z = zM and the weighting factor
// |dt/dx x dt/dphi| for the pins: out[4] = t (3), J.  Wedge oriented for s.
// Returns 0 when the diffracted ray does not reach the plane.
int or_diffraction_point(const double* w16, const double* s, double x, double phi, double zM, double* out) {
    Wedge W;
    W.o = {w16[0], w16[1], w16[2]};
    W.e = {w16[3], w16[4], w16[5]};
    W.n0 = {w16[6], w16[7], w16[8]};
    W.nn = {w16[9], w16[10], w16[11]};
    W.len = w16[12];
    W.n = w16[13];
    W.t0 = cross(W.n0, W.e);
    const V3<double> S{s[0], s[1], s[2]};
    const Wedge R = oriented(W, S);
    D xd(x), pd(phi);
    xd.g[0] = 1.0;
    pd.g[1] = 1.0;
    V3<D> v, ks;
    keller(R, S, xd, pd, &v, &ks);
    if (!(ks.z.v != 0.0)) return 0;
    const D gam = (D(zM) - v.z) / ks.z;
    if (!(gam.v > 0.0)) return 0;
    const V3<D> t{v.x + gam * ks.x, v.y + gam * ks.y, v.z + gam * ks.z};
    const V3<double> tx{t.x.g[0], t.y.g[0], t.z.g[0]}, tp{t.x.g[1], t.y.g[1], t.z.g[1]};
    out[0] = t.x.v; out[1] = t.y.v; out[2] = t.z.v;
    out[3] = norm(cross(tx, tp));
    return 1;
}

}  // extern "C"

extern "C" {

// Diffraction radio map of one transmitter (estimator Eq. radio-map-solver-ci-D-est):
//   C_i += (1 / |M_i|) (L_E n pi / N') e(p) I(p) |dt/dx x dt/dphi|
// over samples_per_wedge = N' lattice samples (x, phi) of every wedge, with
// e(p) = (lambda0 / 4 pi)^2 |E_d|^2 (summed over the two field columns of a
// dual-polarised antenna) and I(p) = 1 when the diffracted ray reaches the map
// and neither the source-to-edge nor the edge-to-plane segment is blocked
// (the wedge's own faces excluded, open intervals shortened by
// 2^-16 max(1, |v|_inf) at the edge end).  mode 0 plain, 1 replay-check of
// the record (GPU visibility bits and cells certified as FP64 near-ties).
// rec: [nw][N'][4] = {bits (1: incident blocked, 2: diffracted blocked;
// -1: no crossing in the map; -2: source behind both faces), ix, iy, 0}.
// counts_out (or null): [3] samples with a crossing, visible samples, wedges.
// slack_out (or null) [ny][nx]: per cell, the sum over deposits of the largest
// change of a deposit's value when its Keller azimuth moves by +-1e-5 rad
// (test error bounds: FP32 may put a sample on the other side of a shadow
// boundary or of a rounding point of N^+-).
// wsel (or null): the positions, in the (tri0, trin) order of or_wedges, of
// the nsel wedges to sample (a subset of the estimator's sum over wedges);
// rec and counts then follow that list.
int or_diffraction_map(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tri_mat,
                       const float* mats, int nm, const or_tx* tx, const or_params* P, int64_t samples_per_wedge,
                       int mode, int32_t* rec, int64_t rec_cap, double* map_out, double* counts_out,
                       or_report* report, double* slack_out, const int64_t* wsel, int64_t nsel) {
    if (samples_per_wedge < 1) return 1;
    Scene S = make_scene(verts, nv, tris, nt, tri_mat, mats, nm);
    std::vector<Wedge> WS = find_wedges(S, verts, tris, nt);
    if (wsel) {
        std::vector<Wedge> sub;
        sub.reserve(nsel > 0 ? (size_t)nsel : 0);
        for (int64_t j = 0; j < nsel; ++j) {
            if (wsel[j] < 0 || wsel[j] >= (int64_t)WS.size()) return 3;
            sub.push_back(WS[wsel[j]]);
        }
        WS.swap(sub);
    }
    const int64_t nw = (int64_t)WS.size(), NS = samples_per_wedge;
    if (rec && rec_cap < nw * NS) return 2;
    MapGeom g = make_geom(*P, 1);
    const double omega = 2.0 * PI * P->freq_hz, k0 = omega / C0;
    const double lam4pi = C0 / P->freq_hz / (4.0 * PI);
    TxC T = make_txc(*tx);
    const int npol = tx->pol == 2 ? 2 : 1;
    const V3<double> s{tx->pos[0], tx->pos[1], tx->pos[2]};
    std::vector<DepList> lists(nw), slacks(slack_out ? nw : 0);
    std::vector<ReplayState> rss(nw);
    for (auto& r : rss) std::memset(&r.rep, 0, sizeof r.rep);
    std::vector<double> cnt(2 * nw, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w = 0; w < nw; ++w) {
        Sink<double> sink{&lists[w]};
        Sink<double> slack_sink{slack_out ? &slacks[w] : nullptr};
        ReplayState& rs = rss[w];
        const Wedge R = oriented(WS[w], s);
        const bool lit = dot(s - R.o, R.n0) >= 0.0;
        const Cx<double> eta0 = permittivity(S.eps[R.mat0], S.sigma[R.mat0], omega);
        const Cx<double> etan = permittivity(S.eps[R.matn], S.sigma[R.matn], omega);
        for (int64_t i = 0; i < NS; ++i) {
            int32_t* rc = rec ? rec + 4 * (w * NS + i) : nullptr;
            if (mode == 1) rs.rep.segments++;
            int code = -2, ix = NO_CELL, iy = NO_CELL;
            double u1, u2;
            wedge_sample(i, NS, &u1, &u2);
            const double x = u1 * R.len, phi = u2 * R.n * PI;
            V3<double> v, ks;
            keller(R, s, x, phi, &v, &ks);
            Crossing<double> cr = crossing(g, v, ks, INFINITY);
            const double vm = std::max(std::fabs(v.x), std::max(std::fabs(v.y), std::fabs(v.z)));
            const double eps = std::ldexp(std::max(1.0, vm), -16);
            const V3<double> sv = v - s;
            const double sprime = norm(sv);
            const V3<double> si = scl(sv, 1.0 / sprime);
            if (lit && !(mode == 1 && rc[0] == -2)) {
                code = -1;
                if (cr.valid) {
                    ix = cr.ix;
                    iy = cr.iy;
                }
                if (mode == 1 && (rc[1] != ix || rc[2] != iy)) {
                    // the GPU's cell (or its finding the crossing in or out of the map)
                    // is adopted only within tol of a cell boundary, the map edge or t_c = 0
                    const double tc = ks.z != 0.0 ? (g.z - v.z) / ks.z : INFINITY;
                    bool ok = std::isfinite(tc) && tc > -1.0;
                    if (ok) {
                        const V3<double> pc = v + scl(ks, tc);
                        const double tol = tie_tol(pc, sprime + std::fabs(tc));
                        const double sh = g.bilinear ? 0.5 : 0.0;
                        const double ux = (pc.x - g.x0) / g.cell - sh, uy = (pc.y - g.y0) / g.cell - sh;
                        const double bx = tol / g.cell;
                        auto near_int = [&](double u) { return std::fabs(u - std::nearbyint(u)) <= bx; };
                        if (rc[1] != NO_CELL && ix != NO_CELL) {
                            ok = std::abs(rc[1] - ix) <= 1 && std::abs(rc[2] - iy) <= 1 &&
                                 (rc[1] == ix || near_int(ux)) && (rc[2] == iy || near_int(uy));
                        } else {
                            ok = near_int(ux) || near_int(uy) || std::fabs(tc) <= tol;
                            if (ok && rc[1] != NO_CELL) {
                                const int ex = (int)std::floor(ux), ey = (int)std::floor(uy);
                                ok = std::abs(rc[1] - ex) <= 1 && std::abs(rc[2] - ey) <= 1;
                            }
                        }
                        if (ok && rc[1] != NO_CELL && !cr.valid) {
                            cr.x = pc.x;
                            cr.y = pc.y;
                            cr.tc_v = tc;
                        }
                    }
                    if (!ok) {
                        rs.fail(w * NS + i, 0, 2, ix, iy, rc[1], rc[2]);
                        continue;
                    }
                    rs.rep.adopted_cell++;
                    ix = rc[1];
                    iy = rc[2];
                }
                if (ix != NO_CELL) {
                    const double gam = cr.tc_v;
                    const bool bi = blocked(S, s, si, eps, sprime - eps, R.tri0, R.trin);
                    const bool bd = blocked(S, v, ks, eps, gam, R.tri0, R.trin);
                    code = (bi ? 1 : 0) | (bd ? 2 : 0);
                    if (mode == 1 && rc[0] != code) {
                        const double tol = tie_tol(v + scl(ks, gam), sprime + gam);
                        const int diff = (rc[0] < 0 ? 3 : rc[0]) ^ code;
                        bool ok = rc[0] >= 0;
                        if (ok && (diff & 1) && !blocked_near_tie(S, s, si, eps, sprime - eps, R.tri0, R.trin, tol))
                            ok = false;
                        if (ok && (diff & 2) && !blocked_near_tie(S, v, ks, eps, gam, R.tri0, R.trin, tol))
                            ok = false;
                        if (!ok) {
                            rs.fail(w * NS + i, 0, 5, code, rc[0], 0, 0);
                            continue;
                        }
                        rs.rep.adopted_hit++;
                        code = rc[0];
                    }
                }
            }
            if (mode == 1 && rc[0] != code) {
                // which side of the 0-face the source lies on is not adopted
                rs.fail(w * NS + i, 0, 6, code, rc[0], 0, 0);
                continue;
            }
            if (rc && mode == 0) {
                rc[0] = code;
                rc[1] = ix;
                rc[2] = iy;
                rc[3] = 0;
            }
            if (ix != NO_CELL) cnt[2 * w] += 1.0;
            if (code != 0 || ix == NO_CELL) continue;
            // weighting factor |dt/dx x dt/dphi| by dual numbers through t(x, phi)
            D xd(x), pd(phi);
            xd.g[0] = 1.0;
            pd.g[1] = 1.0;
            V3<D> vd, kd;
            keller(R, s, xd, pd, &vd, &kd);
            const D gam = (D(g.z) - vd.z) / kd.z;
            const V3<double> tx_{vd.x.g[0] + gam.g[0] * kd.x.v + gam.v * kd.x.g[0],
                                 vd.y.g[0] + gam.g[0] * kd.y.v + gam.v * kd.y.g[0],
                                 vd.z.g[0] + gam.g[0] * kd.z.v + gam.v * kd.z.g[0]};
            const V3<double> tp_{vd.x.g[1] + gam.g[1] * kd.x.v + gam.v * kd.x.g[1],
                                 vd.y.g[1] + gam.g[1] * kd.y.v + gam.v * kd.y.g[1],
                                 vd.z.g[1] + gam.g[1] * kd.z.v + gam.v * kd.z.g[1]};
            const double J = norm(cross(tx_, tp_));
            // incident antenna field in the departure direction s' (App. A.1, Sec. 4.4)
            const std::complex<double> al = array_factor(T, si, k0);
            auto power = [&](const V3<double>& kd_) {
                double pw = 0.0;
                for (int p = 0; p < npol; ++p) {
                    const V3<double> f = tx_field(si, T.R, tx->pattern, tx->pol == 2 ? p : tx->pol);
                    const CV3<double> E{Cx<double>(f.x * al.real(), f.x * al.imag()),
                                        Cx<double>(f.y * al.real(), f.y * al.imag()),
                                        Cx<double>(f.z * al.real(), f.z * al.imag())};
                    std::complex<double> ed[2];
                    utd_field(R, eta0, etan, k0, s, v, kd_, cr.tc_v, E, ed);
                    pw += std::norm(ed[0]) + std::norm(ed[1]);
                }
                return pw;
            };
            const double pw = power(ks);
            const double wgt = lam4pi * lam4pi * J * (R.len * R.n * PI / (double)NS) / (g.cell * g.cell);
            const double value = wgt * pw;
            deposit(g, cr, ix, iy, value, sink);
            if (slack_out) {
                double sl = 0.0;
                for (double dphi : {-1e-5, 1e-5}) {
                    V3<double> v2, k2;
                    keller(R, s, x, phi + dphi, &v2, &k2);
                    sl = std::max(sl, std::fabs(wgt * power(k2) - value));
                }
                Crossing<double> c2 = cr;
                if (g.bilinear) {
                    // the slack goes unweighted to every cell of the stencil
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a)
                            if (ix + a >= 0 && ix + a < g.nx && iy + b >= 0 && iy + b < g.ny)
                                slack_sink.add((iy + b) * g.nx + ix + a, sl);
                } else {
                    deposit(g, c2, ix, iy, sl, slack_sink);
                }
            }
            cnt[2 * w + 1] += 1.0;
        }
    }
    std::memset(map_out, 0, sizeof(double) * (size_t)P->nx * P->ny);
    for (int64_t w = 0; w < nw; ++w)
        for (size_t j = 0; j < lists[w].cell.size(); ++j) map_out[lists[w].cell[j]] += lists[w].val[j];
    if (slack_out) {
        std::memset(slack_out, 0, sizeof(double) * (size_t)P->nx * P->ny);
        for (int64_t w = 0; w < nw; ++w)
            for (size_t j = 0; j < slacks[w].cell.size(); ++j) slack_out[slacks[w].cell[j]] += slacks[w].val[j];
    }
    if (counts_out) {
        counts_out[0] = counts_out[1] = 0.0;
        for (int64_t w = 0; w < nw; ++w) { counts_out[0] += cnt[2 * w]; counts_out[1] += cnt[2 * w + 1]; }
        counts_out[2] = (double)nw;
    }
    if (report) {
        std::memset(report, 0, sizeof *report);
        bool have = false;
        for (int64_t w = 0; w < nw; ++w) {
            const or_report& r = rss[w].rep;
            report->segments += r.segments;
            report->adopted_hit += r.adopted_hit;
            report->adopted_cell += r.adopted_cell;
            report->failures += r.failures;
            if (r.failures && !have) {
                have = true;
                report->fail_ray = r.fail_ray;
                report->fail_kind = r.fail_kind;
                std::memcpy(report->fail_info, r.fail_info, sizeof r.fail_info);
            }
        }
    }
    return 0;
}

// The diffraction map on a mesh measurement surface (one cell per surface
// triangle): a sample's diffracted ray deposits at every surface triangle it
// crosses (t_j > 1e-9) whose segment from the edge is unblocked, with the
// weighting factor taken on that triangle's plane and 1 / A_j for the cell's
// area (Eq. radio-map-solver-ci-D-est with the cell's own measure).  The UTD
// field is evaluated at each crossing's distance.
// rec [nw][N'][4] = {bits (1 incident blocked; -2 source behind both faces),
// crossings found, 0, 0}; replay (mode 1) certifies only the incident bit (the
// per-crossing visibility is recomputed: a near tie goes to the slack).
// slack_out [n_surf]: per cell, the values of crossings within tol of the
// triangle's boundary or of a visibility near tie, plus the +-1e-5 rad
// azimuth change of every deposit.
int or_diffraction_map_mesh(const float* verts, int64_t nv, const int32_t* tris, int64_t nt, const int32_t* tri_mat,
                            const float* mats, int nm, const or_tx* tx, const or_params* P, int64_t samples_per_wedge,
                            const float* surf_verts, const int32_t* surf_tris, int64_t n_surf, int mode, int32_t* rec,
                            int64_t rec_cap, double* map_out, double* slack_out, or_report* report,
                            const int64_t* wsel, int64_t nsel) {
    if (samples_per_wedge < 1) return 1;
    Scene S = make_scene(verts, nv, tris, nt, tri_mat, mats, nm);
    const MeshSurface M = make_surface(surf_verts, surf_tris, n_surf);
    std::vector<Wedge> WS = find_wedges(S, verts, tris, nt);
    if (wsel) {
        // a subset of the wedges, as or_diffraction_map takes it
        std::vector<Wedge> sub;
        sub.reserve(nsel > 0 ? (size_t)nsel : 0);
        for (int64_t j = 0; j < nsel; ++j) {
            if (wsel[j] < 0 || wsel[j] >= (int64_t)WS.size()) return 3;
            sub.push_back(WS[wsel[j]]);
        }
        WS.swap(sub);
    }
    const int64_t nw = (int64_t)WS.size(), NS = samples_per_wedge;
    if (rec && rec_cap < nw * NS) return 2;
    const double omega = 2.0 * PI * P->freq_hz, k0 = omega / C0;
    const double lam4pi = C0 / P->freq_hz / (4.0 * PI);
    TxC T = make_txc(*tx);
    const int npol = tx->pol == 2 ? 2 : 1;
    const V3<double> s{tx->pos[0], tx->pos[1], tx->pos[2]};
    std::vector<DepList> lists(nw), slacks(slack_out ? nw : 0);
    std::vector<ReplayState> rss(nw);
    for (auto& r : rss) std::memset(&r.rep, 0, sizeof r.rep);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w = 0; w < nw; ++w) {
        Sink<double> sink{&lists[w]};
        Sink<double> slack_sink{slack_out ? &slacks[w] : nullptr};
        ReplayState& rs = rss[w];
        const Wedge R = oriented(WS[w], s);
        const bool lit = dot(s - R.o, R.n0) >= 0.0;
        const Cx<double> eta0 = permittivity(S.eps[R.mat0], S.sigma[R.mat0], omega);
        const Cx<double> etan = permittivity(S.eps[R.matn], S.sigma[R.matn], omega);
        for (int64_t i = 0; i < NS; ++i) {
            int32_t* rc = rec ? rec + 4 * (w * NS + i) : nullptr;
            if (mode == 1) rs.rep.segments++;
            double u1, u2;
            wedge_sample(i, NS, &u1, &u2);
            const double x = u1 * R.len, phi = u2 * R.n * PI;
            V3<double> v, ks;
            keller(R, s, x, phi, &v, &ks);
            const double vm = std::max(std::fabs(v.x), std::max(std::fabs(v.y), std::fabs(v.z)));
            const double eps = std::ldexp(std::max(1.0, vm), -16);
            const V3<double> sv = v - s;
            const double sprime = norm(sv);
            const V3<double> si = scl(sv, 1.0 / sprime);
            int code = -2;
            int ncross = 0;
            if (lit) {
                code = blocked(S, s, si, eps, sprime - eps, R.tri0, R.trin) ? 1 : 0;
                if (mode == 1 && rc[0] != code) {
                    const double tol = tie_tol(v, sprime);
                    if (rc[0] < 0 || !blocked_near_tie(S, s, si, eps, sprime - eps, R.tri0, R.trin, tol)) {
                        rs.fail(w * NS + i, 0, 5, code, rc[0], 0, 0);
                        continue;
                    }
                    rs.rep.adopted_hit++;
                    code = rc[0];
                }
            } else if (mode == 1 && rc[0] != -2) {
                rs.fail(w * NS + i, 0, 6, code, rc[0], 0, 0);
                continue;
            }
            if (code == 0) {
                const std::complex<double> al = array_factor(T, si, k0);
                auto power = [&](const V3<double>& kd_, double sobs) {
                    double pw = 0.0;
                    for (int p = 0; p < npol; ++p) {
                        const V3<double> f = tx_field(si, T.R, tx->pattern, tx->pol == 2 ? p : tx->pol);
                        const CV3<double> E{Cx<double>(f.x * al.real(), f.x * al.imag()),
                                            Cx<double>(f.y * al.real(), f.y * al.imag()),
                                            Cx<double>(f.z * al.real(), f.z * al.imag())};
                        std::complex<double> ed[2];
                        utd_field(R, eta0, etan, k0, s, v, kd_, sobs, E, ed);
                        pw += std::norm(ed[0]) + std::norm(ed[1]);
                    }
                    return pw;
                };
                for (int64_t j = 0; j < M.n; ++j) {
                    if (M.inv_area[j] == 0.0) continue;
                    V3<double> pv = cross(ks, M.e2[j]);
                    const double det = dot(M.e1[j], pv);
                    if (det == 0.0) continue;
                    const V3<double> tv = v - M.a[j];
                    const double uu = dot(tv, pv) / det;
                    const V3<double> qv = cross(tv, M.e1[j]);
                    const double vv = dot(ks, qv) / det;
                    const double t = dot(M.e2[j], qv) / det;
                    const double ww = 1.0 - uu - vv;
                    const double tol = tie_tol(v + scl(ks, t), sprime + std::max(t, 0.0));
                    const double tb = tol * M.max_edge[j] * 0.5 * M.inv_area[j];
                    const double mn = std::min(uu, std::min(vv, ww));
                    const bool inside = mn >= 0.0 && t > 1e-9;
                    const bool near = (std::fabs(mn) <= tb && t > -tol) || (mn >= -tb && std::fabs(t - 1e-9) <= tol);
                    if (!inside && !near) continue;
                    if (inside) ++ncross;
                    // visibility of the edge-to-crossing segment
                    const double tt = std::max(t, 0.0);
                    const bool bd = blocked(S, v, ks, eps, tt, R.tri0, R.trin);
                    const bool vis_tie = blocked_near_tie(S, v, ks, eps, tt, R.tri0, R.trin, tol);
                    if (bd && !vis_tie) continue;
                    // weighting factor on the triangle's plane: t(x, phi) = v + gam ks with
                    // n.(t - a) = 0, by dual numbers
                    const V3<double> nj = cross(M.e1[j], M.e2[j]);
                    D xd(x), pd(phi);
                    xd.g[0] = 1.0;
                    pd.g[1] = 1.0;
                    V3<D> vd, kd;
                    keller(R, s, xd, pd, &vd, &kd);
                    const D num = D(dot(nj, M.a[j])) - (vd.x * nj.x + vd.y * nj.y + vd.z * nj.z);
                    const D den = kd.x * nj.x + kd.y * nj.y + kd.z * nj.z;
                    const D gam = num / den;
                    const V3<double> tx_{vd.x.g[0] + gam.g[0] * kd.x.v + gam.v * kd.x.g[0],
                                         vd.y.g[0] + gam.g[0] * kd.y.v + gam.v * kd.y.g[0],
                                         vd.z.g[0] + gam.g[0] * kd.z.v + gam.v * kd.z.g[0]};
                    const V3<double> tp_{vd.x.g[1] + gam.g[1] * kd.x.v + gam.v * kd.x.g[1],
                                         vd.y.g[1] + gam.g[1] * kd.y.v + gam.v * kd.y.g[1],
                                         vd.z.g[1] + gam.g[1] * kd.z.v + gam.v * kd.z.g[1]};
                    const double J = norm(cross(tx_, tp_));
                    const double wgt = lam4pi * lam4pi * J * (R.len * R.n * PI / (double)NS) * M.inv_area[j];
                    if (!(tt > 0.0)) continue;
                    const double value = wgt * power(ks, tt);
                    if (inside && !bd) sink.add((int)j, value);
                    if (slack_out) {
                        double az = 0.0;
                        for (double dphi : {-1e-5, 1e-5}) {
                            V3<double> v2, k2;
                            keller(R, s, x, phi + dphi, &v2, &k2);
                            az = std::max(az, std::fabs(wgt * power(k2, tt) - value));
                        }
                        slack_sink.add((int)j, ((near || vis_tie) ? value : 0.0) + az);
                    }
                }
            }
            if (rc && mode == 0) {
                rc[0] = code;
                rc[1] = ncross;
                rc[2] = 0;
                rc[3] = 0;
            }
        }
    }
    std::memset(map_out, 0, sizeof(double) * (size_t)n_surf);
    for (int64_t w = 0; w < nw; ++w)
        for (size_t j = 0; j < lists[w].cell.size(); ++j) map_out[lists[w].cell[j]] += lists[w].val[j];
    if (slack_out) {
        std::memset(slack_out, 0, sizeof(double) * (size_t)n_surf);
        for (int64_t w = 0; w < nw; ++w)
            for (size_t j = 0; j < slacks[w].cell.size(); ++j) slack_out[slacks[w].cell[j]] += slacks[w].val[j];
    }
    if (report) {
        std::memset(report, 0, sizeof *report);
        bool have = false;
        for (int64_t w = 0; w < nw; ++w) {
            const or_report& r = rss[w].rep;
            report->segments += r.segments;
            report->adopted_hit += r.adopted_hit;
            report->failures += r.failures;
            if (r.failures && !have) {
                have = true;
                report->fail_ray = r.fail_ray;
                report->fail_kind = r.fail_kind;
                std::memcpy(report->fail_info, r.fail_info, sizeof r.fail_info);
            }
        }
    }
    return 0;
}

}  // extern "C"
