// Synthetic transmit arrays (Sec. 4.4): the array factor
//   alpha(k) = sum_a w_a exp(j k0 k.d_a)
// of a ray leaving in direction k, where d_a is element a's position (global
// frame) and w_a its precoding weight.  Phases reach k0 |d| (about 1600 rad
// for a 1024-element half-wavelength array), beyond what an FP32 phase or an
// FP32 lattice direction resolves near the array factor's nulls, so:
//   - the lattice direction is rebuilt as double-float pairs (hi + lo) for
//     array transmitters only (lattice_dir_df);
//   - each element's phase in units of pi, k.d'_a with d' = (2 / lambda0) d
//     stored as hi + lo floats, is reduced modulo 2 with error-free products
//     (FMA) before one sincospif of an argument in [-1, 1];
//   - elements on a regular line (uniform linear arrays, detected on the host)
//     take a blocked Horner recurrence: per block of ULA_BLOCK elements one
//     exact anchor exp(j pi (k.d'_0 + m k.delta')) and powers of
//     z = exp(j pi k.delta') inside the block.
// Double-float arithmetic follows Dekker's and Knuth's error-free
// transformations (TwoSum, TwoProduct by FMA); it needs the file compiled with
// -fmad=false so that no a * b + c is contracted behind its back.
#pragma once

#include "common.cuh"

namespace rmsbr {

constexpr int ULA_BLOCK = 16;

struct df { float h, l; };

static __device__ __forceinline__ df two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
static __device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = a + b;
    return {s, b - (s - a)};
}
static __device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, s.l + (a.l + b.l));
}
static __device__ __forceinline__ df df_mul(df a, df b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p) + (a.h * b.l + a.l * b.h);
    return fast_two_sum(p, e);
}
// an unsigned 64-bit integer v < 2^62 as hi + lo
static __device__ __forceinline__ df df_from_u64(unsigned long long v) {
    const float h = __ull2float_rn(v);
    const long long r = (long long)(v - (unsigned long long)h);
    return {h, __ll2float_rn(r)};
}
// a / b for b > 0: one approximate quotient, one correction from the exact residual
static __device__ __forceinline__ df df_div(df a, df b) {
    const float q = a.h / b.h;
    const float p = q * b.h;
    const float e = fmaf(q, b.h, -p);
    const float r = (((a.h - p) - e) + a.l) - q * b.l;
    return fast_two_sum(q, r / b.h);
}
static __device__ __forceinline__ df df_sqrt(df a) {
    if (a.h <= 0.0f) return {0.0f, 0.0f};
    const float s = sqrtf(a.h);
    const float p = s * s;
    const float e = fmaf(s, s, -p);
    return fast_two_sum(s, (((a.h - p) - e) + a.l) / (2.0f * s));
}

// sin(pi j / 64), cos(pi j / 64) for j = 0..64, each rounded to hi + lo floats
static __device__ const float SINCOS_PI_64[65][4] = {
    {0.0f, 0.0f, 1.0f, 0.0f},
    {0.049067676067352295f, -1.7399343077428853e-09f, 0.9987954497337341f, 6.471438496191695e-09f},
    {0.0980171412229538f, -8.933931927579408e-10f, 0.9951847195625305f, 7.1096666331982306e-09f},
    {0.1467304676771164f, 6.778245520422388e-09f, 0.9891765117645264f, -1.7997453527485163e-09f},
    {0.19509032368659973f, -1.6704715388726754e-09f, 0.9807852506637573f, 2.9739473106360492e-08f},
    {0.24298018217086792f, -2.267604104488896e-09f, 0.9700312614440918f, -8.249547711614014e-09f},
    {0.290284663438797f, 1.3815665056426951e-08f, 0.9569403529167175f, -1.7184508038781132e-08f},
    {0.3368898630142212f, -9.622000973763534e-09f, 0.9415440559387207f, 9.244300436250796e-09f},
    {0.3826834261417389f, 6.2233507236442165e-09f, 0.9238795042037964f, 2.830748968563057e-08f},
    {0.4275550842285156f, 9.201766459909777e-09f, 0.903989315032959f, -2.1909515979245953e-08f},
    {0.4713967442512512f, -7.425253745196869e-09f, 0.8819212913513184f, -2.7002963420841297e-08f},
    {0.5141027569770813f, -1.2783859304477119e-08f, 0.8577286005020142f, 9.498258179974073e-09f},
    {0.5555702447891235f, -1.1769521357507529e-08f, 0.8314695954322815f, 1.687026340846387e-08f},
    {0.5956993103027344f, -5.810301129116624e-09f, 0.803207516670227f, 1.4810417781063734e-08f},
    {0.6343932747840881f, 9.37955757507325e-09f, 0.7730104327201843f, 2.0642552556182636e-08f},
    {0.6715589761734009f, -2.1326382437791835e-08f, 0.7409511208534241f, 4.501535144640911e-09f},
    {0.7071067690849304f, 1.2101617485882343e-08f, 0.7071067690849304f, 1.2101617485882343e-08f},
    {0.7409511208534241f, 4.501535144640911e-09f, 0.6715589761734009f, -2.1326382437791835e-08f},
    {0.7730104327201843f, 2.0642552556182636e-08f, 0.6343932747840881f, 9.37955757507325e-09f},
    {0.803207516670227f, 1.4810417781063734e-08f, 0.5956993103027344f, -5.810300685027414e-09f},
    {0.8314695954322815f, 1.687026340846387e-08f, 0.5555702447891235f, -1.1769521357507529e-08f},
    {0.8577286005020142f, 9.498258179974073e-09f, 0.5141027569770813f, -1.2783859304477119e-08f},
    {0.8819212913513184f, -2.7002963420841297e-08f, 0.4713967442512512f, -7.425253301107659e-09f},
    {0.903989315032959f, -2.1909515979245953e-08f, 0.4275550842285156f, 9.201766459909777e-09f},
    {0.9238795042037964f, 2.830748968563057e-08f, 0.3826834261417389f, 6.2233507236442165e-09f},
    {0.9415440559387207f, 9.244300436250796e-09f, 0.3368898630142212f, -9.622000973763534e-09f},
    {0.9569403529167175f, -1.7184508038781132e-08f, 0.290284663438797f, 1.3815665056426951e-08f},
    {0.9700312614440918f, -8.249547711614014e-09f, 0.24298018217086792f, -2.2676038824442912e-09f},
    {0.9807852506637573f, 2.9739473106360492e-08f, 0.19509032368659973f, -1.670471427850373e-09f},
    {0.9891765117645264f, -1.7997453527485163e-09f, 0.1467304676771164f, 6.778245520422388e-09f},
    {0.9951847195625305f, 7.109666189109021e-09f, 0.0980171412229538f, -8.933930262244871e-10f},
    {0.9987954497337341f, 6.471438496191695e-09f, 0.049067676067352295f, -1.7399341967205828e-09f},
    {1.0f, 0.0f, 0.0f, 0.0f},
    {0.9987954497337341f, 6.471438496191695e-09f, -0.049067676067352295f, 1.7399343077428853e-09f},
    {0.9951847195625305f, 7.1096666331982306e-09f, -0.0980171412229538f, 8.933931372467896e-10f},
    {0.9891765117645264f, -1.7997453527485163e-09f, -0.1467304676771164f, -6.778245076333178e-09f},
    {0.9807852506637573f, 2.9739473106360492e-08f, -0.19509032368659973f, 1.6704715388726754e-09f},
    {0.9700312614440918f, -8.249547711614014e-09f, -0.24298018217086792f, 2.267604104488896e-09f},
    {0.9569403529167175f, -1.7184508038781132e-08f, -0.290284663438797f, -1.3815665056426951e-08f},
    {0.9415440559387207f, 9.244300436250796e-09f, -0.3368898630142212f, 9.622000973763534e-09f},
    {0.9238795042037964f, 2.830748968563057e-08f, -0.3826834261417389f, -6.2233507236442165e-09f},
    {0.903989315032959f, -2.1909515979245953e-08f, -0.4275550842285156f, -9.201766459909777e-09f},
    {0.8819212913513184f, -2.7002963420841297e-08f, -0.4713967442512512f, 7.425253301107659e-09f},
    {0.8577286005020142f, 9.498258179974073e-09f, -0.5141027569770813f, 1.2783859304477119e-08f},
    {0.8314695954322815f, 1.687026340846387e-08f, -0.5555702447891235f, 1.1769521357507529e-08f},
    {0.803207516670227f, 1.4810417781063734e-08f, -0.5956993103027344f, 5.810301129116624e-09f},
    {0.7730104327201843f, 2.0642552556182636e-08f, -0.6343932747840881f, -9.37955757507325e-09f},
    {0.7409511208534241f, 4.501535144640911e-09f, -0.6715589761734009f, 2.1326382437791835e-08f},
    {0.7071067690849304f, 1.2101617485882343e-08f, -0.7071067690849304f, -1.2101617485882343e-08f},
    {0.6715589761734009f, -2.1326382437791835e-08f, -0.7409511208534241f, -4.5015347005517015e-09f},
    {0.6343932747840881f, 9.37955757507325e-09f, -0.7730104327201843f, -2.0642552556182636e-08f},
    {0.5956993103027344f, -5.810300685027414e-09f, -0.803207516670227f, -1.4810417781063734e-08f},
    {0.5555702447891235f, -1.1769521357507529e-08f, -0.8314695954322815f, -1.687026340846387e-08f},
    {0.5141027569770813f, -1.2783859304477119e-08f, -0.8577286005020142f, -9.498258179974073e-09f},
    {0.4713967442512512f, -7.425253301107659e-09f, -0.8819212913513184f, 2.7002963420841297e-08f},
    {0.4275550842285156f, 9.201766459909777e-09f, -0.903989315032959f, 2.1909515979245953e-08f},
    {0.3826834261417389f, 6.223351167733426e-09f, -0.9238795042037964f, -2.830748968563057e-08f},
    {0.3368898630142212f, -9.622000973763534e-09f, -0.9415440559387207f, -9.244299548072377e-09f},
    {0.290284663438797f, 1.3815665056426951e-08f, -0.9569403529167175f, 1.7184508038781132e-08f},
    {0.24298018217086792f, -2.2676038824442912e-09f, -0.9700312614440918f, 8.249547711614014e-09f},
    {0.19509032368659973f, -1.6704710947834656e-09f, -0.9807852506637573f, -2.9739473106360492e-08f},
    {0.1467304676771164f, 6.778245520422388e-09f, -0.9891765117645264f, 1.7997453527485163e-09f},
    {0.0980171412229538f, -8.933929707133359e-10f, -0.9951847195625305f, -7.109666189109021e-09f},
    {0.049067676067352295f, -1.7399343077428853e-09f, -0.9987954497337341f, -6.471438496191695e-09f},
    {0.0f, 0.0f, -1.0f, 0.0f}
};

// sin(pi x), cos(pi x) for x = x.h + x.l in [-1, 1] to ~1e-12: x = j / 64 + r
// with |r| <= 1/128, the table at j and the Taylor series of sin and cos of
// y = pi r (|y| <= 0.0246; the first omitted terms are below 1e-15).
static __device__ __forceinline__ void df_sincospi(df x, df& sn, df& cs) {
    const float jf = rintf(x.h * 64.0f);
    const df r = two_sum(x.h - jf * 0.015625f, x.l);  // x.h - j/64 is exact
    const df y = df_mul(r, df{3.14159274101257324f, -8.74227765734758578e-08f});
    const float y2 = y.h * y.h;
    // sin y = y - y^3/6 + y^5/120 - y^7/5040
    const float ts = y.h * y2 * (-0.166666672f + y2 * (8.33333377e-03f - y2 * 1.98412701e-04f));
    const df sy = df_add(y, df{ts, 0.0f});
    // cos y = 1 - y^2/2 + y^4/24 - y^6/720
    const float p = y.h * y.h;
    const float pe = fmaf(y.h, y.h, -p) + 2.0f * y.h * y.l;
    const float tc = y2 * y2 * (4.16666679e-02f - y2 * 1.38888892e-03f);
    const df c0 = two_sum(1.0f, -0.5f * p);
    const df cy = fast_two_sum(c0.h, c0.l + (tc - 0.5f * pe));
    const int j = (int)jf;
    const int ja = j < 0 ? -j : j;
    const float sg = j < 0 ? -1.0f : 1.0f;
    const df sj{sg * SINCOS_PI_64[ja][0], sg * SINCOS_PI_64[ja][1]};
    const df cj{SINCOS_PI_64[ja][2], SINCOS_PI_64[ja][3]};
    // sin(a + y) = sin a cos y + cos a sin y; cos(a + y) = cos a cos y - sin a sin y
    sn = df_add(df_mul(sj, cy), df_mul(cj, sy));
    const df m = df_mul(sj, sy);
    cs = df_add(df_mul(cj, cy), df{-m.h, -m.l});
}

// The Fibonacci lattice direction of item n of N (Sec. 3.1.1) as double-float
// components: cos theta = 1 - 2n/(N-1), sin theta = 2 sqrt(n (N-1-n)) / (N-1),
// phi = 2 pi frac(n (phi_g - 1)), with frac(n (phi_g - 1)) the 64-bit Weyl
// product n * round(2^64 (phi_g - 1)) mod 2^64.  N >= 2, N < 2^62.
static __device__ __forceinline__ void lattice_dir_df(unsigned long long n, unsigned long long N, df k[3]) {
    const unsigned long long Nm1 = N - 1ULL;
    const df d = df_from_u64(Nm1);
    const df a = df_div(df_from_u64(n), d);          // (1 - cos theta) / 2
    const df b = df_div(df_from_u64(Nm1 - n), d);    // (1 + cos theta) / 2
    const df ct = df_add(b, df{-a.h, -a.l});
    const df st0 = df_sqrt(df_mul(a, b));
    const df st{2.0f * st0.h, 2.0f * st0.l};
    // phi / pi = signed(f) 2^-63 in [-1, 1): 24 high bits exactly, the rest below 2^-23
    const long long f = (long long)(n * 0x9E3779B97F4A7C16ULL);
    const long long fh = f >> 40;                    // arithmetic shift: floor(f / 2^40)
    const df x = two_sum((float)fh * 0x1p-23f, (float)(f & 0xFFFFFFFFFFLL) * 0x1p-63f);
    df sp, cp;
    df_sincospi(x, sp, cp);
    k[0] = df_mul(st, cp);
    k[1] = df_mul(st, sp);
    k[2] = ct;
}

// k.v in units of pi reduced modulo 2 (result in [-1, 1] up to ~1e-7 of
// rounding), for a double-float direction k and an offset v = vh + vl in units
// of lambda0 / 2: each product kh_i vh_i splits exactly into its value and FMA
// error, the values are reduced modulo 2 exactly and summed with TwoSum.
static __device__ __forceinline__ df phase_pi(const df k[3], const float vh[3], const float vl[3]) {
    float small = 0.0f;
    float r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float p = k[i].h * vh[i];
        small += fmaf(k[i].h, vh[i], -p) + (k[i].h * vl[i] + k[i].l * vh[i]);
        r[i] = p - 2.0f * rintf(0.5f * p);
    }
    const df s1 = two_sum(r[0], r[1]);
    const df s2 = two_sum(s1.h, r[2]);
    const float h = s2.h - 2.0f * rintf(0.5f * s2.h);
    return fast_two_sum(h, (s1.l + s2.l) + small);
}

// Table layout per transmitter (at ant + T.ant_begin):
//   T.ant_mode == 0: n_ant records {w re, w im, d'h xyz, d'l xyz};
//   T.ant_mode == 1 (uniform linear array d_a = d_0 + a delta): record 0 holds
//     d'_0, record 1 holds delta' (both as hi, lo in the d' fields), then the
//     weights packed as float2 pairs from record 2 on.
// WIDE (the alpha pre-pass, a kernel of its own): four Horner chains at a time,
// unrolled; the same operations per block and the same order of the block sums
// as the tracer's two rolled chains, so the same bits.
template <bool WIDE = false>
static __device__ __forceinline__ void array_sum(const TxDev& T, const AntDev* __restrict__ ant, const df k[3],
                                                 float& are, float& aim) {
    const AntDev* e = ant + T.ant_begin;
    float ar = 0.0f, ai = 0.0f;
    if (T.ant_mode == 1) {
        const df p0 = phase_pi(k, e[0].dh, e[0].dl);
        const df q = phase_pi(k, e[1].dh, e[1].dl);
        float zs, zc;
        sincospif(q.h + q.l, &zs, &zc);
        const float2* w = reinterpret_cast<const float2*>(e + 2);
        // anchor exp(j pi (p0 + b0 q)) of the block starting at element b0, with b0 q split exactly
        auto anchor = [&](int b0, float& as, float& ac) {
            const float m = (float)b0;
            const float pm = m * q.h;
            const float pr = pm - 2.0f * rintf(0.5f * pm);
            const df s = two_sum(pr, p0.h);
            const float t = s.h - 2.0f * rintf(0.5f * s.h);
            sincospif(t + (s.l + (p0.l + (fmaf(m, q.h, -pm) + m * q.l))), &as, &ac);
        };
        int b0 = 0;
        if constexpr (WIDE) {
            // two pairs of blocks at a time
            for (; b0 + 4 * ULA_BLOCK <= T.n_ant; b0 += 4 * ULA_BLOCK) {
                float hr[4], hi[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float2 wl = w[b0 + c * ULA_BLOCK + ULA_BLOCK - 1];
                    hr[c] = wl.x;
                    hi[c] = wl.y;
                }
#pragma unroll
                for (int i = ULA_BLOCK - 2; i >= 0; --i) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float2 wc = w[b0 + c * ULA_BLOCK + i];
                        const float nr = fmaf(hr[c], zc, fmaf(-hi[c], zs, wc.x));
                        hi[c] = fmaf(hr[c], zs, fmaf(hi[c], zc, wc.y));
                        hr[c] = nr;
                    }
                }
#pragma unroll
                for (int pr = 0; pr < 2; ++pr) {
                    const int c = 2 * pr;
                    float as, ac, bs, bc;
                    anchor(b0 + c * ULA_BLOCK, as, ac);
                    anchor(b0 + (c + 1) * ULA_BLOCK, bs, bc);
                    ar += (ac * hr[c] - as * hi[c]) + (bc * hr[c + 1] - bs * hi[c + 1]);
                    ai += (ac * hi[c] + as * hr[c]) + (bc * hi[c + 1] + bs * hr[c + 1]);
                }
            }
        }
        // full pairs of blocks: two independent Horner chains h = sum_i w_(b+i) z^i (kept
        // rolled: in this form the tracer's hot loop, which shares the kernel, measured
        // 9 % faster than with a single chain or an unrolled pair loop)
        for (; b0 + 2 * ULA_BLOCK <= T.n_ant; b0 += 2 * ULA_BLOCK) {
            float2 wa = w[b0 + ULA_BLOCK - 1], wb = w[b0 + 2 * ULA_BLOCK - 1];
            float ar_ = wa.x, ai_ = wa.y, br_ = wb.x, bi_ = wb.y;
#pragma unroll 1
            for (int i = ULA_BLOCK - 2; i >= 0; --i) {
                wa = w[b0 + i];
                wb = w[b0 + ULA_BLOCK + i];
                const float na = fmaf(ar_, zc, fmaf(-ai_, zs, wa.x));
                ai_ = fmaf(ar_, zs, fmaf(ai_, zc, wa.y));
                ar_ = na;
                const float nb = fmaf(br_, zc, fmaf(-bi_, zs, wb.x));
                bi_ = fmaf(br_, zs, fmaf(bi_, zc, wb.y));
                br_ = nb;
            }
            float as, ac, bs, bc;
            anchor(b0, as, ac);
            anchor(b0 + ULA_BLOCK, bs, bc);
            ar += (ac * ar_ - as * ai_) + (bc * br_ - bs * bi_);
            ai += (ac * ai_ + as * ar_) + (bc * bi_ + bs * br_);
        }
        // the remaining (at most two, the last one ragged) blocks
        for (; b0 < T.n_ant; b0 += ULA_BLOCK) {
            const int b1 = min(b0 + ULA_BLOCK, T.n_ant) - 1;
            float2 wa = w[b1];
            float hr = wa.x, hi = wa.y;
#pragma unroll 4
            for (int a = b1 - 1; a >= b0; --a) {
                wa = w[a];
                const float nr = fmaf(hr, zc, fmaf(-hi, zs, wa.x));
                hi = fmaf(hr, zs, fmaf(hi, zc, wa.y));
                hr = nr;
            }
            float as, ac;
            anchor(b0, as, ac);
            ar += ac * hr - as * hi;
            ai += ac * hi + as * hr;
        }
    } else {
        for (int b0 = 0; b0 < T.n_ant; b0 += ULA_BLOCK) {
            const int b1 = min(b0 + ULA_BLOCK, T.n_ant);
            float br = 0.0f, bi = 0.0f;
            for (int a = b0; a < b1; ++a) {
                const AntDev el = e[a];
                const df ph = phase_pi(k, el.dh, el.dl);
                float sn, cs;
                sincospif(ph.h + ph.l, &sn, &cs);
                br += el.pre * cs - el.pim * sn;
                bi += el.pre * sn + el.pim * cs;
            }
            ar += br;
            ai += bi;
        }
    }
    are = ar;
    aim = ai;
}

// alpha for the ray of lattice item n (the tracer's launch; inlined: a call
// there costs the tracer spills around it)
static __device__ __forceinline__ void array_factor_lattice(const TxDev& T, const AntDev* __restrict__ ant,
                                                         unsigned long long n, float& are, float& aim) {
    df k[3] = {{-1.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};  // N = 1: the kernel's single direction
    if (T.N > 1ULL) lattice_dir_df(n, T.N, k);
    array_sum(T, ant, k, are, aim);
}

// the same alpha through the four-chain form (the pre-pass kernel)
static __device__ __forceinline__ void array_factor_lattice_wide(const TxDev& T, const AntDev* __restrict__ ant,
                                                              unsigned long long n, float& are, float& aim) {
    df k[3] = {{-1.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    if (T.N > 1ULL) lattice_dir_df(n, T.N, k);
    array_sum<true>(T, ant, k, are, aim);
}

// alpha for an FP32 direction (diffraction: the direction to a wedge sample)
static __device__ __noinline__ void array_factor_dir(const TxDev& T, const AntDev* __restrict__ ant, float kx,
                                                     float ky, float kz, float& are, float& aim) {
    const df k[3] = {{kx, 0.0f}, {ky, 0.0f}, {kz, 0.0f}};
    array_sum(T, ant, k, are, aim);
}

}  // namespace rmsbr
