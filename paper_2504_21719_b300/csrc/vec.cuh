// Small complex and 3-vector helpers of the device code (FP32).
#pragma once

#include <cuda_runtime.h>

namespace rmsbr {

// ------------------------------------------------------------------ min / max
// Three-input minimum and maximum (PTX min.f32 / max.f32 with three sources,
// sm_100 and later).  Both are exact, so they equal the two-step fminf /
// fmaxf chains bit for bit on the slab tests' finite distances.
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// ------------------------------------------------------------------ complex
struct cf {
    float r, i;
};
__device__ __forceinline__ cf C(float r, float i = 0.0f) { return {r, i}; }
__device__ __forceinline__ cf operator+(cf a, cf b) { return {a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ cf operator-(cf a, cf b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cf operator*(cf a, cf b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cf operator*(cf a, float s) { return {a.r * s, a.i * s}; }
__device__ __forceinline__ cf cdiv(cf a, cf b) {
    const float inv = 1.0f / (b.r * b.r + b.i * b.i);
    return {(a.r * b.r + a.i * b.i) * inv, (a.i * b.r - a.r * b.i) * inv};
}
__device__ __forceinline__ float cabs2(cf a) { return a.r * a.r + a.i * a.i; }
// conj(a) * b
__device__ __forceinline__ cf cjmul(cf a, cf b) { return {a.r * b.r + a.i * b.i, a.r * b.i - a.i * b.r}; }
// principal square root: sqrt((|z|+x)/2) + j sgn(y) sqrt((|z|-x)/2), with the
// smaller part formed as y / (2 * larger) (Kahan 1987) to avoid cancellation
__device__ __forceinline__ cf csqrt_p(cf z) {
    if (z.r == 0.0f && z.i == 0.0f) return {0.0f, 0.0f};
    const float m = sqrtf(z.r * z.r + z.i * z.i);   // |eta| << 1e19: no overflow
    if (z.r >= 0.0f) {
        const float a = sqrtf(0.5f * (m + z.r));
        return {a, z.i / (2.0f * a)};
    }
    const float b = sqrtf(0.5f * (m - z.r));
    return {fabsf(z.i) / (2.0f * b), copysignf(b, z.i)};
}
// exp(-j w) = exp(Im w) (cos Re w - j sin Re w)
__device__ __forceinline__ cf cexp_mj(cf w) {
    float s, c;
    // reduction by multiples of pi is exact in sincospif; the one rounding of
    // w / pi is below the rounding of w itself
    sincospif(w.r * 0.318309886183790672f, &s, &c);
    const float e = __expf(w.i);
    return {e * c, -e * s};
}

struct f3 {
    float x, y, z;
};
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator*(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ f3 normalize(f3 a) { return a * (1.0f / sqrtf(dot(a, a))); }
__device__ __forceinline__ float sel(f3 v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }
// e^T E for a real unit vector e and a complex 3-vector E
__device__ __forceinline__ cf edot(f3 e, const cf* E) { return E[0] * e.x + E[1] * e.y + E[2] * e.z; }


}  // namespace rmsbr
