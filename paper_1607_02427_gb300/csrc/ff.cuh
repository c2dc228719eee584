// ff.cuh -- float-float ("double-float") arithmetic for the FP32 + two-sum
// precision mode (DEM_FP32_COMP) of the pair kernels.
//
// A value is the unevaluated sum h + l of two floats, |l| <= ulp(h) / 2
// after normalisation: about 48 significant bits on the FP32 pipes (FP64 runs
// at a small fraction of the FP32 rate on this part).  The building blocks
// are the error-free transformations of Knuth (TwoSum: a + b = s + e exactly)
// and of the fused multiply-add (a b = p + e exactly, e = fma(a, b, -p)),
// combined as in Dekker's double-length arithmetic (Numer. Math. 18 (1971)).
// Products and sums drop only terms below about 2^-44 of the result.
//
// In the FP32 + two-sum mode the culls and nearest-point searches run in
// FP32 as in the FP32 mode; each term that survives (r < r_cut) is then
// re-evaluated from the FP64 state split into hi + lo floats: the positions,
// quaternions and geometry tables (pair_kernels.cuh, refined_values).  The
// nearest points' parameters, the separation, the WCA factor, force and
// torque carry float-float precision into the compensated sums; the only
// FP32 rounding left is the final body-to-world rotation of each particle's
// totals, relative to that total.
#pragma once

namespace dem {

struct ff {
    float h, l;
};

__device__ __forceinline__ ff ff_of(float x) { return {x, 0.f}; }

// a + b = s + e exactly (no ordering requirement)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// s + e for |s| >= |e| (or s = 0), renormalised
__device__ __forceinline__ ff ff_norm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return ff_norm(s, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.h, -a.l}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
    return ff_norm(p, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return ff_norm(p, e);
}
// exact scaling by a power of two
__device__ __forceinline__ ff ff_scale2(ff a, float p2) { return {a.h * p2, a.l * p2}; }

// 1 / a: one Newton step x + x (1 - a x) from the FP32 reciprocal
__device__ __forceinline__ ff ff_recip(ff a) {
    const float x = __frcp_rn(a.h);
    const ff ax = ff_mul_f(a, x);
    const ff r = ff_sub(ff_of(1.f), ax);
    return ff_norm(x, __fmul_rn(x, r.h));
}

__device__ __forceinline__ float ff_to_f(ff a) { return __fadd_rn(a.h, a.l); }

// a / b: FP32 quotient, corrected by the float-float remainder
__device__ __forceinline__ ff ff_div(ff a, ff b) {
    const float q1 = __fdiv_rn(a.h, b.h);
    const ff r = ff_sub(a, ff_mul_f(b, q1));
    return ff_norm(q1, __fdiv_rn(r.h, b.h));
}
// clamp to [0, 1] (the decision on the leading part)
__device__ __forceinline__ ff ff_clamp01(ff t) {
    if (t.h < 0.f) return ff_of(0.f);
    if (t.h > 1.f) return ff_of(1.f);
    return t;
}
__device__ __forceinline__ bool ff_lt(ff a, ff b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ ff ff_min(ff a, ff b) { return ff_lt(a, b) ? a : b; }
__device__ __forceinline__ ff ff_max(ff a, ff b) { return ff_lt(a, b) ? b : a; }

// ---- vectors ----
struct ff3 {
    ff x, y, z;
};
__device__ __forceinline__ ff3 ff3_of(float x, float y, float z) {
    return {ff_of(x), ff_of(y), ff_of(z)};
}
// hi + lo float4 pairs (x, y, z; w ignored)
__device__ __forceinline__ ff3 ff3_of(const float4 &h, const float4 &l) {
    return {{h.x, l.x}, {h.y, l.y}, {h.z, l.z}};
}
__device__ __forceinline__ ff3 operator+(ff3 a, ff3 b) {
    return {ff_add(a.x, b.x), ff_add(a.y, b.y), ff_add(a.z, b.z)};
}
__device__ __forceinline__ ff3 operator-(ff3 a, ff3 b) {
    return {ff_sub(a.x, b.x), ff_sub(a.y, b.y), ff_sub(a.z, b.z)};
}
__device__ __forceinline__ ff3 ff3_mul(ff3 a, ff s) {
    return {ff_mul(a.x, s), ff_mul(a.y, s), ff_mul(a.z, s)};
}
__device__ __forceinline__ ff3 ff3_mul_f(ff3 a, float s) {
    return {ff_mul_f(a.x, s), ff_mul_f(a.y, s), ff_mul_f(a.z, s)};
}
__device__ __forceinline__ ff ff3_dot(ff3 a, ff3 b) {
    return ff_add(ff_add(ff_mul(a.x, b.x), ff_mul(a.y, b.y)), ff_mul(a.z, b.z));
}
__device__ __forceinline__ ff3 ff3_cross(ff3 a, ff3 b) {
    return {ff_sub(ff_mul(a.y, b.z), ff_mul(a.z, b.y)), ff_sub(ff_mul(a.z, b.x), ff_mul(a.x, b.z)),
            ff_sub(ff_mul(a.x, b.y), ff_mul(a.y, b.x))};
}
// A + t D (t a float: a searched segment parameter, taken as exact)
__device__ __forceinline__ ff3 ff3_point(ff3 A, ff3 D, float t) { return A + ff3_mul_f(D, t); }
__device__ __forceinline__ ff3 ff3_point(ff3 A, ff3 D, ff t) { return A + ff3_mul(D, t); }

// Rotation of v by the unit quaternion (w, u): v + 2 w (u x v) + 2 u x (u x v).
// conj = true rotates by the conjugate (the inverse rotation).
__device__ __forceinline__ ff3 ff3_rotate(ff w, ff3 u, ff3 v, bool conj) {
    if (conj) u = {ff_neg(u.x), ff_neg(u.y), ff_neg(u.z)};
    ff3 t = ff3_cross(u, v);
    t = {ff_scale2(t.x, 2.f), ff_scale2(t.y, 2.f), ff_scale2(t.z, 2.f)};
    return v + ff3_mul(t, w) + ff3_cross(u, t);
}

}  // namespace dem
