// step_device.cuh -- the per-particle and per-replica pieces of a time step
// (integrate.cu): the scheme of Section "Energy Conservation" of
// arXiv:1607.02427 (second-order velocity Verlet with the free-rotor
// splitting) and the Nose-Hoover thermostat of Section "Assembly".  The
// step kernels of integrate.cu and the cooperative step kernel of
// persistent.cu call the same functions, so both paths do the same
// arithmetic in the same order.
#pragma once

#include "dem_internal.cuh"

namespace dem {
namespace {

// Conversions between double and float by integer operations on the
// IEEE-754 fields, with the results of the conversion instructions (round to
// nearest, ties to even): those run on the FP64 pipe, a small fraction of the
// FP32 rate on this part, and the first half step makes about forty per
// particle.  On large systems that step is bound by the FP64 pipe and the
// integer form is faster; on small ones it is bound by latency and the
// instruction's shorter chain is (StepArgs.int_conv chooses; the results are
// the same).  Results outside the normal float range (subnormal, overflow,
// infinities, NaN), which the state never produces, take the instruction.
__device__ __forceinline__ float f32_of(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
    const int fe = (int)((u >> 52) & 0x7ff) - 896;          // float exponent field
    if (fe >= 1 && fe <= 254) {
        const unsigned long long m = u & 0xfffffffffffffull;
        const unsigned mant = (unsigned)(m >> 29);
        const unsigned long long rest = m & 0x1fffffffull;   // the 29 bits rounded off
        unsigned r = (unsigned)fe << 23 | mant;
        if (rest > 0x10000000ull || (rest == 0x10000000ull && (mant & 1u))) r += 1u;  // carries into the exponent
        return __uint_as_float(sign | r);
    }
    if ((u << 1) == 0ull) return __uint_as_float(sign);     // signed zero
    return (float)x;
}
__device__ __forceinline__ double f64_of(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    if ((b << 1) == 0u) return __longlong_as_double((long long)sign);
    if (e == 0u || e == 0xffu) return (double)x;
    return __longlong_as_double((long long)(sign | (unsigned long long)(e + 896u) << 52 |
                                            (unsigned long long)(b & 0x7fffffu) << 29));
}
__device__ __forceinline__ float cvt_f(double x, bool ic) { return ic ? f32_of(x) : (float)x; }
__device__ __forceinline__ double cvt_d(float x, bool ic) { return ic ? f64_of(x) : (double)x; }
// x = h + l (h = x rounded to float, l = the rest rounded to float)
__device__ __forceinline__ void split_ff_dev(double x, float *h, float *l, bool ic) {
    const float hi = cvt_f(x, ic);
    *h = hi;
    *l = cvt_f(x - cvt_d(hi, ic), ic);
}

__device__ __forceinline__ void quat_rotate_body(double4_32a &q, int k, double c, double s) {
    // r = (c, s e_k); q <- q (x) r ; q = (x:w, y:x, z:y, w:z)
    double w1 = q.x, x1 = q.y, y1 = q.z, z1 = q.w;
    double w2 = c, x2 = k == 0 ? s : 0.0, y2 = k == 1 ? s : 0.0, z2 = k == 2 ? s : 0.0;
    q.x = w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2;
    q.y = w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2;
    q.z = w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2;
    q.w = w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2;
}

__device__ __forceinline__ double comp(const double4_32a &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : v.z);
}
__device__ __forceinline__ void set_comp(double4_32a &v, int k, double x) {
    if (k == 0) v.x = x; else if (k == 1) v.y = x; else v.z = x;
}

// sin h and cos h for |h| <= 1/8 from their Maclaurin series, evaluated by
// Horner's rule in h^2 and truncated after h^9 (sin) and h^10 (cos).  The
// first omitted terms, h^11/11! and h^12/12!, are below 2.4e-17 |h| and
// 3.1e-20: under half an ulp of either result.
__device__ __forceinline__ void sincos_small(double h, double *s, double *c) {
    const double h2 = h * h;
    double ps = 1.0 / 362880.0;
    ps = fma(ps, h2, -1.0 / 5040.0);
    ps = fma(ps, h2, 1.0 / 120.0);
    ps = fma(ps, h2, -1.0 / 6.0);
    *s = fma(ps * h2, h, h);
    double pc = -1.0 / 3628800.0;
    pc = fma(pc, h2, 1.0 / 40320.0);
    pc = fma(pc, h2, -1.0 / 720.0);
    pc = fma(pc, h2, 1.0 / 24.0);
    pc = fma(pc, h2, -0.5);
    *c = fma(pc, h2, 1.0);
}

// One sine-cosine pair of phi/2 serves both the quaternion (half angle) and
// the angular momentum (cos phi = 1 - 2 s^2, sin phi = 2 s c).  FP64 runs at
// a small fraction of the FP32 rate on this part, so the rotation avoids
// divisions (1/I is stored) and, for the usual small angles, the general
// sincos.
__device__ __forceinline__ void free_rotor_axis(double4_32a &q, double4_32a &L, const double *invI,
                                                int k, double dt) {
    if (!(invI[k] > 0.0)) return;
    const double half = 0.5 * dt * comp(L, k) * invI[k];
    double sh, ch;
    if (fabs(half) <= 0.125) sincos_small(half, &sh, &ch);
    else sincos(half, &sh, &ch);
    quat_rotate_body(q, k, ch, sh);
    int a = (k + 1) % 3, b = (k + 2) % 3;
    double c = 1.0 - 2.0 * sh * sh, s = 2.0 * sh * ch;
    double La = comp(L, a), Lb = comp(L, b);
    set_comp(L, a, c * La + s * Lb);
    set_comp(L, b, -s * La + c * Lb);
}

// FP32: sin h and cos h - 1 (|h| <= 1/8: Maclaurin series, truncated where
// the remainder is below 2e-10 of either result; cos h - 1 comes straight
// from the series, so it keeps its relative precision for small h).
__device__ __forceinline__ void sincosm1_f(float h, float *s, float *cm1) {
    if (fabsf(h) <= 0.125f) {
        const float h2 = h * h;
        *s = fmaf(h2 * fmaf(h2, 1.f / 120.f, -1.f / 6.f), h, h);
        *cm1 = h2 * fmaf(h2, fmaf(h2, -1.f / 720.f, 1.f / 24.f), -0.5f);
    } else {
        const float sh = sinf(0.5f * h);
        *s = sinf(h);
        *cm1 = -2.f * sh * sh;
    }
}

// The free rotor of the FP32 modes: the five sub-rotations (z, y, x, y, z)
// run in FP32 as increments, the change dL of the body angular momentum and
// the composite rotation r = 1 + rho (r = r_1 r_2 ... r_5, each r_s =
// (cos h_s, sin h_s e_k)), and are applied to the FP64 state as L += dL and
// q += q rho.  The increments are of order h ~ dt |L| / I, so their FP32
// rounding is of order 1e-7 h: far below the FP32 force error.
__device__ __forceinline__ void free_rotor_f32(double4_32a &q, double4_32a &L, const double *invI,
                                               double dt, bool ic) {
    const float ii[3] = {cvt_f(invI[0], ic), cvt_f(invI[1], ic), cvt_f(invI[2], ic)};
    float Lc[3] = {cvt_f(L.x, ic), cvt_f(L.y, ic), cvt_f(L.z, ic)};
    float dL[3] = {0.f, 0.f, 0.f};
    float rw = 0.f, rv[3] = {0.f, 0.f, 0.f};
    const float hd = (float)(0.25 * dt);
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int k = step == 2 ? 0 : (step == 1 || step == 3 ? 1 : 2);
        if (!(ii[k] > 0.f)) continue;
        const float h = (step == 2 ? 2.f * hd : hd) * Lc[k] * ii[k];
        float sh, cm1;
        sincosm1_f(h, &sh, &cm1);
        // L_b rotates by phi = 2h about k: cos phi - 1 = -2 sh^2, sin phi = 2 sh ch
        const int a = (k + 1) % 3, b = (k + 2) % 3;
        const float c1 = -2.f * sh * sh, s2 = 2.f * sh * (1.f + cm1);
        const float ia = c1 * Lc[a] + s2 * Lc[b], ib = c1 * Lc[b] - s2 * Lc[a];
        Lc[a] += ia; Lc[b] += ib;
        dL[a] += ia; dL[b] += ib;
        // (1 + rho) <- (1 + rho)(1 + sigma), sigma = (cm1, sh e_k)
        float cx[3] = {0.f, 0.f, 0.f};      // rv x e_k
        cx[a] = rv[b];
        cx[b] = -rv[a];
        const float nw = rw + cm1 + (rw * cm1 - rv[k] * sh);
        float nv[3];
#pragma unroll
        for (int m = 0; m < 3; ++m)
            nv[m] = rv[m] + (m == k ? sh : 0.f) + (m == k ? rw * sh : 0.f) + cm1 * rv[m] + sh * cx[m];
        rw = nw;
        rv[0] = nv[0]; rv[1] = nv[1]; rv[2] = nv[2];
    }
    // q rho in FP32, added to the FP64 quaternion; q = (x: w, y: x, z: y, w: z)
    const float qw = cvt_f(q.x, ic), qx = cvt_f(q.y, ic), qy = cvt_f(q.z, ic), qz = cvt_f(q.w, ic);
    const float dw = qw * rw - (qx * rv[0] + qy * rv[1] + qz * rv[2]);
    const float dx = qw * rv[0] + rw * qx + (qy * rv[2] - qz * rv[1]);
    const float dy = qw * rv[1] + rw * qy + (qz * rv[0] - qx * rv[2]);
    const float dz = qw * rv[2] + rw * qz + (qx * rv[1] - qy * rv[0]);
    q.x += cvt_d(dw, ic); q.y += cvt_d(dx, ic); q.z += cvt_d(dy, ic); q.w += cvt_d(dz, ic);
    L.x += cvt_d(dL[0], ic); L.y += cvt_d(dL[1], ic); L.z += cvt_d(dL[2], ic);
}

// x mapped into [0, L) (invL = 1/L)
__device__ __forceinline__ double wrap(double x, double L, double invL) {
    x -= L * floor(x * invL);
    if (x >= L) x -= L;
    else if (x < 0.0) x += L;
    return x;
}

__device__ __forceinline__ double nh_rate(double K, double g, double kT, double tau) {
    return (2.0 * K / (g * kT) - 1.0) / (tau * tau);
}

// Displacement of particle i (at x) since the list build, whose position
// scales with the box (sc = 1 unless a barostat moved it): stored as the FP32
// delta that the pair kernels add to the list separations.  Returns the
// squared displacement for the rebuild test (skin/2)^2, padded by disp_pad
// when the box has shrunk since the build.
__device__ __forceinline__ float since_build(const StepArgs &a, const Rep &rp, int i,
                                             const double4_32a &x) {
    const double4_32a x0 = a.x_last[i];
    const double sc = rp.sc_d;
    double dx = x.x - sc * x0.x, dy = x.y - sc * x0.y, dz = x.z - sc * x0.z;
    dx -= rp.L[0] * rint(dx * rp.inv_L[0]);
    dy -= rp.L[1] * rint(dy * rp.inv_L[1]);
    if (a.dim == 3) dz -= rp.L[2] * rint(dz * rp.inv_L[2]); else dz = 0.0;
    double d2 = dx * dx + dy * dy + dz * dz;
    if (rp.disp_pad > 0.f) {
        const double d = sqrt(d2) + (double)rp.disp_pad;
        d2 = d * d;
    }
    const bool ic = a.int_conv != 0;
    a.delta[i] = make_float4(cvt_f(dx, ic), cvt_f(dy, ic), cvt_f(dz, ic), __int_as_float(a.shape[i]));
    return cvt_f(d2, ic);
}

// Warp max, one atomic per warp (non-negative floats order like their bits);
// every lane of the warp calls it.
__device__ __forceinline__ void max_to_status(const StepArgs &a, float dmax) {
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if ((threadIdx.x & 31) == 0 && dmax > 0.f)
        atomicMax(&a.status->maxdisp2, __float_as_uint(dmax));
}

// FP32 + two-sum mode: the position and the quaternion as hi + lo floats
// (the hi part of the quaternion is quatf).
__device__ __forceinline__ void store_ff_state(float4 *quatf_lo, float4 *xff, int i,
                                               const double4_32a &x, const double4_32a &q,
                                               bool ic = false) {
    float h, l[4];
    split_ff_dev(q.x, &h, &l[0], ic); split_ff_dev(q.y, &h, &l[1], ic);
    split_ff_dev(q.z, &h, &l[2], ic); split_ff_dev(q.w, &h, &l[3], ic);
    quatf_lo[i] = make_float4(l[0], l[1], l[2], l[3]);
    float xh[3], xl[3];
    split_ff_dev(x.x, &xh[0], &xl[0], ic); split_ff_dev(x.y, &xh[1], &xl[1], ic);
    split_ff_dev(x.z, &xh[2], &xl[2], ic);
    xff[2 * i] = make_float4(xh[0], xh[1], xh[2], 0.f);
    xff[2 * i + 1] = make_float4(xl[0], xl[1], xl[2], 0.f);
}

// The first half of a step for particle i of replica rp: the thermostat's
// velocity scale s1 (NVT), the half kick, the drift (with the box dilation
// under NPT), the free rotation, the FP32 copies; returns the squared
// displacement since the list build for the rebuild test.
__device__ __forceinline__ float first_half_particle(const StepArgs &a, int i, const Rep &rp,
                                                     double s1) {
    const ShapeDev &sh = a.shapes[a.shape[i]];
    double4_32a v = a.vel[i], L = a.angmom[i], F = a.force[i], Tq = a.torque[i];
    double4_32a x = a.pos[i], q = a.quat[i];
    if (a.nvt) {
        v.x *= s1; v.y *= s1; v.z *= s1;
        L.x *= s1; L.y *= s1; L.z *= s1;
    }
    if (a.npt) {
        // half kick and drift with the box dilation (the box itself moved
        // by ax in k_box before this kernel)
        const Thermo &t = a.thermo[a.rep[i]];
        const double b = t.bv * sh.inv_mass;
        v.x = t.av * v.x + b * F.x; v.y = t.av * v.y + b * F.y; v.z = t.av * v.z + b * F.z;
        L.x += 0.5 * a.dt * Tq.x; L.y += 0.5 * a.dt * Tq.y; L.z += 0.5 * a.dt * Tq.z;
        x.x = wrap(t.ax * x.x + t.bx * v.x, rp.L[0], rp.inv_L[0]);
        x.y = wrap(t.ax * x.y + t.bx * v.y, rp.L[1], rp.inv_L[1]);
        if (a.dim == 3) x.z = wrap(t.ax * x.z + t.bx * v.z, rp.L[2], rp.inv_L[2]);
    } else {
        const double h = 0.5 * a.dt * sh.inv_mass;
        v.x += h * F.x; v.y += h * F.y; v.z += h * F.z;
        L.x += 0.5 * a.dt * Tq.x; L.y += 0.5 * a.dt * Tq.y; L.z += 0.5 * a.dt * Tq.z;
        x.x = wrap(x.x + a.dt * v.x, rp.L[0], rp.inv_L[0]);
        x.y = wrap(x.y + a.dt * v.y, rp.L[1], rp.inv_L[1]);
        if (a.dim == 3) x.z = wrap(x.z + a.dt * v.z, rp.L[2], rp.inv_L[2]);
    }
    if (a.rotor32) {
        free_rotor_f32(q, L, sh.inv_inertia, a.dt, a.int_conv != 0);
    } else {
        free_rotor_axis(q, L, sh.inv_inertia, 2, 0.5 * a.dt);
        free_rotor_axis(q, L, sh.inv_inertia, 1, 0.5 * a.dt);
        free_rotor_axis(q, L, sh.inv_inertia, 0, a.dt);
        free_rotor_axis(q, L, sh.inv_inertia, 1, 0.5 * a.dt);
        free_rotor_axis(q, L, sh.inv_inertia, 2, 0.5 * a.dt);
    }
    // renormalise: |q|^2 = 1 + e with |e| ~ 1e-10 per step, and
    // 1/sqrt(1 + e) = 1 - e/2 + 3e^2/8 - ... (remainder below 5|e|^3/16,
    // < 3e-18 for |e| < 2e-6; otherwise the general rsqrt)
    const double qq = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w, e2 = qq - 1.0;
    const double inq = fabs(e2) < 2e-6 ? fma(fma(0.375, e2, -0.5), e2, 1.0) : rsqrt(qq);
    q.x *= inq; q.y *= inq; q.z *= inq; q.w *= inq;
    a.pos[i] = x;
    a.vel[i] = v;
    a.angmom[i] = L;
    a.quat[i] = q;
    const bool ic = a.int_conv != 0;
    a.quatf[i] = make_float4(cvt_f(q.x, ic), cvt_f(q.y, ic), cvt_f(q.z, ic), cvt_f(q.w, ic));
    if (a.quatf_lo) store_ff_state(a.quatf_lo, a.xff, i, x, q, ic);
    return since_build(a, rp, i, x);
}

__device__ __forceinline__ double kinetic_of(const ShapeDev &sh, const double4_32a &v,
                                             const double4_32a &L) {
    double k = 0.5 * sh.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
    k += 0.5 * (L.x * L.x * sh.inv_inertia[0] + L.y * L.y * sh.inv_inertia[1] +
                L.z * L.z * sh.inv_inertia[2]);
    return k;
}

__device__ __forceinline__ double kinetic_trans(const ShapeDev &sh, const double4_32a &v) {
    return 0.5 * sh.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
}

// The second half kick of particle i; returns (and stores) its kinetic energy.
__device__ __forceinline__ double second_half_particle(const StepArgs &a, int i) {
    const ShapeDev &sh = a.shapes[a.shape[i]];
    double4_32a v = a.vel[i], L = a.angmom[i], F = a.force[i], Tq = a.torque[i];
    if (a.npt) {
        const Thermo &t = a.thermo[a.rep[i]];
        const double b = t.bv * sh.inv_mass;
        v.x = t.av * v.x + b * F.x; v.y = t.av * v.y + b * F.y; v.z = t.av * v.z + b * F.z;
        a.ket[i] = kinetic_trans(sh, v);
    } else {
        const double h = 0.5 * a.dt * sh.inv_mass;
        v.x += h * F.x; v.y += h * F.y; v.z += h * F.z;
    }
    L.x += 0.5 * a.dt * Tq.x; L.y += 0.5 * a.dt * Tq.y; L.z += 0.5 * a.dt * Tq.z;
    a.vel[i] = v;
    a.angmom[i] = L;
    const double k = kinetic_of(sh, v, L);
    a.ke[i] = k;
    return k;
}

// Fixed-order block sum of x[off..off+n) (deterministic).
__device__ double block_sum(const double *x, int off, int n, int stride, int comp) {
    __shared__ double red[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += x[(size_t)(off + k) * stride + comp];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// One reduction chunk (block-collective): its sums of ke and, under NPT, of
// ket and the virial trace.
__device__ __forceinline__ void chunk_sums_block(const StepArgs &a, int c) {
    const Rep &rp = a.reps[a.chunk_rep[c]];
    const int k0 = (c - rp.chunk_off) * SUM_CHUNK;
    const int off = rp.off + k0, len = min(SUM_CHUNK, rp.n - k0);
    const double K = block_sum(a.ke, off, len, 1, 0);
    double Kt = 0.0, vir = 0.0;
    if (a.npt) {
        Kt = block_sum(a.ket, off, len, 1, 0);
        vir = block_sum(a.virial, off, len, 6, 0) + block_sum(a.virial, off, len, 6, 3) +
              (a.dim == 3 ? block_sum(a.virial, off, len, 6, 5) : 0.0);
    }
    if (threadIdx.x == 0) {
        a.partial[3 * c] = K;
        a.partial[3 * c + 1] = Kt;
        a.partial[3 * c + 2] = vir;
    }
}

// Replica r (block-collective): K = sum of ke, then the second thermostat
// half step of this step and the first half step of the next one.  Small
// replicas (direct_sums) are summed here directly and, under NVT, their
// velocities and angular momenta take this step's second scaling here.
__device__ __forceinline__ void thermo_end_replica(const StepArgs &a, int r) {
    const Rep &rp = a.reps[r];
    __shared__ double s_end;
    double K = a.direct_sums ? block_sum(a.ke, rp.off, rp.n, 1, 0)
                             : block_sum(a.partial, rp.chunk_off, rp.n_chunk, 3, 0);
    if (threadIdx.x == 0) {
        Thermo &t = a.thermo[r];
        const double g = (double)rp.g_dof, d = 0.5 * a.dt;
        if (a.nvt) {
            double xi = t.xi_h + 0.5 * d * nh_rate(K, g, a.kT, a.tau);
            double s2 = exp(-xi * d);
            double eta = t.eta_h + xi * d;
            K *= s2 * s2;
            xi += 0.5 * d * nh_rate(K, g, a.kT, a.tau);
            t.xi = xi; t.eta = eta; t.K = K;
            t.s2 = s2;
            double xh = xi + 0.5 * d * nh_rate(K, g, a.kT, a.tau);
            double s1 = exp(-xh * d);
            t.eta_h = eta + xh * d;
            t.xi_h = xh + 0.5 * d * nh_rate(K * s1 * s1, g, a.kT, a.tau);
            t.s1 = s1;
            s_end = s2;
        } else {
            t.K = K;
        }
    }
    if (a.nvt && a.direct_sums) {
        __syncthreads();
        const double s = s_end;
        for (int k = threadIdx.x; k < rp.n; k += blockDim.x) {
            const int i = rp.off + k;
            double4_32a v = a.vel[i], L = a.angmom[i];
            v.x *= s; v.y *= s; v.z *= s;
            L.x *= s; L.y *= s; L.z *= s;
            a.vel[i] = v;
            a.angmom[i] = L;
        }
    }
}

// The second thermostat scaling of particle i (replicas summed by chunks).
__device__ __forceinline__ void scale_particle(const StepArgs &a, int i) {
    const double s = a.thermo[a.rep[i]].s2;
    double4_32a v = a.vel[i], L = a.angmom[i];
    v.x *= s; v.y *= s; v.z *= s;
    L.x *= s; L.y *= s; L.z *= s;
    a.vel[i] = v;
    a.angmom[i] = L;
}

}  // namespace
}  // namespace dem
