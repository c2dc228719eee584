// integrate.cu -- time integration and reductions (FP64).
//
// Section "Energy Conservation" of arXiv:1607.02427 uses a second-order
// integrator (energy error ~ dt^2, Kamberaj et al. 2005); Section "Assembly"
// a Nose-Hoover thermostat on translational and rotational degrees of
// freedom.  The paper gives no formulas; the scheme here is:
//   * velocity Verlet for the centres;
//   * body-frame angular momentum L_b with the symmetric free-rotor splitting
//     z(dt/2) y(dt/2) x(dt) y(dt/2) z(dt/2): a rotation by phi = L_k/I_k dt
//     about body axis k turns the body by phi and L_b by -phi (the NO_SQUISH
//     splitting, Miller et al., J. Chem. Phys. 116, 8649 (2002));
//   * NVT: T(dt/2) . NVE(dt) . T(dt/2), one friction xi per replica,
//     dxi/dt = (2K/(g kT) - 1)/tau^2, T(delta) = {xi += delta/2 G(K);
//     scale v, L by exp(-xi delta); eta += xi delta; xi += delta/2 G(K)}.
// 2D particles carry a quaternion about z (angle theta = 2 atan2(q_z, q_w))
// and L_b = (0, 0, L_z); only the z sub-rotations act.
#include "dem_internal.cuh"

namespace dem {
namespace {

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
                                               double dt) {
    const float ii[3] = {(float)invI[0], (float)invI[1], (float)invI[2]};
    float Lc[3] = {(float)L.x, (float)L.y, (float)L.z};
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
    const float qw = (float)q.x, qx = (float)q.y, qy = (float)q.z, qz = (float)q.w;
    const float dw = qw * rw - (qx * rv[0] + qy * rv[1] + qz * rv[2]);
    const float dx = qw * rv[0] + rw * qx + (qy * rv[2] - qz * rv[1]);
    const float dy = qw * rv[1] + rw * qy + (qz * rv[0] - qx * rv[2]);
    const float dz = qw * rv[2] + rw * qz + (qx * rv[1] - qy * rv[0]);
    q.x += (double)dw; q.y += (double)dx; q.z += (double)dy; q.w += (double)dz;
    L.x += (double)dL[0]; L.y += (double)dL[1]; L.z += (double)dL[2];
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
    a.delta[i] = make_float4((float)dx, (float)dy, (float)dz, __int_as_float(a.shape[i]));
    return (float)d2;
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
                                               const double4_32a &x, const double4_32a &q) {
    float h, l[4];
    split_ff(q.x, &h, &l[0]); split_ff(q.y, &h, &l[1]);
    split_ff(q.z, &h, &l[2]); split_ff(q.w, &h, &l[3]);
    quatf_lo[i] = make_float4(l[0], l[1], l[2], l[3]);
    float xh[3], xl[3];
    split_ff(x.x, &xh[0], &xl[0]); split_ff(x.y, &xh[1], &xl[1]); split_ff(x.z, &xh[2], &xl[2]);
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
        free_rotor_f32(q, L, sh.inv_inertia, a.dt);
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
    a.quatf[i] = make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
    if (a.quatf_lo) store_ff_state(a.quatf_lo, a.xff, i, x, q);
    return since_build(a, rp, i, x);
}

__global__ void k_first_half(const StepArgs a) {
    float dmax = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const int r = a.rep[i];
        dmax = fmaxf(dmax, first_half_particle(a, i, a.reps[r], a.nvt ? a.thermo[r].s1 : 1.0));
    }
    max_to_status(a, dmax);
}

// The rebuild test after positions were replaced from outside (state upload):
// the displacement of every particle since the list build, as in a step.
__global__ void k_displacement(const StepArgs a) {
    float dmax = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x)
        dmax = fmaxf(dmax, since_build(a, a.reps[a.rep[i]], i, a.pos[i]));
    max_to_status(a, dmax);
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

__global__ void k_second_half(const StepArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x)
        second_half_particle(a, i);
}

__global__ void k_kinetic(const StepArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const ShapeDev &sh = a.shapes[a.shape[i]];
        const double4_32a v = a.vel[i];
        a.ke[i] = kinetic_of(sh, v, a.angmom[i]);
        if (a.ket) a.ket[i] = kinetic_trans(sh, v);
    }
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

// One block per reduction chunk: its sums of ke and, under NPT, of ket and
// the virial trace.
__global__ void k_chunk_sums(const StepArgs a) {
    const int c = blockIdx.x;
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

// One block per replica: K = sum of ke, then the second thermostat half step
// of this step and the first half step of the next one.
__global__ void k_thermo_end(const StepArgs a) {
    const int r = blockIdx.x;
    const Rep &rp = a.reps[r];
    __shared__ double s_end;
    // small replicas: the sum over the particles directly (no chunk partials)
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
    // NVT, small replicas: this step's second thermostat scaling of the
    // replica's velocities and angular momenta here (else k_scale does it)
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

__global__ void k_thermo_begin(const StepArgs a) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_reps) return;
    Thermo &t = a.thermo[r];
    const double g = (double)a.reps[r].g_dof, d = 0.5 * a.dt;
    double xh = t.xi + 0.5 * d * nh_rate(t.K, g, a.kT, a.tau);
    double s1 = exp(-xh * d);
    t.eta_h = t.eta + xh * d;
    t.xi_h = xh + 0.5 * d * nh_rate(t.K * s1 * s1, g, a.kT, a.tau);
    t.s1 = s1;
}

// ---- isotropic barostat (NPT) ----
// sinh(x)/x (Maclaurin series below |x| = 1e-2, remainder < 1e-17)
__device__ __forceinline__ double sinhc(double x) {
    if (fabs(x) < 1e-2) {
        const double x2 = x * x;
        return 1.0 + x2 / 6.0 * (1.0 + x2 / 20.0 * (1.0 + x2 / 42.0));
    }
    return sinh(x) / x;
}

struct NptConst {
    double W;        // barostat mass (N_f + d) kT tau_P^2
    double alpha;    // 1 + d / N_f, N_f = d (N - 1)
    double g1;       // thermostat degrees of freedom: g + 1 (the barostat)
    double V;        // current volume
    double dim;
};

__device__ __forceinline__ NptConst npt_const(const StepArgs &a, const Rep &rp) {
    NptConst c;
    const double nf = a.dim * (rp.n - 1.0);
    c.W = (nf + a.dim) * a.kT * a.tau_P * a.tau_P;
    c.alpha = 1.0 + a.dim / nf;
    c.g1 = (double)rp.g_dof + 1.0;
    c.V = rp.L[0] * rp.L[1] * (a.dim == 3 ? rp.L[2] : 1.0);
    c.dim = (double)a.dim;
    return c;
}

// First half of a step from the canonical state (t.xi, t.eta, t.pe) with the
// replica's translational and rotational kinetic energies Kt, Kr and virial
// trace vir: thermostat T(dt/2) on the particles and the barostat momentum,
// barostat B(dt/2): p_e += dt/2 (alpha 2 K_t + Tr W - d V P), then the
// factors of the dilating half kick, v <- av v + bv F/m, and of the drift,
// x <- ax x + bx v (box <- ax box), each the exact solution of its sub-step.
__device__ void npt_first_half(const StepArgs &a, Thermo &t, const NptConst &c, double Kt,
                               double Kr, double vir) {
    const double d = 0.5 * a.dt;
    double Ktot = Kt + Kr + 0.5 * t.pe * t.pe / c.W;
    const double xh = t.xi + 0.5 * d * nh_rate(Ktot, c.g1, a.kT, a.tau);
    const double s1 = exp(-xh * d);
    t.eta_h = t.eta + xh * d;
    Ktot *= s1 * s1;
    t.xi_h = xh + 0.5 * d * nh_rate(Ktot, c.g1, a.kT, a.tau);
    t.s1 = s1;
    const double pe = t.pe * s1 + d * (c.alpha * 2.0 * Kt * s1 * s1 + vir - c.dim * c.V * a.P);
    t.pe_h = pe;
    const double ve = pe / c.W;
    t.av = exp(-c.alpha * ve * d);
    t.bv = d * exp(-0.5 * c.alpha * ve * d) * sinhc(0.5 * c.alpha * ve * d);
    t.ax = exp(ve * a.dt);
    t.bx = a.dt * exp(0.5 * ve * a.dt) * sinhc(0.5 * ve * a.dt);
}

// Replica sums of the NPT state: total and translational kinetic energy and
// the virial trace (fixed order).
__device__ __forceinline__ void npt_sums(const StepArgs &a, const Rep &rp, double *K, double *Kt,
                                         double *vir) {
    *K = block_sum(a.partial, rp.chunk_off, rp.n_chunk, 3, 0);
    *Kt = block_sum(a.partial, rp.chunk_off, rp.n_chunk, 3, 1);
    *vir = block_sum(a.partial, rp.chunk_off, rp.n_chunk, 3, 2);
}

// One block per replica, end of an NPT step (after the second half kick):
// B(dt/2) and T(dt/2) of this step, then the first half of the next one.
__global__ void k_thermo_end_npt(const StepArgs a) {
    const int r = blockIdx.x;
    const Rep &rp = a.reps[r];
    double K, Kt, vir;
    npt_sums(a, rp, &K, &Kt, &vir);
    if (threadIdx.x == 0) {
        Thermo &t = a.thermo[r];
        const NptConst c = npt_const(a, rp);
        const double d = 0.5 * a.dt;
        double Kr = K - Kt;
        double pe = t.pe_h + d * (c.alpha * 2.0 * Kt + vir - c.dim * c.V * a.P);
        double Ktot = Kt + Kr + 0.5 * pe * pe / c.W;
        double xi = t.xi_h + 0.5 * d * nh_rate(Ktot, c.g1, a.kT, a.tau);
        const double s2 = exp(-xi * d);
        const double eta = t.eta_h + xi * d;
        Ktot *= s2 * s2;
        Kt *= s2 * s2;
        Kr *= s2 * s2;
        pe *= s2;
        xi += 0.5 * d * nh_rate(Ktot, c.g1, a.kT, a.tau);
        t.xi = xi; t.eta = eta; t.pe = pe; t.K = Kt + Kr;
        t.s2 = s2;
        npt_first_half(a, t, c, Kt, Kr, vir);
    }
}

// One block per replica, start of an NPT call: the first half step from the
// canonical state (ke and ket current, forces and virial current).
__global__ void k_thermo_begin_npt(const StepArgs a) {
    const int r = blockIdx.x;
    const Rep &rp = a.reps[r];
    double K, Kt, vir;
    npt_sums(a, rp, &K, &Kt, &vir);
    if (threadIdx.x == 0) {
        Thermo &t = a.thermo[r];
        t.K = K;
        npt_first_half(a, t, npt_const(a, rp), Kt, K - Kt, vir);
    }
}

// One thread per replica, start of an NPT step: the box follows the drift
// factor; the list scale and the rebuild pad follow the box; a box below
// twice the list cutoff or below its cell grid's reach is flagged.
__global__ void k_box(const StepArgs a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= a.n_reps) return;
    Rep &rp = a.reps_rw[r];
    const double ax = a.thermo[r].ax;
    for (int k = 0; k < a.dim; ++k) {
        rp.L[k] *= ax;
        rp.inv_L[k] = 1.0 / rp.L[k];
        if (!(rp.L[k] >= 2.0 * rp.r_list) || (!rp.allpairs && rp.L[k] < rp.nc[k] * rp.r_list))
            a.status->box_limit = 1;
    }
    rep_box_ff(rp);
    const double sc = rp.L[0] / rp.L_build0;
    rp.sc_d = sc;
    rp.sc = (float)sc;
    rp.disp_pad = (float)(0.5 * fmax(0.0, 1.0 - sc) * rp.r_list);
}

__global__ void k_scale(const StepArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        double s = a.thermo[a.rep[i]].s2;
        double4_32a v = a.vel[i], L = a.angmom[i];
        v.x *= s; v.y *= s; v.z *= s;
        L.x *= s; L.y *= s; L.z *= s;
        a.vel[i] = v;
        a.angmom[i] = L;
    }
}

__global__ void k_replica_sums(const Rep *reps, const double *x, int stride, int comps,
                               double *out) {
    const Rep &rp = reps[blockIdx.x];
    for (int c = 0; c < comps; ++c) {
        double s = block_sum(x, rp.off, rp.n, stride, c);
        if (threadIdx.x == 0) out[blockIdx.x * comps + c] = s;
    }
}

}  // namespace

// ---- small helpers for state conversion ----
namespace {
struct M3 { double m[3][3]; };
__device__ __forceinline__ M3 qmat(const double4_32a &q) {
    double w = q.x, x = q.y, y = q.z, z = q.w;
    M3 R;
    R.m[0][0] = 1 - 2 * (y * y + z * z); R.m[0][1] = 2 * (x * y - w * z); R.m[0][2] = 2 * (x * z + w * y);
    R.m[1][0] = 2 * (x * y + w * z); R.m[1][1] = 1 - 2 * (x * x + z * z); R.m[1][2] = 2 * (y * z - w * x);
    R.m[2][0] = 2 * (x * z - w * y); R.m[2][1] = 2 * (y * z + w * x); R.m[2][2] = 1 - 2 * (x * x + y * y);
    return R;
}

__global__ void k_prepare(int n, int dim, double4_32a *pos, double4_32a *quat, float4 *quatf,
                          float4 *quatf_lo, float4 *xff, double4_32a *angmom, const int *rep,
                          const Rep *reps, int world_to_body) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Rep &rp = reps[rep[i]];
        double4_32a x = pos[i];
        x.x = wrap(x.x, rp.L[0], rp.inv_L[0]);
        x.y = wrap(x.y, rp.L[1], rp.inv_L[1]);
        x.z = dim == 3 ? wrap(x.z, rp.L[2], rp.inv_L[2]) : 0.0;
        pos[i] = x;
        double4_32a q = quat[i];
        double nq = sqrt(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
        q.x /= nq; q.y /= nq; q.z /= nq; q.w /= nq;
        quat[i] = q;
        quatf[i] = make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
        if (quatf_lo) store_ff_state(quatf_lo, xff, i, x, q);
        if (world_to_body) {
            double4_32a L = angmom[i];
            if (dim == 3) {
                M3 R = qmat(q);
                double bx = R.m[0][0] * L.x + R.m[1][0] * L.y + R.m[2][0] * L.z;
                double by = R.m[0][1] * L.x + R.m[1][1] * L.y + R.m[2][1] * L.z;
                double bz = R.m[0][2] * L.x + R.m[1][2] * L.y + R.m[2][2] * L.z;
                angmom[i] = make_double4_32a(bx, by, bz, 0.0);
            } else {
                angmom[i] = make_double4_32a(0.0, 0.0, L.z, 0.0);
            }
        }
    }
}

// Input state into the packed arrays.  A particle whose imported values
// are not all finite, or whose quaternion has zero norm, is recorded in
// status->bad_input (1 + its index) and given a harmless state (centre at
// the origin, identity orientation, at rest), so that the kernels that
// follow in the same call run on finite data; the call then fails.
__global__ void k_import(int n, int dim, const double *pos_in, const double *orient_in,
                         const double *vel_in, const double *angmom_in, double4_32a *pos,
                         double4_32a *quat, double4_32a *vel, double4_32a *angmom,
                         Status *status) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        bool bad = false;
        if (dim == 3) {
            if (pos_in) {
                double4_32a x = make_double4_32a(pos_in[3 * i], pos_in[3 * i + 1], pos_in[3 * i + 2], 0.0);
                if (!(isfinite(x.x) && isfinite(x.y) && isfinite(x.z))) { bad = true; x = make_double4_32a(0, 0, 0, 0); }
                pos[i] = x;
            }
            if (vel_in) {
                double4_32a v = make_double4_32a(vel_in[3 * i], vel_in[3 * i + 1], vel_in[3 * i + 2], 0.0);
                if (!(isfinite(v.x) && isfinite(v.y) && isfinite(v.z))) { bad = true; v = make_double4_32a(0, 0, 0, 0); }
                vel[i] = v;
            }
            if (orient_in) {
                double4_32a q = make_double4_32a(orient_in[4 * i], orient_in[4 * i + 1], orient_in[4 * i + 2],
                                                 orient_in[4 * i + 3]);
                const double q2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
                if (!(isfinite(q2) && q2 > 0.0)) { bad = true; q = make_double4_32a(1, 0, 0, 0); }
                quat[i] = q;
            }
            if (angmom_in) {
                double4_32a L = make_double4_32a(angmom_in[3 * i], angmom_in[3 * i + 1], angmom_in[3 * i + 2], 0.0);
                if (!(isfinite(L.x) && isfinite(L.y) && isfinite(L.z))) { bad = true; L = make_double4_32a(0, 0, 0, 0); }
                angmom[i] = L;
            }
        } else {
            if (pos_in) {
                double4_32a x = make_double4_32a(pos_in[2 * i], pos_in[2 * i + 1], 0.0, 0.0);
                if (!(isfinite(x.x) && isfinite(x.y))) { bad = true; x = make_double4_32a(0, 0, 0, 0); }
                pos[i] = x;
            }
            if (vel_in) {
                double4_32a v = make_double4_32a(vel_in[2 * i], vel_in[2 * i + 1], 0.0, 0.0);
                if (!(isfinite(v.x) && isfinite(v.y))) { bad = true; v = make_double4_32a(0, 0, 0, 0); }
                vel[i] = v;
            }
            if (orient_in) {
                double th = orient_in[i];
                if (!isfinite(th)) { bad = true; th = 0.0; }
                quat[i] = make_double4_32a(cos(0.5 * th), 0.0, 0.0, sin(0.5 * th));
            }
            if (angmom_in) {
                double L = angmom_in[i];
                if (!isfinite(L)) { bad = true; L = 0.0; }
                angmom[i] = make_double4_32a(0.0, 0.0, L, 0.0);
            }
        }
        if (bad && status) atomicMax(&status->bad_input, i + 1);
    }
}

__global__ void k_export(int n, int dim, const double4_32a *pos, const double4_32a *quat,
                         const double4_32a *vel, const double4_32a *angmom, double *pos_out,
                         double *orient_out, double *vel_out, double *angmom_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double4_32a q = quat[i];
        if (dim == 3) {
            if (pos_out) { double4_32a x = pos[i]; pos_out[3 * i] = x.x; pos_out[3 * i + 1] = x.y; pos_out[3 * i + 2] = x.z; }
            if (vel_out) { double4_32a v = vel[i]; vel_out[3 * i] = v.x; vel_out[3 * i + 1] = v.y; vel_out[3 * i + 2] = v.z; }
            if (orient_out) { orient_out[4 * i] = q.x; orient_out[4 * i + 1] = q.y; orient_out[4 * i + 2] = q.z; orient_out[4 * i + 3] = q.w; }
            if (angmom_out) {
                M3 R = qmat(q);
                double4_32a L = angmom[i];
                angmom_out[3 * i] = R.m[0][0] * L.x + R.m[0][1] * L.y + R.m[0][2] * L.z;
                angmom_out[3 * i + 1] = R.m[1][0] * L.x + R.m[1][1] * L.y + R.m[1][2] * L.z;
                angmom_out[3 * i + 2] = R.m[2][0] * L.x + R.m[2][1] * L.y + R.m[2][2] * L.z;
            }
        } else {
            if (pos_out) { double4_32a x = pos[i]; pos_out[2 * i] = x.x; pos_out[2 * i + 1] = x.y; }
            if (vel_out) { double4_32a v = vel[i]; vel_out[2 * i] = v.x; vel_out[2 * i + 1] = v.y; }
            if (orient_out) orient_out[i] = 2.0 * atan2(q.w, q.x);
            if (angmom_out) angmom_out[i] = angmom[i].z;
        }
    }
}

__global__ void k_export_forces(int n, int dim, const double4_32a *force, const double4_32a *torque_b,
                                const double4_32a *quat, double *force_out, double *torque_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double4_32a F = force[i], T = torque_b[i];
        if (dim == 3) {
            if (force_out) { force_out[3 * i] = F.x; force_out[3 * i + 1] = F.y; force_out[3 * i + 2] = F.z; }
            if (torque_out) {
                M3 R = qmat(quat[i]);
                torque_out[3 * i] = R.m[0][0] * T.x + R.m[0][1] * T.y + R.m[0][2] * T.z;
                torque_out[3 * i + 1] = R.m[1][0] * T.x + R.m[1][1] * T.y + R.m[1][2] * T.z;
                torque_out[3 * i + 2] = R.m[2][0] * T.x + R.m[2][1] * T.y + R.m[2][2] * T.z;
            }
        } else {
            if (force_out) { force_out[2 * i] = F.x; force_out[2 * i + 1] = F.y; }
            if (torque_out) torque_out[i] = T.z;
        }
    }
}

__global__ void k_rescale(int n, int dim, double4_32a *pos, double4_32a *x_last, const int *rep,
                          const double *scale3) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double *s = scale3 + 3 * rep[i];
        double4_32a x = pos[i];
        x.x *= s[0]; x.y *= s[1];
        if (dim == 3) x.z *= s[2];
        pos[i] = x;
        x_last[i] = x;
    }
}

inline int grid_for(int n, int block) {
    int g = (n + block - 1) / block;
    return g > 0 ? g : 1;
}

// Threads per block of the per-particle step kernels: 256, or fewer (down to
// one warp) while blocks of 256 would leave SMs idle.  FP64 runs at a few
// flops per clock per SM on this part, so a small system's integrator work
// is spread over as many SMs as it can fill.
int particle_block(int n) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    int b = 256;
    while (b > 32 && (n + b - 1) / b < sms) b >>= 1;
    return b;
}

}  // namespace

cudaError_t launch_first_half(const StepArgs &a, cudaStream_t s) {
    const int b = particle_block(a.n);
    k_first_half<<<grid_for(a.n, b), b, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_displacement(const StepArgs &a, cudaStream_t s) {
    const int b = particle_block(a.n);
    k_displacement<<<grid_for(a.n, b), b, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_second_half(const StepArgs &a, cudaStream_t s) {
    const int b = particle_block(a.n);
    k_second_half<<<grid_for(a.n, b), b, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_kinetic(const StepArgs &a, cudaStream_t s) {
    const int b = particle_block(a.n);
    k_kinetic<<<grid_for(a.n, b), b, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_thermo_end(const StepArgs &a, cudaStream_t s) {
    if (a.npt) k_thermo_end_npt<<<a.n_reps, 256, 0, s>>>(a);
    else k_thermo_end<<<a.n_reps, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_chunk_sums(const StepArgs &a, cudaStream_t s) {
    k_chunk_sums<<<a.n_chunks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_box(const StepArgs &a, cudaStream_t s) {
    k_box<<<(a.n_reps + 127) / 128, 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_thermo_begin(const StepArgs &a, cudaStream_t s) {
    if (a.npt) k_thermo_begin_npt<<<a.n_reps, 256, 0, s>>>(a);
    else k_thermo_begin<<<grid_for(a.n_reps, 128), 128, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_scale(const StepArgs &a, cudaStream_t s) {
    const int b = particle_block(a.n);
    k_scale<<<grid_for(a.n, b), b, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_replica_sums(int n_reps, const Rep *reps, const double *per_particle,
                                int stride, int comps, double *out, cudaStream_t s) {
    k_replica_sums<<<n_reps, 256, 0, s>>>(reps, per_particle, stride, comps, out);
    return cudaGetLastError();
}
cudaError_t launch_prepare_state(int n, int dim, double4_32a *pos, double4_32a *quat, float4 *quatf,
                                 float4 *quatf_lo, float4 *xff,
                                 double4_32a *angmom, const int *rep, const Rep *reps,
                                 int world_to_body, cudaStream_t s) {
    k_prepare<<<grid_for(n, 256), 256, 0, s>>>(n, dim, pos, quat, quatf, quatf_lo, xff, angmom, rep,
                                               reps, world_to_body);
    return cudaGetLastError();
}
cudaError_t launch_import_state(int n, int dim, const double *pos_in, const double *orient_in,
                                const double *vel_in, const double *angmom_in, double4_32a *pos,
                                double4_32a *quat, double4_32a *vel, double4_32a *angmom,
                                Status *status, cudaStream_t s) {
    k_import<<<grid_for(n, 256), 256, 0, s>>>(n, dim, pos_in, orient_in, vel_in, angmom_in, pos,
                                              quat, vel, angmom, status);
    return cudaGetLastError();
}
cudaError_t launch_export_state(int n, int dim, const double4_32a *pos, const double4_32a *quat,
                                const double4_32a *vel, const double4_32a *angmom, double *pos_out,
                                double *orient_out, double *vel_out, double *angmom_out,
                                cudaStream_t s) {
    k_export<<<grid_for(n, 256), 256, 0, s>>>(n, dim, pos, quat, vel, angmom, pos_out, orient_out,
                                              vel_out, angmom_out);
    return cudaGetLastError();
}
cudaError_t launch_export_forces(int n, int dim, const double4_32a *force, const double4_32a *torque_b,
                                 const double4_32a *quat, double *force_out, double *torque_out,
                                 cudaStream_t s) {
    k_export_forces<<<grid_for(n, 256), 256, 0, s>>>(n, dim, force, torque_b, quat, force_out,
                                                     torque_out);
    return cudaGetLastError();
}
cudaError_t launch_rescale(int n, int dim, double4_32a *pos, double4_32a *x_last, const int *rep,
                           const double *scale3, cudaStream_t s) {
    k_rescale<<<grid_for(n, 256), 256, 0, s>>>(n, dim, pos, x_last, rep, scale3);
    return cudaGetLastError();
}

}  // namespace dem
