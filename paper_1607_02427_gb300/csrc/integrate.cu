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
#include "step_device.cuh"

namespace dem {
namespace {

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

// One block per reduction chunk.
__global__ void k_chunk_sums(const StepArgs a) { chunk_sums_block(a, blockIdx.x); }

// One block per replica.
__global__ void k_thermo_end(const StepArgs a) { thermo_end_replica(a, blockIdx.x); }

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
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x)
        scale_particle(a, i);
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

// Self-check of the integer-operation conversions (f32_of, f64_of) against
// the conversion instructions: input k of a launch is bits of a counter-based
// hash (splitmix64) of seed + k, taken as a double (with every fourth input
// put on a rounding tie) and, its low word, as a float.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__global__ void k_check_conversions(unsigned long long n, unsigned long long seed,
                                    unsigned long long *bad) {
    unsigned long long nb0 = 0, nb1 = 0;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long r = splitmix64(seed + k);
        unsigned long long u = r;
        if ((k & 3) == 1)   // a tie: the 29 bits below a float's last place are 1000...0
            u = (r & 0xffffffffe0000000ull) | 0x10000000ull;
        else if ((k & 3) == 2)   // exponents around the float range
            u = (r & 0x800fffffffffffffull) | (unsigned long long)(860 + (r >> 52) % 340) << 52;
        const double x = __longlong_as_double((long long)u);
        const float a = f32_of(x), b = __double2float_rn(x);
        if (!(a != a && b != b) && __float_as_uint(a) != __float_as_uint(b)) ++nb0;
        const float f = __uint_as_float((unsigned)r);
        const double c = f64_of(f), d = (double)f;
        if (!(c != c && d != d) && __double_as_longlong(c) != __double_as_longlong(d)) ++nb1;
    }
    if (nb0) atomicAdd(bad, nb0);
    if (nb1) atomicAdd(bad + 1, nb1);
}

// The FP32 (and float-float) copies of positions and orientations from the
// FP64 state, which is left as it is (a state restored from a snapshot).
__global__ void k_refresh_copies(int n, const double4_32a *pos, const double4_32a *quat,
                                 float4 *quatf, float4 *quatf_lo, float4 *xff) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double4_32a q = quat[i];
        quatf[i] = make_float4((float)q.x, (float)q.y, (float)q.z, (float)q.w);
        if (quatf_lo) store_ff_state(quatf_lo, xff, i, pos[i], q);
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
cudaError_t launch_check_conversions(unsigned long long n, unsigned long long seed,
                                    unsigned long long *bad, cudaStream_t s) {
    k_check_conversions<<<1216, 256, 0, s>>>(n, seed, bad);
    return cudaGetLastError();
}
cudaError_t launch_refresh_copies(int n, const double4_32a *pos, const double4_32a *quat,
                                  float4 *quatf, float4 *quatf_lo, float4 *xff, cudaStream_t s) {
    k_refresh_copies<<<grid_for(n, 256), 256, 0, s>>>(n, pos, quat, quatf, quatf_lo, xff);
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

// ---- self-check of the conversions (C ABI) ----
extern "C" int dem_check_conversions(unsigned long long n, unsigned long long seed,
                                     unsigned long long *mismatches) {
    if (!mismatches) {
        dem::set_global_error("dem_check_conversions: mismatches is NULL");
        return DEM_ERR_ARG;
    }
    unsigned long long *bad = nullptr;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMalloc(&bad, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess && n > 0) e = dem::launch_check_conversions(n, seed, bad, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mismatches, bad, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    if (bad) cudaFree(bad);
    if (e != cudaSuccess) {
        dem::set_global_error(std::string("dem_check_conversions: ") + cudaGetErrorString(e));
        return DEM_ERR_CUDA;
    }
    return DEM_OK;
}
