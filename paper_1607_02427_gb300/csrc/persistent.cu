// persistent.cu -- many time steps of a small system in one cooperative
// kernel launch.
//
// A step of a system of a few thousand particles takes a few tens of
// microseconds as a chain of separate kernels (first half step, list check,
// pair kernel, second half step, thermostat), and most of that is the
// latency of each launch and of its slowest thread.  Here one cooperative
// launch runs the steps of Section "Algorithm" of arXiv:1607.02427
// (velocity Verlet with the free-rotor splitting, Section "Energy
// Conservation"; Nose-Hoover, Section "Assembly") with grid-wide barriers
// between the phases of a step:
//   P1  first half step of every particle (thermostat scale, half kick,
//       drift, free rotor, displacement since the list build)    barrier
//       if some particle moved more than skin/2 since the list build, or a
//       rebuild was requested, the kernel stops here: the host rebuilds the
//       list (the cell binning and list kernels) and relaunches it from P2
//   P2  every list entry (i, k) in its own thread: range test, pair setup
//       and all terms of the pair (Eq. DEM / Eq. DEM_2D) into the entry's
//       partial sums                                               barrier
//   P3  per particle: its entries' partials summed in list order, the
//       outputs, the second half kick and the kinetic energy
//   NVT: barrier, chunk sums (replicas of more than 2048 particles; barrier),
//       the thermostat of each replica, barrier, and (chunked replicas) the
//       second velocity scaling
// P1, P3 and the scaling map particle i to the same thread, so a particle's
// second half kick and its next first half step need no barrier between
// them.  That map deals the particles to the blocks in turn (particle i to
// block i mod grid): a small system's FP64 integrator work, which runs at a
// small fraction of the FP32 rate on this part, is spread over every SM.
// A pair's partial sums and the order in which a particle adds them are
// those of the WARP decomposition (pair.cu), and the integrator pieces are
// the functions of integrate.cu.  In the FP32 modes the trajectory is
// bit-identical to the step kernels' with the WARP decomposition; in FP64
// the compiler fuses some multiply-adds of the FP64 free rotor differently
// in the two kernels, and the trajectories agree to rounding (1e-13 after
// 100 steps of a dense cluster).
//
// Every barrier wait is bounded: a block that waits past the time limit
// records a timeout, marks the launch aborted and returns; every other block
// returns at its next barrier.  The host then reports DEM_ERR_TIMEOUT and
// restores the state from before the call.
#include "pair_kernels.cuh"
#include "step_device.cuh"

namespace dem {
namespace {

constexpr int COOP_BLOCK = 256;           // the thermostat's block sums assume 256 threads
constexpr unsigned SPIN_MAX = 1u << 27;   // backstop of the time limit (>= 4 s of 32 ns sleeps)

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait.  Returns false when the launch is
// aborted (this block or another waited past the limit).  Block-collective.
__device__ bool grid_barrier(CoopCtl *ctl, long long limit_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &ctl->bar_gen;
        volatile int *abort = &ctl->abort;
        int ok = *abort == 0;
        if (ok) {
            const unsigned g = *gen;
            __threadfence();
            if (atomicAdd(&ctl->bar_count, 1u) == gridDim.x - 1) {
                atomicExch(&ctl->bar_count, 0u);
                __threadfence();
                atomicAdd(&ctl->bar_gen, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                for (unsigned spin = 0; *gen == g; ++spin) {
                    if (*abort) {
                        ok = 0;
                        break;
                    }
                    if (spin >= SPIN_MAX || global_ns() - t0 > (unsigned long long)limit_ns) {
                        atomicExch(&ctl->timeout, 1);
                        atomicExch(&ctl->abort, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Warp maximum of non-negative floats into *dst (one atomic per warp).
__device__ __forceinline__ void warp_max_to(unsigned *dst, float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(dst, __float_as_uint(v));
}

template <class T, bool COMP, int DIM>
__global__ void __launch_bounds__(COOP_BLOCK, 1) k_coop_steps(const CoopArgs c) {
    using R4 = typename R4T<T>::type;
    constexpr bool REF = COMP && std::is_same<T, float>::value;
    extern __shared__ __align__(32) unsigned char smem[];
    const PairArgs &a = c.p;
    const StepArgs &sa = c.s;
    CoopCtl *ctl = c.ctl;
    if (c.test_stall && blockIdx.x == 0) return;   // test hook: block 0 never arrives
    R4 *tab = reinterpret_cast<R4 *>(smem);
    Geom *geo = reinterpret_cast<Geom *>(tab + a.table_len);
    int *itab = reinterpret_cast<int *>(geo + a.n_geoms);
    stage_tables<T>(a, tab, geo, itab);
    const int n = a.n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const int pid = threadIdx.x * gridDim.x + blockIdx.x;   // first particle of this thread
    if (c.resume && tid == 0) {
        // the list was rebuilt after this launch's first half step
        a.status->maxdisp2 = 0u;
        a.status->rebuild = 0;
    }
    // the longest list of this launch (the list changes only between launches)
    int kl = 0;
    for (int i = tid; i < n; i += nthr) kl = max(kl, a.nn[i]);
    for (int o = 16; o > 0; o >>= 1) kl = max(kl, __shfl_xor_sync(0xffffffffu, kl, o));
    if ((threadIdx.x & 31) == 0 && kl > 0) atomicMax(&ctl->kmax, kl);
    if (!grid_barrier(ctl, c.limit_ns)) return;
    const int kmax = *(volatile int *)&ctl->kmax;
    const long long n_entries = (long long)kmax * n;
    const size_t plane = (size_t)a.cap * n;       // values per partial component
    T *part = reinterpret_cast<T *>(c.part);
    const T eps = (T)a.eps, par_eps = (T)a.par_eps;

    for (int step = 0; step < c.n_steps; ++step) {
        if (step > 0 || !c.resume) {
            // ---- P1: first half step ----
            float dmax = 0.f;
            for (int i = pid; i < n; i += nthr) {
                const int r = sa.rep[i];
                dmax = fmaxf(dmax, first_half_particle(sa, i, sa.reps[r], sa.nvt ? sa.thermo[r].s1 : 1.0));
            }
            warp_max_to(&ctl->maxd[step & 1], dmax);
            if (!grid_barrier(ctl, c.limit_ns)) return;
            const float m2 = __uint_as_float(*(volatile unsigned *)&ctl->maxd[step & 1]);
            if (m2 > c.half_skin2 || *(volatile int *)&a.status->rebuild != 0) {
                if (tid == 0) {
                    ctl->steps_done = step;
                    ctl->stop = 1;
                    a.status->rebuild = 1;
                }
                return;
            }
        }
        // the other slot is the next step's maximum (every block has read it)
        if (tid == 0) ctl->maxd[(step + 1) & 1] = 0u;

        // ---- P2: one list entry per thread ----
        for (long long e = tid; e < n_entries; e += nthr) {
            const int k = (int)(e / n), i = (int)(e - (long long)k * n);
            unsigned char on = 0;
            if (k < a.nn[i]) {
                const ShapeDev &shi = a.shapes[a.shape[i]];
                const Geom &gi = geo[shi.geom];
                const Owner<T> own = make_owner<T>(a, i, shi, gi);
                const float4 ent = a.nlist[e];
                PairGeom<T> pg;
                int j;
                if (in_range<T>(a, ent, own, &j, &pg)) {
                    const Geom &gj = geo[pg.gj];
                    const M33<T> Ri = orientation<T>(a, i);
                    PairWork<T> w;
                    w.M = mul_tn(Ri, orientation_j<T>(a, j, pg));
                    w.dl = mul_t(Ri, pg.d);
                    w.rc = (T)WCA_CUT * pg.sig;
                    w.sig2 = pg.sig * pg.sig;
                    w.gj = pg.gj;
                    w.jref = j < i;
                    w.i = i;
                    w.j = j;
                    PathCount pc;
                    if (pair_setup<T, false>(tab, itab, gi, gj, &w, &pc)) {
                        on = 1;
                        if constexpr (REF) {
                            FFPartSink ps;
                            ps.zero();
                            eval_pair<T, DIM, false, true>(tab, itab, gi, gj, w, eps, par_eps, ps, &pc, &a);
#pragma unroll
                            for (int q = 0; q < 6; ++q) {
                                part[q * plane + e] = ps.f[q].s;
                                part[(6 + q) * plane + e] = ps.f[q].c;
                            }
#pragma unroll
                            for (int q = 0; q < 7; ++q) part[(12 + q) * plane + e] = ps.v[q];
                        } else {
                            PartSink<T> ps;
                            ps.zero();
                            eval_pair<T, DIM, false, false>(tab, itab, gi, gj, w, eps, par_eps, ps, &pc);
#pragma unroll
                            for (int q = 0; q < 13; ++q) part[q * plane + e] = ps.v[q];
                        }
                    }
                }
            }
            c.act[e] = on;
        }
        if (!grid_barrier(ctl, c.limit_ns)) return;

        // ---- P3: per-particle sums, outputs, second half step ----
        for (int i = pid; i < n; i += nthr) {
            SumSink<T, COMP> S;
            S.zero();
            const int nn = a.nn[i];
            for (int k = 0; k < nn; ++k) {
                const size_t e = (size_t)k * n + i;
                if (!c.act[e]) continue;
                if constexpr (REF) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) S.v[q].merge(part[q * plane + e], part[(6 + q) * plane + e]);
#pragma unroll
                    for (int q = 0; q < 7; ++q) S.v[6 + q].add(part[(12 + q) * plane + e]);
                } else {
                    T v[13];
#pragma unroll
                    for (int q = 0; q < 13; ++q) v[q] = part[q * plane + e];
                    S.add(v);
                }
            }
            finish_particle(a, i, S, orientation<T>(a, i));
            second_half_particle(sa, i);
        }

        // ---- thermostat ----
        if (sa.nvt) {
            if (!grid_barrier(ctl, c.limit_ns)) return;
            if (!sa.direct_sums) {
                for (int ch = blockIdx.x; ch < sa.n_chunks; ch += gridDim.x) chunk_sums_block(sa, ch);
                if (!grid_barrier(ctl, c.limit_ns)) return;
            }
            for (int r = blockIdx.x; r < sa.n_reps; r += gridDim.x) thermo_end_replica(sa, r);
            if (!grid_barrier(ctl, c.limit_ns)) return;
            if (!sa.direct_sums)
                for (int i = pid; i < n; i += nthr) scale_particle(sa, i);
        }
    }
    if (tid == 0) {
        ctl->steps_done = c.n_steps;
        ctl->stop = 0;
    }
}

template <class K> int coop_blocks_per_sm(K kernel, size_t smem) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, COOP_BLOCK, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return b;
}

template <class T, bool COMP> int coop_per_sm(int dim, size_t smem) {
    return dim == 2 ? coop_blocks_per_sm(k_coop_steps<T, COMP, 2>, smem)
                    : coop_blocks_per_sm(k_coop_steps<T, COMP, 3>, smem);
}

template <class T, bool COMP> const void *coop_kernel(int dim) {
    if (dim == 2) return reinterpret_cast<const void *>(k_coop_steps<T, COMP, 2>);
    return reinterpret_cast<const void *>(k_coop_steps<T, COMP, 3>);
}

}  // namespace

size_t coop_partial_bytes(int precision, int n, int cap) {
    const size_t pw = precision == DEM_FP32_COMP ? 19 : 13;
    const size_t el = precision == DEM_FP64 ? sizeof(double) : sizeof(float);
    return pw * el * (size_t)cap * (size_t)n;
}

int coop_grid(int precision, int dim, int n, int cap, size_t smem) {
    int per_sm = 0;
    switch (precision) {
        case DEM_FP64: per_sm = coop_per_sm<double, false>(dim, smem); break;
        case DEM_FP32: per_sm = coop_per_sm<float, false>(dim, smem); break;
        default: per_sm = coop_per_sm<float, true>(dim, smem);
    }
    if (per_sm < 1) return 0;
    // one block per SM: every SM takes a share of the per-particle FP64 work,
    // and a barrier waits for no more blocks than there are SMs
    (void)n;
    (void)cap;
    return sm_count();
}

cudaError_t launch_coop_steps(const CoopArgs &c, int precision, int dim, int grid, size_t smem,
                              cudaStream_t s) {
    const void *k = precision == DEM_FP64 ? coop_kernel<double, false>(dim)
                    : precision == DEM_FP32 ? coop_kernel<float, false>(dim)
                                            : coop_kernel<float, true>(dim);
    void *args[] = {const_cast<CoopArgs *>(&c)};
    return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(COOP_BLOCK), args, smem, s);
}

}  // namespace dem
