// pair.cu -- pair feature kernels: force, torque, energy and virial of every
// particle from all feature pairs with its neighbours (Eq. DEM in 3D,
// Eq. DEM_2D in 2D, WCA of Eq. LJ / Eq. WCA), Section "Algorithm" of
// arXiv:1607.02427 re-designed for sm_103a.
//
// Work decomposition (owner computes over a full neighbour list; only
// particle i's sums are written, so no atomics and a fixed summation order):
//   THREAD  one thread per particle i walks its neighbours j.
//   WARP    one warp per particle i; the pair setups of 32 list entries are
//           made by 32 lanes, then the (neighbour, vertex) and (neighbour,
//           edge) work items and, after the cheap culls, the surviving
//           (vertex, face) and (edge, edge) tests are spread evenly over the
//           lanes with warp scans; shuffle trees combine the lane sums.
//
// Separation.  FP32 modes: x_j - x_i = d0 + delta_j - delta_i, where d0 is
// the FP32 minimum-image separation stored in the list entry when the list
// was built (taken in FP64 there) and delta the FP32 displacement since the
// build: no FP64 arithmetic in the kernel (FP64 throughput is ~1/64 of FP32
// on this part).  FP64 mode: x_j - x_i from the FP64 positions, minimum image
// by comparison with half the box.
//
// Exact culls (each skips only terms that are zero because r* >= r_cut):
//   pair:    |x_ij| >= R_i + R_j + r_cut         (all features lie within R)
//   vertex:  |p - x_owner| >= R_owner + r_cut    (p cannot reach any face)
//   edge:    |c_e - x_i| >= R_i + h_e + r_cut    (the edge cannot reach i)
//   face:    |signed plane distance| >= r_cut
//   edges:   |c_1 - c_2| >= h_1 + h_2 + r_cut    (edge bounding spheres)
#include <type_traits>

#include "pair_common.cuh"

namespace dem {
namespace {

constexpr double WCA_CUT = 1.122462048309373;   // 2^(1/6)
constexpr unsigned FULL = 0xffffffffu;

template <class T> __device__ __forceinline__ const typename R4T<T>::type *table_ptr(const PairArgs &a) {
    return reinterpret_cast<const typename R4T<T>::type *>(a.table);
}

// Copy the geometry table into shared memory (once per block).
template <class T>
__device__ __forceinline__ void stage_tables(const PairArgs &a, typename R4T<T>::type *tab,
                                             Geom *geo, int *itab) {
    const typename R4T<T>::type *src = table_ptr<T>(a);
    for (int k = threadIdx.x; k < a.table_len; k += blockDim.x) tab[k] = src[k];
    const int *gsrc = reinterpret_cast<const int *>(a.geoms);
    int *gdst = reinterpret_cast<int *>(geo);
    int gwords = a.n_geoms * (int)(sizeof(Geom) / sizeof(int));
    for (int k = threadIdx.x; k < gwords; k += blockDim.x) gdst[k] = gsrc[k];
    for (int k = threadIdx.x; k < a.itable_len; k += blockDim.x) itab[k] = a.itable[k];
}

// Particle i's data for the range tests of its list entries.
template <class T> struct Owner {
    float4 delta;        // FP32 modes
    double4_32a x;       // FP64 mode
    T R, rnd;
    T sig_all;           // the one sigma of all pairs, or 0 (sigma_ij = r_i + r_j)
    const Rep *rp;
};

template <class T> struct PairGeom {
    V3<T> d;             // x_j - x_i (minimum image), world frame
    T sig;               // sigma_ij
    int gj;              // geometry of j
};

// Bounding-sphere range test of list entry e of owner o.
template <class T>
__device__ __forceinline__ bool in_range(const PairArgs &a, const float4 &e, const Owner<T> &o,
                                         int *jout, PairGeom<T> *pg) {
    const int j = __float_as_int(e.w);
    *jout = j;
    const ShapeDev &shj = a.shapes[__ldg(a.shape + j)];
    if constexpr (std::is_same<T, float>::value) {
        const float4 dj = a.delta[j];
        const float dx = e.x + (dj.x - o.delta.x);
        const float dy = e.y + (dj.y - o.delta.y);
        const float dz = e.z + (dj.z - o.delta.z);
        const float sig = o.sig_all > 0.f ? o.sig_all : o.rnd + shj.rounding_f;
        const float lim = o.R + shj.R + (float)WCA_CUT * sig;
        if (!(dx * dx + dy * dy + dz * dz < lim * lim)) return false;
        pg->d = v3<float>(dx, dy, dz);
        pg->sig = sig;
    } else {
        const double4_32a xj = a.pos[j];
        const Rep &rp = *o.rp;
        double d[3] = {xj.x - o.x.x, xj.y - o.x.y, a.dim == 3 ? xj.z - o.x.z : 0.0};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (d[k] > 0.5 * rp.L[k]) d[k] -= rp.L[k];
            else if (d[k] < -0.5 * rp.L[k]) d[k] += rp.L[k];
        }
        const double sig = o.sig_all > 0.0 ? o.sig_all : o.rnd + shj.rounding;
        const double lim = (double)o.R + (double)shj.R + WCA_CUT * sig;
        if (!(d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < lim * lim)) return false;
        pg->d = v3<double>(d[0], d[1], d[2]);
        pg->sig = sig;
    }
    pg->gj = shj.geom;
    return true;
}

template <class T> __device__ __forceinline__ M33<T> orientation(const PairArgs &a, int i);
template <> __device__ __forceinline__ M33<float> orientation<float>(const PairArgs &a, int i) {
    float4 q = a.quatf[i];
    return quat_mat<float>(q.x, q.y, q.z, q.w);
}
template <> __device__ __forceinline__ M33<double> orientation<double>(const PairArgs &a, int i) {
    double4_32a q = a.quat[i];
    return quat_mat<double>(q.x, q.y, q.z, q.w);
}

template <class T>
__device__ __forceinline__ Owner<T> make_owner(const PairArgs &a, int i, const ShapeDev &shi,
                                               const Geom &gi) {
    Owner<T> o;
    o.rp = &a.reps[a.rep[i]];
    o.R = (T)gi.R;
    o.sig_all = a.sigma > 0.0 ? (T)a.sigma : T(0);
    if constexpr (std::is_same<T, float>::value) {
        o.delta = a.delta[i];
        o.rnd = shi.rounding_f;
    } else {
        o.x = a.pos[i];
        o.rnd = shi.rounding;
    }
    return o;
}

// Totals of particle i: force rotated to the world frame, torque in the
// body frame, energy, virial rotated to the world frame (R W R^T), all in T;
// out = {F(3), tau(3), U, W(6)}.
template <class T, bool COMP>
__device__ __forceinline__ void totals(const Sums<T, COMP> &S, const M33<T> &R, T out[13]) {
    T tot[13];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        tot[k] = S.f[k].s + S.f[k].comp();
        tot[3 + k] = S.t[k].s + S.t[k].comp();
    }
    tot[6] = S.u.s + S.u.comp();
#pragma unroll
    for (int k = 0; k < 6; ++k) tot[7 + k] = S.w[k].s + S.w[k].comp();
    const V3<T> fw = mul(R, v3<T>(tot[0], tot[1], tot[2]));
    out[0] = fw.x; out[1] = fw.y; out[2] = fw.z;
    out[3] = tot[3]; out[4] = tot[4]; out[5] = tot[5];
    out[6] = tot[6];
    const T B[3][3] = {{tot[7], tot[8], tot[9]}, {tot[8], tot[10], tot[11]}, {tot[9], tot[11], tot[12]}};
    T RB[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            RB[r][c] = R.m[r][0] * B[0][c] + R.m[r][1] * B[1][c] + R.m[r][2] * B[2][c];
    const int idx[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int r = idx[k][0], c = idx[k][1];
        out[7 + k] = RB[r][0] * R.m[c][0] + RB[r][1] * R.m[c][1] + RB[r][2] * R.m[c][2];
    }
}

// Store value k of the 13 totals of particle i.
__device__ __forceinline__ void store_value(const PairArgs &a, int i, int k, double v) {
    if (k < 3) reinterpret_cast<double *>(a.force + i)[k] = v;
    else if (k < 6) reinterpret_cast<double *>(a.torque + i)[k - 3] = v;
    else if (k == 6) a.energy[i] = v;
    else a.virial[6 * (size_t)i + (k - 7)] = v;
    if (!isfinite(v)) atomicExch(&a.status->nonfinite, 1);
}

// All terms of the ordered pair (i, j) (i's geometry gi, j's gj), evaluated
// in i's frame, accumulated into S.  Returns the number of feature pairs
// the definition (Eq. DEM / Eq. DEM_2D) assigns to the pair.
template <class T, bool COMP, int DIM, bool COUNT>
__device__ __forceinline__ unsigned int pair_terms(const typename R4T<T>::type *tab,
                                                   const int *itab, const Geom &gi,
                                                   const Geom &gj, const M33<T> &M, V3<T> dl,
                                                   T rc, T sig2, T eps, T par_eps,
                                                   Sums<T, COMP> &S, PathCount *pc) {
    using R4 = typename R4T<T>::type;
    const T rc2 = rc * rc;
    T U, wf;
    if (gi.nv == 1 && gj.nv == 1) {             // sphere / disk limit: central WCA
        V3<T> pi = xyz<T>(tab[gi.v_off]);
        V3<T> pj = dl + mul(M, xyz<T>(tab[gj.v_off]));
        V3<T> rv = pi - pj;
        T r2 = dot(rv, rv);
        if (r2 < rc2) {
            wf = wca_factor(r2, sig2, eps, &U);
            add_term_body(S, pi, rv * wf, dl, U);
        }
        return 1u;
    }
    const T reach_i = T(gi.R) + rc, reach_j = T(gj.R) + rc;
    if constexpr (DIM == 2) {
        // V_j x E_i (Eq. DEM_2D, second sum), in i's frame
        for (int b = 0; b < gj.nv; ++b) {
            V3<T> p = dl + mul(M, xyz<T>(tab[gj.v_off + b]));
            bump<COUNT>(pc, C_VTX);
            if (!(dot(p, p) < reach_i * reach_i)) continue;
            for (int e = 0; e < gi.ne; ++e) {
                R4 ea = tab[gi.e_off + 2 * e], ed = tab[gi.e_off + 2 * e + 1];
                V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                V3<T> c = A + D * T(0.5) - p;
                T lim = ea.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(c, c) < lim * lim)) continue;
                bump<COUNT>(pc, C_PTSEG);
                V3<T> q = A + D * clamp01(dot(p - A, D) * ed.w);
                V3<T> rv = q - p;
                T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    wf = wca_factor(r2, sig2, eps, &U);
                    add_term_body(S, q, rv * wf, dl, U);
                }
            }
        }
        // V_i x E_j (Eq. DEM_2D, first sum), in j's frame
        for (int a_ = 0; a_ < gi.nv; ++a_) {
            V3<T> u = xyz<T>(tab[gi.v_off + a_]);
            V3<T> p = mul_t(M, u - dl);
            bump<COUNT>(pc, C_VTX);
            if (!(dot(p, p) < reach_j * reach_j)) continue;
            for (int e = 0; e < gj.ne; ++e) {
                R4 ea = tab[gj.e_off + 2 * e], ed = tab[gj.e_off + 2 * e + 1];
                V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                V3<T> c = A + D * T(0.5) - p;
                T lim = ea.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(c, c) < lim * lim)) continue;
                bump<COUNT>(pc, C_PTSEG);
                V3<T> q = A + D * clamp01(dot(p - A, D) * ed.w);
                V3<T> rv = p - q;
                T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    bump<COUNT>(pc, C_JTERMS);
                    wf = wca_factor(r2, sig2, eps, &U);
                    add_term_body(S, u, mul(M, rv * wf), dl, U);
                }
            }
        }
        return (unsigned)(gi.nv * gj.ne + gj.nv * gi.ne);
    } else {
        // 3D.  V_j x F_i (Eq. DEM, third sum), in i's frame
        for (int b = 0; b < gj.nv; ++b) {
            V3<T> p = dl + mul(M, xyz<T>(tab[gj.v_off + b]));
            bump<COUNT>(pc, C_VTX);
            if (!(dot(p, p) < reach_i * reach_i)) continue;
            for (int f = 0; f < gi.nf; ++f) {
                V3<T> q;
                T r2;
                if (!face_nearest<T, COUNT>(tab, itab, gi.f_off + f, gi.fi_off + 2 * f, p, rc, &q, &r2, pc))
                    continue;
                if (r2 < rc2) {
                    wf = wca_factor(r2, sig2, eps, &U);
                    add_term_body(S, q, (q - p) * wf, dl, U);
                }
            }
        }
        // V_i x F_j (Eq. DEM, second sum), in j's frame
        for (int a_ = 0; a_ < gi.nv; ++a_) {
            V3<T> u = xyz<T>(tab[gi.v_off + a_]);
            V3<T> p = mul_t(M, u - dl);
            bump<COUNT>(pc, C_VTX);
            if (!(dot(p, p) < reach_j * reach_j)) continue;
            for (int f = 0; f < gj.nf; ++f) {
                V3<T> q;
                T r2;
                if (!face_nearest<T, COUNT>(tab, itab, gj.f_off + f, gj.fi_off + 2 * f, p, rc, &q, &r2, pc))
                    continue;
                if (r2 < rc2) {
                    bump<COUNT>(pc, C_JTERMS);
                    wf = wca_factor(r2, sig2, eps, &U);
                    add_term_body(S, u, mul(M, (p - q) * wf), dl, U);
                }
            }
        }
        // E_i x E_j (Eq. DEM, first sum), in i's frame
        for (int eb = 0; eb < (gi.ne > 0 ? gj.ne : 0); ++eb) {
            R4 ba = tab[gj.e_off + 2 * eb], bd = tab[gj.e_off + 2 * eb + 1];
            V3<T> A2 = dl + mul(M, xyz<T>(ba));
            V3<T> D2 = mul(M, xyz<T>(bd));
            V3<T> C2 = A2 + D2 * T(0.5);
            T reach = reach_i + ba.w;
            bump<COUNT>(pc, C_EDGE);
            if (!(dot(C2, C2) < reach * reach)) continue;
            for (int ea = 0; ea < gi.ne; ++ea) {
                R4 aa = tab[gi.e_off + 2 * ea], ad = tab[gi.e_off + 2 * ea + 1];
                V3<T> A1 = xyz<T>(aa), D1 = xyz<T>(ad);
                V3<T> dc = A1 + D1 * T(0.5) - C2;
                T lim = aa.w + ba.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(dc, dc) < lim * lim)) continue;
                bump<COUNT>(pc, C_SEGSEG);
                V3<T> P1, P2;
                segment_nearest<T>(A1, D1, ad.w, A2, D2, bd.w, par_eps, &P1, &P2);
                V3<T> rv = P1 - P2;
                T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    wf = wca_factor(r2, sig2, eps, &U);
                    add_term_body(S, P1, rv * wf, dl, U);
                }
            }
        }
        return (unsigned)(gi.ne * gj.ne + gi.nv * gj.nf + gj.nv * gi.nf);
    }
}

// ---------------------------------------------------------------------------
// THREAD decomposition
// ---------------------------------------------------------------------------
template <class T, bool COMP, int DIM, bool COUNT>
__global__ void __launch_bounds__(THREADS) k_pair_thread(const PairArgs a) {
    using R4 = typename R4T<T>::type;
    extern __shared__ __align__(32) unsigned char smem[];
    R4 *tab = reinterpret_cast<R4 *>(smem);
    Geom *geo = reinterpret_cast<Geom *>(tab + a.table_len);
    int *itab = reinterpret_cast<int *>(geo + a.n_geoms);
    stage_tables<T>(a, tab, geo, itab);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && !COUNT) {
        // the list (if it was due) has been rebuilt by now: clear the request
        a.status->maxdisp2 = 0u;
        a.status->rebuild = 0;
    }
    const T eps = (T)a.eps;
    const T par_eps = (T)a.par_eps;
    PathCount pc;
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k) pc.v[k] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const ShapeDev &shi = a.shapes[a.shape[i]];
        const Geom gi = geo[shi.geom];
        const Owner<T> own = make_owner<T>(a, i, shi, gi);
        const M33<T> Ri = orientation<T>(a, i);
        Sums<T, COMP> S;
        S.zero();
        const int nn = a.nn[i];
        for (int k = 0; k < nn; ++k) {
            const float4 e = a.nlist[(size_t)k * a.n + i];
            PairGeom<T> pg;
            int j;
            bump<COUNT>(&pc, C_NEIGH);
            if (!in_range<T>(a, e, own, &j, &pg)) continue;
            const M33<T> Rj = orientation<T>(a, j);
            const M33<T> M = mul_tn(Ri, Rj);
            const V3<T> dl = mul_t(Ri, pg.d);
            const T rc = (T)WCA_CUT * pg.sig;
            unsigned nf = pair_terms<T, COMP, DIM, COUNT>(tab, itab, gi, geo[pg.gj], M, dl, rc,
                                                          pg.sig * pg.sig, eps, par_eps, S, &pc);
            bump<COUNT>(&pc, C_PAIRS);
            bump<COUNT>(&pc, C_FPE, nf);
        }
        bump<COUNT>(&pc, C_TERMS, S.nterm);
        T out[13];
        totals(S, Ri, out);
#pragma unroll
        for (int k = 0; k < 13; ++k) store_value(a, i, k, (double)out[k]);
    }
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k)
            if (pc.v[k]) atomicAdd(a.counters + k, (unsigned long long)pc.v[k]);
}

template <class T, bool COMP, int DIM>
cudaError_t launch_thread(const PairArgs &a, int block, bool count, size_t smem, cudaStream_t s) {
    int grid = (a.n + block - 1) / block;
    if (grid < 1) grid = 1;
    if (count) {
        auto k = k_pair_thread<T, COMP, DIM, true>;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, s>>>(a);
    } else {
        auto k = k_pair_thread<T, COMP, DIM, false>;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, s>>>(a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// WARP decomposition
//
// One warp per particle i (grid-stride over particles, persistent grid).  The
// neighbour list is taken 32 entries at a time; each lane tests one entry
// for the bounding-sphere range and, if in range, writes the pair setup
// (M = R_i^T R_j, dl, r_cut, sigma^2, j's geometry) to a per-warp slot.
// Then two compacted phases share the pair work evenly across the lanes:
//   vertices: items = (slot, vertex of j or of i); each lane maps its vertex
//     into the face owner's frame and tests its reach; the survivors' (vertex,
//     face) tests (2D: (vertex, edge)) are re-spread over all lanes with a
//     warp scan of their counts, the vertex data moving by shuffles;
//   edges (3D): items = (slot, edge of j); each lane maps its edge into i's
//     frame and tests its reach; the survivors' (edge of j, edge of i) tests
//     are re-spread the same way.
// Each lane keeps private sums; a fixed shuffle tree combines them (two-sum
// merge in the compensated mode), so results are deterministic.  The 13
// totals are rotated on lane 0 and written by 13 lanes at once.
// ---------------------------------------------------------------------------
template <class T> struct Slot {
    T m[9];
    T dl[3];
    T rc, sig2;
    int gj;
    int pad;
};

// Exclusive warp scan of v; *total = the warp's sum.
__device__ __forceinline__ int warp_excl_scan(int v, int lane, int *total) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(FULL, x, 31);
    return x - v;
}

// Largest k in [0, n) with off[k] <= t (off non-decreasing, off[0] = 0): the
// owner of item t when owner k holds items [off[k], off[k+1]).
__device__ __forceinline__ int owner_of(const int *off, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class T> __device__ __forceinline__ M33<T> slot_m(const Slot<T> &s) {
    M33<T> M;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) M.m[r][c] = s.m[3 * r + c];
    return M;
}

template <class T, bool COMP> __device__ __forceinline__ void merge_down(Acc<T, COMP> &x, int o) {
    const T s = __shfl_down_sync(FULL, x.s, o);
    const T c = __shfl_down_sync(FULL, x.comp(), o);
    x.merge(s, c);
}

template <class T, bool COMP>
__device__ __forceinline__ void warp_sum(Sums<T, COMP> &S) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            merge_down(S.f[k], o);
            merge_down(S.t[k], o);
        }
        merge_down(S.u, o);
#pragma unroll
        for (int k = 0; k < 6; ++k) merge_down(S.w[k], o);
        S.nterm += __shfl_down_sync(FULL, S.nterm, o);
    }
}

template <class T, bool COMP, int DIM, bool COUNT>
__global__ void __launch_bounds__(128) k_pair_warp(const PairArgs a) {
    using R4 = typename R4T<T>::type;
    extern __shared__ __align__(32) unsigned char smem[];
    R4 *tab = reinterpret_cast<R4 *>(smem);
    Geom *geo = reinterpret_cast<Geom *>(tab + a.table_len);
    int *itab = reinterpret_cast<int *>(geo + a.n_geoms);
    size_t tb = (size_t)a.table_len * sizeof(R4) + sizeof(Geom) * a.n_geoms +
                sizeof(int) * a.itable_len;
    tb = (tb + 31) & ~(size_t)31;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    Slot<T> *slots = reinterpret_cast<Slot<T> *>(smem + tb) + w * 32;
    int *offs = reinterpret_cast<int *>(reinterpret_cast<Slot<T> *>(smem + tb) + wpb * 32) + w * 64;
    int *loffs = offs + 32;
    stage_tables<T>(a, tab, geo, itab);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && !COUNT) {
        a.status->maxdisp2 = 0u;
        a.status->rebuild = 0;
    }
    const T eps = (T)a.eps;
    const T par_eps = (T)a.par_eps;
    PathCount pc;
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k) pc.v[k] = 0;
    for (int i = blockIdx.x * wpb + w; i < a.n; i += gridDim.x * wpb) {
        const ShapeDev &shi = a.shapes[a.shape[i]];
        const Geom gi = geo[shi.geom];
        const Owner<T> own = make_owner<T>(a, i, shi, gi);
        const M33<T> Ri = orientation<T>(a, i);
        Sums<T, COMP> S;
        S.zero();
        const int nn = a.nn[i];
        for (int base = 0; base < nn; base += 32) {
            // ---- pair setups of up to 32 list entries ----
            const int k = base + lane;
            PairGeom<T> pg;
            bool inr = false;
            int j = 0;
            if (k < nn) {
                const float4 e = a.nlist[(size_t)k * a.n + i];
                bump<COUNT>(&pc, C_NEIGH);
                inr = in_range<T>(a, e, own, &j, &pg);
            }
            const unsigned m = __ballot_sync(FULL, inr);
            const int ns = __popc(m);
            if (ns == 0) continue;
            if (inr) {
                const int my = __popc(m & ((1u << lane) - 1u));
                const M33<T> Rj = orientation<T>(a, j);
                const M33<T> M = mul_tn(Ri, Rj);
                const V3<T> dl = mul_t(Ri, pg.d);
                Slot<T> &sl = slots[my];
#pragma unroll
                for (int r = 0; r < 3; ++r)
#pragma unroll
                    for (int c = 0; c < 3; ++c) sl.m[3 * r + c] = M.m[r][c];
                sl.dl[0] = dl.x; sl.dl[1] = dl.y; sl.dl[2] = dl.z;
                sl.rc = (T)WCA_CUT * pg.sig;
                sl.sig2 = pg.sig * pg.sig;
                sl.gj = pg.gj;
                const Geom &gj = geo[pg.gj];
                if (gi.nv == 1 && gj.nv == 1) {
                    // sphere / disk limit: the one central term, by this lane
                    const V3<T> pi = xyz<T>(tab[gi.v_off]);
                    const V3<T> rv = pi - (dl + mul(M, xyz<T>(tab[gj.v_off])));
                    const T r2 = dot(rv, rv);
                    if (r2 < sl.rc * sl.rc) {
                        T U;
                        const T wf = wca_factor(r2, sl.sig2, eps, &U);
                        add_term_body(S, pi, rv * wf, dl, U);
                    }
                    bump<COUNT>(&pc, C_FPE, 1u);
                } else if (DIM == 2) {
                    bump<COUNT>(&pc, C_FPE, (unsigned)(gi.nv * gj.ne + gj.nv * gi.ne));
                } else {
                    bump<COUNT>(&pc, C_FPE, (unsigned)(gi.ne * gj.ne + gi.nv * gj.nf + gj.nv * gi.nf));
                }
                bump<COUNT>(&pc, C_PAIRS);
            }
            __syncwarp();

            // ---- vertex phase ----
            {
                int c = 0;
                if (lane < ns) {
                    const Geom &gj = geo[slots[lane].gj];
                    c = (gi.nv == 1 && gj.nv == 1) ? 0 : gj.nv + gi.nv;
                }
                int tot;
                const int ex = warp_excl_scan(c, lane, &tot);
                offs[lane] = ex;
                __syncwarp();
                for (int t0 = 0; t0 < tot; t0 += 32) {
                    const int t = t0 + lane;
                    bool surv = false;
                    V3<T> p = v3<T>(T(0), T(0), T(0));
                    int s = 0, dir = 0, vid = 0, nfc = 0;
                    if (t < tot) {
                        s = owner_of(offs, ns, t);
                        const Slot<T> &sl = slots[s];
                        const Geom &gj = geo[sl.gj];
                        const M33<T> M = slot_m(sl);
                        const V3<T> dl = v3<T>(sl.dl[0], sl.dl[1], sl.dl[2]);
                        vid = t - offs[s];
                        T reach;
                        if (vid < gj.nv) {          // vertex of j against i's faces
                            dir = 0;
                            p = dl + mul(M, xyz<T>(tab[gj.v_off + vid]));
                            reach = T(gi.R) + sl.rc;
                            nfc = DIM == 3 ? gi.nf : gi.ne;
                        } else {                    // vertex of i against j's faces
                            dir = 1;
                            vid -= gj.nv;
                            p = mul_t(M, xyz<T>(tab[gi.v_off + vid]) - dl);
                            reach = T(gj.R) + sl.rc;
                            nfc = DIM == 3 ? gj.nf : gj.ne;
                        }
                        bump<COUNT>(&pc, C_VTX);
                        surv = dot(p, p) < reach * reach;
                    }
                    int ftot;
                    const int fex = warp_excl_scan(surv ? nfc : 0, lane, &ftot);
                    loffs[lane] = fex;
                    __syncwarp();
                    for (int u0 = 0; u0 < ftot; u0 += 32) {
                        const int u = u0 + lane;
                        const int L = owner_of(loffs, 32, u < ftot ? u : ftot - 1);
                        const T px = __shfl_sync(FULL, p.x, L);
                        const T py = __shfl_sync(FULL, p.y, L);
                        const T pz = __shfl_sync(FULL, p.z, L);
                        const int os = __shfl_sync(FULL, s, L);
                        const int od = __shfl_sync(FULL, dir, L);
                        const int ov = __shfl_sync(FULL, vid, L);
                        if (u < ftot) {
                            const int f = u - loffs[L];
                            const Slot<T> &sl = slots[os];
                            const Geom &go = od == 0 ? gi : geo[sl.gj];
                            const T rc = sl.rc;
                            const V3<T> P = v3<T>(px, py, pz);
                            V3<T> q;
                            T r2;
                            bool hit;
                            if constexpr (DIM == 3) {
                                hit = face_nearest<T, COUNT>(tab, itab, go.f_off + f, go.fi_off + 2 * f,
                                                             P, rc, &q, &r2, &pc) && r2 < rc * rc;
                            } else {
                                const R4 ea = tab[go.e_off + 2 * f], ed = tab[go.e_off + 2 * f + 1];
                                const V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                                const V3<T> cc = A + D * T(0.5) - P;
                                const T lim = ea.w + rc;
                                bump<COUNT>(&pc, C_SPHERE);
                                hit = false;
                                if (dot(cc, cc) < lim * lim) {
                                    bump<COUNT>(&pc, C_PTSEG);
                                    q = A + D * clamp01(dot(P - A, D) * ed.w);
                                    const V3<T> rr = P - q;
                                    r2 = dot(rr, rr);
                                    hit = r2 < rc * rc;
                                }
                            }
                            if (hit) {
                                T U;
                                const T wf = wca_factor(r2, sl.sig2, eps, &U);
                                const V3<T> dl = v3<T>(sl.dl[0], sl.dl[1], sl.dl[2]);
                                if (od == 0) {
                                    add_term_body(S, q, (q - P) * wf, dl, U);
                                } else {
                                    bump<COUNT>(&pc, C_JTERMS);
                                    add_term_body(S, xyz<T>(tab[gi.v_off + ov]),
                                                  mul(slot_m(sl), (P - q) * wf), dl, U);
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            }

            // ---- edge phase (3D) ----
            if constexpr (DIM == 3) {
                int c = 0;
                if (lane < ns) {
                    const Geom &gj = geo[slots[lane].gj];
                    c = (gi.nv == 1 && gj.nv == 1) || gi.ne == 0 ? 0 : gj.ne;
                }
                int tot;
                const int ex = warp_excl_scan(c, lane, &tot);
                offs[lane] = ex;
                __syncwarp();
                for (int t0 = 0; t0 < tot; t0 += 32) {
                    const int t = t0 + lane;
                    bool surv = false;
                    V3<T> A2 = v3<T>(T(0), T(0), T(0)), D2 = A2;
                    T h2 = T(0), ic = T(0);
                    int s = 0;
                    if (t < tot) {
                        s = owner_of(offs, ns, t);
                        const Slot<T> &sl = slots[s];
                        const Geom &gj = geo[sl.gj];
                        const M33<T> M = slot_m(sl);
                        const V3<T> dl = v3<T>(sl.dl[0], sl.dl[1], sl.dl[2]);
                        const int eb = t - offs[s];
                        const R4 ba = tab[gj.e_off + 2 * eb], bd = tab[gj.e_off + 2 * eb + 1];
                        A2 = dl + mul(M, xyz<T>(ba));
                        D2 = mul(M, xyz<T>(bd));
                        h2 = ba.w;
                        ic = bd.w;
                        const V3<T> C2 = A2 + D2 * T(0.5);
                        const T reach = T(gi.R) + sl.rc + h2;
                        bump<COUNT>(&pc, C_EDGE);
                        surv = dot(C2, C2) < reach * reach;
                    }
                    int etot;
                    const int eex = warp_excl_scan(surv ? gi.ne : 0, lane, &etot);
                    loffs[lane] = eex;
                    __syncwarp();
                    for (int u0 = 0; u0 < etot; u0 += 32) {
                        const int u = u0 + lane;
                        const int L = owner_of(loffs, 32, u < etot ? u : etot - 1);
                        const V3<T> a2 = v3<T>(__shfl_sync(FULL, A2.x, L), __shfl_sync(FULL, A2.y, L),
                                               __shfl_sync(FULL, A2.z, L));
                        const V3<T> d2 = v3<T>(__shfl_sync(FULL, D2.x, L), __shfl_sync(FULL, D2.y, L),
                                               __shfl_sync(FULL, D2.z, L));
                        const T oh = __shfl_sync(FULL, h2, L);
                        const T oic = __shfl_sync(FULL, ic, L);
                        const int os = __shfl_sync(FULL, s, L);
                        if (u < etot) {
                            const int ea = u - loffs[L];
                            const Slot<T> &sl = slots[os];
                            const T rc = sl.rc;
                            const R4 aa = tab[gi.e_off + 2 * ea], ad = tab[gi.e_off + 2 * ea + 1];
                            const V3<T> A1 = xyz<T>(aa), D1 = xyz<T>(ad);
                            const V3<T> dc = A1 + D1 * T(0.5) - (a2 + d2 * T(0.5));
                            const T lim = aa.w + oh + rc;
                            bump<COUNT>(&pc, C_SPHERE);
                            if (dot(dc, dc) < lim * lim) {
                                bump<COUNT>(&pc, C_SEGSEG);
                                V3<T> P1, P2;
                                segment_nearest<T>(A1, D1, ad.w, a2, d2, oic, par_eps, &P1, &P2);
                                const V3<T> rv = P1 - P2;
                                const T r2 = dot(rv, rv);
                                if (r2 < rc * rc) {
                                    T U;
                                    const T wf = wca_factor(r2, sl.sig2, eps, &U);
                                    add_term_body(S, P1, rv * wf,
                                                  v3<T>(sl.dl[0], sl.dl[1], sl.dl[2]), U);
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
            }
            __syncwarp();
        }
        warp_sum(S);
        T out[13];
        if (lane == 0) {
            bump<COUNT>(&pc, C_TERMS, S.nterm);
            totals(S, Ri, out);
        }
        // lane k stores value k: the 13 conversions to FP64 run side by side
        T mine = T(0);
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            const T v = __shfl_sync(FULL, lane == 0 ? out[k] : T(0), 0);
            if (lane == k) mine = v;
        }
        if (lane < 13) store_value(a, i, lane, (double)mine);
    }
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k)
            if (pc.v[k]) atomicAdd(a.counters + k, (unsigned long long)pc.v[k]);
}

// Resident blocks per SM of a kernel (cached per kernel, block and smem size).
template <class K> int blocks_per_sm(K kernel, int block, size_t smem) {
    struct Entry { const void *fn; int block; size_t smem; int blocks; };
    static Entry cache[64];
    static int used = 0;
    const void *fn = reinterpret_cast<const void *>(kernel);
    for (int k = 0; k < used; ++k)
        if (cache[k].fn == fn && cache[k].block == block && cache[k].smem == smem)
            return cache[k].blocks;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, block, smem) != cudaSuccess || b < 1)
        b = 1;
    if (used < 64) cache[used++] = {fn, block, smem, b};
    return b;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

template <class T, bool COMP, int DIM>
cudaError_t launch_warp(const PairArgs &a, bool count, size_t smem_tables, cudaStream_t s) {
    const int block = 128;
    size_t smem = ((smem_tables + 31) & ~(size_t)31) + (block / 32) * (32 * sizeof(Slot<T>) + 64 * sizeof(int));
    auto launch = [&](auto kernel) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        long long need = (a.n + (block / 32) - 1) / (block / 32);
        long long cap = (long long)blocks_per_sm(kernel, block, smem) * sm_count();
        int grid = (int)(need < cap ? need : cap);
        if (grid < 1) grid = 1;
        kernel<<<grid, block, smem, s>>>(a);
    };
    if (count) launch(k_pair_warp<T, COMP, DIM, true>);
    else launch(k_pair_warp<T, COMP, DIM, false>);
    return cudaGetLastError();
}

template <class T, bool COMP>
cudaError_t dispatch_dim(const PairArgs &a, int decomp, int block, bool count, size_t smem,
                         cudaStream_t s) {
    if (decomp == DEM_DECOMP_WARP) {
        if (a.dim == 2) return launch_warp<T, COMP, 2>(a, count, smem, s);
        return launch_warp<T, COMP, 3>(a, count, smem, s);
    }
    if (a.dim == 2) return launch_thread<T, COMP, 2>(a, block, count, smem, s);
    return launch_thread<T, COMP, 3>(a, block, count, smem, s);
}

}  // namespace

size_t pair_smem_bytes(const PairArgs &a, int precision) {
    size_t rec = precision == DEM_FP64 ? sizeof(double4_32a) : sizeof(float4);
    return rec * a.table_len + sizeof(Geom) * a.n_geoms + sizeof(int) * a.itable_len;
}

cudaError_t launch_pair(const PairArgs &a, int precision, int decomp, int block, bool count,
                        cudaStream_t s) {
    size_t smem = pair_smem_bytes(a, precision);
    if (block <= 0) block = THREADS;
    if (block > THREADS) block = THREADS;
    switch (precision) {
        case DEM_FP64: return dispatch_dim<double, false>(a, decomp, block, count, smem, s);
        case DEM_FP32: return dispatch_dim<float, false>(a, decomp, block, count, smem, s);
        default: return dispatch_dim<float, true>(a, decomp, block, count, smem, s);
    }
}

}  // namespace dem
