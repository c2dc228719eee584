// pair.cu -- pair feature kernels: force, torque, energy and virial of every
// particle from all feature pairs with its neighbours (Eq. DEM in 3D,
// Eq. DEM_2D in 2D, WCA of Eq. LJ / Eq. WCA), Section "Algorithm" of
// arXiv:1607.02427 re-designed for sm_103a.
//
// Work decomposition (owner computes over a full neighbour list; only
// particle i's sums are written, so no atomics and a fixed summation order):
//   THREAD  one thread per particle i walks its neighbours j.
//   WARP    one warp per 32 particles, one lane per active pair: the lanes
//           scan the list entries of the 32 particles, the pairs that pass
//           the culls below are queued in ballot order, 32 queued pairs are
//           evaluated at a time (one per lane), and each particle's lane
//           adds its pairs' partial sums in queue order.
//
// Separation.  FP32 modes: x_j - x_i = d0 + delta_j - delta_i, where d0 is
// the FP32 minimum-image separation stored in the list entry when the list
// was built (taken in FP64 there) and delta the FP32 displacement since the
// build: no FP64 arithmetic in the kernel (FP64 throughput is ~1/64 of FP32
// on this part).  FP64 mode: x_j - x_i from the FP64 positions, minimum image
// by comparison with half the box.
//
// Culls (each skips only terms that are zero because every point pair of
// the two features is at least r_cut apart):
//   pair:    |x_ij| >= R_i + R_j + r_cut         (all features lie within R)
//   pair:    separating axis along u = x_ij / |x_ij|: |x_ij| - h_i - h_j >=
//            r_cut, with h_i, h_j the supports of the inner shapes towards
//            each other (projections of the vertices on u)
//   feature: a feature of i whose largest projection on u is at most
//            |x_ij| - h_j - r_cut cannot reach j (likewise for j); vertex
//            masks come from the projections, edge and face masks from the
//            vertex-membership masks of the geometry table
//   vertex:  |p - x_owner| >= R_owner + r_cut    (p cannot reach any face)
//   edge:    |c_e - x_i| >= R_i + h_e + r_cut    (the edge cannot reach i)
//   face:    |signed plane distance| >= r_cut
//   edges:   |c_1 - c_2| >= h_1 + h_2 + r_cut    (edge bounding spheres)
//   edges:   distance of the two carrier lines >= r_cut


#include "pair_kernels.cuh"

namespace dem {
namespace {

// ---------------------------------------------------------------------------
// THREAD decomposition
// ---------------------------------------------------------------------------
template <class T, bool COMP, int DIM, bool COUNT, class MK = unsigned>
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
        SumSink<T, COMP> S;
        S.zero();
        const int nn = a.nn[i];
        for (int k = 0; k < nn; ++k) {
            const float4 e = a.nlist[(size_t)k * a.n + i];
            PairGeom<T> pg;
            int j;
            bump<COUNT>(&pc, C_NEIGH);
            if (!in_range<T>(a, e, own, &j, &pg)) continue;
            const Geom &gj = geo[pg.gj];
            bump<COUNT>(&pc, C_PAIRS);
            bump<COUNT>(&pc, C_FPE, defined_feature_pairs(DIM, gi, gj));
            PairWork<T, MK> w;
            w.M = mul_tn(Ri, orientation_j<T>(a, j, pg));
            w.dl = mul_t(Ri, pg.d);
            w.rc = (T)WCA_CUT * pg.sig;
            w.sig2 = pg.sig * pg.sig;
            w.gj = pg.gj;
            w.jref = j < i;
            w.i = i;
            w.j = j;
            if (!pair_setup<T, COUNT>(tab, itab, gi, gj, &w, &pc)) continue;
            bump<COUNT>(&pc, C_ACTIVE);
            eval_pair<T, DIM, COUNT, COMP && std::is_same<T, float>::value>(tab, itab, gi, gj, w, eps,
                                                                            par_eps, S, &pc, &a);
        }
        finish_particle(a, i, S, Ri);
    }
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k)
            if (pc.v[k]) atomicAdd(a.counters + k, (unsigned long long)pc.v[k]);
}

template <class T, bool COMP, int DIM>
cudaError_t launch_thread(const PairArgs &a, int block, bool count, size_t smem, cudaStream_t s) {
    int grid = (a.n + block - 1) / block;
    if (grid < 1) grid = 1;
    auto launch = [&](auto k) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, block, smem, s>>>(a);
    };
    // shapes with more than 32 vertices, edges or faces: two-level masks
    if (a.mask_words > 1) {
        if (count) launch(k_pair_thread<T, COMP, DIM, true, WideMask<WIDE_WORDS>>);
        else launch(k_pair_thread<T, COMP, DIM, false, WideMask<WIDE_WORDS>>);
    } else {
        if (count) launch(k_pair_thread<T, COMP, DIM, true>);
        else launch(k_pair_thread<T, COMP, DIM, false>);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// WARP decomposition: 32 particles per warp, one lane per active pair
// ---------------------------------------------------------------------------
constexpr int PQ = 64;   // ring of queued pairs (one round adds at most 32)

template <class T> struct alignas(16) QPair {
    T m[12];             // row r: M[r][0..2], dl[r] at m[4r + 3]; reused for the partial
    T rc, sig2;
    int gj, owner;       // owner: the particle's lane in the warp
    unsigned vim, vjm, eim, ejm, fim, fjm;
    int jref;            // j < i: j's edge is the parallel-edge rule's reference
    int j;               // the neighbour (FP32 + two-sum refinement)
};
template <class T> struct alignas(16) PInfo {   // one particle of the warp
    T r[9];              // R_i
    T x[3];              // FP32: delta_i; FP64: position
    T R, rnd, sig_all;
    int geom, rep, nn;
    float sc;            // FP32 list separation scale of the replica
};
template <class T> struct WarpSmem {
    QPair<T> q[PQ];
    PInfo<T> p[32];
    int offs[32];
};

// lane add its pairs' partials in queue order.
// In the FP32 + two-sum mode a pair's partials are float-float for force and
// torque: the 6 leading parts go to m[0..5], their compensations to
// m[6..11], and the 7 other sums to rc, sig2 and the first five masks.
template <class T, bool COMP, int DIM, bool COUNT>
__device__ __forceinline__ void run_batch(WarpSmem<T> &ws, int qh, int nb, int lane,
                                          const typename R4T<T>::type *tab, const int *itab,
                                          const Geom *geo, T eps, T par_eps,
                                          SumSink<T, COMP> &S, PathCount *pc, const PairArgs &a,
                                          int base) {
    constexpr bool REF = COMP && std::is_same<T, float>::value;
    if (lane < nb) {
        QPair<T> &qp = ws.q[(qh + lane) & (PQ - 1)];
        PairWork<T> w;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) w.M.m[r][c] = qp.m[4 * r + c];
        w.dl = v3<T>(qp.m[3], qp.m[7], qp.m[11]);
        w.rc = qp.rc;
        w.sig2 = qp.sig2;
        w.gj = qp.gj;
        w.vim = qp.vim; w.vjm = qp.vjm; w.eim = qp.eim; w.ejm = qp.ejm;
        w.fim = qp.fim; w.fjm = qp.fjm;
        w.jref = qp.jref;
        w.i = base + qp.owner;
        w.j = qp.j;
        if constexpr (REF) {
            FFPartSink part;
            part.zero();
            eval_pair<T, DIM, COUNT, true>(tab, itab, geo[ws.p[qp.owner].geom], geo[qp.gj], w, eps,
                                           par_eps, part, pc, &a);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                qp.m[k] = part.f[k].s;
                qp.m[6 + k] = part.f[k].c;
            }
            qp.rc = part.v[0];
            qp.sig2 = part.v[1];
            qp.vim = __float_as_uint(part.v[2]);
            qp.vjm = __float_as_uint(part.v[3]);
            qp.eim = __float_as_uint(part.v[4]);
            qp.ejm = __float_as_uint(part.v[5]);
            qp.fim = __float_as_uint(part.v[6]);
        } else {
            PartSink<T> part;
            part.zero();
            eval_pair<T, DIM, COUNT, false>(tab, itab, geo[ws.p[qp.owner].geom], geo[qp.gj], w, eps,
                                            par_eps, part, pc);
#pragma unroll
            for (int k = 0; k < 12; ++k) qp.m[k] = part.v[k];
            qp.rc = part.v[12];
        }
    }
    __syncwarp();
    for (int e = 0; e < nb; ++e) {
        const QPair<T> &qp = ws.q[(qh + e) & (PQ - 1)];
        if (qp.owner == lane) {
            if constexpr (REF) {
#pragma unroll
                for (int k = 0; k < 6; ++k) S.v[k].merge(qp.m[k], qp.m[6 + k]);
                const float rest[7] = {qp.rc, qp.sig2, __uint_as_float(qp.vim), __uint_as_float(qp.vjm),
                                       __uint_as_float(qp.eim), __uint_as_float(qp.ejm),
                                       __uint_as_float(qp.fim)};
#pragma unroll
                for (int k = 0; k < 7; ++k) S.v[6 + k].add(rest[k]);
            } else {
                T v[13];
#pragma unroll
                for (int k = 0; k < 12; ++k) v[k] = qp.m[k];
                v[12] = qp.rc;
                S.add(v);
            }
        }
    }
    __syncwarp();
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
    tb = (tb + 127) & ~(size_t)127;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    WarpSmem<T> &ws = reinterpret_cast<WarpSmem<T> *>(smem + tb)[w];
    stage_tables<T>(a, tab, geo, itab);
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && !COUNT) {
        a.status->maxdisp2 = 0u;
        a.status->rebuild = 0;
    }
    const T eps = (T)a.eps;
    const T par_eps = (T)a.par_eps;
    const T sig_all = a.sigma > 0.0 ? (T)a.sigma : T(0);
    PathCount pc;
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k) pc.v[k] = 0;
    const int nwarps = gridDim.x * wpb;
    for (int base = (blockIdx.x * wpb + w) * 32; base < a.n; base += nwarps * 32) {
        // ---- this lane's particle ----
        const int i_me = base + lane;
        const bool mine = i_me < a.n;
        M33<T> Rme;
        int nn_me = 0;
        if (mine) {
            const ShapeDev &shi = a.shapes[a.shape[i_me]];
            Rme = orientation<T>(a, i_me);
            PInfo<T> &pi = ws.p[lane];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) pi.r[3 * r + c] = Rme.m[r][c];
            if constexpr (std::is_same<T, float>::value) {
                const float4 dd = a.delta[i_me];
                pi.x[0] = dd.x; pi.x[1] = dd.y; pi.x[2] = dd.z;
                pi.rnd = shi.rounding_f;
            } else {
                const double4_32a xx = a.pos[i_me];
                pi.x[0] = xx.x; pi.x[1] = xx.y; pi.x[2] = xx.z;
                pi.rnd = shi.rounding;
            }
            pi.R = (T)geo[shi.geom].R;
            pi.sig_all = sig_all;
            pi.geom = shi.geom;
            pi.rep = a.rep[i_me];
            pi.sc = a.reps[pi.rep].sc;
            nn_me = a.nn[i_me];
            pi.nn = nn_me;
        }
        SumSink<T, COMP> S;
        S.zero();
        int total;
        ws.offs[lane] = warp_excl_scan(nn_me, lane, &total);
        __syncwarp();
        int qh = 0, qt = 0;
        // ---- scan the list entries of the 32 particles ----
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            bool active = false;
            PairWork<T> wk;
            int pl = 0;
            if (t < total) {
                pl = owner_of(ws.offs, 32, t);
                const int k = t - ws.offs[pl];
                const int i = base + pl;
                const PInfo<T> &pi = ws.p[pl];
                const Geom &gi = geo[pi.geom];
                Owner<T> own;
                own.rp = &a.reps[pi.rep];
                own.sc = pi.sc;
                own.R = pi.R;
                own.rnd = pi.rnd;
                own.sig_all = pi.sig_all;
                own.geom = pi.geom;
                if constexpr (std::is_same<T, float>::value)
                    own.delta = make_float4(pi.x[0], pi.x[1], pi.x[2], 0.f);
                else
                    own.x = make_double4_32a(pi.x[0], pi.x[1], pi.x[2], 0.0);
                const float4 e = a.nlist[(size_t)k * a.n + i];
                bump<COUNT>(&pc, C_NEIGH);
                PairGeom<T> pg;
                int j;
                if (in_range<T>(a, e, own, &j, &pg)) {
                    const Geom &gj = geo[pg.gj];
                    bump<COUNT>(&pc, C_PAIRS);
                    bump<COUNT>(&pc, C_FPE, defined_feature_pairs(DIM, gi, gj));
                    M33<T> Ri;
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) Ri.m[r][c] = pi.r[3 * r + c];
                    wk.M = mul_tn(Ri, orientation_j<T>(a, j, pg));
                    wk.dl = mul_t(Ri, pg.d);
                    wk.rc = (T)WCA_CUT * pg.sig;
                    wk.sig2 = pg.sig * pg.sig;
                    wk.gj = pg.gj;
                    wk.jref = j < i;
                    wk.j = j;
                    active = pair_setup<T, COUNT>(tab, itab, gi, gj, &wk, &pc);
                    if (active) bump<COUNT>(&pc, C_ACTIVE);
                }
            }
            const unsigned m = __ballot_sync(FULL, active);
            if (active) {
                QPair<T> &qp = ws.q[(qt + __popc(m & ((1u << lane) - 1u))) & (PQ - 1)];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) qp.m[4 * r + c] = wk.M.m[r][c];
                }
                qp.m[3] = wk.dl.x; qp.m[7] = wk.dl.y; qp.m[11] = wk.dl.z;
                qp.rc = wk.rc;
                qp.sig2 = wk.sig2;
                qp.gj = wk.gj;
                qp.owner = pl;
                qp.vim = wk.vim; qp.vjm = wk.vjm; qp.eim = wk.eim; qp.ejm = wk.ejm;
                qp.fim = wk.fim; qp.fjm = wk.fjm;
                qp.jref = wk.jref;
                qp.j = wk.j;
            }
            qt += __popc(m);
            __syncwarp();
            if (qt - qh >= 32) {
                run_batch<T, COMP, DIM, COUNT>(ws, qh, 32, lane, tab, itab, geo, eps, par_eps, S, &pc,
                                               a, base);
                qh += 32;
            }
        }
        if (qt > qh)
            run_batch<T, COMP, DIM, COUNT>(ws, qh, qt - qh, lane, tab, itab, geo, eps, par_eps, S, &pc,
                                           a, base);
        if (mine) finish_particle(a, i_me, S, Rme);
        __syncwarp();
    }
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k)
            if (pc.v[k]) atomicAdd(a.counters + k, (unsigned long long)pc.v[k]);
}

// Resident blocks per SM of a kernel (cached per kernel, block and smem size).
template <class T, bool COMP, int DIM>
cudaError_t launch_warp(const PairArgs &a, bool count, size_t smem_tables, cudaStream_t s) {
    const int block = 128;
    size_t smem = ((smem_tables + 127) & ~(size_t)127) + (block / 32) * sizeof(WarpSmem<T>);
    auto launch = [&](auto kernel) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        long long need = (a.n + block - 1) / block;        // 32 particles per warp
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
    if (decomp == DEM_DECOMP_WARP && a.mask_words == 1) {
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
    // the queue-based decompositions carry one-word masks: contexts with
    // larger shapes run THREAD (the context refuses other choices for them)
    if (a.mask_words == 1 && decomp == DEM_DECOMP_STAGED) return launch_pair_staged(a, precision, count, smem, s);
    if (a.mask_words == 1 && decomp == DEM_DECOMP_SPLIT) return launch_pair_split(a, precision, count, smem, s);
    if (block <= 0) block = THREADS;
    if (block > THREADS) block = THREADS;
    switch (precision) {
        case DEM_FP64: return dispatch_dim<double, false>(a, decomp, block, count, smem, s);
        case DEM_FP32: return dispatch_dim<float, false>(a, decomp, block, count, smem, s);
        default: return dispatch_dim<float, true>(a, decomp, block, count, smem, s);
    }
}

}  // namespace dem