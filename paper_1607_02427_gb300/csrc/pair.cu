// pair.cu -- pair feature kernels: force, torque, energy and virial of every
// particle from all feature pairs with its neighbours (Eq. DEM in 3D,
// Eq. DEM_2D in 2D, WCA of Eq. LJ / Eq. WCA), Section "Algorithm" of
// arXiv:1607.02427 re-designed for sm_103a.
//
// Work decomposition (owner computes over a full neighbour list; only
// particle i's sums are written, so no atomics and a fixed summation order):
//   THREAD  one thread per particle i walks its neighbours j.
//   WARP    one warp per particle i; lane l takes neighbours l, l+32, ...
//           for the per-pair setup, then the warp shares the (neighbour,
//           outer feature) work items; warp-shuffle sums at the end.
//   TILED   one warp per particle i; for each neighbour j the lanes take the
//           features of i and j as in the paper's thread decomposition
//           (vertex threads and edge threads), then shuffle-sum.
//
// Exact culls (each skips only terms that are zero because r* >= r_cut):
//   pair:    |x_ij| >= R_i + R_j + r_cut         (all features lie within R)
//   vertex:  |p - x_owner| >= R_owner + r_cut    (p cannot reach any face)
//   edge:    |c_e - x_i| >= R_i + h_e + r_cut    (the edge cannot reach i)
//   face:    |signed plane distance| >= r_cut
//   edges:   |c_1 - c_2| >= h_1 + h_2 + r_cut    (edge bounding spheres)
#include "pair_common.cuh"

namespace dem {
namespace {

constexpr double WCA_CUT = 1.122462048309373;   // 2^(1/6)

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

struct PairGeom {
    double dx, dy, dz;   // d = x_j - x_i (minimum image, FP64)
    int gj;              // geometry of j
    float Rj;
    double sig;          // sigma_ij
};

// Minimum-image separation and the bounding-sphere test of pair (i, j).
__device__ __forceinline__ bool pair_in_range(const PairArgs &a, int j, double4_32a xi, float Ri,
                                              double rnd_i, const Rep &rp, PairGeom *pg) {
    double4_32a xj = a.pos[j];
    double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    dx -= rp.L[0] * rint(dx / rp.L[0]);
    dy -= rp.L[1] * rint(dy / rp.L[1]);
    if (a.dim == 3) dz -= rp.L[2] * rint(dz / rp.L[2]); else dz = 0.0;
    int sj = __ldg(a.shape + j);
    const ShapeDev &shj = a.shapes[sj];
    double sig = a.sigma > 0.0 ? a.sigma : rnd_i + shj.rounding;
    double rc = WCA_CUT * sig;
    double lim = (double)Ri + (double)shj.R + rc;
    if (!(dx * dx + dy * dy + dz * dz < lim * lim)) return false;
    pg->dx = dx; pg->dy = dy; pg->dz = dz;
    pg->gj = shj.geom;
    pg->Rj = shj.R;
    pg->sig = sig;
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
    if (gi.nv == 1 && gj.nv == 1) {             // sphere / disk limit: central WCA
        V3<T> pi = xyz<T>(tab[gi.v_off]);
        V3<T> pj = dl + mul(M, xyz<T>(tab[gj.v_off]));
        V3<T> rv = pi - pj;
        T r2 = dot(rv, rv);
        if (r2 < rc2) wca_term(S, pi, rv, r2, sig2, eps);
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
                T t = clamp01(dot(p - A, D) * ed.w);
                V3<T> q = A + D * t;
                V3<T> rv = q - p;
                T r2 = dot(rv, rv);
                if (r2 < rc2) wca_term(S, q, rv, r2, sig2, eps);
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
                T t = clamp01(dot(p - A, D) * ed.w);
                V3<T> q = A + D * t;
                V3<T> rv = p - q;
                T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    bump<COUNT>(pc, C_JTERMS);
                    wca_term_jframe(S, M, u, rv, r2, sig2, eps);
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
            if (r2 < rc2) wca_term(S, q, q - p, r2, sig2, eps);
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
                wca_term_jframe(S, M, u, p - q, r2, sig2, eps);
            }
        }
    }
    // E_i x E_j (Eq. DEM, first sum), in i's frame
    for (int eb = 0; eb < gj.ne; ++eb) {
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
            if (r2 < rc2) wca_term(S, P1, rv, r2, sig2, eps);
        }
    }
    return (unsigned)(gi.ne * gj.ne + gi.nv * gj.nf + gj.nv * gi.nf);
    }
}

// Write particle i's results: force rotated to the world frame (FP64),
// torque in i's body frame, energy, virial; flag non-finite values.
template <class T, bool COMP>
__device__ __forceinline__ void store_particle(const PairArgs &a, int i, Sums<T, COMP> &S,
                                               const double *W) {
    double4_32a q = a.quat[i];
    M33<double> R = quat_mat<double>(q.x, q.y, q.z, q.w);
    V3<double> fb = v3<double>(S.f[0].get(), S.f[1].get(), S.f[2].get());
    V3<double> fw = mul(R, fb);
    double tx = S.t[0].get(), ty = S.t[1].get(), tz = S.t[2].get();
    a.force[i] = make_double4_32a(fw.x, fw.y, fw.z, 0.0);
    a.torque[i] = make_double4_32a(tx, ty, tz, 0.0);
    a.energy[i] = S.u;
#pragma unroll
    for (int k = 0; k < 6; ++k) a.virial[6 * i + k] = W[k];
    double chk = fw.x + fw.y + fw.z + tx + ty + tz + S.u;
    if (!isfinite(chk)) atomicExch(&a.status->nonfinite, 1);
}

// Virial of one ordered pair: W_i += 1/2 sym(x_ij (x) f), x_ij = -d, f = R_i f_pair.
template <class T, bool COMP>
__device__ __forceinline__ void pair_virial(const M33<double> &Rd, const PairGeom &pg,
                                            const Sums<T, COMP> &S, double *W) {
    V3<double> f = mul(Rd, v3<double>((double)S.fp.x, (double)S.fp.y, (double)S.fp.z));
    double x = -pg.dx, y = -pg.dy, z = -pg.dz;
    W[0] += 0.5 * x * f.x;
    W[1] += 0.25 * (x * f.y + y * f.x);
    W[2] += 0.25 * (x * f.z + z * f.x);
    W[3] += 0.5 * y * f.y;
    W[4] += 0.25 * (y * f.z + z * f.y);
    W[5] += 0.5 * z * f.z;
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
        const int si = a.shape[i];
        const ShapeDev &shi = a.shapes[si];
        const Geom gi = geo[shi.geom];
        const double rnd_i = shi.rounding;
        const Rep &rp = a.reps[a.rep[i]];
        const double4_32a xi = a.pos[i];
        const M33<T> Ri = orientation<T>(a, i);
        double4_32a qd = a.quat[i];
        const M33<double> Rd = quat_mat<double>(qd.x, qd.y, qd.z, qd.w);
        Sums<T, COMP> S;
        S.zero();
        double W[6] = {0, 0, 0, 0, 0, 0};
        const int nn = a.nn[i];
        for (int k = 0; k < nn; ++k) {
            const int j = a.nlist[(size_t)k * a.n + i];
            PairGeom pg;
            bump<COUNT>(&pc, C_NEIGH);
            if (!pair_in_range(a, j, xi, gi.R, rnd_i, rp, &pg)) continue;
            const M33<T> Rj = orientation<T>(a, j);
            const M33<T> M = mul_tn(Ri, Rj);
            const V3<T> dl = mul_t(Ri, v3<T>((T)pg.dx, (T)pg.dy, (T)pg.dz));
            const T sig = (T)pg.sig;
            const T rc = (T)(WCA_CUT * pg.sig);
            S.fp = v3<T>(T(0), T(0), T(0));
            unsigned before = S.nterm;
            unsigned nf = pair_terms<T, COMP, DIM, COUNT>(tab, itab, gi, geo[pg.gj], M, dl, rc,
                                                          sig * sig, eps, par_eps, S, &pc);
            if (S.nterm != before) pair_virial(Rd, pg, S, W);
            bump<COUNT>(&pc, C_PAIRS);
            bump<COUNT>(&pc, C_FPE, nf);
        }
        bump<COUNT>(&pc, C_TERMS, S.nterm);
        store_particle(a, i, S, W);
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

template <class T, bool COMP>
cudaError_t dispatch_dim(const PairArgs &a, int decomp, int block, bool count, size_t smem,
                         cudaStream_t s) {
    (void)decomp;
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
