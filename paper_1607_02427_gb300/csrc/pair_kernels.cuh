// pair_kernels.cuh -- device pieces shared by the pair-kernel decompositions
// (pair.cu, pair_staged.cu): list-entry range test, pair setup with the
// separating-axis culls, the terms of Eq. DEM / Eq. DEM_2D, per-particle
// outputs, warp scans and occupancy queries.  See pair.cu for the frames,
// the FP32 separation scheme and the list of culls.
#pragma once

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
    float sc;            // FP32 modes: list separation scale (1 unless a barostat moved the box)
    float4 delta;        // FP32 modes
    double4_32a x;       // FP64 mode
    T R, rnd;
    T sig_all;           // the one sigma of all pairs, or 0 (sigma_ij = r_i + r_j)
    int geom;
    const Rep *rp;
};

template <class T> struct PairGeom {
    V3<T> d;             // x_j - x_i (minimum image), world frame
    T sig;               // sigma_ij
    int gj;              // geometry of j
    float4 qj;           // FP32 modes: j's orientation (loaded with its displacement)
};

// Bounding-sphere range test of list entry e of owner o.
template <class T>
__device__ __forceinline__ bool in_range(const PairArgs &a, const float4 &e, const Owner<T> &o,
                                         int *jout, PairGeom<T> *pg) {
    const int j = __float_as_int(e.w);
    *jout = j;
    if constexpr (std::is_same<T, float>::value) {
        // one round of gathers: the displacement (w: shape index) and the
        // orientation, which the pair setup needs when the test passes
        const float4 dj = a.delta[j];
        pg->qj = a.quatf[j];
        const ShapeDev &shj = a.shapes[__float_as_int(dj.w)];
        pg->gj = shj.geom;
        const float dx = fmaf(e.x, o.sc, dj.x - o.delta.x);
        const float dy = fmaf(e.y, o.sc, dj.y - o.delta.y);
        const float dz = fmaf(e.z, o.sc, dj.z - o.delta.z);
        const float sig = o.sig_all > 0.f ? o.sig_all : o.rnd + shj.rounding_f;
        const float lim = o.R + shj.R + (float)WCA_CUT * sig;
        if (!(dx * dx + dy * dy + dz * dz < lim * lim)) return false;
        pg->d = v3<float>(dx, dy, dz);
        pg->sig = sig;
    } else {
        const ShapeDev &shj = a.shapes[__ldg(a.shape + j)];
        pg->gj = shj.geom;
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

// Orientation of the neighbour of an in-range list entry.
template <class T>
__device__ __forceinline__ M33<T> orientation_j(const PairArgs &a, int j, const PairGeom<T> &pg) {
    if constexpr (std::is_same<T, float>::value) return quat_mat<float>(pg.qj.x, pg.qj.y, pg.qj.z, pg.qj.w);
    else return orientation<T>(a, j);
}

// Orientation quaternion (w, x, y, z) of the neighbour of an in-range list
// entry, and the relative quaternion conj(qa) qb (R(conj(qa) qb) = R_a^T R_b).
template <class T>
__device__ __forceinline__ typename R4T<T>::type quat_j(const PairArgs &a, int j,
                                                        const PairGeom<T> &pg) {
    if constexpr (std::is_same<T, float>::value) return pg.qj;
    else return a.quat[j];
}
template <class T, class R4>
__device__ __forceinline__ void relative_quat(const R4 &qa, const R4 &qb, T *q) {
    const T aw = qa.x, ax = -qa.y, ay = -qa.z, az = -qa.w;   // conj(qa)
    const T bw = qb.x, bx = qb.y, by = qb.z, bz = qb.w;
    q[0] = aw * bw - ax * bx - ay * by - az * bz;
    q[1] = aw * bx + ax * bw + ay * bz - az * by;
    q[2] = aw * by - ax * bz + ay * bw + az * bx;
    q[3] = aw * bz + ax * by - ay * bx + az * bw;
}

template <class T>
__device__ __forceinline__ Owner<T> make_owner(const PairArgs &a, int i, const ShapeDev &shi,
                                               const Geom &gi) {
    Owner<T> o;
    o.rp = &a.reps[a.rep[i]];
    o.sc = o.rp->sc;
    o.R = (T)gi.R;
    o.geom = shi.geom;
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

template <class T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return 1.0 / sqrt(x); }

// ---------------------------------------------------------------------------
// Pair setup: separating axis along the centre line and the feature masks
// ---------------------------------------------------------------------------
template <class T> struct PairWork {
    M33<T> M;            // R_i^T R_j
    V3<T> dl;            // x_j - x_i in i's frame
    T q[4];              // STAGED / SPLIT: conj(q_i) q_j, whose rotation matrix is M
    T sig;               // sigma_ij
    T rc, sig2;
    int gj;
    int jref;            // 1 when j < i: j's edge is the parallel-edge rule's reference
    unsigned vim, vjm;   // vertices of i / of j that can reach the other
    unsigned eim, ejm;   // edges
    unsigned fim, fjm;   // faces
};

__device__ __forceinline__ unsigned low_bits(int n) { return n >= 32 ? FULL : ((1u << n) - 1u); }

// Mask of the features (edges or faces) with a vertex in vmask, from the
// per-vertex incidence masks inc.
__device__ __forceinline__ unsigned feature_mask(const int *inc, unsigned vmask) {
    unsigned m = 0;
    for (unsigned v = vmask; v; v &= v - 1u) m |= (unsigned)inc[__ffs(v) - 1];
    return m;
}

// Returns false when the pair is separated along its centre line by at least
// r_cut (all of its terms are zero).
template <class T, bool COUNT>
__device__ __forceinline__ bool pair_setup(const typename R4T<T>::type *tab, const int *itab,
                                           const Geom &gi, const Geom &gj, PairWork<T> *w,
                                           PathCount *pc) {
    w->vim = low_bits(gi.nv);
    w->vjm = low_bits(gj.nv);
    w->eim = low_bits(gi.ne);
    w->ejm = low_bits(gj.ne);
    w->fim = low_bits(gi.nf);
    w->fjm = low_bits(gj.nf);
    const T d2 = dot(w->dl, w->dl);
    if (gi.nv == 1 && gj.nv == 1) return true;           // sphere limit: one term
    if (!(d2 > T(0))) return true;                         // coincident centres
    const T inv = rsqrt_t(d2);
    const T dn = d2 * inv;                                 // |x_ij|
    const V3<T> u = w->dl * inv;                           // i's frame
    const V3<T> uj = mul_t(w->M, u);                       // the same axis in j's frame
    // support of j towards i: max over j's vertices of -(v . uj)
    T hj = T(-3.0e38);
    for (int k = 0; k < gj.nv; ++k) hj = fmax(hj, -dot(xyz<T>(tab[gj.v_off + k]), uj));
    // support of i towards j, and i's vertices that reach j's slab
    const T lo_i = dn - hj - w->rc;
    T hi = T(-3.0e38);
    unsigned vim = 0;
    for (int k = 0; k < gi.nv; ++k) {
        const T p = dot(xyz<T>(tab[gi.v_off + k]), u);
        hi = fmax(hi, p);
        if (p > lo_i) vim |= 1u << k;
    }
    bump<COUNT>(pc, C_PROJ, (unsigned)(gi.nv + 2 * gj.nv));
    if (!(dn - hi - hj < w->rc)) return false;
    const T hi_j = hi + w->rc - dn;                        // j's vertices: v . uj < hi_j
    unsigned vjm = 0;
    for (int k = 0; k < gj.nv; ++k)
        if (dot(xyz<T>(tab[gj.v_off + k]), uj) < hi_j) vjm |= 1u << k;
    w->vim = vim;
    w->vjm = vjm;
    w->eim = feature_mask(itab + gi.vem_off, vim);
    w->ejm = feature_mask(itab + gj.vem_off, vjm);
    w->fim = feature_mask(itab + gi.vfm_off, vim);
    w->fjm = feature_mask(itab + gj.vfm_off, vjm);
    return true;
}

// The 13 values of one term: force f and torque pi x f in i's frame, half
// the energy, the body-frame virial 1/2 sym((-dl) (x) f).
template <class T>
__device__ __forceinline__ void term_values(V3<T> pi, V3<T> f, V3<T> dl, T U, T *v) {
    const V3<T> tq = cross(pi, f);
    v[0] = f.x; v[1] = f.y; v[2] = f.z;
    v[3] = tq.x; v[4] = tq.y; v[5] = tq.z;
    v[6] = T(0.5) * U;
    const T x = -dl.x, y = -dl.y, z = -dl.z;
    v[7] = T(0.5) * x * f.x;
    v[8] = T(0.25) * (x * f.y + y * f.x);
    v[9] = T(0.25) * (x * f.z + z * f.x);
    v[10] = T(0.5) * y * f.y;
    v[11] = T(0.25) * (y * f.z + z * f.y);
    v[12] = T(0.5) * z * f.z;
}

// Sinks of the terms: the particle's compensated sums, or a pair's partial.
template <class T, bool COMP> struct SumSink {
    Acc<T, COMP> v[13];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 13; ++k) v[k].zero();
    }
    __device__ __forceinline__ void add(const T *x) {
#pragma unroll
        for (int k = 0; k < 13; ++k) v[k].add(x[k]);
    }
    __device__ __forceinline__ T total(int k) const { return v[k].s + v[k].comp(); }
};
template <class T> struct PartSink {
    T v[13];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 13; ++k) v[k] = T(0);
    }
    __device__ __forceinline__ void add(const T *x) {
#pragma unroll
        for (int k = 0; k < 13; ++k) v[k] += x[k];
    }
};

// All terms of an active pair (Eq. DEM / Eq. DEM_2D restricted to the
// masked features, which carry every non-zero term), in i's frame.
template <class T, int DIM, bool COUNT, class Sink>
__device__ __forceinline__ void eval_pair(const typename R4T<T>::type *tab, const int *itab,
                                          const Geom &gi, const Geom &gj, const PairWork<T> &w,
                                          T eps, T par_eps, Sink &sink, PathCount *pc) {
    using R4 = typename R4T<T>::type;
    const T rc = w.rc, rc2 = rc * rc;
    const V3<T> dl = w.dl;
    T U, wf, tv[13];
    if (gi.nv == 1 && gj.nv == 1) {             // sphere / disk limit: central WCA
        const V3<T> pi = xyz<T>(tab[gi.v_off]);
        const V3<T> rv = pi - (dl + mul(w.M, xyz<T>(tab[gj.v_off])));
        const T r2 = dot(rv, rv);
        if (r2 < rc2) {
            wf = wca_factor(r2, w.sig2, eps, &U);
            term_values(pi, rv * wf, dl, U, tv);
            sink.add(tv);
            bump<COUNT>(pc, C_TERMS);
        }
        return;
    }
    const T reach_i = T(gi.R) + rc, reach_j = T(gj.R) + rc;
    // vertex of j against the faces (2D: edges) of i, in i's frame
    for (unsigned mb = w.vjm; mb; mb &= mb - 1u) {
        const int b = __ffs(mb) - 1;
        const V3<T> p = dl + mul(w.M, xyz<T>(tab[gj.v_off + b]));
        bump<COUNT>(pc, C_VTX);
        if (!(dot(p, p) < reach_i * reach_i)) continue;
        if constexpr (DIM == 3) {
            for (unsigned mf = w.fim; mf; mf &= mf - 1u) {
                const int f = __ffs(mf) - 1;
                V3<T> q;
                T r2;
                if (!face_nearest<T, COUNT>(tab, itab, gi.f_off + f, gi.fi_off + 2 * f, p, rc, &q, &r2, pc))
                    continue;
                if (r2 < rc2) {
                    wf = wca_factor(r2, w.sig2, eps, &U);
                    term_values(q, (q - p) * wf, dl, U, tv);
                    sink.add(tv);
                    bump<COUNT>(pc, C_TERMS);
                }
            }
        } else {
            for (unsigned me = w.eim; me; me &= me - 1u) {
                const int e = __ffs(me) - 1;
                const R4 ea = tab[gi.e_off + 2 * e], ed = tab[gi.e_off + 2 * e + 1];
                const V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                const V3<T> c = A + D * T(0.5) - p;
                const T lim = ea.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(c, c) < lim * lim)) continue;
                bump<COUNT>(pc, C_PTSEG);
                const V3<T> q = A + D * clamp01(dot(p - A, D) * ed.w);
                const V3<T> rv = q - p;
                const T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    wf = wca_factor(r2, w.sig2, eps, &U);
                    term_values(q, rv * wf, dl, U, tv);
                    sink.add(tv);
                    bump<COUNT>(pc, C_TERMS);
                }
            }
        }
    }
    // vertex of i against the faces (2D: edges) of j, in j's frame
    for (unsigned ma = w.vim; ma; ma &= ma - 1u) {
        const int ai = __ffs(ma) - 1;
        const V3<T> u = xyz<T>(tab[gi.v_off + ai]);
        const V3<T> p = mul_t(w.M, u - dl);
        bump<COUNT>(pc, C_VTX);
        if (!(dot(p, p) < reach_j * reach_j)) continue;
        if constexpr (DIM == 3) {
            for (unsigned mf = w.fjm; mf; mf &= mf - 1u) {
                const int f = __ffs(mf) - 1;
                V3<T> q;
                T r2;
                if (!face_nearest<T, COUNT>(tab, itab, gj.f_off + f, gj.fi_off + 2 * f, p, rc, &q, &r2, pc))
                    continue;
                if (r2 < rc2) {
                    wf = wca_factor(r2, w.sig2, eps, &U);
                    term_values(u, mul(w.M, (p - q) * wf), dl, U, tv);
                    sink.add(tv);
                    bump<COUNT>(pc, C_TERMS);
                    bump<COUNT>(pc, C_JTERMS);
                }
            }
        } else {
            for (unsigned me = w.ejm; me; me &= me - 1u) {
                const int e = __ffs(me) - 1;
                const R4 ea = tab[gj.e_off + 2 * e], ed = tab[gj.e_off + 2 * e + 1];
                const V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                const V3<T> c = A + D * T(0.5) - p;
                const T lim = ea.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(c, c) < lim * lim)) continue;
                bump<COUNT>(pc, C_PTSEG);
                const V3<T> q = A + D * clamp01(dot(p - A, D) * ed.w);
                const V3<T> rv = p - q;
                const T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    wf = wca_factor(r2, w.sig2, eps, &U);
                    term_values(u, mul(w.M, rv * wf), dl, U, tv);
                    sink.add(tv);
                    bump<COUNT>(pc, C_TERMS);
                    bump<COUNT>(pc, C_JTERMS);
                }
            }
        }
    }
    if constexpr (DIM == 3) {
        // edges of j against the edges of i, in i's frame
        const unsigned eim = w.eim;
        for (unsigned mb = eim ? w.ejm : 0u; mb; mb &= mb - 1u) {
            const int eb = __ffs(mb) - 1;
            const R4 ba = tab[gj.e_off + 2 * eb], bd = tab[gj.e_off + 2 * eb + 1];
            const V3<T> A2 = dl + mul(w.M, xyz<T>(ba));
            const V3<T> D2 = mul(w.M, xyz<T>(bd));
            const V3<T> C2 = A2 + D2 * T(0.5);
            const T reach = reach_i + ba.w;
            bump<COUNT>(pc, C_EDGE);
            if (!(dot(C2, C2) < reach * reach)) continue;
            for (unsigned ma = eim; ma; ma &= ma - 1u) {
                const int ea = __ffs(ma) - 1;
                const R4 aa = tab[gi.e_off + 2 * ea], ad = tab[gi.e_off + 2 * ea + 1];
                const V3<T> A1 = xyz<T>(aa), D1 = xyz<T>(ad);
                const V3<T> dc = A1 + D1 * T(0.5) - C2;
                const T lim = aa.w + ba.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(dc, dc) < lim * lim)) continue;
                // carrier lines farther apart than r_cut: the segments are too
                const V3<T> nrm = cross(D1, D2);
                const T n2 = dot(nrm, nrm);
                const T sep = dot(A2 - A1, nrm);
                bump<COUNT>(pc, C_LINE);
                if (sep * sep >= rc2 * n2 && n2 > par_eps * dot(D1, D1) * dot(D2, D2)) continue;
                bump<COUNT>(pc, C_SEGSEG);
                V3<T> P1, P2;
                segment_nearest<T>(A1, D1, ad.w, A2, D2, bd.w, par_eps, w.jref != 0, &P1, &P2);
                const V3<T> rv = P1 - P2;
                const T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    wf = wca_factor(r2, w.sig2, eps, &U);
                    term_values(P1, rv * wf, dl, U, tv);
                    sink.add(tv);
                    bump<COUNT>(pc, C_TERMS);
                }
            }
        }
    }
}

// Number of feature pairs Eq. DEM / Eq. DEM_2D assigns to a pair.
__device__ __forceinline__ unsigned defined_feature_pairs(int dim, const Geom &gi, const Geom &gj) {
    if (gi.nv == 1 && gj.nv == 1) return 1u;
    if (dim == 2) return (unsigned)(gi.nv * gj.ne + gj.nv * gi.ne);
    return (unsigned)(gi.ne * gj.ne + gi.nv * gj.nf + gj.nv * gi.nf);
}

// World-frame outputs of particle i from its body-frame totals:
// out = {F (rotated), tau (body), U, W (R W R^T)}.
template <class T>
__device__ __forceinline__ void world_outputs(const T *tot, const M33<T> &R, T *out) {
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
    out[7] = RB[0][0] * R.m[0][0] + RB[0][1] * R.m[0][1] + RB[0][2] * R.m[0][2];
    out[8] = RB[0][0] * R.m[1][0] + RB[0][1] * R.m[1][1] + RB[0][2] * R.m[1][2];
    out[9] = RB[0][0] * R.m[2][0] + RB[0][1] * R.m[2][1] + RB[0][2] * R.m[2][2];
    out[10] = RB[1][0] * R.m[1][0] + RB[1][1] * R.m[1][1] + RB[1][2] * R.m[1][2];
    out[11] = RB[1][0] * R.m[2][0] + RB[1][1] * R.m[2][1] + RB[1][2] * R.m[2][2];
    out[12] = RB[2][0] * R.m[2][0] + RB[2][1] * R.m[2][1] + RB[2][2] * R.m[2][2];
}

__device__ __forceinline__ void store_outputs(const PairArgs &a, int i, const double *v) {
    double *f = reinterpret_cast<double *>(a.force + i);
    double *t = reinterpret_cast<double *>(a.torque + i);
    f[0] = v[0]; f[1] = v[1]; f[2] = v[2];
    t[0] = v[3]; t[1] = v[4]; t[2] = v[5];
    a.energy[i] = v[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) a.virial[6 * (size_t)i + k] = v[7 + k];
    double chk = 0.0;
#pragma unroll
    for (int k = 0; k < 13; ++k) chk += v[k];
    if (!isfinite(chk)) atomicExch(&a.status->nonfinite, 1);
}

template <class T, bool COMP>
__device__ __forceinline__ void finish_particle(const PairArgs &a, int i, const SumSink<T, COMP> &S,
                                                const M33<T> &R) {
    T tot[13], out[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) tot[k] = S.total(k);
    world_outputs(tot, R, out);
    double v[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) v[k] = (double)out[k];
    store_outputs(a, i, v);
}


// Items t0 .. t0+31 of consecutive ranges [off_p, off_p + c_p), range p held
// by lane p: the range of item t0 + lane, for all lanes at once.  Each range
// with items in the round marks the lane of its first one there (who: 32
// ints of the warp's shared memory); a lane's range is the last mark at or
// below it.  Warp-collective; lanes past the last item get an arbitrary range.
__device__ __forceinline__ int round_owner(int off_me, int c_me, int t0, int lane, int *who) {
    const int s = off_me - t0, e = s + c_me;
    unsigned bit = 0u;
    if (c_me > 0 && e > 0 && s < 32) {
        const int b = s > 0 ? s : 0;
        who[b] = lane;
        bit = 1u << b;
    }
    const unsigned starts = __reduce_or_sync(FULL, bit);
    __syncwarp();
    const unsigned upto = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;
    const unsigned m = starts & upto;
    const int own = m ? who[31 - __clz(m)] : 0;
    __syncwarp();
    return own;
}

__device__ __forceinline__ int owner_of(const int *off, int n, int t) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

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

// Evaluate queued pairs [qh, qh + nb) (one per lane), then let each owner

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


}  // namespace
}  // namespace dem
