// pair_kernels.cuh -- device pieces shared by the pair-kernel decompositions
// (pair.cu, pair_staged.cu): list-entry range test, pair setup with the
// separating-axis culls, the terms of Eq. DEM / Eq. DEM_2D, per-particle
// outputs, warp scans and occupancy queries.  See pair.cu for the frames,
// the FP32 separation scheme and the list of culls.
#pragma once

#include <type_traits>

#include "ff.cuh"
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
// ---------------------------------------------------------------------------
// Feature masks.  Shapes with at most 32 vertices, edges and faces use one
// 32-bit word per mask (every decomposition).  Larger shapes (up to 128 of
// each) use a two-level mask of four words: the culls and loops skip the
// empty words, then walk the set bits of the others (THREAD decomposition).
// The incidence rows of the geometry table (the edges / faces of each vertex)
// have one word per mask word.
// ---------------------------------------------------------------------------
template <int W> struct WideMask {
    unsigned w[W];
};
template <class MK> struct MaskWords;
template <> struct MaskWords<unsigned> { static constexpr int value = 1; };
template <int W> struct MaskWords<WideMask<W>> { static constexpr int value = W; };

__device__ __forceinline__ unsigned low_bits(int n) { return n >= 32 ? FULL : ((1u << n) - 1u); }
__device__ __forceinline__ void mask_low(unsigned *m, int n) { *m = low_bits(n); }
template <int W> __device__ __forceinline__ void mask_low(WideMask<W> *m, int n) {
#pragma unroll
    for (int k = 0; k < W; ++k) m->w[k] = n >= 32 * (k + 1) ? FULL : (n > 32 * k ? low_bits(n - 32 * k) : 0u);
}
__device__ __forceinline__ void mask_zero(unsigned *m) { *m = 0u; }
template <int W> __device__ __forceinline__ void mask_zero(WideMask<W> *m) {
#pragma unroll
    for (int k = 0; k < W; ++k) m->w[k] = 0u;
}
__device__ __forceinline__ void mask_set(unsigned *m, int b) { *m |= 1u << b; }
template <int W> __device__ __forceinline__ void mask_set(WideMask<W> *m, int b) {
    m->w[b >> 5] |= 1u << (b & 31);
}
__device__ __forceinline__ bool mask_any(unsigned m) { return m != 0u; }
template <int W> __device__ __forceinline__ bool mask_any(const WideMask<W> &m) {
    unsigned a = 0u;
#pragma unroll
    for (int k = 0; k < W; ++k) a |= m.w[k];
    return a != 0u;
}
// f(b) for every set bit b, in increasing order
template <class F> __device__ __forceinline__ void for_each_bit(unsigned m, F f) {
    for (; m; m &= m - 1u) f(__ffs(m) - 1);
}
template <int W, class F> __device__ __forceinline__ void for_each_bit(const WideMask<W> &m, F f) {
    for (int k = 0; k < W; ++k)
        for (unsigned b = m.w[k]; b; b &= b - 1u) f(32 * k + __ffs(b) - 1);
}

template <class T, class MK = unsigned> struct PairWork {
    M33<T> M;            // R_i^T R_j
    V3<T> dl;            // x_j - x_i in i's frame
    int i, j;            // the particles (FP32 + two-sum refinement)
    T q[4];              // STAGED / SPLIT: conj(q_i) q_j, whose rotation matrix is M
    T sig;               // sigma_ij
    T rc, sig2;
    int gj;
    int jref;            // 1 when j < i: j's edge is the parallel-edge rule's reference
    MK vim, vjm;         // vertices of i / of j that can reach the other
    MK eim, ejm;         // edges
    MK fim, fjm;         // faces
};

// Mask of the features (edges or faces) with a vertex in vmask, from the
// per-vertex incidence masks inc (one row of mask words per vertex).
__device__ __forceinline__ unsigned feature_mask(const int *inc, unsigned vmask) {
    unsigned m = 0;
    for (unsigned v = vmask; v; v &= v - 1u) m |= (unsigned)inc[__ffs(v) - 1];
    return m;
}
template <int W>
__device__ __forceinline__ WideMask<W> feature_mask(const int *inc, const WideMask<W> &vmask) {
    WideMask<W> m;
    mask_zero(&m);
    for_each_bit(vmask, [&](int v) {
#pragma unroll
        for (int k = 0; k < W; ++k) m.w[k] |= (unsigned)inc[W * v + k];
    });
    return m;
}

// Returns false when the pair is separated along its centre line by at least
// r_cut (all of its terms are zero).
template <class T, bool COUNT, class MK>
__device__ __forceinline__ bool pair_setup(const typename R4T<T>::type *tab, const int *itab,
                                           const Geom &gi, const Geom &gj, PairWork<T, MK> *w,
                                           PathCount *pc) {
    mask_low(&w->vim, gi.nv);
    mask_low(&w->vjm, gj.nv);
    mask_low(&w->eim, gi.ne);
    mask_low(&w->ejm, gj.ne);
    mask_low(&w->fim, gi.nf);
    mask_low(&w->fjm, gj.nf);
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
    MK vim;
    mask_zero(&vim);
    for (int k = 0; k < gi.nv; ++k) {
        const T p = dot(xyz<T>(tab[gi.v_off + k]), u);
        hi = fmax(hi, p);
        if (p > lo_i) mask_set(&vim, k);
    }
    bump<COUNT>(pc, C_PROJ, (unsigned)(gi.nv + 2 * gj.nv));
    if (!(dn - hi - hj < w->rc)) return false;
    const T hi_j = hi + w->rc - dn;                        // j's vertices: v . uj < hi_j
    MK vjm;
    mask_zero(&vjm);
    for (int k = 0; k < gj.nv; ++k)
        if (dot(xyz<T>(tab[gj.v_off + k]), uj) < hi_j) mask_set(&vjm, k);
    w->vim = vim;
    w->vjm = vjm;
    w->eim = feature_mask(itab + gi.vem_off, vim);
    w->ejm = feature_mask(itab + gj.vem_off, vjm);
    w->fim = feature_mask(itab + gi.vfm_off, vim);
    w->fjm = feature_mask(itab + gj.vfm_off, vjm);
    return true;
}

// ---------------------------------------------------------------------------
// FP32 + two-sum mode: each term with r < r_cut re-evaluated in float-float
// ---------------------------------------------------------------------------
// The search found the term's features and, in FP32, the parameters of its
// nearest points.  The refinement rebuilds both nearest points in i's body
// frame from the FP64 state split into hi + lo floats (ff.cuh): j's points
// are mapped with the quaternions of both particles and the minimum-image
// separation, x_i + R_i p_i = x_j + R_j p_j taken in float-float.  The
// search's parameters decide only the branch: a parameter it clamped to an
// end of its segment is exact, an interior one is recomputed in float-float
// as the search defined it (the foot of a perpendicular, the stationary
// point of an edge pair, the midpoint of the parallel-edge rule's overlap).
// The distance is stationary in those parameters, but the lever arm of the
// torque is not: its error would be first order in them.
enum TermKind {
    TK_SPH = 0,    // one-vertex shapes: the centres' vertices
    TK_VF_I = 1,   // vertex b of j against face a of i
    TK_VF_J = 2,   // vertex a of i against face b of j
    TK_EE = 3,     // edge a of i at s against edge b of j at t
    TK_VE_I = 4,   // 2D: vertex b of j against edge a of i at t
    TK_VE_J = 5    // 2D: vertex a of i against edge b of j at t
};
struct TermSpec {
    int kind, a, b;
    FaceHit hit;       // vertex-face terms: inside the face, or face edge k at t;
                       // edge pairs: hit.inside = 1 when the parallel-edge rule applied
    float s, t;
    int jref;          // j's edge is the rule's reference (j < i)
};

struct FFPair {
    ff qiw, qjw;       // quaternions (w, u) of i and j
    ff3 qiu, qju;
    ff3 d;             // x_j - x_i (minimum image), world frame
    ff sig2;           // sigma_ij^2
};

__device__ __forceinline__ ff min_image_ff(ff x, float L, float L_lo) {
    const float n = rintf(__fdiv_rn(x.h, L));
    return n != 0.f ? ff_sub(x, ff_mul_f(ff{L, L_lo}, n)) : x;
}

__device__ __forceinline__ FFPair load_ffpair(const PairArgs &a, int i, int j) {
    FFPair p;
    const float4 qih = a.quatf[i], qil = a.quatf_lo[i], qjh = a.quatf[j], qjl = a.quatf_lo[j];
    p.qiw = {qih.x, qil.x};
    p.qiu = {{qih.y, qil.y}, {qih.z, qil.z}, {qih.w, qil.w}};
    p.qjw = {qjh.x, qjl.x};
    p.qju = {{qjh.y, qjl.y}, {qjh.z, qjl.z}, {qjh.w, qjl.w}};
    ff3 d = ff3_of(a.xff[2 * j], a.xff[2 * j + 1]) - ff3_of(a.xff[2 * i], a.xff[2 * i + 1]);
    const Rep &rp = a.reps[a.rep[i]];
    // the image is decided on the hi part: the pair is within its range,
    // well inside half a box, so the choice is never close
    p.d.x = min_image_ff(d.x, rp.Lf[0], rp.Lf_lo[0]);
    p.d.y = min_image_ff(d.y, rp.Lf[1], rp.Lf_lo[1]);
    p.d.z = a.dim == 3 ? min_image_ff(d.z, rp.Lf[2], rp.Lf_lo[2]) : d.z;
    ff sig;
    if (a.sigma > 0.0) {
        sig = {a.sigma_f, a.sigma_lo};
    } else {
        const ShapeDev &si = a.shapes[a.shape[i]], &sj = a.shapes[a.shape[j]];
        sig = ff_add({si.rounding_f, si.rounding_lo}, {sj.rounding_f, sj.rounding_lo});
    }
    p.sig2 = ff_mul(sig, sig);
    return p;
}

// Geometry records as hi (shared-memory table) + lo (device table)
struct FFTab {
    const float4 *tab, *lo;
    const int *itab;
    __device__ __forceinline__ ff3 rec(int k) const { return ff3_of(tab[k], lo[k]); }
    __device__ __forceinline__ ff recw(int k) const { return {tab[k].w, lo[k].w}; }
    __device__ __forceinline__ ff3 vertex(const Geom &g, int v) const { return rec(g.v_off + v); }
    // edge e: start A, direction D, 1/|D|^2
    __device__ __forceinline__ void edge(const Geom &g, int e, ff3 *A, ff3 *D, ff *inv) const {
        *A = rec(g.e_off + 2 * e);
        *D = rec(g.e_off + 2 * e + 1);
        *inv = recw(g.e_off + 2 * e + 1);
    }
    // edge k of face f: start A, direction E, 1/|E|^2
    __device__ __forceinline__ void face_edge(const Geom &g, int f, int k, ff3 *A, ff3 *E,
                                              ff *inv) const {
        const int fe = itab[g.fi_off + 2 * f];
        *A = rec(fe + 3 * k);
        *E = rec(fe + 3 * k + 1);
        *inv = recw(fe + 3 * k + 1);
    }
    // signed distance of p from face f's plane
    __device__ __forceinline__ ff plane(const Geom &g, int f, ff3 p, ff3 *n) const {
        const int k = g.f_off + f;
        *n = rec(k);
        return ff_sub(ff3_dot(*n, p), recw(k));
    }
};

// j's body point in i's frame, i's body point in j's frame, and j's body
// directions in i's frame
__device__ __forceinline__ ff3 to_i(const FFPair &p, ff3 Pj) {
    return ff3_rotate(p.qiw, p.qiu, p.d + ff3_rotate(p.qjw, p.qju, Pj, false), true);
}
__device__ __forceinline__ ff3 to_j(const FFPair &p, ff3 Pi) {
    return ff3_rotate(p.qjw, p.qju, ff3_rotate(p.qiw, p.qiu, Pi, false) - p.d, true);
}
__device__ __forceinline__ ff3 dir_to_i(const FFPair &p, ff3 v) {
    return ff3_rotate(p.qiw, p.qiu, ff3_rotate(p.qjw, p.qju, v, false), true);
}

// Parameter of the foot of P on A + u D (inv = 1/|D|^2) in [0, 1]: the
// search's u is kept when it clamped (an end of the segment), else recomputed.
__device__ __forceinline__ ff foot(ff3 P, ff3 A, ff3 D, ff inv, float u) {
    if (!(u > 0.f && u < 1.f)) return ff_of(u);
    return ff_clamp01(ff_mul(ff3_dot(P - A, D), inv));
}

// Nearest points of i's edge A1 + s D1 and j's edge A2 + t D2 (both in i's
// frame) as segment_nearest defines them, with the search's branch.
__device__ __forceinline__ void refine_edges(ff3 A1, ff3 D1, ff ia, ff3 A2, ff3 D2, ff ic,
                                             const TermSpec &sp, ff *s, ff *t) {
    const ff3 W = A1 - A2;
    const ff b = ff3_dot(D1, D2), d = ff3_dot(D1, W), e = ff3_dot(D2, W);
    if (sp.hit.inside) {           // the parallel-edge rule: midpoint of the overlap
        ff t0, t1;
        if (sp.jref) {
            t0 = ff_mul(e, ic);
            t1 = ff_mul(ff_add(e, b), ic);
        } else {
            t0 = ff_mul(ff_neg(d), ia);
            t1 = ff_mul(ff_sub(b, d), ia);
        }
        const ff lo = ff_max(ff_of(0.f), ff_min(t0, t1)), hi = ff_min(ff_of(1.f), ff_max(t0, t1));
        if (!ff_lt(hi, lo)) {
            const ff mid = ff_scale2(ff_add(lo, hi), 0.5f);
            if (sp.jref) {
                *t = mid;
                *s = ff_clamp01(ff_mul(ff_sub(ff_mul(mid, b), d), ia));
            } else {
                *s = mid;
                *t = ff_clamp01(ff_mul(ff_add(e, ff_mul(mid, b)), ic));
            }
            return;
        }
        // no overlap: an endpoint pair, below
    }
    const bool s_in = sp.s > 0.f && sp.s < 1.f, t_in = sp.t > 0.f && sp.t < 1.f;
    if (s_in && t_in) {            // the stationary point of the quadratic
        const ff a = ff3_dot(D1, D1), c = ff3_dot(D2, D2);
        const ff den = ff_sub(ff_mul(a, c), ff_mul(b, b));
        *s = ff_div(ff_sub(ff_mul(b, e), ff_mul(c, d)), den);
        *t = ff_div(ff_sub(ff_mul(a, e), ff_mul(b, d)), den);
    } else if (s_in) {             // t at an end: the optimal s for it
        *t = ff_of(sp.t);
        *s = ff_clamp01(ff_mul(ff_sub(ff_mul(*t, b), d), ia));
    } else if (t_in) {             // s at an end: the optimal t for it
        *s = ff_of(sp.s);
        *t = ff_clamp01(ff_mul(ff_add(e, ff_mul(*s, b)), ic));
    } else {
        *s = ff_of(sp.s);
        *t = ff_of(sp.t);
    }
}

// The term's nearest points in i's frame: rv = p_i - p_j and the lever arm
// p_i (i's point relative to its centre).  Every kind maps one point and one
// direction of j's feature into i's frame (the costly part: four float-float
// rotations, the same instructions for every lane of a warp); the kind
// decides only which records are read and how the nearest points follow.
__device__ __forceinline__ void refine_points(const FFTab &T, const Geom &gi, const Geom &gj,
                                              const FFPair &p, const TermSpec &sp, ff3 *rv,
                                              ff3 *arm) {
    const ff3 zero = ff3_of(0.f, 0.f, 0.f);
    ff3 Ai = zero, Di = zero, Pj = zero, Dj = zero;   // i's feature, j's feature (body frames)
    ff ci = ff_of(0.f), cj = ff_of(0.f);              // 1/|D|^2, or i's plane offset
    switch (sp.kind) {
        case TK_SPH:
            Ai = T.vertex(gi, 0);
            Pj = T.vertex(gj, 0);
            break;
        case TK_VF_I:
            Pj = T.vertex(gj, sp.b);
            if (sp.hit.inside) {                      // Ai: i's face normal, ci: offset
                Ai = T.rec(gi.f_off + sp.a);
                ci = T.recw(gi.f_off + sp.a);
            } else {
                T.face_edge(gi, sp.a, sp.hit.k, &Ai, &Di, &ci);
            }
            break;
        case TK_VF_J:
            Ai = T.vertex(gi, sp.a);
            if (sp.hit.inside) {                      // Pj: a point of j's face, Dj: its normal
                T.face_edge(gj, sp.b, 0, &Pj, &Dj, &cj);
                Dj = T.rec(gj.f_off + sp.b);
            } else {
                T.face_edge(gj, sp.b, sp.hit.k, &Pj, &Dj, &cj);
            }
            break;
        case TK_EE:
            T.edge(gi, sp.a, &Ai, &Di, &ci);
            T.edge(gj, sp.b, &Pj, &Dj, &cj);
            break;
        case TK_VE_I:
            T.edge(gi, sp.a, &Ai, &Di, &ci);
            Pj = T.vertex(gj, sp.b);
            break;
        default:   // TK_VE_J
            Ai = T.vertex(gi, sp.a);
            T.edge(gj, sp.b, &Pj, &Dj, &cj);
            break;
    }
    // j's point and direction in i's frame: R_i^T (d + R_j Pj), R_i^T R_j Dj.
    // One rotation body in a loop (r: Pj and Dj by q_j, then both by the
    // conjugate of q_i): the instruction cache holds it once.
    ff3 Q = Pj, E = Dj;
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
        const bool jr = r < 2, second = r & 1;
        const ff w = jr ? p.qjw : p.qiw;
        ff3 u = jr ? p.qju : p.qiu;
        if (!jr) u = {ff_neg(u.x), ff_neg(u.y), ff_neg(u.z)};
        const ff3 v = second ? E : Q;
        ff3 out = ff3_rotate(w, u, v, false);
        if (r == 0) out = out + p.d;
        if (second) E = out;
        else Q = out;
    }
    ff3 pi = Ai, pj = Q;
    switch (sp.kind) {
        case TK_VF_I:
            if (sp.hit.inside) {                      // projection minus the vertex: -h n
                const ff h = ff_sub(ff3_dot(Ai, Q), ci);
                *rv = ff3_mul(Ai, ff_neg(h));
                *arm = Q + *rv;
                return;
            }
            pi = ff3_point(Ai, Di, foot(Q, Ai, Di, ci, sp.hit.t));
            break;
        case TK_VF_J:
            if (sp.hit.inside) {                      // the vertex minus its projection: h n
                const ff h = ff3_dot(E, Ai - Q);
                *rv = ff3_mul(E, h);
                *arm = Ai;
                return;
            }
            pj = ff3_point(Q, E, foot(Ai, Q, E, cj, sp.hit.t));
            break;
        case TK_EE: {
            ff s, t;
            refine_edges(Ai, Di, ci, Q, E, cj, sp, &s, &t);
            pi = ff3_point(Ai, Di, s);
            pj = ff3_point(Q, E, t);
            break;
        }
        case TK_VE_I:
            pi = ff3_point(Ai, Di, foot(Q, Ai, Di, ci, sp.t));
            break;
        case TK_VE_J:
            pj = ff3_point(Q, E, foot(Ai, Q, E, cj, sp.t));
            break;
        default:
            break;
    }
    *rv = pi - pj;
    *arm = pi;
}

// The refined term's values: force and torque (i's frame) as float-float,
// half the energy and the virial as floats.  Returns false when the refined
// distance is not below r_cut (the search's FP32 test let it through at the
// edge; its WCA term is zero there).
__device__ __forceinline__ bool refined_values(const FFTab &T, const Geom &gi, const Geom &gj,
                                               const FFPair &p, const TermSpec &sp, float rc2,
                                               float eps, V3<float> dl, ff *vf, float *v) {
    ff3 rv, arm;
    refine_points(T, gi, gj, p, sp, &rv, &arm);
    const ff r2 = ff3_dot(rv, rv);
    if (!(r2.h < rc2)) return false;
    const ff ir2 = ff_recip(r2);
    const ff s2 = ff_mul(p.sig2, ir2);
    const ff s6 = ff_mul(ff_mul(s2, s2), s2);
    const ff s12 = ff_mul(s6, s6);
    const float U = 4.f * eps * ff_to_f(ff_sub(s12, s6)) + eps;
    const ff wf = ff_mul_f(ff_mul(ff_sub(ff_scale2(s12, 2.f), s6), ir2), 24.f * eps);
    const ff3 f = ff3_mul(rv, wf);
    const ff3 tq = ff3_cross(arm, f);
    vf[0] = f.x; vf[1] = f.y; vf[2] = f.z;
    vf[3] = tq.x; vf[4] = tq.y; vf[5] = tq.z;
    v[0] = 0.5f * U;
    const float fx = ff_to_f(f.x), fy = ff_to_f(f.y), fz = ff_to_f(f.z);
    const float x = -dl.x, y = -dl.y, z = -dl.z;
    v[1] = 0.5f * x * fx;
    v[2] = 0.25f * (x * fy + y * fx);
    v[3] = 0.25f * (x * fz + z * fx);
    v[4] = 0.5f * y * fy;
    v[5] = 0.25f * (y * fz + z * fy);
    v[6] = 0.5f * z * fz;
    return true;
}

// refined_values behind a call: THREAD and WARP evaluate terms from six
// places, which then share one copy of the code in the instruction cache.
__device__ __noinline__ bool refined_values_call(const FFTab &T, const Geom &gi, const Geom &gj,
                                                 const FFPair &p, const TermSpec &sp, float rc2,
                                                 float eps, V3<float> dl, ff *vf, float *v) {
    return refined_values(T, gi, gj, p, sp, rc2, eps, dl, vf, v);
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
    // a refined term (FP32 + two-sum): force and torque as float-float, the
    // energy and virial as floats
    __device__ __forceinline__ void add_ff(const ff *vf, const float *x) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k].add_ff(vf[k]);
#pragma unroll
        for (int k = 0; k < 7; ++k) v[6 + k].add(x[k]);
    }
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
// A pair's partial sums in the FP32 + two-sum mode (WARP decomposition):
// float-float for force and torque, floats for the rest.
struct FFPartSink {
    Acc<float, true> f[6];
    float v[7];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int k = 0; k < 6; ++k) f[k].zero();
#pragma unroll
        for (int k = 0; k < 7; ++k) v[k] = 0.f;
    }
    __device__ __forceinline__ void add_ff(const ff *vf, const float *x) {
#pragma unroll
        for (int k = 0; k < 6; ++k) f[k].add_ff(vf[k]);
#pragma unroll
        for (int k = 0; k < 7; ++k) v[k] += x[k];
    }
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
// masked features, which carry every non-zero term), in i's frame.  REF (the
// FP32 + two-sum mode): each term found is re-evaluated in float-float
// (refined_values) and added to the sink as float-float; pa then gives the
// state, and w.i, w.j the particles.
template <class T, int DIM, bool COUNT, bool REF, class Sink, class MK>
__device__ __forceinline__ void eval_pair(const typename R4T<T>::type *tab, const int *itab,
                                          const Geom &gi, const Geom &gj, const PairWork<T, MK> &w,
                                          T eps, T par_eps, Sink &sink, PathCount *pc,
                                          const PairArgs *pa = nullptr) {
    using R4 = typename R4T<T>::type;
    const T rc = w.rc, rc2 = rc * rc;
    const V3<T> dl = w.dl;
    T U, wf, tv[13];
    FFPair fp;
    FFTab ft;
    if constexpr (REF) {
        fp = load_ffpair(*pa, w.i, w.j);
        ft = {reinterpret_cast<const float4 *>(tab), pa->table_lo, itab};
    }
    auto refined = [&](int kind, int fa, int fb, FaceHit hit, float ps, float pt) {
        if constexpr (REF) {
            const TermSpec sp = {kind, fa, fb, hit, ps, pt, w.jref};
            ff vf[6];
            float v[7];
            if (refined_values_call(ft, gi, gj, fp, sp, (float)rc2, (float)eps, dl, vf, v))
                sink.add_ff(vf, v);
        }
    };
    const FaceHit nohit = {0, 0, 0.f};
    if (gi.nv == 1 && gj.nv == 1) {             // sphere / disk limit: central WCA
        const V3<T> pi = xyz<T>(tab[gi.v_off]);
        const V3<T> rv = pi - (dl + mul(w.M, xyz<T>(tab[gj.v_off])));
        const T r2 = dot(rv, rv);
        if (r2 < rc2) {
            if constexpr (REF) {
                refined(TK_SPH, 0, 0, nohit, 0.f, 0.f);
            } else {
                wf = wca_factor(r2, w.sig2, eps, &U);
                term_values(pi, rv * wf, dl, U, tv);
                sink.add(tv);
            }
            bump<COUNT>(pc, C_TERMS);
        }
        return;
    }
    const T reach_i = T(gi.R) + rc, reach_j = T(gj.R) + rc;
    // vertex of j against the faces (2D: edges) of i, in i's frame
    for_each_bit(w.vjm, [&](int b) {
        const V3<T> p = dl + mul(w.M, xyz<T>(tab[gj.v_off + b]));
        bump<COUNT>(pc, C_VTX);
        if (!(dot(p, p) < reach_i * reach_i)) return;
        if constexpr (DIM == 3) {
            for_each_bit(w.fim, [&](int f) {
                V3<T> q;
                T r2;
                FaceHit hit;
                if (!face_nearest<T, COUNT>(tab, itab, gi.f_off + f, gi.fi_off + 2 * f, p, rc, &q, &r2, pc,
                                            &hit))
                    return;
                if (r2 < rc2) {
                    if constexpr (REF) {
                        refined(TK_VF_I, f, b, hit, 0.f, 0.f);
                    } else {
                        wf = wca_factor(r2, w.sig2, eps, &U);
                        term_values(q, (q - p) * wf, dl, U, tv);
                        sink.add(tv);
                    }
                    bump<COUNT>(pc, C_TERMS);
                }
            });
        } else {
            for_each_bit(w.eim, [&](int e) {
                const R4 ea = tab[gi.e_off + 2 * e], ed = tab[gi.e_off + 2 * e + 1];
                const V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                const V3<T> c = A + D * T(0.5) - p;
                const T lim = ea.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(c, c) < lim * lim)) return;
                bump<COUNT>(pc, C_PTSEG);
                const T t = clamp01(dot(p - A, D) * ed.w);
                const V3<T> q = A + D * t;
                const V3<T> rv = q - p;
                const T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    if constexpr (REF) {
                        refined(TK_VE_I, e, b, nohit, 0.f, (float)t);
                    } else {
                        wf = wca_factor(r2, w.sig2, eps, &U);
                        term_values(q, rv * wf, dl, U, tv);
                        sink.add(tv);
                    }
                    bump<COUNT>(pc, C_TERMS);
                }
            });
        }
    });
    // vertex of i against the faces (2D: edges) of j, in j's frame
    for_each_bit(w.vim, [&](int ai) {
        const V3<T> u = xyz<T>(tab[gi.v_off + ai]);
        const V3<T> p = mul_t(w.M, u - dl);
        bump<COUNT>(pc, C_VTX);
        if (!(dot(p, p) < reach_j * reach_j)) return;
        if constexpr (DIM == 3) {
            for_each_bit(w.fjm, [&](int f) {
                V3<T> q;
                T r2;
                FaceHit hit;
                if (!face_nearest<T, COUNT>(tab, itab, gj.f_off + f, gj.fi_off + 2 * f, p, rc, &q, &r2, pc,
                                            &hit))
                    return;
                if (r2 < rc2) {
                    if constexpr (REF) {
                        refined(TK_VF_J, ai, f, hit, 0.f, 0.f);
                    } else {
                        wf = wca_factor(r2, w.sig2, eps, &U);
                        term_values(u, mul(w.M, (p - q) * wf), dl, U, tv);
                        sink.add(tv);
                    }
                    bump<COUNT>(pc, C_TERMS);
                    bump<COUNT>(pc, C_JTERMS);
                }
            });
        } else {
            for_each_bit(w.ejm, [&](int e) {
                const R4 ea = tab[gj.e_off + 2 * e], ed = tab[gj.e_off + 2 * e + 1];
                const V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                const V3<T> c = A + D * T(0.5) - p;
                const T lim = ea.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(c, c) < lim * lim)) return;
                bump<COUNT>(pc, C_PTSEG);
                const T t = clamp01(dot(p - A, D) * ed.w);
                const V3<T> q = A + D * t;
                const V3<T> rv = p - q;
                const T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    if constexpr (REF) {
                        refined(TK_VE_J, ai, e, nohit, 0.f, (float)t);
                    } else {
                        wf = wca_factor(r2, w.sig2, eps, &U);
                        term_values(u, mul(w.M, rv * wf), dl, U, tv);
                        sink.add(tv);
                    }
                    bump<COUNT>(pc, C_TERMS);
                    bump<COUNT>(pc, C_JTERMS);
                }
            });
        }
    });
    if constexpr (DIM == 3) {
        // edges of j against the edges of i, in i's frame
        if (mask_any(w.eim)) for_each_bit(w.ejm, [&](int eb) {
            const R4 ba = tab[gj.e_off + 2 * eb], bd = tab[gj.e_off + 2 * eb + 1];
            const V3<T> A2 = dl + mul(w.M, xyz<T>(ba));
            const V3<T> D2 = mul(w.M, xyz<T>(bd));
            const V3<T> C2 = A2 + D2 * T(0.5);
            const T reach = reach_i + ba.w;
            bump<COUNT>(pc, C_EDGE);
            if (!(dot(C2, C2) < reach * reach)) return;
            for_each_bit(w.eim, [&](int ea) {
                const R4 aa = tab[gi.e_off + 2 * ea], ad = tab[gi.e_off + 2 * ea + 1];
                const V3<T> A1 = xyz<T>(aa), D1 = xyz<T>(ad);
                const V3<T> dc = A1 + D1 * T(0.5) - C2;
                const T lim = aa.w + ba.w + rc;
                bump<COUNT>(pc, C_SPHERE);
                if (!(dot(dc, dc) < lim * lim)) return;
                // carrier lines farther apart than r_cut: the segments are too
                const V3<T> nrm = cross(D1, D2);
                const T n2 = dot(nrm, nrm);
                const T sep = dot(A2 - A1, nrm);
                bump<COUNT>(pc, C_LINE);
                if (sep * sep >= rc2 * n2 && n2 > par_eps * dot(D1, D1) * dot(D2, D2)) return;
                bump<COUNT>(pc, C_SEGSEG);
                V3<T> P1, P2;
                T ps, pt;
                int par;
                segment_nearest<T>(A1, D1, ad.w, A2, D2, bd.w, par_eps, w.jref != 0, &P1, &P2, &ps,
                                   &pt, &par);
                const V3<T> rv = P1 - P2;
                const T r2 = dot(rv, rv);
                if (r2 < rc2) {
                    if constexpr (REF) {
                        refined(TK_EE, ea, eb, FaceHit{par, 0, 0.f}, (float)ps, (float)pt);
                    } else {
                        wf = wca_factor(r2, w.sig2, eps, &U);
                        term_values(P1, rv * wf, dl, U, tv);
                        sink.add(tv);
                    }
                    bump<COUNT>(pc, C_TERMS);
                }
            });
        });
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
