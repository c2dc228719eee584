// pair_common.cuh -- device arithmetic of the feature-pair terms (Eq. DEM,
// Eq. DEM_2D, Eq. LJ / Eq. WCA, parallel-edge rule of Section "Model"),
// shared by the pair-kernel decompositions in pair.cu.
//
// Frames: every term of the ordered pair (i, j) is evaluated in i's body
// frame, where i's features are constants of the geometry table.  j's
// vertices and edges are mapped in with M = R_i^T R_j and dl = R_i^T d
// (d = x_j - x_i, minimum image).  Vertex(i)-face(j) terms are evaluated in
// j's body frame instead (j's faces are then table constants) and their
// force is mapped back with M.
#pragma once

#include "dem_internal.cuh"
#include "ff.cuh"

namespace dem {

template <class T> struct R4T;
template <> struct R4T<float> { using type = float4; };
template <> struct R4T<double> { using type = double4_32a; };

template <class T> struct V3 { T x, y, z; };

template <class T> __device__ __forceinline__ V3<T> v3(T x, T y, T z) { return {x, y, z}; }
template <class T> __device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) {
    return {a.x + b.x, a.y + b.y, a.z + b.z};
}
template <class T> __device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) {
    return {a.x - b.x, a.y - b.y, a.z - b.z};
}
template <class T> __device__ __forceinline__ V3<T> operator*(V3<T> a, T s) {
    return {a.x * s, a.y * s, a.z * s};
}
template <class T> __device__ __forceinline__ T dot(V3<T> a, V3<T> b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <class T> __device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T, class R4> __device__ __forceinline__ V3<T> xyz(const R4 &r) {
    return {r.x, r.y, r.z};
}
template <class T> __device__ __forceinline__ T clamp01(T t) {
    return t < T(0) ? T(0) : (t > T(1) ? T(1) : t);
}

template <class T> struct M33 { T m[3][3]; };

// Rotation matrix (body -> world) of the unit quaternion (w, x, y, z).
template <class T> __device__ __forceinline__ M33<T> quat_mat(T w, T x, T y, T z) {
    M33<T> R;
    R.m[0][0] = T(1) - T(2) * (y * y + z * z);
    R.m[0][1] = T(2) * (x * y - w * z);
    R.m[0][2] = T(2) * (x * z + w * y);
    R.m[1][0] = T(2) * (x * y + w * z);
    R.m[1][1] = T(1) - T(2) * (x * x + z * z);
    R.m[1][2] = T(2) * (y * z - w * x);
    R.m[2][0] = T(2) * (x * z - w * y);
    R.m[2][1] = T(2) * (y * z + w * x);
    R.m[2][2] = T(1) - T(2) * (x * x + y * y);
    return R;
}
template <class T> __device__ __forceinline__ V3<T> mul(const M33<T> &R, V3<T> v) {
    return {R.m[0][0] * v.x + R.m[0][1] * v.y + R.m[0][2] * v.z,
            R.m[1][0] * v.x + R.m[1][1] * v.y + R.m[1][2] * v.z,
            R.m[2][0] * v.x + R.m[2][1] * v.y + R.m[2][2] * v.z};
}
template <class T> __device__ __forceinline__ V3<T> mul_t(const M33<T> &R, V3<T> v) {
    return {R.m[0][0] * v.x + R.m[1][0] * v.y + R.m[2][0] * v.z,
            R.m[0][1] * v.x + R.m[1][1] * v.y + R.m[2][1] * v.z,
            R.m[0][2] * v.x + R.m[1][2] * v.y + R.m[2][2] * v.z};
}
// A^T B
template <class T> __device__ __forceinline__ M33<T> mul_tn(const M33<T> &A, const M33<T> &B) {
    M33<T> C;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            C.m[r][c] = A.m[0][r] * B.m[0][c] + A.m[1][r] * B.m[1][c] + A.m[2][r] * B.m[2][c];
    return C;
}

// ---- summation ----
// Plain sum in T, or (float, COMP) an error-free two-sum accumulation: the
// rounding error of every addition is carried in c (Knuth's TwoSum, adds
// only, so FMA contraction cannot change it; the _rn intrinsics keep the
// compiler from re-associating).
template <class T, bool COMP> struct Acc {
    T s;
    __device__ __forceinline__ void zero() { s = T(0); }
    __device__ __forceinline__ void add(T x) { s += x; }
    // merge another lane's accumulator (os, oc); oc is unused without two-sum
    __device__ __forceinline__ void merge(T os, T) { s += os; }
    __device__ __forceinline__ T comp() const { return T(0); }
    __device__ __forceinline__ double get() const { return (double)s; }
};
template <> struct Acc<float, true> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float t = __fadd_rn(s, x);
        float bp = __fsub_rn(t, s);
        float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        s = t;
        c = __fadd_rn(c, e);
    }
    // two-sum of the leading parts, the trailing parts added to the error
    __device__ __forceinline__ void merge(float os, float oc) {
        float t = __fadd_rn(s, os);
        float bp = __fsub_rn(t, s);
        float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(os, bp));
        s = t;
        c = __fadd_rn(__fadd_rn(c, oc), e);
    }
    __device__ __forceinline__ float comp() const { return c; }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
    // a float-float addend h + l: h by two-sum, l into the compensation
    __device__ __forceinline__ void add_ff(ff x) {
        float t = __fadd_rn(s, x.h);
        float bp = __fsub_rn(t, s);
        float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x.h, bp));
        s = t;
        c = __fadd_rn(c, __fadd_rn(e, x.l));
    }
};

// WCA of one feature pair (Eq. LJ, Eq. WCA) at squared nearest-point distance
// r2 < r_cut^2: returns w with the force on i equal to w (p_i - p_j), and
// *U = 4 eps ((s/r)^12 - (s/r)^6) + eps (the shift removes U_LJ(r_cut) = -eps).
template <class T>
__device__ __forceinline__ T wca_factor(T r2, T sig2, T eps, T *U) {
    T ir2 = T(1) / r2;
    T s2 = sig2 * ir2;
    T s6 = s2 * s2 * s2;
    T s12 = s6 * s6;
    *U = T(4) * eps * (s12 - s6) + eps;
    return T(24) * eps * (T(2) * s12 - s6) * ir2;
}

// Work counters of a counting launch (see dem_get_counters).
enum {
    C_PAIRS = 0,       // ordered pairs within the bounding-sphere range
    C_FPE = 1,         // feature pairs Eq. DEM / Eq. DEM_2D assigns to them
    C_TERMS = 2,       // terms with r < r_cut (WCA evaluated)
    C_VTX = 3,         // vertex transforms (+ reach test)
    C_PLANE = 4,       // face-plane tests
    C_INPLANE = 5,     // in-plane edge tests of faces
    C_PTSEG = 6,       // point-segment nearest points
    C_EDGE = 7,        // edge transforms (+ reach test)
    C_SPHERE = 8,      // edge bounding-sphere tests
    C_SEGSEG = 9,      // segment-segment nearest points
    C_NEIGH = 10,      // neighbour-list entries scanned
    C_INSIDE = 11,     // vertex-face projections inside the face
    C_JTERMS = 12,     // terms evaluated in j's frame
    C_ACTIVE = 15,     // pairs that pass the separating-axis test
    C_PROJ = 16,       // vertex projections of the separating-axis test
    C_LINE = 17,       // carrier-line distance tests of edge pairs
    NCOUNT = 20
};
struct PathCount {
    unsigned int v[NCOUNT];
};
template <bool COUNT>
__device__ __forceinline__ void bump(PathCount *pc, int k, unsigned int n = 1) {
    if constexpr (COUNT) pc->v[k] += n;
}

// Nearest point q on a convex face to p (both in the face owner's frame).
// Returns false when |signed plane distance| >= rc: then r* >= rc and the
// term is exactly zero.  Otherwise *r2 = |p - q|^2.  Inside the face (all
// in-plane edge tests >= 0) q is the projection; else q is the nearest
// point on the edges whose test fails (the nearest boundary point of a
// convex polygon lies on such an edge).
// The nearest point after a passed plane test (nf the face record, h the
// signed plane distance of p).
// Where the nearest point of a vertex-face term lies: inside the face (the
// projection), or on face edge k at parameter t.
struct FaceHit {
    int inside, k;
    float t;
};

template <class T, bool COUNT, class R4>
__device__ __forceinline__ void face_rest(const R4 *tab, const int *itab, int face_int,
                                          const R4 &nf, V3<T> p, T h, V3<T> *q, T *r2,
                                          PathCount *pc, FaceHit *hit = nullptr);

template <class T, bool COUNT, class R4>
__device__ __forceinline__ bool face_nearest(const R4 *tab, const int *itab, int face_rec,
                                             int face_int, V3<T> p, T rc, V3<T> *q, T *r2,
                                             PathCount *pc, FaceHit *hit = nullptr) {
    R4 nf = tab[face_rec];
    T h = nf.x * p.x + nf.y * p.y + nf.z * p.z - nf.w;
    bump<COUNT>(pc, C_PLANE);
    if (!(fabs(h) < rc)) return false;
    face_rest<T, COUNT>(tab, itab, face_int, nf, p, h, q, r2, pc, hit);
    return true;
}

template <class T, bool COUNT, class R4>
__device__ __forceinline__ void face_rest(const R4 *tab, const int *itab, int face_int,
                                          const R4 &nf, V3<T> p, T h, V3<T> *q, T *r2,
                                          PathCount *pc, FaceHit *hit) {
    int fe = itab[face_int], cnt = itab[face_int + 1];
    bool inside = true;
    T best = T(3.0e38);
    V3<T> bq = p;
    int bk = 0;
    T bt = T(0);
    bump<COUNT>(pc, C_INPLANE, (unsigned)cnt);
    for (int k = 0; k < cnt; ++k) {
        R4 m = tab[fe + 3 * k + 2];
        T s = m.x * p.x + m.y * p.y + m.z * p.z - m.w;
        if (s < T(0)) {
            inside = false;
            bump<COUNT>(pc, C_PTSEG);
            R4 a = tab[fe + 3 * k], e = tab[fe + 3 * k + 1];
            V3<T> A = xyz<T>(a), E = xyz<T>(e);
            T t = clamp01(dot(p - A, E) * e.w);
            V3<T> c = A + E * t;
            V3<T> dd = p - c;
            T d2 = dot(dd, dd);
            if (d2 < best) { best = d2; bq = c; bk = k; bt = t; }
        }
    }
    if (inside) {
        bump<COUNT>(pc, C_INSIDE);
        *q = p - xyz<T>(nf) * h;
        *r2 = h * h;
    } else {
        *q = bq;
        *r2 = best;
    }
    if (hit) *hit = {inside ? 1 : 0, bk, (float)bt};
}

// Nearest points of segments [A1, A1 + D1] and [A2, A2 + D2] (inv_a =
// 1/|D1|^2, inv_c = 1/|D2|^2).  Not nearly parallel: the constrained
// minimiser of the convex quadratic |W + s D1 - t D2|^2 over [0,1]^2,
// taking s from the unconstrained solution clamped to [0,1], the optimal t
// for that s, and if that t leaves [0,1], t clamped and the optimal s for it
// (each step solves one linear condition of the quadratic).  Nearly
// parallel (|D1 x D2|^2 <= par_eps |D1|^2 |D2|^2): the parallel-edge rule
// of Section "Model": the midpoint of the overlap of the other segment's
// projection on the reference segment, and its nearest point on the other
// segment; with no overlap, the nearest of the four endpoint-to-segment
// pairs.  Unless the edges are exactly parallel the rule's result depends on
// which segment is the reference, so both orders of a particle pair must
// name the same one (else F_ij != -F_ji): the edge of the particle with the
// lower index.  ref2 = false: segment 1 is the reference; ref2 = true:
// segment 2 is.
template <class T>
__device__ __forceinline__ void segment_nearest(V3<T> A1, V3<T> D1, T inv_a, V3<T> A2,
                                                V3<T> D2, T inv_c, T par_eps, bool ref2,
                                                V3<T> *P1, V3<T> *P2, T *s_out = nullptr,
                                                T *t_out = nullptr, int *par_out = nullptr) {
    V3<T> W = A1 - A2;
    T a = dot(D1, D1), b = dot(D1, D2), c = dot(D2, D2);
    T d = dot(D1, W), e = dot(D2, W);
    V3<T> cr = cross(D1, D2);
    T den = dot(cr, cr);
    T s, t;
    if (den > par_eps * a * c) {
        s = clamp01((b * e - c * d) / den);
        t = (b * s + e) * inv_c;
        if (t < T(0)) {
            t = T(0);
            s = clamp01(-d * inv_a);
        } else if (t > T(1)) {
            t = T(1);
            s = clamp01((b - d) * inv_a);
        }
    } else {
        // the other segment's endpoints projected on the reference's line
        T t0, t1;
        if (ref2) { t0 = e * inv_c; t1 = (e + b) * inv_c; }
        else { t0 = -d * inv_a; t1 = (b - d) * inv_a; }
        T lo = fmax(T(0), fmin(t0, t1)), hi = fmin(T(1), fmax(t0, t1));
        if (lo <= hi) {
            if (ref2) {
                t = T(0.5) * (lo + hi);
                s = clamp01((t * b - d) * inv_a);
            } else {
                s = T(0.5) * (lo + hi);
                t = clamp01((e + s * b) * inv_c);
            }
        } else {
            // four endpoint-to-segment candidates in a fixed order
            T best = T(3.0e38);
            s = T(0);
            t = T(0);
            {
                T tt = clamp01(e * inv_c);  // A1 vs segment 2
                V3<T> r = W - D2 * tt;
                T d2 = dot(r, r);
                if (d2 < best) { best = d2; s = T(0); t = tt; }
            }
            {
                T tt = clamp01((e + b) * inv_c);  // A1 + D1 vs segment 2
                V3<T> r = W + D1 - D2 * tt;
                T d2 = dot(r, r);
                if (d2 < best) { best = d2; s = T(1); t = tt; }
            }
            {
                T ss = clamp01(-d * inv_a);  // A2 vs segment 1
                V3<T> r = W + D1 * ss;
                T d2 = dot(r, r);
                if (d2 < best) { best = d2; s = ss; t = T(0); }
            }
            {
                T ss = clamp01((b - d) * inv_a);  // A2 + D2 vs segment 1
                V3<T> r = W + D1 * ss - D2;
                T d2 = dot(r, r);
                if (d2 < best) { best = d2; s = ss; t = T(1); }
            }
        }
    }
    *P1 = A1 + D1 * s;
    *P2 = A2 + D2 * t;
    if (s_out) *s_out = s;
    if (t_out) *t_out = t;
    if (par_out) *par_out = den > par_eps * a * c ? 0 : 1;
}

}  // namespace dem
