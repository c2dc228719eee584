// pair_staged.cu -- STAGED decomposition of the pair kernel (Eq. DEM,
// Eq. DEM_2D; Section "Algorithm" of arXiv:1607.02427 re-designed for
// sm_103a).
//
// One warp owns a group of particles at a time (32 in the fused kernel; 32,
// 16, 8 or 4 in SPLIT) and streams their feature-pair work through per-warp
// shared-memory rings, so that every stage runs with full warps on uniform
// work instead of one lane walking all features of a pair:
//
//   scan     lanes take the group's list entries: range test, pair
//            setup (M, dl, separating-axis test, feature masks); the pairs
//            that pass are appended to the pair ring in ballot order.
//   batch    32 queued pairs at a time:
//     sphere   one-vertex pairs (sphere / disk limit): the one central term.
//     vertex   lanes take (pair, vertex) items of both orders (j's masked
//              vertices against i's faces, i's against j's): the vertex is
//              mapped into the other body's frame once, reach-tested, then
//              the warp walks the items' face masks in step; 3D: a plane test
//              per (vertex, face), survivors queued; 2D: the edge
//              bounding-sphere test and the point-segment nearest point.
//     face     queued (vertex, face) candidates, 32 at a time: in-plane
//              tests and the nearest point on the face.
//     edge     lanes take (pair, edge of j) items: the edge is mapped into
//              i's frame once and reach-tested, then the warp walks i's
//              masked edges in step: bounding-sphere and carrier-line tests,
//              survivors queued.
//     segment  queued edge pairs, 32 at a time: segment-segment nearest
//              points.
//   terms    queued terms (r < r_cut), 32 at a time: WCA force, torque,
//            energy and virial in i's frame; terms of the same owner are
//            added by the owner's lane in queue order (shuffles), so each
//            particle's sum has a fixed order.
//
// The arithmetic of every test and term is that of eval_pair (shared
// helpers in pair_kernels.cuh / pair_common.cuh); only the work order
// differs.  Rings hold at most 63 entries (a round adds at most 32 and a
// stage runs as soon as 32 are queued).
#include "pair_kernels.cuh"

namespace dem {
namespace {

constexpr int RING = 64;
constexpr int SBLOCK = 128;

// Records are rows of R4 (float4 / double4) so that they move with vector
// shared-memory accesses.
template <class T> struct SPair {      // a queued active pair
    typename R4T<T>::type row[3];      // (M[r][0], M[r][1], M[r][2], dl[r]): M = R_i^T R_j,
                                       // dl = x_j - x_i in i's frame
    T rc, sig2;
    int gj, owner;                     // j's geometry; the owner's lane
    unsigned vim, vjm, eim, ejm, fim, fjm;
    int gi;                            // i's geometry
    int jref;                          // bit 0: j < i (j's edge is the parallel-edge rule's
                                       // reference); bits 1..: j
};
template <class T> struct SInfo {      // one particle of the warp
    typename R4T<T>::type row[3];      // (R_i[r][0..2], x[r]); x: FP32 delta_i, FP64 position
    typename R4T<T>::type q;           // q_i (w, x, y, z)
    T rnd;
    int geom, rep;
    float sc;                          // FP32 list separation scale of the replica
};
// Per-warp shared memory of the batch stages and of the list scan.
template <class T, int PR> struct BatchSmem {   // PR: pair ring entries (a power of 2)
    SPair<T> pr[PR];
    // The rings hold their records' fields in separate arrays, so that the
    // lanes' 16-byte accesses to consecutive slots are contiguous.
    union {
        struct {                          // (vertex, face) after the plane test
            typename R4T<T>::type p[RING];   // the vertex in the face owner's frame;
                                             // w: its signed plane distance
            int code[RING];                  // pair | side << 5 | vertex << 6 | face << 11
        } vf;
        struct {                          // edge pair after the sphere and line tests
            typename R4T<T>::type a2[RING];  // j's edge start in i's frame; w: code =
                                             // pair | edge of i << 5 | edge of j << 10
            typename R4T<T>::type d2[RING];  // j's edge direction in i's frame
        } ee;
    } fq;
    struct {                              // terms with r < r_cut
        typename R4T<T>::type q[RING];       // the point on i's feature (i's frame); w: r^2
                                             // FP32 + two-sum: (s, t, r_cut^2, spec code)
        typename R4T<T>::type rv[RING];      // i's point minus j's point (i's frame); w: pair
                                             // FP32 + two-sum: (dl, j)
        int info[RING];                      // FP32 + two-sum: owner | gi << 8 | gj << 16 |
                                             // jref << 24 (the term outlives its pair's slot)
    } tq;
    int boffs[32];                     // item offsets of the batch's pairs
    int who[32];                       // pair whose items start at lane k of a round
    unsigned gmask[32];                // per owner: lanes holding its terms
};
// An active pair as SPLIT's scan kernel writes it to device memory: the
// relative orientation as a quaternion instead of M, sigma instead of r_cut
// and sigma^2, the geometries, owner lane and rule reference packed in one
// word, and only the vertex masks (the edge and face masks are the features
// of those vertices).  The feature kernel expands it into an SPair.
template <class T> struct alignas(16) GRec {
    T q[4];                            // q_rel = conj(q_i) q_j: M = R(q_rel) = R_i^T R_j
    T dl[3];                           // x_j - x_i in i's frame
    T sig;                             // sigma_ij
    unsigned ids;                      // gi | gj << 8 | owner << 16 | jref << 21
    unsigned vim, vjm;
    int j;                             // the neighbour
};
static_assert(MAX_GEOMS <= 256, "GRec packs geometry indices in 8 bits");

template <class T> struct ScanSmem {
    SInfo<T> info[32];
    int offs[32];                      // list offsets of the group's particles
    int who[32];                       // particle whose entries start at lane k of a round
};
template <class T> struct StagedSmem {
    BatchSmem<T, RING> b;
    ScanSmem<T> s;
};

// Position of the n-th (from 0) set bit of m (n < popc(m)).
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
    int pos = 0;
    int c = __popc(m & 0xffffu);
    if (n >= c) { n -= c; m >>= 16; pos += 16; }
    c = __popc(m & 0xffu);
    if (n >= c) { n -= c; m >>= 8; pos += 8; }
    c = __popc(m & 0xfu);
    if (n >= c) { n -= c; m >>= 4; pos += 4; }
    c = __popc(m & 0x3u);
    if (n >= c) { n -= c; m >>= 2; pos += 2; }
    if (n >= (int)(m & 1u)) pos += 1;
    return pos;
}

// Ring slot of this lane's entry when the lanes in m append at tail.
__device__ __forceinline__ int ring_slot(unsigned m, int lane, int tail) {
    return (tail + __popc(m & ((1u << lane) - 1u))) & (RING - 1);
}

// M and dl of a queued pair, or R_i and x of a particle (three vector loads).
template <class R4, class T>
__device__ __forceinline__ void load_rows(const R4 *row, M33<T> *M, V3<T> *x) {
    const R4 r0 = row[0], r1 = row[1], r2 = row[2];
    M->m[0][0] = r0.x; M->m[0][1] = r0.y; M->m[0][2] = r0.z;
    M->m[1][0] = r1.x; M->m[1][1] = r1.y; M->m[1][2] = r1.z;
    M->m[2][0] = r2.x; M->m[2][1] = r2.y; M->m[2][2] = r2.z;
    *x = v3<T>(r0.w, r1.w, r2.w);
}
template <class R4, class T>
__device__ __forceinline__ void store_rows(R4 *row, const M33<T> &M, V3<T> x) {
    row[0] = {M.m[0][0], M.m[0][1], M.m[0][2], x.x};
    row[1] = {M.m[1][0], M.m[1][1], M.m[1][2], x.y};
    row[2] = {M.m[2][0], M.m[2][1], M.m[2][2], x.z};
}
template <class T> __device__ __forceinline__ M33<T> pair_m(const SPair<T> &P) {
    M33<T> M;
    V3<T> dl;
    load_rows(P.row, &M, &dl);
    return M;
}
template <class T> __device__ __forceinline__ V3<T> pair_dl(const SPair<T> &P) {
    return v3<T>(P.row[0].w, P.row[1].w, P.row[2].w);
}

// Every stage has one call site (code size: the stages of 16 warps per SM
// must share the instruction cache).  batch() is a loop whose body does one
// action per turn: consumers first, so that no ring reaches 64 entries,
// then steps of the current producer until its ring holds 32 entries or
// its items are done.
template <class T, bool COMP, int DIM, bool COUNT, int PR = RING, bool SPILL = false> struct Staged {
    using R4 = typename R4T<T>::type;
    const PairArgs &a;
    const R4 *tab;
    const Geom *geo;
    const int *itab;
    BatchSmem<T, PR> &ws;
    const int lane;
    const T eps, par_eps;
    PathCount pc;
    SumSink<T, COMP> S;                // this lane's particle
    // FP32 + two-sum: the term ring carries each term's features and
    // parameters (spec_code), and run_terms re-evaluates it in float-float
    static constexpr bool REF = COMP && std::is_same<T, float>::value;
    int base = 0;                      // first particle of the warp's group
    const float4 *tab_lo = nullptr;    // REF: the table's low parts (shared memory)
    // SPILL (REF in SPLIT's feature kernel): terms go to the warp's region of
    // the term buffer (tcur records so far) instead of the term ring
    long long region = 0;
    int tcur = 0;
    int ph = 0, np = 0;                // pair ring: head, queued pairs
    int fh = 0, ft = 0;                // feature ring (vertex-face or edge items)
    int th = 0, tt = 0;                // term ring
    // this lane's item: vertex phase (pair, side, vertex) with va = the
    // vertex in the other body's frame; edge phase (pair, j's edge) with
    // va, vb, vc = its start, direction and centre in i's frame
    unsigned cm = 0u;                  // features of the other shape left to test
    int cp = 0, cside = 0, cidx = 0, coff = 0;
    int citems = 0;                    // items of this lane's pair in the current phase
    V3<T> va, vb, vc;
    T crb = T(0), crc = T(0);          // j's edge radius; r_cut

    __device__ __forceinline__ Staged(const PairArgs &a_, const R4 *tab_, const Geom *geo_,
                                      const int *itab_, BatchSmem<T, PR> &ws_, int lane_)
        : a(a_), tab(tab_), geo(geo_), itab(itab_), ws(ws_), lane(lane_), eps((T)a_.eps),
          par_eps((T)a_.par_eps) {
        if constexpr (COUNT)
            for (int k = 0; k < NCOUNT; ++k) pc.v[k] = 0;
    }

    __device__ __forceinline__ SPair<T> &pair(int p) { return ws.pr[(ph + p) & (PR - 1)]; }
    __device__ __forceinline__ const Geom &geom_i(const SPair<T> &P) { return geo[P.gi]; }
    __device__ __forceinline__ static bool spheres(const Geom &gi, const Geom &gj) {
        return gi.nv == 1 && gj.nv == 1;
    }

    // term spec (REF): pair | kind << 5 | a << 8 | b << 15 | face edge << 22 | inside << 26
    __device__ __forceinline__ static int spec_code(int p, int kind, int fa, int fb, FaceHit h) {
        return p | kind << 5 | fa << 8 | fb << 15 | h.k << 22 | h.inside << 26;
    }
    // A refined term's record carries everything run_terms_refined needs from
    // its pair, so that terms may wait in the ring past their batch (the
    // refinement then runs on full warps) until the group of particles ends.
    __device__ __forceinline__ void push_spec(bool ok, int code, float ps, float pt, int p) {
        const unsigned m = __ballot_sync(FULL, ok);
        if constexpr (SPILL) {
            if (ok) {
                const int k = tcur + __popc(m & ((1u << lane) - 1u));
                if (k < a.term_capw) {
                    const SPair<T> &P = pair(p);
                    const V3<T> dl = pair_dl(P);
                    const long long r = region + k;
                    a.term_a[r] = make_float4(ps, pt, (float)(P.rc * P.rc), __int_as_float(code));
                    a.term_b[r] = make_float4(dl.x, dl.y, dl.z, __int_as_float(P.jref >> 1));
                    a.term_info[r] = P.owner | P.gi << 8 | P.gj << 16 | (P.jref & 1) << 24;
                }
            }
            tcur += __popc(m);
            return;
        }
        if (ok) {
            const int s = ring_slot(m, lane, tt);
            const SPair<T> &P = pair(p);
            const V3<T> dl = pair_dl(P);
            ws.tq.q[s] = {ps, pt, (float)(P.rc * P.rc), __int_as_float(code)};
            ws.tq.rv[s] = {dl.x, dl.y, dl.z, __int_as_float(P.jref >> 1)};
            ws.tq.info[s] = P.owner | P.gi << 8 | P.gj << 16 | (P.jref & 1) << 24;
        }
        tt += __popc(m);
        __syncwarp();
    }

    // ---- ring appends (the caller's loop consumes) ----
    __device__ __forceinline__ void push_term(bool ok, V3<T> q, V3<T> rv, T r2, int p) {
        const unsigned m = __ballot_sync(FULL, ok);
        if (ok) {
            const int s = ring_slot(m, lane, tt);
            ws.tq.q[s] = {q.x, q.y, q.z, r2};
            ws.tq.rv[s] = {rv.x, rv.y, rv.z, (T)p};
        }
        tt += __popc(m);
        __syncwarp();
    }
    __device__ __forceinline__ void push_face(bool ok, V3<T> pv, T h, int code) {
        const unsigned m = __ballot_sync(FULL, ok);
        if (ok) {
            const int s = ring_slot(m, lane, ft);
            ws.fq.vf.p[s] = {pv.x, pv.y, pv.z, h};
            ws.fq.vf.code[s] = code;
        }
        ft += __popc(m);
        __syncwarp();
    }
    __device__ __forceinline__ void push_edge(bool ok, V3<T> A2, V3<T> D2, int code) {
        const unsigned m = __ballot_sync(FULL, ok);
        if (ok) {
            const int s = ring_slot(m, lane, ft);
            ws.fq.ee.a2[s] = {A2.x, A2.y, A2.z, (T)code};
            ws.fq.ee.d2[s] = {D2.x, D2.y, D2.z, T(0)};
        }
        ft += __popc(m);
        __syncwarp();
    }

    // ---- consumers ----
    // n queued terms: values in i's frame, added by the owners' lanes in
    // queue order
    __device__ __forceinline__ void run_terms(int n) {
        if constexpr (REF) {
            if constexpr (!SPILL) run_terms_refined(n);
            return;
        }
        T v[13];
        const bool has = lane < n;
        int owner = 32 + lane;                    // lanes without a term: distinct keys
        if (has) {
            const int s = (th + lane) & (RING - 1);
            const auto tq = ws.tq.q[s], trv = ws.tq.rv[s];
            const SPair<T> &P = pair((int)trv.w);
            owner = P.owner;
            T U;
            const T wf = wca_factor(tq.w, P.sig2, eps, &U);
            term_values(v3<T>(tq.x, tq.y, tq.z), v3<T>(trv.x, trv.y, trv.z) * wf, pair_dl(P), U, v);
        } else {
#pragma unroll
            for (int k = 0; k < 13; ++k) v[k] = T(0);
        }
        th += n;
        const unsigned grp = __match_any_sync(FULL, owner);
        if (has && lane == __ffs(grp) - 1) ws.gmask[owner] = grp;
        __syncwarp();
        unsigned rest = ws.gmask[lane];
        const int cnt = __popc(rest);
        const int rounds = (int)__reduce_max_sync(FULL, (unsigned)cnt);
        for (int r = 0; r < rounds; ++r) {
            const int src = rest ? __ffs(rest) - 1 : lane;
            rest &= rest - 1u;
            T x[13];
#pragma unroll
            for (int k = 0; k < 13; ++k) x[k] = __shfl_sync(FULL, v[k], src);
            if (r < cnt) S.add(x);
        }
        ws.gmask[lane] = 0u;
        __syncwarp();
    }

    // REF: n queued term specs, re-evaluated in float-float (refined_values),
    // added by the owners' lanes in queue order (force and torque as
    // float-float)
    __device__ __forceinline__ void run_terms_refined(int n) {
        ff vf[6];
        float v[7];
        const bool has = lane < n;
        int owner = 32 + lane;                    // lanes without a term: distinct keys
        bool ok = false;
        if (has) {
            const int s = (th + lane) & (RING - 1);
            const float4 sp = reinterpret_cast<const float4 &>(ws.tq.q[s]);
            const float4 sr = reinterpret_cast<const float4 &>(ws.tq.rv[s]);
            const int code = __float_as_int(sp.w), info = ws.tq.info[s];
            owner = info & 255;
            const TermSpec ts = {(code >> 5) & 7, (code >> 8) & 127, (code >> 15) & 127,
                                 {(code >> 26) & 1, (code >> 22) & 15, sp.y}, sp.x, sp.y,
                                 (info >> 24) & 1};
            const FFPair fp = load_ffpair(a, base + owner, __float_as_int(sr.w));
            const FFTab ft = {reinterpret_cast<const float4 *>(tab), tab_lo, itab};
            ok = refined_values(ft, geo[(info >> 8) & 255], geo[(info >> 16) & 255], fp, ts, sp.z,
                                (float)eps, v3<float>(sr.x, sr.y, sr.z), vf, v);
        }
        if (!ok) {
#pragma unroll
            for (int k = 0; k < 6; ++k) vf[k] = ff_of(0.f);
#pragma unroll
            for (int k = 0; k < 7; ++k) v[k] = 0.f;
        }
        th += n;
        const unsigned grp = __match_any_sync(FULL, owner);
        if (has && lane == __ffs(grp) - 1) ws.gmask[owner] = grp;
        __syncwarp();
        unsigned rest = ws.gmask[lane];
        const int cnt = __popc(rest);
        const int rounds = (int)__reduce_max_sync(FULL, (unsigned)cnt);
        for (int r = 0; r < rounds; ++r) {
            const int src = rest ? __ffs(rest) - 1 : lane;
            rest &= rest - 1u;
            ff xf[6];
            float x[7];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                xf[k].h = __shfl_sync(FULL, vf[k].h, src);
                xf[k].l = __shfl_sync(FULL, vf[k].l, src);
            }
#pragma unroll
            for (int k = 0; k < 7; ++k) x[k] = __shfl_sync(FULL, v[k], src);
            if (r < cnt) S.add_ff(xf, x);
        }
        ws.gmask[lane] = 0u;
        __syncwarp();
    }

    // n queued (vertex, face) candidates: nearest point on the face
    __device__ __forceinline__ void run_faces(int n) {
        bool ok = false;
        V3<T> q = v3<T>(0, 0, 0), rv = q;
        T r2 = T(0);
        int p = 0, tcode = 0;
        FaceHit hit = {0, 0, 0.f};
        if (lane < n) {
            const int s = (fh + lane) & (RING - 1);
            const auto ip = ws.fq.vf.p[s];
            const int code = ws.fq.vf.code[s];
            p = code & 31;
            const int side = (code >> 5) & 1, vtx = (code >> 6) & 31, f = (code >> 11) & 31;
            const SPair<T> &P = pair(p);
            const Geom &gi = geom_i(P);
            const Geom &gf = side ? geo[P.gj] : gi;
            const V3<T> pv = v3<T>(ip.x, ip.y, ip.z);
            V3<T> qq;
            T rr;
            face_rest<T, COUNT>(tab, itab, gf.fi_off + 2 * f, tab[gf.f_off + f], pv, ip.w, &qq, &rr,
                                &pc, &hit);
            if (rr < P.rc * P.rc) {
                ok = true;
                r2 = rr;
                bump<COUNT>(&pc, C_TERMS);
                if (side == 0) {
                    q = qq;
                    rv = qq - pv;
                    tcode = spec_code(p, TK_VF_I, f, vtx, hit);
                } else {
                    bump<COUNT>(&pc, C_JTERMS);
                    q = xyz<T>(tab[gi.v_off + vtx]);
                    rv = mul(pair_m(P), pv - qq);
                    tcode = spec_code(p, TK_VF_J, vtx, f, hit);
                }
            }
        }
        fh += n;
        __syncwarp();
        if constexpr (REF) push_spec(ok, tcode, 0.f, hit.t, p);
        else push_term(ok, q, rv, r2, p);
    }

    // n queued edge pairs: segment-segment nearest points
    __device__ __forceinline__ void run_segments(int n) {
        bool ok = false;
        V3<T> q = v3<T>(0, 0, 0), rv = q;
        T r2 = T(0);
        int p = 0, tcode = 0, par = 0;
        T ps = T(0), pt = T(0);
        if (lane < n) {
            const int s = (fh + lane) & (RING - 1);
            const auto a2 = ws.fq.ee.a2[s], d2 = ws.fq.ee.d2[s];
            const int code = (int)a2.w;
            p = code & 31;
            const int ea = (code >> 5) & 31, eb = (code >> 10) & 31;
            const SPair<T> &P = pair(p);
            const Geom &gi = geom_i(P), &gj = geo[P.gj];
            const R4 aa = tab[gi.e_off + 2 * ea], ad = tab[gi.e_off + 2 * ea + 1];
            const T inv_c = tab[gj.e_off + 2 * eb + 1].w;
            V3<T> P1, P2;
            bump<COUNT>(&pc, C_SEGSEG);
            segment_nearest<T>(xyz<T>(aa), xyz<T>(ad), ad.w, v3<T>(a2.x, a2.y, a2.z),
                               v3<T>(d2.x, d2.y, d2.z), inv_c, par_eps, (P.jref & 1) != 0, &P1, &P2,
                               &ps, &pt, &par);
            const V3<T> d = P1 - P2;
            const T rr = dot(d, d);
            if (rr < P.rc * P.rc) {
                ok = true;
                bump<COUNT>(&pc, C_TERMS);
                q = P1;
                rv = d;
                r2 = rr;
                tcode = spec_code(p, TK_EE, ea, eb, FaceHit{par, 0, 0.f});
            }
        }
        fh += n;
        __syncwarp();
        if constexpr (REF) push_spec(ok, tcode, (float)ps, (float)pt, p);
        else push_term(ok, q, rv, r2, p);
    }

    // ---- producers ----
    // one-vertex pairs (sphere / disk limit): the one central term
    __device__ __forceinline__ void sphere_terms(int nb) {
        bool ok = false;
        V3<T> q = v3<T>(0, 0, 0), rv = q;
        T r2 = T(0);
        if (lane < nb) {
            const SPair<T> &P = pair(lane);
            const Geom &gi = geom_i(P), &gj = geo[P.gj];
            if (spheres(gi, gj)) {
                q = xyz<T>(tab[gi.v_off]);
                M33<T> M;
                V3<T> dl;
                load_rows(P.row, &M, &dl);
                rv = q - (dl + mul(M, xyz<T>(tab[gj.v_off])));
                r2 = dot(rv, rv);
                ok = r2 < P.rc * P.rc;
                if (ok) bump<COUNT>(&pc, C_TERMS);
            }
        }
        if constexpr (REF) push_spec(ok, spec_code(lane, TK_SPH, 0, 0, FaceHit{0, 0, 0.f}), 0.f, 0.f, lane);
        else push_term(ok, q, rv, r2, lane);
    }

    // item offsets of the batch's pairs for a phase; returns the item count
    __device__ __forceinline__ int phase_items(int nb, bool edges) {
        int c = 0;
        if (lane < nb) {
            const SPair<T> &P = pair(lane);
            const Geom &gi = geom_i(P), &gj = geo[P.gj];
            if (!spheres(gi, gj)) {
                if (edges) {
                    if (P.eim) c = __popc(P.ejm);
                } else {
                    const unsigned oA = DIM == 3 ? P.fim : P.eim, oB = DIM == 3 ? P.fjm : P.ejm;
                    c = (oA ? __popc(P.vjm) : 0) + (oB ? __popc(P.vim) : 0);
                }
            }
        }
        int total;
        ws.boffs[lane] = warp_excl_scan(c, lane, &total);
        citems = c;
        __syncwarp();
        return total;
    }

    // the pair of item t0 + lane of the current phase (warp-collective)
    __device__ __forceinline__ int item_pair(int t0) {
        return round_owner(ws.boffs[lane], citems, t0, lane, ws.who);
    }

    // take vertex item t0 + lane (if below total): map the vertex, reach test
    __device__ __forceinline__ void load_vertex_item(int t0, int total) {
        cm = 0u;
        const int own = item_pair(t0);
        const int t = t0 + lane;
        if (t >= total) return;
        cp = own;
        const int k = t - ws.boffs[cp];
        const SPair<T> &P = pair(cp);
        const Geom &gi = geom_i(P), &gj = geo[P.gj];
        const unsigned oA = DIM == 3 ? P.fim : P.eim;
        const int nA = oA ? __popc(P.vjm) : 0;
        M33<T> M;
        V3<T> dl;
        load_rows(P.row, &M, &dl);
        crc = P.rc;
        T reach;
        unsigned m;
        if (k < nA) {
            cside = 0;
            cidx = nth_set_bit(P.vjm, k);
            va = dl + mul(M, xyz<T>(tab[gj.v_off + cidx]));
            reach = T(gi.R) + crc;
            m = oA;
            coff = DIM == 3 ? gi.f_off : gi.e_off;
        } else {
            cside = 1;
            cidx = nth_set_bit(P.vim, k - nA);
            va = mul_t(M, xyz<T>(tab[gi.v_off + cidx]) - dl);
            reach = T(gj.R) + crc;
            m = DIM == 3 ? P.fjm : P.ejm;
            coff = DIM == 3 ? gj.f_off : gj.e_off;
        }
        bump<COUNT>(&pc, C_VTX);
        if (dot(va, va) < reach * reach) cm = m;
    }

    // one face (3D: plane test, survivors queued) or edge (2D: sphere test
    // and point-segment nearest point, terms queued) of each lane's item
    __device__ __forceinline__ void vertex_step() {
        bool ok = false;
        int f = 0;
        if constexpr (DIM == 3) {
            T h = T(0);
            if (cm) {
                f = __ffs(cm) - 1;
                cm &= cm - 1u;
                const R4 nf = tab[coff + f];
                h = nf.x * va.x + nf.y * va.y + nf.z * va.z - nf.w;
                bump<COUNT>(&pc, C_PLANE);
                ok = fabs(h) < crc;
            }
            push_face(ok, va, h, cp | (cside << 5) | (cidx << 6) | (f << 11));
        } else {
            V3<T> q = v3<T>(0, 0, 0), rv = q;
            T r2 = T(0);
            T tt2 = T(0);
            int code = 0;
            if (cm) {
                f = __ffs(cm) - 1;
                cm &= cm - 1u;
                const R4 ea = tab[coff + 2 * f], ed = tab[coff + 2 * f + 1];
                const V3<T> A = xyz<T>(ea), D = xyz<T>(ed);
                const V3<T> c = A + D * T(0.5) - va;
                const T lim = ea.w + crc;
                bump<COUNT>(&pc, C_SPHERE);
                if (dot(c, c) < lim * lim) {
                    bump<COUNT>(&pc, C_PTSEG);
                    tt2 = clamp01(dot(va - A, D) * ed.w);
                    const V3<T> qq = A + D * tt2;
                    const V3<T> d = va - qq;
                    r2 = dot(d, d);
                    if (r2 < crc * crc) {
                        ok = true;
                        bump<COUNT>(&pc, C_TERMS);
                        if (cside == 0) {
                            q = qq;
                            rv = qq - va;
                            code = spec_code(cp, TK_VE_I, f, cidx, FaceHit{0, 0, 0.f});
                        } else {
                            bump<COUNT>(&pc, C_JTERMS);
                            const SPair<T> &P = pair(cp);
                            q = xyz<T>(tab[geom_i(P).v_off + cidx]);
                            rv = mul(pair_m(P), d);
                            code = spec_code(cp, TK_VE_J, cidx, f, FaceHit{0, 0, 0.f});
                        }
                    }
                }
            }
            if constexpr (REF) push_spec(ok, code, 0.f, (float)tt2, cp);
            else push_term(ok, q, rv, r2, cp);
        }
    }

    // take edge item t0 + lane (if below total): j's edge into i's frame, reach test
    __device__ __forceinline__ void load_edge_item(int t0, int total) {
        cm = 0u;
        const int own = item_pair(t0);
        const int t = t0 + lane;
        if (t >= total) return;
        cp = own;
        const SPair<T> &P = pair(cp);
        const Geom &gi = geom_i(P), &gj = geo[P.gj];
        cidx = nth_set_bit(P.ejm, t - ws.boffs[cp]);
        const R4 ba = tab[gj.e_off + 2 * cidx], bd = tab[gj.e_off + 2 * cidx + 1];
        M33<T> M;
        V3<T> dl;
        load_rows(P.row, &M, &dl);
        va = dl + mul(M, xyz<T>(ba));
        vb = mul(M, xyz<T>(bd));
        vc = va + vb * T(0.5);
        crb = ba.w;
        crc = P.rc;
        coff = gi.e_off;
        const T reach = T(gi.R) + crc + crb;
        bump<COUNT>(&pc, C_EDGE);
        if (dot(vc, vc) < reach * reach) cm = P.eim;
    }

    // one edge of i against each lane's j edge: sphere and carrier-line
    // tests, survivors queued
    __device__ __forceinline__ void edge_step() {
        bool ok = false;
        int ea = 0;
        if (cm) {
            ea = __ffs(cm) - 1;
            cm &= cm - 1u;
            const R4 aa = tab[coff + 2 * ea], ad = tab[coff + 2 * ea + 1];
            const V3<T> A1 = xyz<T>(aa), D1 = xyz<T>(ad);
            const V3<T> dc = A1 + D1 * T(0.5) - vc;
            const T lim = aa.w + crb + crc;
            bump<COUNT>(&pc, C_SPHERE);
            if (dot(dc, dc) < lim * lim) {
                const V3<T> nrm = cross(D1, vb);
                const T n2 = dot(nrm, nrm);
                const T sep = dot(va - A1, nrm);
                bump<COUNT>(&pc, C_LINE);
                ok = !(sep * sep >= crc * crc * n2 && n2 > par_eps * dot(D1, D1) * dot(vb, vb));
            }
        }
        push_edge(ok, va, vb, cp | (ea << 5) | (cidx << 10));
    }

    // the terms still queued, at the end of a group of particles
    __device__ __forceinline__ void flush_terms() {
        while (tt > th) run_terms(tt - th < 32 ? tt - th : 32);
    }

    // ---- one batch of nb queued pairs ----
    __device__ __forceinline__ void batch(int nb) {
        // phase 0: sphere terms; 1: vertex items; 2: edge items; 3: done
        int phase = 0, t0 = 0, total = 0;
        cm = 0u;
        for (;;) {
            // cm changes only in producer turns: one vote serves this turn
            const bool any_cm = __any_sync(FULL, cm);
            // (refined terms carry their pair's data and may wait for later
            // batches: flush_terms runs the rest when the group ends)
            if (tt - th >= 32 || (!REF && phase == 3 && tt > th)) {
                run_terms(tt - th < 32 ? tt - th : 32);
                continue;
            }
            const bool produced = t0 >= total && !any_cm;
            if (ft - fh >= 32 || (produced && ft > fh)) {
                const int n = ft - fh < 32 ? ft - fh : 32;
                if (DIM == 3 && phase == 2) run_segments(n);
                else run_faces(n);
                continue;
            }
            if (phase == 3) break;
            if (produced) {
                ++phase;
                if (phase == 1) {
                    sphere_terms(nb);
                    total = phase_items(nb, false);
                } else if (phase == 2) {
                    total = DIM == 3 ? phase_items(nb, true) : 0;
                } else {
                    total = 0;
                }
                t0 = 0;
                continue;
            }
            if (!any_cm) {
                if (phase == 1) load_vertex_item(t0, total);
                else load_edge_item(t0, total);
                t0 += 32;
                continue;
            }
            // producer steps while the ring they feed has room for 32 more
            // (3D steps feed the feature ring, 2D vertex steps the term ring)
            if (DIM == 3 && phase == 2) {
                do edge_step();
                while (ft - fh < 32 && __any_sync(FULL, cm));
            } else if constexpr (DIM == 3) {
                do vertex_step();
                while (ft - fh < 32 && __any_sync(FULL, cm));
            } else {
                do vertex_step();
                while (tt - th < 32 && __any_sync(FULL, cm));
            }
        }
        ph = (ph + nb) & (PR - 1);
        np -= nb;
    }
};

// ---- the list scan (shared by STAGED and the SPLIT scan kernel) ----

// Lane's particle i (or none) into the warp's scan table; returns its list
// length.
template <class T>
__device__ __forceinline__ int scan_particle(const PairArgs &a, ScanSmem<T> &ss, int lane, int i) {
    if (i >= a.n) return 0;
    const ShapeDev &shi = a.shapes[a.shape[i]];
    const M33<T> R = orientation<T>(a, i);
    SInfo<T> &pi = ss.info[lane];
    if constexpr (std::is_same<T, float>::value) {
        const float4 dd = a.delta[i];
        store_rows(pi.row, R, v3<float>(dd.x, dd.y, dd.z));
        pi.rnd = shi.rounding_f;
        pi.q = a.quatf[i];
    } else {
        const double4_32a xx = a.pos[i];
        store_rows(pi.row, R, v3<double>(xx.x, xx.y, xx.z));
        pi.rnd = shi.rounding;
        pi.q = a.quat[i];
    }
    pi.geom = shi.geom;
    pi.rep = a.rep[i];
    pi.sc = a.reps[pi.rep].sc;
    return a.nn[i];
}

// List entry t of the warp's particles base, base+1, ... (of the particle in
// lane pl): the range test and the pair setup (separating-axis test, feature
// masks).  Returns whether the pair is active; *gi is the owner's geometry.
template <class T, int DIM, bool COUNT>
__device__ __forceinline__ bool scan_entry(const PairArgs &a, const typename R4T<T>::type *tab,
                                           const int *itab, const Geom *geo, const ScanSmem<T> &ss,
                                           int base, int t, int pl, T sig_all, PairWork<T> *wk,
                                           int *gi_out, PathCount *pc) {
    const int k = t - ss.offs[pl];
    const int i = base + pl;
    const SInfo<T> &pi = ss.info[pl];
    const Geom &gi = geo[pi.geom];
    *gi_out = pi.geom;
    M33<T> Ri;
    V3<T> xi;
    load_rows(pi.row, &Ri, &xi);
    Owner<T> own;
    own.rp = &a.reps[pi.rep];
    own.sc = pi.sc;
    own.R = (T)gi.R;
    own.rnd = pi.rnd;
    own.sig_all = sig_all;
    own.geom = pi.geom;
    if constexpr (std::is_same<T, float>::value)
        own.delta = make_float4(xi.x, xi.y, xi.z, 0.f);
    else
        own.x = make_double4_32a(xi.x, xi.y, xi.z, 0.0);
    const float4 e = a.nlist[(size_t)k * a.n + i];
    bump<COUNT>(pc, C_NEIGH);
    PairGeom<T> pg;
    int j;
    if (!in_range<T>(a, e, own, &j, &pg)) return false;
    const Geom &gj = geo[pg.gj];
    bump<COUNT>(pc, C_PAIRS);
    bump<COUNT>(pc, C_FPE, defined_feature_pairs(DIM, gi, gj));
    // M = R_i^T R_j = R(conj(q_i) q_j): the relative quaternion is what
    // SPLIT's records carry, and the scan's culls use the same M
    relative_quat<T>(pi.q, quat_j<T>(a, j, pg), wk->q);
    wk->M = quat_mat<T>(wk->q[0], wk->q[1], wk->q[2], wk->q[3]);
    wk->dl = mul_t(Ri, pg.d);
    wk->sig = pg.sig;
    wk->rc = (T)WCA_CUT * pg.sig;
    wk->sig2 = pg.sig * pg.sig;
    wk->gj = pg.gj;
    wk->jref = j < i;
    wk->i = i;
    wk->j = j;
    const bool active = pair_setup<T, COUNT>(tab, itab, gi, gj, wk, pc);
    if (active) bump<COUNT>(pc, C_ACTIVE);
    return active;
}

template <class T>
__device__ __forceinline__ void store_grec(GRec<T> &G, const PairWork<T> &wk, int owner, int gi) {
    G.q[0] = wk.q[0]; G.q[1] = wk.q[1]; G.q[2] = wk.q[2]; G.q[3] = wk.q[3];
    G.dl[0] = wk.dl.x; G.dl[1] = wk.dl.y; G.dl[2] = wk.dl.z;
    G.sig = wk.sig;
    G.ids = (unsigned)gi | (unsigned)wk.gj << 8 | (unsigned)owner << 16 | (unsigned)wk.jref << 21;
    G.vim = wk.vim;
    G.vjm = wk.vjm;
    G.j = wk.j;
}

// The SPair of a GRec: M from the relative quaternion, r_cut and sigma^2
// from sigma (the expressions the scan used), the edge and face masks from
// the vertex masks (the features with a vertex in them, as pair_setup
// derives them).
template <class T>
__device__ __forceinline__ void expand_grec(SPair<T> &P, const GRec<T> &G, const Geom *geo,
                                            const int *itab) {
    const M33<T> M = quat_mat<T>(G.q[0], G.q[1], G.q[2], G.q[3]);
    store_rows(P.row, M, v3<T>(G.dl[0], G.dl[1], G.dl[2]));
    P.rc = (T)WCA_CUT * G.sig;
    P.sig2 = G.sig * G.sig;
    P.gi = (int)(G.ids & 255u);
    P.gj = (int)((G.ids >> 8) & 255u);
    P.owner = (int)((G.ids >> 16) & 31u);
    P.jref = (int)((G.ids >> 21) & 1u) | G.j << 1;
    P.vim = G.vim;
    P.vjm = G.vjm;
    const Geom &gi = geo[P.gi], &gj = geo[P.gj];
    P.eim = feature_mask(itab + gi.vem_off, G.vim);
    P.ejm = feature_mask(itab + gj.vem_off, G.vjm);
    P.fim = feature_mask(itab + gi.vfm_off, G.vim);
    P.fjm = feature_mask(itab + gj.vfm_off, G.vjm);
}

template <class T>
__device__ __forceinline__ void store_record(SPair<T> &P, const PairWork<T> &wk, int owner, int gi) {
    store_rows(P.row, wk.M, wk.dl);
    P.rc = wk.rc;
    P.sig2 = wk.sig2;
    P.gj = wk.gj;
    P.owner = owner;
    P.vim = wk.vim; P.vjm = wk.vjm; P.eim = wk.eim; P.ejm = wk.ejm;
    P.fim = wk.fim; P.fjm = wk.fjm;
    P.gi = gi;
    P.jref = wk.jref | wk.j << 1;
}

// Shared-memory tables of a pair block: geometry records, geometries, int
// table; returns the bytes they take (rounded to 128).
template <class T>
__device__ __forceinline__ size_t table_layout(const PairArgs &a, unsigned char *smem,
                                               typename R4T<T>::type **tab, Geom **geo, int **itab) {
    using R4 = typename R4T<T>::type;
    *tab = reinterpret_cast<R4 *>(smem);
    *geo = reinterpret_cast<Geom *>(*tab + a.table_len);
    *itab = reinterpret_cast<int *>(*geo + a.n_geoms);
    size_t tb = (size_t)a.table_len * sizeof(R4) + sizeof(Geom) * a.n_geoms +
                sizeof(int) * a.itable_len;
    return (tb + 127) & ~(size_t)127;
}

// FP32 + two-sum: the table's low parts follow the tables in shared memory
// (the refinement reads them for every term); returns the bytes they take.
__device__ __forceinline__ size_t stage_table_lo(const PairArgs &a, unsigned char *at,
                                                 const float4 **lo) {
    float4 *dst = reinterpret_cast<float4 *>(at);
    for (int k = threadIdx.x; k < a.table_len; k += blockDim.x) dst[k] = a.table_lo[k];
    *lo = dst;
    return ((size_t)a.table_len * sizeof(float4) + 127) & ~(size_t)127;
}
__host__ __device__ size_t table_lo_bytes(const PairArgs &a, bool ref) {
    return ref ? ((size_t)a.table_len * sizeof(float4) + 127) & ~(size_t)127 : 0;
}

// ---- STAGED: scan and batches in one kernel ----
template <class T, bool COMP, int DIM, bool COUNT>
__global__ void __launch_bounds__(SBLOCK, std::is_same<T, float>::value ? 4 : 2)
    k_pair_staged(const PairArgs a) {
    using R4 = typename R4T<T>::type;
    extern __shared__ __align__(32) unsigned char smem[];
    R4 *tab;
    Geom *geo;
    int *itab;
    size_t tb = table_layout<T>(a, smem, &tab, &geo, &itab);
    const float4 *tlo = nullptr;
    if constexpr (COMP && std::is_same<T, float>::value) tb += stage_table_lo(a, smem + tb, &tlo);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    StagedSmem<T> &ws = reinterpret_cast<StagedSmem<T> *>(smem + tb)[w];
    stage_tables<T>(a, tab, geo, itab);
    ws.b.gmask[lane] = 0u;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && !COUNT) {
        a.status->maxdisp2 = 0u;
        a.status->rebuild = 0;
    }
    const T sig_all = a.sigma > 0.0 ? (T)a.sigma : T(0);
    Staged<T, COMP, DIM, COUNT> st(a, tab, geo, itab, ws.b, lane);
    st.tab_lo = tlo;
    const int nwarps = gridDim.x * wpb;
    for (int base = (blockIdx.x * wpb + w) * 32; base < a.n; base += nwarps * 32) {
        const int i_me = base + lane;
        const int nn_me = scan_particle<T>(a, ws.s, lane, i_me);
        st.S.zero();
        st.base = base;
        int total;
        ws.s.offs[lane] = warp_excl_scan(nn_me, lane, &total);
        __syncwarp();
        // one batch call site: batches run when 32 pairs are queued and at
        // the end of the particles' lists
        int t0 = 0;
        for (;;) {
            if (st.np >= 32 || (t0 >= total && st.np > 0)) {
                st.batch(st.np < 32 ? st.np : 32);
                continue;
            }
            if (t0 >= total) break;
            const int t = t0 + lane;
            const int pl = round_owner(ws.s.offs[lane], nn_me, t0, lane, ws.s.who);
            t0 += 32;
            bool active = false;
            PairWork<T> wk;
            int gi = 0;
            if (t < total)
                active = scan_entry<T, DIM, COUNT>(a, tab, itab, geo, ws.s, base, t, pl, sig_all,
                                                   &wk, &gi, &st.pc);
            const unsigned m = __ballot_sync(FULL, active);
            if (active) store_record(ws.b.pr[ring_slot(m, lane, st.ph + st.np)], wk, pl, gi);
            st.np += __popc(m);
            __syncwarp();
        }
        st.flush_terms();
        if (i_me < a.n) {
            M33<T> R;
            V3<T> x;
            load_rows(ws.s.info[lane].row, &R, &x);
            finish_particle(a, i_me, st.S, R);
        }
        __syncwarp();
    }
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k)
            if (st.pc.v[k]) atomicAdd(a.counters + k, (unsigned long long)st.pc.v[k]);
}

// ---- SPLIT: a scan kernel writes the active pairs of each group of G
// particles to HBM (group g at recs + g G cap, in the order STAGED queues
// them), a feature kernel evaluates them.  The scan is bound by the latency
// of the neighbour gathers and runs with a small footprint at a higher
// occupancy; the feature kernel keeps the batch stages. ----
template <class T> struct ScanBlockSmem {
    ScanSmem<T> s;
    GRec<T> stage[32];                 // this chunk's active pairs, in ballot order
};

template <class T, int DIM, bool COUNT>
__global__ void __launch_bounds__(SBLOCK) k_pair_scan(const PairArgs a) {
    using R4 = typename R4T<T>::type;
    extern __shared__ __align__(32) unsigned char smem[];
    R4 *tab;
    Geom *geo;
    int *itab;
    const size_t tb = table_layout<T>(a, smem, &tab, &geo, &itab);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    ScanBlockSmem<T> &ws = reinterpret_cast<ScanBlockSmem<T> *>(smem + tb)[w];
    stage_tables<T>(a, tab, geo, itab);
    __syncthreads();
    const T sig_all = a.sigma > 0.0 ? (T)a.sigma : T(0);
    PathCount pc;
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k) pc.v[k] = 0;
    constexpr int QW = sizeof(GRec<T>) / sizeof(uint4);
    const int nwarps = gridDim.x * wpb;
    const int G = a.group;   // particles per warp (lanes G..31 hold none)
    for (int base = a.p_lo + (blockIdx.x * wpb + w) * G; base < a.p_hi; base += nwarps * G) {
        const int g = base / G;
        const int nn_me = scan_particle<T>(a, ws.s, lane, lane < G ? base + lane : a.n);
        int total;
        ws.s.offs[lane] = warp_excl_scan(nn_me, lane, &total);
        __syncwarp();
        uint4 *out = reinterpret_cast<uint4 *>(reinterpret_cast<GRec<T> *>(a.recs) +
                                               (size_t)g * G * a.cap);
        int cnt = 0;
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            const int pl = t < total ? owner_of(ws.s.offs, 32, t) : 0;
            bool active = false;
            PairWork<T> wk;
            int gi = 0;
            if (t < total)
                active = scan_entry<T, DIM, COUNT>(a, tab, itab, geo, ws.s, base, t, pl, sig_all,
                                                   &wk, &gi, &pc);
            const unsigned m = __ballot_sync(FULL, active);
            if (active) store_grec(ws.stage[__popc(m & ((1u << lane) - 1u))], wk, pl, gi);
            __syncwarp();
            // the chunk's records out, one 16-byte word per lane per round
            const uint4 *src = reinterpret_cast<const uint4 *>(ws.stage);
            const int words = __popc(m) * QW;
            for (int q = lane; q < words; q += 32) out[(size_t)cnt * QW + q] = src[q];
            cnt += __popc(m);
            __syncwarp();
        }
        if (lane == 0) a.rec_count[g] = cnt;
    }
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k)
            if (pc.v[k]) atomicAdd(a.counters + k, (unsigned long long)pc.v[k]);
}

constexpr int APPLY_PR = 32;   // the feature kernel holds one batch of records at a time

// Blocks per SM of the feature kernel: 5 in FP32 (96 registers), 2 in FP64.
// (In the FP32 + two-sum mode it only records the terms; the term kernel
// refines them.)
template <class T, bool COMP> constexpr int apply_blocks() {
    return std::is_same<T, float>::value ? 5 : 2;
}

// ---- SPLIT, FP32 + two-sum: the term kernel ----
// One warp per P consecutive particles (P / G groups of the feature kernel;
// P = 32 on large systems, down to G on small ones).  The terms of its
// groups form one pool; each chunk of up to
// TERM_CHUNK of them is put in order of term kind (stable: within a kind,
// the order the feature kernel found them), so that the lanes of a round
// mostly run the same code, and pooling keeps the rounds full when a group
// has few terms.  32 at a time the terms are refined in float-float
// (refined_values) and added by their owners' lanes in that order; then
// each lane writes its particle's outputs.  The kernel holds only this
// code, so the refinement runs out of a small instruction footprint, with
// its own registers.
constexpr int TERM_CHUNK = 256;   // terms of a warp sorted at a time

template <int DIM>
__global__ void __launch_bounds__(SBLOCK, 4) k_pair_terms(const PairArgs a) {
    extern __shared__ __align__(32) unsigned char smem[];
    float4 *tab;
    Geom *geo;
    int *itab;
    size_t tb = table_layout<float>(a, smem, &tab, &geo, &itab);
    const float4 *tlo;
    stage_table_lo(a, smem + tb, &tlo);
    stage_tables<float>(a, tab, geo, itab);
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5, w = threadIdx.x >> 5;
    int *wsm = reinterpret_cast<int *>(smem + tb + table_lo_bytes(a, true)) + (32 + 2 * TERM_CHUNK + 16) * w;
    int *gmask = wsm;                       // 32
    int *srt_r = wsm + 32;                  // TERM_CHUNK: record of the sorted term
    int *srt_o = srt_r + TERM_CHUNK;        // TERM_CHUNK: its owner (particle lane)
    int *goff = srt_o + TERM_CHUNK;         // 8 group offsets in the pool, 8 group starts
    gmask[lane] = 0;
    __syncthreads();
    const FFTab ft = {tab, tlo, itab};
    const float eps = (float)a.eps;
    const int G = a.group, P = a.term_ppw, ng = P / G;   // P particles (ng groups) per warp
    const int nwarps = gridDim.x * wpb;
    for (int base = a.p_lo + (blockIdx.x * wpb + w) * P; base < a.p_hi; base += nwarps * P) {
        SumSink<float, true> S;
        S.zero();
        // the pool: the terms of the warp's groups, group after group
        int cnt_me = 0, start_me = 0;
        if (lane < ng && base + lane * G < a.n) {
            const int g = base / G + lane;
            cnt_me = a.term_cnt[g];
            start_me = a.term_start[g];
        }
        int total;
        const int off_me = warp_excl_scan(cnt_me, lane, &total);
        if (lane < 8) {
            goff[lane] = lane < ng ? off_me : 0x7fffffff;
            goff[8 + lane] = start_me;
        }
        __syncwarp();
        for (int c0 = 0; c0 < total; c0 += TERM_CHUNK) {
            const int nc = min(TERM_CHUNK, total - c0);
            // counting sort of the chunk by term kind (stable)
            int base_k = 0;
            for (int kind = 0; kind < 8; ++kind) {   // every 3-bit kind: each term is placed
                for (int m = 0; m < nc; m += 32) {
                    const int p = c0 + m + lane;
                    bool mine = false;
                    int r = 0, h = 0;
                    if (m + lane < nc) {
                        while (h + 1 < ng && goff[h + 1] <= p) ++h;
                        r = goff[8 + h] + (p - goff[h]);
                        mine = ((__float_as_int(a.term_a[r].w) >> 5) & 7) == kind;
                    }
                    const unsigned bm = __ballot_sync(FULL, mine);
                    if (mine) {
                        const int q = base_k + __popc(bm & ((1u << lane) - 1u));
                        srt_r[q] = r;
                        srt_o[q] = h * G + (a.term_info[r] & 255);
                    }
                    base_k += __popc(bm);
                }
            }
            __syncwarp();
            for (int t0 = 0; t0 < nc; t0 += 32) {
                const bool has = t0 + lane < nc;
                int owner = 32 + lane;            // lanes without a term: distinct keys
                bool ok = false;
                ff vf[6];
                float v[7];
                if (has) {
                    const int r = srt_r[t0 + lane];
                    owner = srt_o[t0 + lane];
                    const float4 sp = a.term_a[r], sr = a.term_b[r];
                    const int code = __float_as_int(sp.w), info = a.term_info[r];
                    const TermSpec ts = {(code >> 5) & 7, (code >> 8) & 127, (code >> 15) & 127,
                                         {(code >> 26) & 1, (code >> 22) & 15, sp.y}, sp.x, sp.y,
                                         (info >> 24) & 1};
                    const FFPair fp = load_ffpair(a, base + owner, __float_as_int(sr.w));
                    ok = refined_values(ft, geo[(info >> 8) & 255], geo[(info >> 16) & 255], fp, ts,
                                        sp.z, eps, v3<float>(sr.x, sr.y, sr.z), vf, v);
                }
                if (!ok) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) vf[k] = ff_of(0.f);
#pragma unroll
                    for (int k = 0; k < 7; ++k) v[k] = 0.f;
                }
                // each owner's lane adds its terms in the round's order
                const unsigned grp = __match_any_sync(FULL, owner);
                if (has && lane == __ffs(grp) - 1) gmask[owner] = (int)grp;
                __syncwarp();
                unsigned rest = (unsigned)gmask[lane];
                const int cntm = __popc(rest);
                const int rounds = (int)__reduce_max_sync(FULL, (unsigned)cntm);
                for (int rr = 0; rr < rounds; ++rr) {
                    const int src = rest ? __ffs(rest) - 1 : lane;
                    rest &= rest - 1u;
                    ff xf[6];
                    float x[7];
#pragma unroll
                    for (int k = 0; k < 6; ++k) {
                        xf[k].h = __shfl_sync(FULL, vf[k].h, src);
                        xf[k].l = __shfl_sync(FULL, vf[k].l, src);
                    }
#pragma unroll
                    for (int k = 0; k < 7; ++k) x[k] = __shfl_sync(FULL, v[k], src);
                    if (rr < cntm) S.add_ff(xf, x);
                }
                gmask[lane] = 0;
                __syncwarp();
            }
        }
        const int i = base + lane;
        if (lane < P && i < a.n) finish_particle(a, i, S, orientation<float>(a, i));
        __syncwarp();
    }
}

template <class T, bool COMP, int DIM, bool COUNT>
__global__ void __launch_bounds__(SBLOCK, apply_blocks<T, COMP>())
    k_pair_apply(const PairArgs a) {
    using R4 = typename R4T<T>::type;
    extern __shared__ __align__(32) unsigned char smem[];
    R4 *tab;
    Geom *geo;
    int *itab;
    const size_t tb = table_layout<T>(a, smem, &tab, &geo, &itab);
    const float4 *tlo = nullptr;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    BatchSmem<T, APPLY_PR> &ws = reinterpret_cast<BatchSmem<T, APPLY_PR> *>(smem + tb)[w];
    stage_tables<T>(a, tab, geo, itab);
    ws.gmask[lane] = 0u;
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0 && !COUNT) {
        a.status->maxdisp2 = 0u;
        a.status->rebuild = 0;
    }
    constexpr bool REF = COMP && std::is_same<T, float>::value;
    Staged<T, COMP, DIM, COUNT, APPLY_PR, REF> st(a, tab, geo, itab, ws, lane);
    st.tab_lo = tlo;
    if constexpr (REF) st.region = (long long)(blockIdx.x * wpb + w) * a.term_capw;
    constexpr int QW = sizeof(GRec<T>) / sizeof(uint4);
    // the compact records land at the end of the ring's storage, from where
    // each lane expands one into its SPair slot (all reads before all writes)
    static_assert(sizeof(GRec<T>) <= sizeof(SPair<T>), "records must fit in the ring");
    static_assert(sizeof(SPair<T>) % 16 == 0, "ring slots must keep 16-byte alignment");
    GRec<T> *gbuf = reinterpret_cast<GRec<T> *>(reinterpret_cast<unsigned char *>(ws.pr) +
                                                APPLY_PR * sizeof(SPair<T>) - APPLY_PR * sizeof(GRec<T>));
    const int nwarps = gridDim.x * wpb;
    const int G = a.group;   // particles per warp (lanes G..31 own none)
    for (int base = a.p_lo + (blockIdx.x * wpb + w) * G; base < a.p_hi; base += nwarps * G) {
        const int g = base / G;
        const int cnt = a.rec_count[g];
        const uint4 *in = reinterpret_cast<const uint4 *>(reinterpret_cast<const GRec<T> *>(a.recs) +
                                                          (size_t)g * G * a.cap);
        // the records of this warp's next group into L2 while this one runs
        // (its first 32 records: one 128-byte line per lane at most)
        const int gn = g + nwarps;
        if ((long long)gn * G < a.n) {
            const int cn = min(a.rec_count[gn], 32);
            const char *nx = reinterpret_cast<const char *>(reinterpret_cast<const GRec<T> *>(a.recs) +
                                                            (size_t)gn * G * a.cap);
            const int lines = (cn * (int)sizeof(GRec<T>) + 127) / 128;
            if (lane < lines) asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + 128 * lane));
        }
        st.S.zero();
        st.base = base;
        const int gstart = st.tcur;
        for (int b0 = 0; b0 < cnt; b0 += 32) {
            const int nb = cnt - b0 < 32 ? cnt - b0 : 32;
            // records b0.. into the staging area: asynchronous 16-byte
            // global-to-shared copies, all in flight at once, then one wait
            uint4 *dst = reinterpret_cast<uint4 *>(gbuf);
            for (int q = lane; q < nb * QW; q += 32) {
                const unsigned s = (unsigned)__cvta_generic_to_shared(dst + q);
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s),
                             "l"(in + (size_t)b0 * QW + q)
                             : "memory");
            }
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
            __syncwarp();
            // the ring is empty here: the batch's pairs take slots 0 .. nb-1
            GRec<T> gr;
            if (lane < nb) gr = gbuf[lane];
            __syncwarp();
            st.ph = 0;
            if (lane < nb) expand_grec(ws.pr[lane], gr, geo, itab);
            __syncwarp();
            st.np = nb;
            st.batch(nb);
        }
        if constexpr (REF) {
            // the group's terms for the term kernel: only the records that
            // were stored (the region holds term_capw); on an overflow the
            // evaluation is redone with a larger buffer
            if (lane == 0) {
                const int stored_end = min(st.tcur, a.term_capw);
                a.term_start[g] = (int)(st.region + gstart);
                a.term_cnt[g] = max(0, stored_end - gstart);
                if (st.tcur > a.term_capw) atomicMax(&a.status->term_overflow, st.tcur);
            }
        } else {
            st.flush_terms();
            const int i_me = base + lane;
            if (lane < G && i_me < a.n) finish_particle(a, i_me, st.S, orientation<T>(a, i_me));
        }
        __syncwarp();
    }
    if constexpr (COUNT)
        for (int k = 0; k < NCOUNT; ++k)
            if (st.pc.v[k]) atomicAdd(a.counters + k, (unsigned long long)st.pc.v[k]);
}

template <class T, bool COMP, int DIM>
cudaError_t launch_dim(const PairArgs &a, bool count, size_t smem_tables, cudaStream_t s) {
    const size_t smem = ((smem_tables + 127) & ~(size_t)127) +
                        table_lo_bytes(a, COMP && std::is_same<T, float>::value) +
                        (SBLOCK / 32) * sizeof(StagedSmem<T>);
    auto launch = [&](auto kernel) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const long long need = (a.n + SBLOCK - 1) / SBLOCK;   // 32 particles per warp
        const long long cap = (long long)blocks_per_sm(kernel, SBLOCK, smem) * sm_count();
        int grid = (int)(need < cap ? need : cap);
        if (grid < 1) grid = 1;
        kernel<<<grid, SBLOCK, smem, s>>>(a);
    };
    if (count) launch(k_pair_staged<T, COMP, DIM, true>);
    else launch(k_pair_staged<T, COMP, DIM, false>);
    return cudaGetLastError();
}

template <class T, bool COMP>
cudaError_t launch_prec(const PairArgs &a, bool count, size_t smem_tables, cudaStream_t s) {
    if (a.dim == 2) return launch_dim<T, COMP, 2>(a, count, smem_tables, s);
    return launch_dim<T, COMP, 3>(a, count, smem_tables, s);
}

template <class T, bool COMP, int DIM>
cudaError_t launch_split_slice(const PairArgs &a, bool count, size_t smem_tables, cudaStream_t s) {
    const size_t t = (smem_tables + 127) & ~(size_t)127;
    const size_t smem1 = t + (SBLOCK / 32) * sizeof(ScanBlockSmem<T>);
    const size_t smem2 = t + (SBLOCK / 32) * sizeof(BatchSmem<T, APPLY_PR>);
    const int np = a.p_hi - a.p_lo;
    const int warps = (np + a.group - 1) / a.group;      // a.group particles per warp
    const long long need = (warps + SBLOCK / 32 - 1) / (SBLOCK / 32);
    auto launch = [&](auto kernel, size_t smem) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        const long long cap = (long long)blocks_per_sm(kernel, SBLOCK, smem) * sm_count();
        int grid = (int)(need < cap ? need : cap);
        if (grid < 1) grid = 1;
        kernel<<<grid, SBLOCK, smem, s>>>(a);
    };
    if (count) {
        launch(k_pair_scan<T, DIM, true>, smem1);
        launch(k_pair_apply<T, COMP, DIM, true>, smem2);
    } else {
        launch(k_pair_scan<T, DIM, false>, smem1);
        launch(k_pair_apply<T, COMP, DIM, false>, smem2);
    }
    if constexpr (COMP && std::is_same<T, float>::value) {
        // the term kernel: one warp per P particles, P = 32 when that fills
        // the resident warps, else halved down to the group size, so that a
        // small system's terms spread over more warps (the time of a warp's
        // chain of rounds sets the kernel's time there)
        const size_t smem3 = t + table_lo_bytes(a, true) + (SBLOCK / 32) * (32 + 2 * TERM_CHUNK + 16) * sizeof(int);
        auto kernel = k_pair_terms<DIM>;
        if (smem3 > 48 * 1024)
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem3);
        const long long cap3 = (long long)blocks_per_sm(kernel, SBLOCK, smem3) * sm_count();
        PairArgs b = a;
        b.term_ppw = 32;
        while (b.term_ppw > a.group && (long long)np < (long long)b.term_ppw * cap3 * (SBLOCK / 32))
            b.term_ppw >>= 1;
        const long long per_block = (long long)b.term_ppw * (SBLOCK / 32);
        const long long need3 = ((long long)np + per_block - 1) / per_block;
        int grid3 = (int)(need3 < cap3 ? need3 : cap3);
        if (grid3 < 1) grid3 = 1;
        kernel<<<grid3, SBLOCK, smem3, s>>>(b);
    }
    return cudaGetLastError();
}

// The SPLIT kernels over [0, n), slice after slice (slices of a multiple of
// 32 particles, so that no group of the scan or warp of the term kernel
// straddles two).
template <class T, bool COMP, int DIM>
cudaError_t launch_split_dim(const PairArgs &a, bool count, size_t smem_tables, cudaStream_t s) {
    const int S = a.slice > 0 ? (a.slice + 31) / 32 * 32 : a.n;
    for (int p0 = 0; p0 < a.n; p0 += S) {
        PairArgs b = a;
        b.p_lo = p0;
        b.p_hi = a.n - p0 < S ? a.n : p0 + S;
        const cudaError_t e = launch_split_slice<T, COMP, DIM>(b, count, smem_tables, s);
        if (e != cudaSuccess) return e;
        if (a.n == 0) break;
    }
    return cudaGetLastError();
}

template <class T, bool COMP>
cudaError_t launch_split_prec(const PairArgs &a, bool count, size_t smem_tables, cudaStream_t s) {
    if (a.dim == 2) return launch_split_dim<T, COMP, 2>(a, count, smem_tables, s);
    return launch_split_dim<T, COMP, 3>(a, count, smem_tables, s);
}

}  // namespace

cudaError_t launch_pair_staged(const PairArgs &a, int precision, bool count, size_t smem_tables,
                               cudaStream_t s) {
    switch (precision) {
        case DEM_FP64: return launch_prec<double, false>(a, count, smem_tables, s);
        case DEM_FP32: return launch_prec<float, false>(a, count, smem_tables, s);
        default: return launch_prec<float, true>(a, count, smem_tables, s);
    }
}

size_t pair_record_bytes(int precision) {
    return precision == DEM_FP64 ? sizeof(GRec<double>) : sizeof(GRec<float>);
}

// Particles per warp of the SPLIT kernels: 32, or fewer (16, 8, 4) while
// that leaves less than one wave of the feature kernel (five blocks of four
// warps on every SM), so that a small system spreads over the whole GPU.
int split_apply_max_warps() { return apply_blocks<float, true>() * sm_count() * (SBLOCK / 32); }

int split_group(int n) {
    const int wave = 5 * (SBLOCK / 32) * sm_count();
    int G = 32;
    while (G > 4 && (n + G - 1) / G < wave) G >>= 1;
    return G;
}

cudaError_t launch_pair_split(const PairArgs &a0, int precision, bool count, size_t smem_tables,
                              cudaStream_t s) {
    PairArgs a = a0;
    if (a.group != 4 && a.group != 8 && a.group != 16 && a.group != 32) a.group = split_group(a.n);
    switch (precision) {
        case DEM_FP64: return launch_split_prec<double, false>(a, count, smem_tables, s);
        case DEM_FP32: return launch_split_prec<float, false>(a, count, smem_tables, s);
        default: return launch_split_prec<float, true>(a, count, smem_tables, s);
    }
}

}  // namespace dem
