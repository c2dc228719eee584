// api.cu -- the C ABI of libdem (include/dem.h): context lifetime, shape
// preprocessing, state transfer and the per-step launch sequence, replayed
// as a captured CUDA graph.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "dem_internal.cuh"

using namespace dem;

namespace {

constexpr double WCA_CUT = 1.122462048309373;   // 2^(1/6)
constexpr double CELL_MARGIN = 0.05;           // fraction a box may shrink before its grid is redone
constexpr int MAX_NLIST_CAP = 768;             // list slots per particle (the build sorts in shared memory)
thread_local std::string g_create_error;

// ---------------------------------------------------------------------------
// Shape preprocessing (host)
// ---------------------------------------------------------------------------
struct HostGeom {
    int dim = 3;
    std::vector<double> v;                // nv * 3
    std::vector<std::vector<int>> faces;  // 3D
    std::vector<std::pair<int, int>> edges;
    double R = 0.0;
};

struct HostShape {
    int geom = 0;
    double rounding = 0, mass = 1, inertia[3] = {0, 0, 0};
    double R = 0;
    double volume = 0, offdiag = 0;
};

struct D3 { double x, y, z; };
static D3 d3(const double *p) { return {p[0], p[1], p[2]}; }
static D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
static D3 add(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
static D3 scl(D3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
static double dotp(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static D3 crossp(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
static double norm(D3 a) { return sqrt(dotp(a, a)); }

// Whether the closed 2D segments ab and cd share a point (crossing, touching
// or overlapping), with a tolerance relative to their lengths.
static bool segments_meet_2d(D3 a, D3 b, D3 c, D3 d) {
    auto orient = [](D3 p, D3 q, D3 r) {
        return (q.x - p.x) * (r.y - p.y) - (q.y - p.y) * (r.x - p.x);
    };
    const double tol = 1e-12 * std::max(dotp(sub(b, a), sub(b, a)), dotp(sub(d, c), sub(d, c)));
    auto sgn = [&](double v) { return v > tol ? 1 : (v < -tol ? -1 : 0); };
    auto within = [](D3 p, D3 q, D3 r) {   // r on the line pq: inside the box of pq?
        return std::min(p.x, q.x) <= r.x && r.x <= std::max(p.x, q.x) &&
               std::min(p.y, q.y) <= r.y && r.y <= std::max(p.y, q.y);
    };
    const int o1 = sgn(orient(a, b, c)), o2 = sgn(orient(a, b, d));
    const int o3 = sgn(orient(c, d, a)), o4 = sgn(orient(c, d, b));
    if (o1 * o2 < 0 && o3 * o4 < 0) return true;
    return (o1 == 0 && within(a, b, c)) || (o2 == 0 && within(a, b, d)) ||
           (o3 == 0 && within(c, d, a)) || (o4 == 0 && within(c, d, b));
}

// Validate one shape, derive its geometry (edges, circumradius) and, when
// not given, the principal moments of the uniform inner solid.  The
// integrals use the divergence theorem over a fan of simplices from the
// origin: for a tetrahedron (0, a, b, c),
//   int x x^T dV = det/120 (a a^T + b b^T + c c^T + s s^T), s = a + b + c,
// and for a triangle (0, a, b), int x x^T dA = det/24 (a a^T + b b^T + s s^T).
static int preprocess_shape(const dem_shape &s, HostGeom *g, HostShape *h, std::string *err) {
    char buf[256];
    auto fail = [&](const char *fmt, ...) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        *err = buf;
        return DEM_ERR_ARG;
    };
    if (s.dim != 2 && s.dim != 3) return fail("shape dim must be 2 or 3");
    if (s.n_verts < 1 || s.n_verts > MAX_VERTS) return fail("shape needs 1..%d vertices", MAX_VERTS);
    if (!s.verts) return fail("shape vertices missing");
    if (!(s.rounding_radius > 0.0)) return fail("rounding radius must be > 0");
    if (!(s.mass > 0.0)) return fail("mass must be > 0");
    g->dim = s.dim;
    g->v.assign(3 * s.n_verts, 0.0);
    for (int k = 0; k < s.n_verts; ++k)
        for (int a = 0; a < s.dim; ++a) {
            double x = s.verts[s.dim * k + a];
            if (!isfinite(x)) return fail("non-finite vertex");
            g->v[3 * k + a] = x;
        }
    g->R = 0.0;
    for (int k = 0; k < s.n_verts; ++k) g->R = std::max(g->R, norm(d3(&g->v[3 * k])));
    const int nv = s.n_verts;
    double I[3][3] = {{0}};
    double vol = 0.0;
    D3 cen = {0, 0, 0};
    if (s.dim == 2) {
        if (nv == 2) g->edges.push_back({0, 1});
        if (nv >= 3) {
            for (int k = 0; k < nv; ++k) g->edges.push_back({k, (k + 1) % nv});
            // simple (no two edges meet except neighbours at their shared
            // vertex) and counter-clockwise (positive area); it may be concave
            double area2 = 0.0;
            for (int k = 0; k < nv; ++k) {
                D3 a = d3(&g->v[3 * k]), b = d3(&g->v[3 * ((k + 1) % nv)]);
                area2 += a.x * b.y - a.y * b.x;
                if (!(norm(sub(b, a)) > 0.0)) return fail("2D polygon has a zero-length edge");
            }
            if (!(area2 > 0.0)) return fail("2D polygon must be counter-clockwise (positive area)");
            // no vertex where the boundary folds back on itself
            for (int k = 0; k < nv; ++k) {
                D3 m = d3(&g->v[3 * k]);
                D3 u = sub(d3(&g->v[3 * ((k + nv - 1) % nv)]), m), w = sub(d3(&g->v[3 * ((k + 1) % nv)]), m);
                if (fabs(u.x * w.y - u.y * w.x) <= 1e-12 * norm(u) * norm(w) && dotp(u, w) > 0.0)
                    return fail("2D polygon folds back on itself at vertex %d", k);
            }
            // no two edges that are not neighbours meet
            for (int k = 0; k < nv; ++k)
                for (int l = k + 2; l < nv; ++l) {
                    if (k == 0 && l == nv - 1) continue;
                    if (segments_meet_2d(d3(&g->v[3 * k]), d3(&g->v[3 * ((k + 1) % nv)]),
                                         d3(&g->v[3 * l]), d3(&g->v[3 * ((l + 1) % nv)])))
                        return fail("2D polygon must be simple (edges %d and %d meet)", k, l);
                }
            for (int k = 0; k < nv; ++k) {
                D3 a = d3(&g->v[3 * k]), b = d3(&g->v[3 * ((k + 1) % nv)]);
                double det = a.x * b.y - a.y * b.x;
                vol += det / 2.0;
                cen = add(cen, scl(add(a, b), det / 6.0));
                D3 sv = add(a, b);
                double xx = a.x * a.x + b.x * b.x + sv.x * sv.x;
                double yy = a.y * a.y + b.y * b.y + sv.y * sv.y;
                double xy = a.x * a.y + b.x * b.y + sv.x * sv.y;
                I[0][0] += det / 24.0 * yy;   // int y^2
                I[1][1] += det / 24.0 * xx;   // int x^2
                I[0][1] -= det / 24.0 * xy;
                I[2][2] += det / 24.0 * (xx + yy);
            }
        }
        if (nv == 2) {   // thin rod: I_z = m L^2 / 12 about its midpoint
            D3 a = d3(&g->v[0]), b = d3(&g->v[3]);
            double L = norm(sub(b, a));
            I[2][2] = L * L / 12.0;
            vol = 1.0;   // mass normalisation below uses the per-length measure
            cen = scl(add(a, b), 0.5);
        }
    } else {
        if (nv == 1) {
            if (s.n_faces != 0) return fail("a one-vertex 3D shape has no faces");
        } else {
            if (s.n_faces < 4 || !s.face_offsets || !s.face_verts)
                return fail("3D polyhedron needs >= 4 faces");
            for (int f = 0; f < s.n_faces; ++f) {
                int b = s.face_offsets[f], e = s.face_offsets[f + 1];
                if (e - b < 3 || e - b > MAX_FACE_VERTS)
                    return fail("face %d must have 3..%d vertices", f, MAX_FACE_VERTS);
                std::vector<int> loop;
                for (int k = b; k < e; ++k) {
                    int idx = s.face_verts[k];
                    if (idx < 0 || idx >= nv) return fail("face vertex index out of range");
                    loop.push_back(idx);
                }
                g->faces.push_back(loop);
            }
            // edges: distinct vertex pairs adjacent on a face loop
            for (auto &loop : g->faces)
                for (size_t k = 0; k < loop.size(); ++k) {
                    int a = loop[k], b = loop[(k + 1) % loop.size()];
                    std::pair<int, int> e = {std::min(a, b), std::max(a, b)};
                    if (std::find(g->edges.begin(), g->edges.end(), e) == g->edges.end())
                        g->edges.push_back(e);
                }
            if ((int)g->edges.size() > MAX_EDGES) return fail("more than %d edges", MAX_EDGES);
            if ((int)g->faces.size() > MAX_FACES) return fail("more than %d faces", MAX_FACES);
            // a closed surface with consistently oriented faces: every
            // directed face edge a->b appears once, and b->a once on another face
            {
                std::vector<std::pair<int, int>> directed;
                for (auto &loop : g->faces)
                    for (size_t k = 0; k < loop.size(); ++k)
                        directed.push_back({loop[k], loop[(k + 1) % loop.size()]});
                std::sort(directed.begin(), directed.end());
                for (size_t k = 0; k + 1 < directed.size(); ++k)
                    if (directed[k] == directed[k + 1])
                        return fail("faces are not consistently oriented (an edge is traversed "
                                    "twice in the same direction)");
                for (auto &e : directed)
                    if (!std::binary_search(directed.begin(), directed.end(),
                                            std::make_pair(e.second, e.first)))
                        return fail("polyhedron is not closed (edge %d-%d bounds one face)",
                                    e.first, e.second);
            }
            // faces planar and convex (the nearest point on a face relies on
            // it; the polyhedron itself may be concave), counter-clockwise seen
            // from outside (the enclosed volume is positive; checked below)
            double scale = g->R > 0 ? g->R : 1.0;
            for (auto &loop : g->faces) {
                size_t m = loop.size();
                D3 n = {0, 0, 0};
                for (size_t k = 0; k < m; ++k)
                    n = add(n, crossp(d3(&g->v[3 * loop[k]]), d3(&g->v[3 * loop[(k + 1) % m]])));
                double ln = norm(n);
                if (!(ln > 0)) return fail("degenerate face");
                n = scl(n, 1.0 / ln);
                D3 a0 = d3(&g->v[3 * loop[0]]);
                for (size_t k = 0; k < m; ++k)
                    if (fabs(dotp(sub(d3(&g->v[3 * loop[k]]), a0), n)) > 1e-9 * scale)
                        return fail("face is not planar");
                for (size_t k = 0; k < m; ++k) {
                    D3 p = d3(&g->v[3 * loop[k]]), q = d3(&g->v[3 * loop[(k + 1) % m]]),
                       r = d3(&g->v[3 * loop[(k + 2) % m]]);
                    if (dotp(crossp(sub(q, p), sub(r, q)), n) <= 0.0) return fail("face is not convex");
                }
                // solid integrals over the fan tetrahedra (origin, a0, a_k, a_k+1)
                for (size_t k = 1; k + 1 < m; ++k) {
                    D3 a = a0, b = d3(&g->v[3 * loop[k]]), c = d3(&g->v[3 * loop[k + 1]]);
                    double det = dotp(a, crossp(b, c));
                    vol += det / 6.0;
                    cen = add(cen, scl(add(add(a, b), c), det / 24.0));
                    D3 sv = add(add(a, b), c);
                    double P[3][3];
                    const D3 vs[4] = {a, b, c, sv};
                    for (int r_ = 0; r_ < 3; ++r_)
                        for (int c_ = 0; c_ < 3; ++c_) {
                            double acc = 0;
                            for (int t = 0; t < 4; ++t) {
                                const double *pt = &vs[t].x;
                                acc += pt[r_] * pt[c_];
                            }
                            P[r_][c_] = det / 120.0 * acc;
                        }
                    double tr = P[0][0] + P[1][1] + P[2][2];
                    for (int r_ = 0; r_ < 3; ++r_)
                        for (int c_ = 0; c_ < 3; ++c_) I[r_][c_] += (r_ == c_ ? tr : 0.0) - P[r_][c_];
                }
            }
        }
    }
    if (s.dim == 3 && nv > 1 && !(vol > 0.0))
        return fail("faces must be counter-clockwise seen from outside (enclosed volume <= 0)");
    h->R = g->R;
    h->rounding = s.rounding_radius;
    h->mass = s.mass;
    h->volume = vol;
    double off = 0.0, trace = 0.0;
    if (vol > 0.0) {
        for (int r_ = 0; r_ < 3; ++r_)
            for (int c_ = 0; c_ < 3; ++c_) I[r_][c_] *= s.mass / vol;
        cen = scl(cen, 1.0 / vol);
        off = std::max(fabs(I[0][1]), std::max(fabs(I[0][2]), fabs(I[1][2])));
        trace = I[0][0] + I[1][1] + I[2][2];
    }
    h->offdiag = off;
    if (s.inertia) {
        if (s.dim == 3) {
            for (int k = 0; k < 3; ++k) {
                if (!(s.inertia[k] >= 0.0)) return fail("inertia must be >= 0");
                h->inertia[k] = s.inertia[k];
            }
        } else {
            if (!(s.inertia[0] >= 0.0)) return fail("inertia must be >= 0");
            h->inertia[0] = h->inertia[1] = 0.0;
            h->inertia[2] = s.inertia[0];
        }
    } else {
        if (vol > 0.0 && norm(cen) > 1e-9 * (g->R > 0 ? g->R : 1.0))
            return fail("vertices must be centred on the centre of mass");
        // in 2D only I_z is used, so any body frame will do
        if (s.dim == 3 && off > 1e-9 * (trace > 0 ? trace : 1.0))
            return fail("shape is not in principal axes; pass the inertia explicitly");
        if (s.dim == 3) {
            for (int k = 0; k < 3; ++k) h->inertia[k] = I[k][k];
        } else {
            h->inertia[0] = h->inertia[1] = 0.0;
            h->inertia[2] = I[2][2];
        }
    }
    return DEM_OK;
}

bool same_geom(const HostGeom &a, const HostGeom &b) {
    return a.dim == b.dim && a.v == b.v && a.faces == b.faces;
}

}  // namespace

// The message dem_last_error(NULL) returns, for entry points without a context.
void dem::set_global_error(const std::string &msg) { g_create_error = msg; }

namespace {

// Geometry tables in the layout the pair kernels read (see Geom): FP64
// records and their FP32 copies, the int table (face ranges, and the vertex
// membership masks of every edge and face used by the separating-axis
// culls), and the per-shape records.
void build_tables(const std::vector<HostGeom> &geoms, const std::vector<HostShape> &hs,
                  HostTables *t) {
    t->td.clear(); t->itab.clear(); t->geoms.clear(); t->shapes.clear();
    t->Rmax = 0; t->rnd_max = 0;
    // one-word feature masks unless some shape has more than 32 vertices,
    // edges or faces
    t->mask_words = 1;
    for (auto &g : geoms)
        if ((int)(g.v.size() / 3) > NARROW_FEATURES || (int)g.edges.size() > NARROW_FEATURES ||
            (int)g.faces.size() > NARROW_FEATURES)
            t->mask_words = WIDE_WORDS;
    const int words = t->mask_words;
    for (auto &g : geoms) {
        Geom G = {};
        G.nv = (int)(g.v.size() / 3);
        G.ne = (int)g.edges.size();
        G.nf = (int)g.faces.size();
        // conservative (slightly enlarged) radii for the exact culls
        G.R = (float)(g.R * (1.0 + 1e-6) + 1e-7);
        t->Rmax = std::max(t->Rmax, (double)G.R);
        G.v_off = (int)t->td.size();
        for (int k = 0; k < G.nv; ++k)
            t->td.push_back(make_double4_32a(g.v[3 * k], g.v[3 * k + 1], g.v[3 * k + 2], 0.0));
        G.e_off = (int)t->td.size();
        for (auto &e : g.edges) {
            D3 a = d3(&g.v[3 * e.first]), b = d3(&g.v[3 * e.second]);
            D3 d = sub(b, a);
            double ln = norm(d);
            t->td.push_back(make_double4_32a(a.x, a.y, a.z, 0.5 * ln * (1.0 + 1e-5) + 1e-6));
            t->td.push_back(make_double4_32a(d.x, d.y, d.z, 1.0 / (ln * ln)));
        }
        G.f_off = (int)t->td.size();
        std::vector<D3> normals;
        for (auto &loop : g.faces) {
            size_t m = loop.size();
            D3 n = {0, 0, 0};
            for (size_t k = 0; k < m; ++k)
                n = add(n, crossp(d3(&g.v[3 * loop[k]]), d3(&g.v[3 * loop[(k + 1) % m]])));
            n = scl(n, 1.0 / norm(n));
            normals.push_back(n);
            t->td.push_back(make_double4_32a(n.x, n.y, n.z, dotp(n, d3(&g.v[3 * loop[0]]))));
        }
        G.fe_off = (int)t->td.size();
        G.fi_off = (int)t->itab.size();
        int nfe = 0;
        for (size_t f = 0; f < g.faces.size(); ++f) {
            auto &loop = g.faces[f];
            size_t m = loop.size();
            t->itab.push_back((int)t->td.size());
            t->itab.push_back((int)m);
            for (size_t k = 0; k < m; ++k) {
                D3 a = d3(&g.v[3 * loop[k]]), b = d3(&g.v[3 * loop[(k + 1) % m]]);
                D3 e = sub(b, a);
                D3 mm = crossp(normals[f], e);
                mm = scl(mm, 1.0 / norm(mm));
                t->td.push_back(make_double4_32a(a.x, a.y, a.z, 0.0));
                t->td.push_back(make_double4_32a(e.x, e.y, e.z, 1.0 / dotp(e, e)));
                t->td.push_back(make_double4_32a(mm.x, mm.y, mm.z, dotp(mm, a)));
                ++nfe;
            }
        }
        G.nfe = nfe;
        // incidence masks: per vertex, bit k set when the vertex bounds edge / face k
        // (rows of `words` words: feature k is bit k % 32 of word k / 32)
        G.vem_off = (int)t->itab.size();
        for (int v = 0; v < G.nv; ++v) {
            std::vector<unsigned> m(words, 0u);
            for (size_t k = 0; k < g.edges.size(); ++k)
                if (g.edges[k].first == v || g.edges[k].second == v) m[k / 32] |= 1u << (k % 32);
            for (int w = 0; w < words; ++w) t->itab.push_back((int)m[w]);
        }
        G.vfm_off = (int)t->itab.size();
        for (int v = 0; v < G.nv; ++v) {
            std::vector<unsigned> m(words, 0u);
            for (size_t f = 0; f < g.faces.size(); ++f)
                for (int u : g.faces[f])
                    if (u == v) m[f / 32] |= 1u << (f % 32);
            for (int w = 0; w < words; ++w) t->itab.push_back((int)m[w]);
        }
        t->geoms.push_back(G);
    }
    if (t->itab.empty()) { t->itab.push_back(0); t->itab.push_back(0); }
    t->tf.resize(t->td.size());
    t->tf_lo.resize(t->td.size());
    for (size_t k = 0; k < t->td.size(); ++k) {
        float4 h, l;
        split_ff(t->td[k].x, &h.x, &l.x); split_ff(t->td[k].y, &h.y, &l.y);
        split_ff(t->td[k].z, &h.z, &l.z); split_ff(t->td[k].w, &h.w, &l.w);
        t->tf[k] = h;
        t->tf_lo[k] = l;
    }
    for (auto &h : hs) {
        ShapeDev sd = {};
        sd.geom = h.geom;
        sd.R = t->geoms[h.geom].R;
        sd.rounding = h.rounding;
        split_ff(h.rounding, &sd.rounding_f, &sd.rounding_lo);
        sd.mass = h.mass;
        sd.inv_mass = 1.0 / h.mass;
        for (int k = 0; k < 3; ++k) {
            sd.inertia[k] = h.inertia[k];
            sd.inv_inertia[k] = h.inertia[k] > 0.0 ? 1.0 / h.inertia[k] : 0.0;
        }
        t->rnd_max = std::max(t->rnd_max, h.rounding);
        t->shapes.push_back(sd);
    }
}

}  // namespace

// Host copies of the geometry tables (same layout as a context's), for the
// entry point that evaluates forces without a context (noalloc.cu).
int dem::make_host_tables(const dem_shape *shapes, int n_shapes, HostTables *t,
                          std::string *err) {
    std::vector<HostGeom> geoms;
    std::vector<HostShape> hs;
    for (int s = 0; s < n_shapes; ++s) {
        HostGeom g;
        HostShape h;
        int rc = preprocess_shape(shapes[s], &g, &h, err);
        if (rc) return rc;
        if (shapes[s].dim != shapes[0].dim) { *err = "all shapes must have the same dim"; return DEM_ERR_ARG; }
        int gid = -1;
        for (size_t k = 0; k < geoms.size(); ++k)
            if (same_geom(geoms[k], g)) { gid = (int)k; break; }
        if (gid < 0) {
            if ((int)geoms.size() >= MAX_GEOMS) { *err = "too many distinct geometries"; return DEM_ERR_ARG; }
            gid = (int)geoms.size();
            geoms.push_back(g);
        }
        h.geom = gid;
        hs.push_back(h);
    }
    t->dim = shapes[0].dim;
    build_tables(geoms, hs, t);
    return DEM_OK;
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct dem_ctx {
    int dim = 3, n_shapes = 0, R = 0, N = 0, precision = DEM_FP32_COMP;
    double eps = 1.0, sigma = 0.0;
    std::vector<HostGeom> geoms;
    std::vector<HostShape> shapes;
    std::vector<int> sizes, offs;
    int max_rep = 0;                  // largest replica
    std::vector<double> box;   // R * 3
    std::vector<Rep> reps;
    std::vector<int> shape_host;
    std::vector<int> ids_in;          // dem_set_state: device shape ids copied to the host
    int n_cells = 0;
    // parameters
    double skin = -1, par_eps = 1e-6;
    int decomp = DEM_DECOMP_THREAD, block = 0, use_graph = 1, cap = 0, cell_cap = 0;
    bool cap_fixed = false;   // capacity set explicitly: grown only on overflow
    // stream / graph
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr;
    double g_dt = 0, g_kT = 0, g_tau = 0, g_P = 0, g_tauP = 0;
    int g_ens = -1;
    // thermostat / barostat parameters of the last NVT or NPT call (conserved quantity)
    double last_kT = 1.0, last_tau = 1.0, last_P = 0.0, last_tauP = 1.0;
    int last_ens = DEM_NVE;
    // barostat (dem_set_barostat) and the steps per NPT chunk
    double P = 0.0, tau_P = 0.0;
    int npt_chunk = 100;
    int split_G = 0;                  // SPLIT particles per warp (0: from N)
    int split_slice = 0;              // SPLIT particles per slice (0: all at once)
    bool split_user = false;          // split_G set by the caller (the autotuner keeps it)
    // device memory
    double4_32a *pos = nullptr, *vel = nullptr, *quat = nullptr, *angmom = nullptr;
    double4_32a *force = nullptr, *torque = nullptr, *x_last = nullptr;
    float4 *quatf = nullptr;
    float4 *quatf_lo = nullptr, *xff = nullptr;   // FP32 + two-sum: hi + lo state
    float4 *d_table_lo = nullptr;                 // FP32 + two-sum: table low parts
    int *shape = nullptr, *rep = nullptr, *nn = nullptr;
    float4 *nlist = nullptr, *delta = nullptr, *posf = nullptr;
    int *cell_count = nullptr, *cell_slots = nullptr;
    double *energy = nullptr, *virial = nullptr, *ke = nullptr, *ket = nullptr;
    void *recs = nullptr;             // SPLIT: active-pair records
    int *rec_count = nullptr;
    // SPLIT, FP32 + two-sum: the term buffer (term_capw records per warp of
    // the feature kernel) and each group's first record and count
    float4 *term_a = nullptr, *term_b = nullptr;
    int *term_info = nullptr, *term_start = nullptr, *term_cnt = nullptr;
    int term_capw = 0;
    size_t term_recs = 0;
    size_t rec_bytes = 0;
    int n_chunks = 0;                 // replica-sum chunks (SUM_CHUNK particles)
    int *chunk_rep = nullptr;
    double *partial = nullptr;        // n_chunks * 3
    double *staging = nullptr;        // N * 4 doubles
    double *red = nullptr;            // R * 6 doubles
    double *scale3 = nullptr;         // R * 3
    Status *status = nullptr;
    Thermo *thermo = nullptr;
    Rep *d_reps = nullptr;
    ShapeDev *d_shapes = nullptr;
    Geom *d_geoms = nullptr;
    void *d_table = nullptr;
    int *d_itable = nullptr;
    unsigned long long *d_counters = nullptr;
    int table_len = 0, itable_len = 0, n_geoms = 0;
    int mask_words = 1;               // WIDE_WORDS: a shape has more than 32 features
    // snapshot for the overflow retry
    double4_32a *snap = nullptr;
    Thermo *snap_thermo = nullptr;
    Rep *snap_reps = nullptr;
    bool have_state = false;
    long long rebuilds = 0;
    // kernel launches issued (a graph replay counts each of its kernels)
    long long launches = 0;
    int kernels_per_step = 0;
    // CUDA-event timing of the pair kernel inside the stepped run
    bool profile = false;
    cudaEvent_t cap_ev[2] = {nullptr, nullptr};
    cudaGraph_t graph_src = nullptr;
    cudaGraphNode_t ev_node[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> ev_pool;
    double prof_ms = 0.0;
    long long prof_n = 0;
    std::vector<float> tune_ms;   // pair-kernel ms of each autotuner candidate
    // cooperative multi-step kernel (persistent.cu): -1 = as dem_autotune
    // timed it (before that: for systems of at most COOP_AUTO_MAX_N
    // particles), 0 = never, 1 = whenever it can run
    int persistent = -1;
    int coop_auto = -1;               // -1: by size; 0 / 1: chosen by dem_autotune
    float tune_step_ms[2] = {-1.f, -1.f};   // dem_autotune: ms per step, graph / cooperative
    bool coop_used = false;           // the last dem_step ran the cooperative kernel
    double coop_wait_ms = 1000.0;     // barrier wait limit
    int coop_test_stall = 0;          // test hook: the next launch stalls one block
    CoopCtl *coop_ctl = nullptr;
    void *coop_part = nullptr;
    size_t coop_part_bytes = 0;
    unsigned char *coop_act = nullptr;
    size_t coop_act_bytes = 0;
    std::string err;
};

namespace {

int set_err(dem_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return set_err(ctx, e_ == cudaErrorMemoryAllocation ? DEM_ERR_NOMEM : DEM_ERR_CUDA, \
                           "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// Host-to-device copy ordered on the context's stream (a non-blocking stream:
// copies on the legacy stream would not be ordered with its kernels), done
// when it returns, so that the host buffer may go.
cudaError_t upload(dem_ctx *ctx, void *dst, const void *src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e;
}

template <class T> cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

void free_graph(dem_ctx *ctx) {
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    if (ctx->graph_src) cudaGraphDestroy(ctx->graph_src);
    ctx->graph = nullptr;
    ctx->graph_src = nullptr;
    ctx->ev_node[0] = ctx->ev_node[1] = nullptr;
    ctx->g_ens = -1;
}

// Upload geometry tables (FP64 and FP32 copies) and per-shape records.
int upload_tables(dem_ctx *ctx) {
    HostTables t;
    t.dim = ctx->dim;
    build_tables(ctx->geoms, ctx->shapes, &t);
    ctx->table_len = (int)t.td.size();
    ctx->itable_len = (int)t.itab.size();
    ctx->mask_words = t.mask_words;
    if (ctx->mask_words > 1) ctx->decomp = DEM_DECOMP_THREAD;
    ctx->n_geoms = (int)t.geoms.size();
    CK(dalloc(&ctx->d_geoms, t.geoms.size()));
    CK(upload(ctx, ctx->d_geoms, t.geoms.data(), sizeof(Geom) * t.geoms.size()));
    CK(dalloc(&ctx->d_itable, t.itab.size()));
    CK(upload(ctx, ctx->d_itable, t.itab.data(), sizeof(int) * t.itab.size()));
    if (ctx->precision == DEM_FP64) {
        CK(dalloc((double4_32a **)&ctx->d_table, t.td.size()));
        CK(upload(ctx, ctx->d_table, t.td.data(), sizeof(double4_32a) * t.td.size()));
    } else {
        CK(dalloc((float4 **)&ctx->d_table, t.tf.size()));
        CK(upload(ctx, ctx->d_table, t.tf.data(), sizeof(float4) * t.tf.size()));
        if (ctx->precision == DEM_FP32_COMP) {
            CK(dalloc(&ctx->d_table_lo, t.tf_lo.size()));
            CK(upload(ctx, ctx->d_table_lo, t.tf_lo.data(), sizeof(float4) * t.tf_lo.size()));
        }
    }
    CK(dalloc(&ctx->d_shapes, t.shapes.size()));
    CK(upload(ctx, ctx->d_shapes, t.shapes.data(), sizeof(ShapeDev) * t.shapes.size()));
    return DEM_OK;
}

double sigma_pair(const dem_ctx *ctx, int a, int b) {
    return ctx->sigma > 0 ? ctx->sigma : ctx->shapes[a].rounding + ctx->shapes[b].rounding;
}

double max_sigma(const dem_ctx *ctx) {
    double m = 0;
    for (int a = 0; a < ctx->n_shapes; ++a) m = std::max(m, sigma_pair(ctx, a, a));
    return m;
}

// Default neighbour-list skin: the largest sigma_ij, at most 0.4 (lengths in
// the units of the shapes).  A skin of a whole sigma for unit spheres lists
// seven times the interaction volume; 0.4 keeps rebuilds tens of steps apart
// at kT = 1, dt = 1e-3.
constexpr double SKIN_CAP = 0.4;
// Largest replica whose thermostat block sums and scales it directly.
constexpr int DIRECT_MAX = 2048;
double default_skin(const dem_ctx *ctx) { return std::min(max_sigma(ctx), SKIN_CAP); }

// Cell grids, list cutoffs and degrees of freedom of every replica (needs the
// shape of each particle).  Reallocates cell arrays and the list.
int setup_replicas(dem_ctx *ctx) {
    if (ctx->skin < 0) ctx->skin = default_skin(ctx);
    std::vector<Rep> reps(ctx->R);
    int cell_off = 0;
    double worst_ratio = 0;   // expected neighbours estimate
    double worst_cell = 0;
    for (int r = 0; r < ctx->R; ++r) {
        Rep &rp = reps[r];
        rp.off = ctx->offs[r];
        rp.n = ctx->sizes[r];
        double Rmax = 0, rnd_max = 0;
        double g = ctx->dim * (rp.n - 1.0);
        for (int i = rp.off; i < rp.off + rp.n; ++i) {
            const HostShape &sh = ctx->shapes[ctx->shape_host[i]];
            Rmax = std::max(Rmax, (double)ctx->geoms[sh.geom].R);
            rnd_max = std::max(rnd_max, sh.rounding);
            for (int k = 0; k < 3; ++k) g += sh.inertia[k] > 0.0 ? 1.0 : 0.0;
        }
        rp.g_dof = (int)g;
        double sig = ctx->sigma > 0 ? ctx->sigma : 2 * rnd_max;
        double rlist = pair_range(Rmax, sig, ctx->skin);
        double vol = 1.0;
        rp.allpairs = 0;
        for (int a = 0; a < 3; ++a) {
            rp.L[a] = a < ctx->dim ? ctx->box[3 * r + a] : 1.0;
            rp.inv_L[a] = 1.0 / rp.L[a];
            if (a < ctx->dim) {
                if (!(rp.L[a] >= 2.0 * rlist))
                    return set_err(ctx, DEM_ERR_BOX,
                                   "replica %d: box edge %g below twice the list cutoff %g", r,
                                   rp.L[a], rlist);
                // cells keep a margin so that a barostat may shrink the box by
                // CELL_MARGIN before the grid has to be rebuilt on the host
                rp.nc[a] = (int)floor(rp.L[a] * (1.0 - CELL_MARGIN) / rlist);
                if (rp.nc[a] < 3) rp.allpairs = 1;
                vol *= rp.L[a];
            } else {
                rp.nc[a] = 1;
            }
        }
        rp.r_list = rlist;
        rep_box_ff(rp);
        rp.L_build0 = rp.L[0];
        rp.sc_d = 1.0;
        rp.sc = 1.f;
        rp.disp_pad = 0.f;
        double rho = rp.n / vol;
        double expect = ctx->dim == 3 ? 4.18879 * rlist * rlist * rlist * rho : 3.14159 * rlist * rlist * rho;
        worst_ratio = std::max(worst_ratio, expect);
        if (rp.allpairs) {
            rp.nc[0] = rp.nc[1] = rp.nc[2] = 1;
            rp.cell_off = cell_off;   // no cells used
        } else {
            rp.cell_off = cell_off;
            cell_off += rp.nc[0] * rp.nc[1] * rp.nc[2];
            double cv = vol / (rp.nc[0] * rp.nc[1] * rp.nc[2]);
            worst_cell = std::max(worst_cell, rho * cv);
        }
    }
    // reduction chunks
    std::vector<int> chunk_rep;
    for (int r = 0; r < ctx->R; ++r) {
        reps[r].chunk_off = (int)chunk_rep.size();
        reps[r].n_chunk = std::max(1, (reps[r].n + SUM_CHUNK - 1) / SUM_CHUNK);
        for (int c = 0; c < reps[r].n_chunk; ++c) chunk_rep.push_back(r);
    }
    if ((int)chunk_rep.size() != ctx->n_chunks || !ctx->chunk_rep) {
        ctx->n_chunks = (int)chunk_rep.size();
        if (ctx->chunk_rep) cudaFree(ctx->chunk_rep);
        if (ctx->partial) cudaFree(ctx->partial);
        CK(dalloc(&ctx->chunk_rep, (size_t)ctx->n_chunks));
        CK(dalloc(&ctx->partial, 3 * (size_t)ctx->n_chunks));
        free_graph(ctx);
    }
    CK(upload(ctx, ctx->chunk_rep, chunk_rep.data(), sizeof(int) * ctx->n_chunks));
    ctx->reps = reps;
    int want_cap = (int)(2.0 * worst_ratio + 16);
    want_cap = (want_cap + 7) / 8 * 8;
    int want_cell = (int)(2.5 * worst_cell + 8);
    want_cap = std::min(want_cap, MAX_NLIST_CAP);
    if ((want_cap > ctx->cap && !ctx->cap_fixed) || !ctx->nlist) {
        ctx->cap = std::max(ctx->cap, ctx->cap_fixed ? 1 : want_cap);
        if (ctx->nlist) cudaFree(ctx->nlist);
        CK(dalloc(&ctx->nlist, (size_t)ctx->cap * ctx->N));
        free_graph(ctx);
    }
    if (want_cell > ctx->cell_cap || cell_off != ctx->n_cells || !ctx->cell_count) {
        ctx->cell_cap = std::max(ctx->cell_cap, want_cell);
        ctx->n_cells = cell_off;
        if (ctx->cell_count) cudaFree(ctx->cell_count);
        if (ctx->cell_slots) cudaFree(ctx->cell_slots);
        CK(dalloc(&ctx->cell_count, (size_t)std::max(cell_off, 1)));
        CK(dalloc(&ctx->cell_slots, (size_t)std::max(cell_off, 1) * ctx->cell_cap));
        free_graph(ctx);
    }
    CK(upload(ctx, ctx->d_reps, reps.data(), sizeof(Rep) * ctx->R));
    return DEM_OK;
}

// Particles per warp group of the SPLIT kernels: the one set, else from N.
int ctx_split_group(const dem_ctx *ctx) {
    return ctx->split_G > 0 ? ctx->split_G : split_group(ctx->N);
}

PairArgs pair_args(dem_ctx *ctx) {
    PairArgs a = {};
    a.n = ctx->N; a.dim = ctx->dim; a.cap = ctx->cap;
    a.pos = ctx->pos; a.quat = ctx->quat; a.quatf = ctx->quatf;
    a.shape = ctx->shape; a.rep = ctx->rep; a.reps = ctx->d_reps; a.shapes = ctx->d_shapes;
    a.geoms = ctx->d_geoms; a.n_geoms = ctx->n_geoms;
    a.table = ctx->d_table; a.table_len = ctx->table_len;
    a.itable = ctx->d_itable; a.itable_len = ctx->itable_len;
    a.nlist = ctx->nlist; a.nn = ctx->nn; a.delta = ctx->delta;
    a.force = ctx->force; a.torque = ctx->torque; a.energy = ctx->energy; a.virial = ctx->virial;
    a.eps = ctx->eps; a.sigma = ctx->sigma; a.par_eps = ctx->par_eps;
    a.status = ctx->status;
    a.counters = ctx->d_counters;
    a.recs = ctx->recs;
    a.rec_count = ctx->rec_count;
    a.group = ctx_split_group(ctx);
    a.slice = ctx->split_slice;
    a.p_lo = 0;
    a.p_hi = ctx->N;
    a.mask_words = ctx->mask_words;
    if (ctx->precision == DEM_FP32_COMP) {
        a.quatf_lo = ctx->quatf_lo;
        a.xff = ctx->xff;
        a.table_lo = ctx->d_table_lo;
        split_ff(ctx->sigma > 0 ? ctx->sigma : 0.0, &a.sigma_f, &a.sigma_lo);
        a.term_a = ctx->term_a; a.term_b = ctx->term_b; a.term_info = ctx->term_info;
        a.term_start = ctx->term_start; a.term_cnt = ctx->term_cnt;
        a.term_capw = ctx->term_capw;
    }
    return a;
}

// SPLIT decomposition: record buffers for the current list capacity (never
// allocated during a stream capture: every path that launches calls this
// first).
int ensure_recs(dem_ctx *ctx, int decomp) {
    if (decomp != DEM_DECOMP_SPLIT) return DEM_OK;
    const size_t G = (size_t)ctx_split_group(ctx);
    const size_t groups = ((size_t)ctx->N + G - 1) / G;
    const size_t need = groups * G * (size_t)ctx->cap * pair_record_bytes(ctx->precision);
    if (need > ctx->rec_bytes || !ctx->recs) {
        if (ctx->recs) cudaFree(ctx->recs);
        ctx->recs = nullptr;
        ctx->rec_bytes = 0;
        if (cudaMalloc(&ctx->recs, need) != cudaSuccess) {
            cudaGetLastError();
            return set_err(ctx, DEM_ERR_NOMEM, "SPLIT needs %zu bytes of pair records", need);
        }
        ctx->rec_bytes = need;
        free_graph(ctx);
    }
    // counts for the smallest group size, so that any group size fits
    if (!ctx->rec_count) CK(dalloc(&ctx->rec_count, ((size_t)ctx->N + 3) / 4));
    if (ctx->precision == DEM_FP32_COMP) {
        // the term buffer: a region of term_capw records per warp of the
        // feature kernel.  Start: sixteen terms per particle on average, about
        // five times what dense fluids of the shapes here produce, so that a
        // warp whose groups lie in the densest replicas fits; an overflow
        // grows it and redoes the call.
        const int maxw = split_apply_max_warps();
        if (ctx->term_capw == 0)
            ctx->term_capw = (int)std::max<long long>(512, (16LL * ctx->N + maxw - 1) / maxw);
        const size_t recs = (size_t)ctx->term_capw * maxw;
        if (recs > ctx->term_recs) {
            cudaFree(ctx->term_a); cudaFree(ctx->term_b); cudaFree(ctx->term_info);
            ctx->term_a = ctx->term_b = nullptr;
            ctx->term_info = nullptr;
            ctx->term_recs = 0;
            if (cudaMalloc(&ctx->term_a, sizeof(float4) * recs) != cudaSuccess ||
                cudaMalloc(&ctx->term_b, sizeof(float4) * recs) != cudaSuccess ||
                cudaMalloc(&ctx->term_info, sizeof(int) * recs) != cudaSuccess) {
                cudaGetLastError();
                return set_err(ctx, DEM_ERR_NOMEM, "SPLIT needs %zu term records", recs);
            }
            ctx->term_recs = recs;
            free_graph(ctx);
        }
        if (!ctx->term_start) {
            CK(dalloc(&ctx->term_start, ((size_t)ctx->N + 3) / 4));
            CK(dalloc(&ctx->term_cnt, ((size_t)ctx->N + 3) / 4));
        }
    }
    return DEM_OK;
}

NlistArgs nlist_args(dem_ctx *ctx) {
    NlistArgs a = {};
    a.n = ctx->N; a.dim = ctx->dim; a.cap = ctx->cap; a.cell_cap = ctx->cell_cap;
    a.pos = ctx->pos; a.shape = ctx->shape; a.rep = ctx->rep; a.reps = ctx->d_reps;
    a.shapes = ctx->d_shapes; a.sigma = ctx->sigma; a.skin = ctx->skin;
    a.cell_count = ctx->cell_count; a.cell_slots = ctx->cell_slots;
    a.nlist = ctx->nlist; a.nn = ctx->nn; a.x_last = ctx->x_last; a.status = ctx->status;
    a.delta = ctx->delta;
    a.half_skin2 = (float)(0.25 * ctx->skin * ctx->skin);
    a.reps_rw = ctx->d_reps;
    a.posf = ctx->posf;
    return a;
}

StepArgs step_args(dem_ctx *ctx, double dt, int ens, double kT, double tau) {
    StepArgs a = {};
    a.n = ctx->N; a.dim = ctx->dim; a.n_reps = ctx->R; a.dt = dt;
    a.nvt = ens == DEM_NVT || ens == DEM_NPT;
    a.npt = ens == DEM_NPT;
    a.P = ctx->P; a.tau_P = ctx->tau_P;
    a.kT = kT; a.tau = tau;
    a.pos = ctx->pos; a.vel = ctx->vel; a.quat = ctx->quat; a.angmom = ctx->angmom;
    a.x_last = ctx->x_last; a.quatf = ctx->quatf; a.delta = ctx->delta;
    a.force = ctx->force; a.torque = ctx->torque;
    a.shape = ctx->shape; a.rep = ctx->rep; a.reps = ctx->d_reps; a.shapes = ctx->d_shapes;
    a.ke = ctx->ke; a.thermo = ctx->thermo; a.status = ctx->status;
    a.rotor32 = ctx->precision != DEM_FP64;
    a.ket = ctx->ket; a.virial = ctx->virial; a.reps_rw = ctx->d_reps;
    a.n_chunks = ctx->n_chunks; a.chunk_rep = ctx->chunk_rep; a.partial = ctx->partial;
    // replicas of at most DIRECT_MAX particles: the thermostat kernel (one
    // block per replica) sums the kinetic energies itself and, under NVT,
    // applies the step's second scaling (the NPT kernels take the chunk
    // partials)
    a.direct_sums = !a.npt && ctx->max_rep <= DIRECT_MAX;
    a.quatf_lo = ctx->quatf_lo;
    a.xff = ctx->xff;
    // the integer-operation conversions pay where the first half step is
    // bound by the FP64 pipe, on large systems
    a.int_conv = ctx->N >= 32768;
    return a;
}

// List build (if due) and the pair kernel; e0/e1 (optional) bracket the pair
// kernel with CUDA events on the context's stream.
int launch_forces(dem_ctx *ctx, bool count, cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr) {
    NlistArgs na = nlist_args(ctx);
    CK(launch_cells(na, ctx->n_cells, ctx->stream));
    CK(launch_nlist(na, ctx->stream));
    // under stream capture the events are external records (they become
    // event-record nodes of the graph); launched directly, plain records
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (e0 || e1) CK(cudaStreamIsCapturing(ctx->stream, &cap));
    const unsigned ev_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                   : cudaEventRecordDefault;
    if (e0) CK(cudaEventRecordWithFlags(e0, ctx->stream, ev_flags));
    CK(launch_pair(pair_args(ctx), ctx->precision, ctx->decomp, ctx->block, count, ctx->stream));
    if (e1) CK(cudaEventRecordWithFlags(e1, ctx->stream, ev_flags));
    // SPLIT: scan and feature kernels, and in the FP32 + two-sum mode the term kernel
    const int slice32 = (ctx->split_slice + 31) / 32 * 32;
    const int slices = slice32 > 0 ? (ctx->N + slice32 - 1) / slice32 : 1;
    ctx->launches += 2 + (ctx->decomp == DEM_DECOMP_SPLIT
                              ? (ctx->precision == DEM_FP32_COMP ? 3 : 2) * slices : 1);
    return DEM_OK;
}

int launch_step(dem_ctx *ctx, double dt, int ens, double kT, double tau,
                cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr) {
    StepArgs sa = step_args(ctx, dt, ens, kT, tau);
    if (ens == DEM_NPT) {
        CK(launch_box(sa, ctx->stream));
        ctx->launches += 1;
    }
    CK(launch_first_half(sa, ctx->stream));
    int rc = launch_forces(ctx, false, e0, e1);
    if (rc) return rc;
    CK(launch_second_half(sa, ctx->stream));
    ctx->launches += 2;
    if (ens != DEM_NVE) {
        if (!sa.direct_sums) {
            CK(launch_chunk_sums(sa, ctx->stream));
            ctx->launches += 1;
        }
        CK(launch_thermo_end(sa, ctx->stream));
        ctx->launches += 1;
        if (!sa.direct_sums) {   // else k_thermo_end scaled the small replicas
            CK(launch_scale(sa, ctx->stream));
            ctx->launches += 1;
        }
    }
    return DEM_OK;
}

int read_status(dem_ctx *ctx, Status *st) {
    CK(cudaMemcpyAsync(st, ctx->status, sizeof(Status), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->rebuilds = st->rebuilds;
    return DEM_OK;
}

int clear_flags(dem_ctx *ctx) {
    // nlist_overflow, cell_overflow, nonfinite; box_limit; term_overflow
    CK(cudaMemsetAsync(&ctx->status->nlist_overflow, 0, 3 * sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(&ctx->status->box_limit, 0, sizeof(int), ctx->stream));
    CK(cudaMemsetAsync(&ctx->status->term_overflow, 0, sizeof(int), ctx->stream));
    return DEM_OK;
}

int force_rebuild(dem_ctx *ctx) {
    int one = 1;
    CK(cudaMemcpyAsync(&ctx->status->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

// Grow list / cell capacities after an overflow; returns 1 if grown.
int grow(dem_ctx *ctx, const Status &st, int *grown) {
    *grown = 0;
    if (st.nlist_overflow > ctx->cap) {
        if (st.nlist_overflow > MAX_NLIST_CAP)
            return set_err(ctx, DEM_ERR_NLIST_OVERFLOW,
                           "%d neighbours within the list cutoff (at most %d are supported)",
                           st.nlist_overflow, MAX_NLIST_CAP);
        ctx->cap = std::min(MAX_NLIST_CAP, (st.nlist_overflow * 3 / 2 + 7) / 8 * 8);
        cudaFree(ctx->nlist);
        CK(dalloc(&ctx->nlist, (size_t)ctx->cap * ctx->N));
        *grown = 1;
    }
    if (st.cell_overflow > ctx->cell_cap) {
        ctx->cell_cap = st.cell_overflow * 3 / 2 + 4;
        cudaFree(ctx->cell_slots);
        CK(dalloc(&ctx->cell_slots, (size_t)std::max(ctx->n_cells, 1) * ctx->cell_cap));
        *grown = 1;
    }
    if (st.term_overflow > ctx->term_capw) {
        // the next ensure_recs allocates the larger buffer
        ctx->term_capw = st.term_overflow * 3 / 2 + 64;
        *grown = 1;
    }
    if (*grown) free_graph(ctx);
    return DEM_OK;
}

// Evaluate forces at the current state; grow and redo on overflow.
int compute_forces(dem_ctx *ctx) {
    for (int attempt = 0; attempt < 4; ++attempt) {
        int rc = ensure_recs(ctx, ctx->decomp);
        if (rc) return rc;
        rc = clear_flags(ctx);
        if (rc) return rc;
        rc = launch_forces(ctx, false);
        if (rc) return rc;
        Status st;
        rc = read_status(ctx, &st);
        if (rc) return rc;
        if (st.nlist_overflow > ctx->cap || st.cell_overflow > ctx->cell_cap ||
            st.term_overflow > ctx->term_capw) {
            int grown;
            rc = grow(ctx, st, &grown);
            if (rc) return rc;
            rc = force_rebuild(ctx);
            if (rc) return rc;
            continue;
        }
        if (st.bad_input)
            return set_err(ctx, DEM_ERR_ARG, "particle %d: non-finite position, orientation, "
                           "velocity or angular momentum, or a zero quaternion", st.bad_input - 1);
        if (st.nonfinite) return set_err(ctx, DEM_ERR_NONFINITE, "non-finite force or energy");
        return DEM_OK;
    }
    return set_err(ctx, DEM_ERR_NLIST_OVERFLOW, "neighbour list kept overflowing");
}

int snapshot(dem_ctx *ctx, bool restore) {
    size_t n = (size_t)ctx->N;
    if (!ctx->snap) {
        CK(dalloc(&ctx->snap, 7 * n));
        CK(dalloc(&ctx->snap_thermo, (size_t)ctx->R));
        CK(dalloc(&ctx->snap_reps, (size_t)ctx->R));
    }
    double4_32a *arrs[7] = {ctx->pos, ctx->vel, ctx->quat, ctx->angmom, ctx->force, ctx->torque, ctx->x_last};
    for (int k = 0; k < 7; ++k) {
        if (restore)
            CK(cudaMemcpyAsync(arrs[k], ctx->snap + k * n, sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        else
            CK(cudaMemcpyAsync(ctx->snap + k * n, arrs[k], sizeof(double4_32a) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (restore) {
        CK(cudaMemcpyAsync(ctx->thermo, ctx->snap_thermo, sizeof(Thermo) * ctx->R, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_reps, ctx->snap_reps, sizeof(Rep) * ctx->R, cudaMemcpyDeviceToDevice, ctx->stream));
    } else {
        CK(cudaMemcpyAsync(ctx->snap_thermo, ctx->thermo, sizeof(Thermo) * ctx->R, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->snap_reps, ctx->d_reps, sizeof(Rep) * ctx->R, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    if (restore) {
        // the float copies of the restored state (left bit for bit as saved)
        CK(launch_refresh_copies(ctx->N, ctx->pos, ctx->quat, ctx->quatf, ctx->quatf_lo, ctx->xff,
                                 ctx->stream));
    }
    return DEM_OK;
}

// Capture one step as a CUDA graph (re-captured when the step parameters,
// buffers or the profiling switch change).  With profiling on, the graph
// carries two event-record nodes around the pair kernel; before every replay
// they are pointed at a fresh pair of events.
int get_graph(dem_ctx *ctx, double dt, int ens, double kT, double tau) {
    if (ctx->graph && ctx->g_dt == dt && ctx->g_ens == ens && ctx->g_kT == kT &&
        ctx->g_tau == tau && ctx->g_P == ctx->P && ctx->g_tauP == ctx->tau_P &&
        (ctx->ev_node[0] != nullptr) == ctx->profile)
        return DEM_OK;
    free_graph(ctx);
    if (ctx->profile && !ctx->cap_ev[0]) {
        CK(cudaEventCreate(&ctx->cap_ev[0]));
        CK(cudaEventCreate(&ctx->cap_ev[1]));
    }
    cudaGraph_t g;
    long long l0 = ctx->launches;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = ctx->profile ? launch_step(ctx, dt, ens, kT, tau, ctx->cap_ev[0], ctx->cap_ev[1])
                          : launch_step(ctx, dt, ens, kT, tau);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    ctx->launches = l0;
    if (rc) return rc;
    CK(e);
    size_t nn = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    int kernels = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        CK(cudaGraphNodeGetType(nd, &t));
        if (t == cudaGraphNodeTypeKernel) ++kernels;
        if (t == cudaGraphNodeTypeEventRecord) {
            cudaEvent_t ev;
            CK(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            if (ev == ctx->cap_ev[0]) ctx->ev_node[0] = nd;
            if (ev == ctx->cap_ev[1]) ctx->ev_node[1] = nd;
        }
    }
    ctx->kernels_per_step = kernels;
    e = cudaGraphInstantiate(&ctx->graph, g, 0);
    ctx->graph_src = g;
    CK(e);
    if (ctx->profile && (!ctx->ev_node[0] || !ctx->ev_node[1]))
        return set_err(ctx, DEM_ERR_CUDA, "profiling events missing from the captured step");
    ctx->g_dt = dt; ctx->g_ens = ens; ctx->g_kT = kT; ctx->g_tau = tau;
    ctx->g_P = ctx->P; ctx->g_tauP = ctx->tau_P;
    return DEM_OK;
}

int ensure_events(dem_ctx *ctx, size_t n) {
    while (ctx->ev_pool.size() < n) {
        cudaEvent_t ev;
        CK(cudaEventCreate(&ev));
        ctx->ev_pool.push_back(ev);
    }
    return DEM_OK;
}

bool valid(const dem_ctx *ctx) { return ctx != nullptr; }

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

int dem_shape_info(const dem_shape *shape, double *out) {
    if (!shape || !out) return DEM_ERR_ARG;
    HostGeom g;
    HostShape h;
    std::string err;
    int rc = preprocess_shape(*shape, &g, &h, &err);
    if (rc) { g_create_error = err; return rc; }
    out[0] = g.R;
    out[1] = (double)g.edges.size();
    if (shape->dim == 3) { out[2] = h.inertia[0]; out[3] = h.inertia[1]; out[4] = h.inertia[2]; }
    else { out[2] = h.inertia[2]; out[3] = 0; out[4] = 0; }
    out[5] = h.volume;
    out[6] = h.offdiag;
    return DEM_OK;
}

const char *dem_last_error(const dem_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void dem_destroy(dem_ctx *ctx) {
    if (!ctx) return;
    free_graph(ctx);
    void *ptrs[] = {ctx->pos, ctx->vel, ctx->quat, ctx->angmom, ctx->force, ctx->torque,
                    ctx->x_last, ctx->quatf, ctx->delta, ctx->shape, ctx->rep, ctx->nlist, ctx->nn,
                    ctx->cell_count, ctx->cell_slots, ctx->energy, ctx->virial, ctx->ke,
                    ctx->staging, ctx->red, ctx->scale3, ctx->status, ctx->thermo, ctx->d_reps,
                    ctx->d_shapes, ctx->d_geoms, ctx->d_table, ctx->d_itable, ctx->d_counters,
                    ctx->snap, ctx->snap_thermo, ctx->snap_reps, ctx->ket, ctx->chunk_rep,
                    ctx->partial, ctx->posf, ctx->recs, ctx->rec_count, ctx->quatf_lo, ctx->xff,
                    ctx->d_table_lo, ctx->term_a, ctx->term_b, ctx->term_info, ctx->term_start,
                    ctx->term_cnt, ctx->coop_ctl, ctx->coop_part, ctx->coop_act};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto ev : ctx->ev_pool) cudaEventDestroy(ev);
    for (auto ev : ctx->cap_ev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

int dem_create(dem_ctx **out, const dem_shape *shapes, int n_shapes, double epsilon, double sigma,
               const double *box, int n_replicas, const int *replica_sizes, int precision) {
    if (!out) return set_err(nullptr, DEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!shapes || n_shapes < 1) return set_err(nullptr, DEM_ERR_ARG, "no shapes");
    if (!box || !replica_sizes || n_replicas < 1) return set_err(nullptr, DEM_ERR_ARG, "no replicas");
    if (precision != DEM_FP64 && precision != DEM_FP32 && precision != DEM_FP32_COMP)
        return set_err(nullptr, DEM_ERR_ARG, "unknown precision %d", precision);
    if (!(epsilon > 0.0)) return set_err(nullptr, DEM_ERR_ARG, "epsilon must be > 0");
    dem_ctx *ctx = new dem_ctx();
    ctx->dim = shapes[0].dim;
    ctx->n_shapes = n_shapes;
    ctx->eps = epsilon;
    ctx->sigma = sigma > 0 ? sigma : 0.0;
    ctx->precision = precision;
    ctx->R = n_replicas;
    for (int s = 0; s < n_shapes; ++s) {
        if (shapes[s].dim != ctx->dim) {
            delete ctx;
            return set_err(nullptr, DEM_ERR_ARG, "all shapes must have the same dim");
        }
        HostGeom g;
        HostShape h;
        std::string err;
        int rc = preprocess_shape(shapes[s], &g, &h, &err);
        if (rc) {
            delete ctx;
            return set_err(nullptr, rc, "shape %d: %s", s, err.c_str());
        }
        int gid = -1;
        for (size_t k = 0; k < ctx->geoms.size(); ++k)
            if (same_geom(ctx->geoms[k], g)) { gid = (int)k; break; }
        if (gid < 0) {
            if ((int)ctx->geoms.size() >= MAX_GEOMS) {
                delete ctx;
                return set_err(nullptr, DEM_ERR_ARG, "more than %d distinct geometries", MAX_GEOMS);
            }
            gid = (int)ctx->geoms.size();
            ctx->geoms.push_back(g);
        }
        h.geom = gid;
        ctx->shapes.push_back(h);
    }
    int N = 0;
    for (int r = 0; r < n_replicas; ++r) {
        if (replica_sizes[r] < 1) {
            delete ctx;
            return set_err(nullptr, DEM_ERR_ARG, "replica %d is empty", r);
        }
        ctx->offs.push_back(N);
        ctx->sizes.push_back(replica_sizes[r]);
        ctx->max_rep = std::max(ctx->max_rep, replica_sizes[r]);
        N += replica_sizes[r];
        for (int a = 0; a < 3; ++a) {
            double L = a < ctx->dim ? box[ctx->dim * r + a] : 1.0;
            if (!(L > 0.0) || !isfinite(L)) {
                delete ctx;
                return set_err(nullptr, DEM_ERR_ARG, "replica %d: bad box", r);
            }
            ctx->box.push_back(L);
        }
    }
    ctx->N = N;
    // device buffers
    int rc = [&]() -> int {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
        size_t n = N;
        CK(dalloc(&ctx->pos, n)); CK(dalloc(&ctx->vel, n)); CK(dalloc(&ctx->quat, n));
        CK(dalloc(&ctx->angmom, n)); CK(dalloc(&ctx->force, n)); CK(dalloc(&ctx->torque, n));
        CK(dalloc(&ctx->x_last, n)); CK(dalloc(&ctx->quatf, n)); CK(dalloc(&ctx->delta, n));
        CK(dalloc(&ctx->posf, n));
        if (ctx->precision == DEM_FP32_COMP) {
            CK(dalloc(&ctx->quatf_lo, n));
            CK(dalloc(&ctx->xff, 2 * n));
        }
        CK(cudaMemsetAsync(ctx->delta, 0, sizeof(float4) * n, ctx->stream));
        CK(dalloc(&ctx->shape, n)); CK(dalloc(&ctx->rep, n)); CK(dalloc(&ctx->nn, n));
        CK(dalloc(&ctx->energy, n)); CK(dalloc(&ctx->virial, 6 * n)); CK(dalloc(&ctx->ke, n)); CK(dalloc(&ctx->ket, n));
        CK(dalloc(&ctx->staging, 4 * n));
        CK(dalloc(&ctx->red, 6 * (size_t)ctx->R)); CK(dalloc(&ctx->scale3, 3 * (size_t)ctx->R));
        CK(dalloc(&ctx->status, 1)); CK(dalloc(&ctx->thermo, (size_t)ctx->R));
        CK(dalloc(&ctx->d_reps, (size_t)ctx->R)); CK(dalloc(&ctx->d_counters, DEM_N_COUNTERS));
        CK(cudaMemsetAsync(ctx->status, 0, sizeof(Status), ctx->stream));
        CK(cudaMemsetAsync(ctx->thermo, 0, sizeof(Thermo) * ctx->R, ctx->stream));
        CK(cudaMemsetAsync(ctx->nn, 0, sizeof(int) * n, ctx->stream));
        CK(cudaMemsetAsync(ctx->force, 0, sizeof(double4_32a) * n, ctx->stream));
        CK(cudaMemsetAsync(ctx->torque, 0, sizeof(double4_32a) * n, ctx->stream));
        std::vector<int> rep(n);
        for (int r = 0; r < ctx->R; ++r)
            for (int k = 0; k < ctx->sizes[r]; ++k) rep[ctx->offs[r] + k] = r;
        CK(upload(ctx, ctx->rep, rep.data(), sizeof(int) * n));
        return upload_tables(ctx);
    }();
    if (rc) {
        std::string e = ctx->err;
        dem_destroy(ctx);
        return set_err(nullptr, rc, "%s", e.c_str());
    }
    *out = ctx;
    return DEM_OK;
}

int dem_set_stream(dem_ctx *ctx, void *stream) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    ctx->own_stream = false;
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    free_graph(ctx);
    return DEM_OK;
}

int dem_set_param(dem_ctx *ctx, const char *name, double value) {
    if (!valid(ctx) || !name) return DEM_ERR_ARG;
    std::string n(name);
    if (n == "skin") {
        if (!(value > 0)) return set_err(ctx, DEM_ERR_ARG, "skin must be > 0");
        ctx->skin = value;
        if (ctx->have_state) {
            int rc = setup_replicas(ctx);
            if (rc) return rc;
            rc = force_rebuild(ctx);
            if (rc) return rc;
        }
    } else if (n == "npt_chunk") {
        if (!(value >= 1) || value > 1e9) return set_err(ctx, DEM_ERR_ARG, "npt_chunk must be >= 1");
        ctx->npt_chunk = (int)value;
    } else if (n == "split_group") {
        const int G = (int)value;
        if (value != (double)G || (G != 0 && G != 4 && G != 8 && G != 16 && G != 32))
            return set_err(ctx, DEM_ERR_ARG, "split_group must be 0, 4, 8, 16 or 32");
        ctx->split_G = G;
        ctx->split_user = G != 0;
    } else if (n == "par_eps") {
        if (!(value >= 0)) return set_err(ctx, DEM_ERR_ARG, "par_eps must be >= 0");
        ctx->par_eps = value;
    } else if (n == "decomp") {
        int d = (int)value;
        if (d < DEM_DECOMP_AUTO || d > DEM_DECOMP_SPLIT) return set_err(ctx, DEM_ERR_ARG, "bad decomp");
        if (ctx->mask_words > 1 && d != DEM_DECOMP_AUTO && d != DEM_DECOMP_THREAD)
            return set_err(ctx, DEM_ERR_ARG, "shapes with more than 32 vertices, edges or faces "
                           "run the THREAD decomposition only");
        ctx->decomp = d == DEM_DECOMP_AUTO ? DEM_DECOMP_THREAD : d;
    } else if (n == "block") {
        int b = (int)value;
        if (b < 0 || b > 1024 || b % 32) return set_err(ctx, DEM_ERR_ARG, "bad block");
        ctx->block = b;
    } else if (n == "graph") {
        ctx->use_graph = value != 0;
    } else if (n == "profile") {
        ctx->profile = value != 0;
        ctx->prof_ms = 0.0;
        ctx->prof_n = 0;
    } else if (n == "nlist_cap") {
        int c = (int)value;
        if (c < 1 || c > MAX_NLIST_CAP) return set_err(ctx, DEM_ERR_ARG, "bad nlist_cap");
        ctx->cap = c;
        ctx->cap_fixed = true;
        if (ctx->nlist) cudaFree(ctx->nlist);
        ctx->nlist = nullptr;
        CK(dalloc(&ctx->nlist, (size_t)ctx->cap * ctx->N));
        if (ctx->have_state) {
            int rc = force_rebuild(ctx);
            if (rc) return rc;
        }
    } else if (n == "persistent") {
        int v = (int)value;
        if (v < -1 || v > 1) return set_err(ctx, DEM_ERR_ARG, "bad persistent (-1, 0 or 1)");
        if (v == 1 && ctx->mask_words > 1)
            return set_err(ctx, DEM_ERR_ARG, "the cooperative step kernel takes shapes of at "
                           "most 32 vertices, edges and faces");
        ctx->persistent = v;
        ctx->coop_auto = -1;
    } else if (n == "persistent_wait_ms") {
        if (!(value >= 1.0 && value <= 10000.0))
            return set_err(ctx, DEM_ERR_ARG, "persistent_wait_ms must be in [1, 10000]");
        ctx->coop_wait_ms = value;
    } else if (n == "persistent_test_stall") {
        ctx->coop_test_stall = value != 0;
    } else if (n == "split_slice") {
        if (!(value >= 0 && value <= 1e9)) return set_err(ctx, DEM_ERR_ARG, "bad split_slice");
        ctx->split_slice = (int)value;
    } else if (n == "term_cap") {
        int c = (int)value;
        if (c < 1 || c > (1 << 24)) return set_err(ctx, DEM_ERR_ARG, "bad term_cap");
        ctx->term_capw = c;
        cudaFree(ctx->term_a); cudaFree(ctx->term_b); cudaFree(ctx->term_info);
        ctx->term_a = ctx->term_b = nullptr;
        ctx->term_info = nullptr;
        ctx->term_recs = 0;
    } else {
        return set_err(ctx, DEM_ERR_ARG, "unknown parameter '%s'", name);
    }
    free_graph(ctx);
    return DEM_OK;
}

int dem_get_param(dem_ctx *ctx, const char *name, double *value) {
    if (!valid(ctx) || !name || !value) return DEM_ERR_ARG;
    std::string n(name);
    if (n == "skin") *value = ctx->skin < 0 ? default_skin(ctx) : ctx->skin;
    else if (n == "par_eps") *value = ctx->par_eps;
    else if (n == "npt_chunk") *value = ctx->npt_chunk;
    else if (n == "split_group") *value = ctx_split_group(ctx);
    else if (n == "decomp") *value = ctx->decomp;
    else if (n == "block") *value = ctx->block;
    else if (n == "graph") *value = ctx->use_graph;
    else if (n == "profile") *value = ctx->profile;
    else if (n == "pair_ms_total") *value = ctx->prof_ms;
    else if (n == "pair_launches") *value = (double)ctx->prof_n;
    else if (n == "launches") *value = (double)ctx->launches;
    else if (n.rfind("autotune_ms_", 0) == 0) {
        size_t k = (size_t)atoi(n.c_str() + 12);
        if (k >= ctx->tune_ms.size()) return set_err(ctx, DEM_ERR_ARG, "no such autotune result");
        *value = ctx->tune_ms[k];
    }
    else if (n == "nlist_cap") *value = ctx->cap;
    else if (n == "term_cap") *value = ctx->term_capw;
    else if (n == "split_slice") *value = ctx->split_slice;
    else if (n == "persistent") *value = ctx->persistent;
    else if (n == "persistent_used") *value = ctx->coop_used;
    else if (n == "persistent_auto") *value = ctx->coop_auto;
    else if (n == "autotune_step_ms_graph") *value = ctx->tune_step_ms[0];
    else if (n == "autotune_step_ms_persistent") *value = ctx->tune_step_ms[1];
    else if (n == "persistent_wait_ms") *value = ctx->coop_wait_ms;
    else if (n == "n_cells") *value = ctx->n_cells;
    else if (n == "allpairs_replicas") {
        int k = 0;
        for (auto &r : ctx->reps) k += r.allpairs;
        *value = k;
    } else return set_err(ctx, DEM_ERR_ARG, "unknown parameter '%s'", name);
    return DEM_OK;
}

int dem_set_state(dem_ctx *ctx, const int *shape_id, const double *pos, const double *orient,
                  const double *vel, const double *angmom, int device_ptrs) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!shape_id || !pos || !orient || !vel || !angmom)
        return set_err(ctx, DEM_ERR_ARG, "dem_set_state: all arrays are required");
    const size_t n = ctx->N;
    const int dim = ctx->dim;
    const int *ids = shape_id;
    if (device_ptrs) {
        ctx->ids_in.resize(n);
        CK(cudaMemcpyAsync(ctx->ids_in.data(), shape_id, sizeof(int) * n, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ids = ctx->ids_in.data();
    }
    // The same shape of every particle keeps the replica tables, the cell grid
    // and the neighbour list: the list stays valid while every particle is
    // within skin/2 of its position at the build, which the device tests
    // below as in a step.  New shapes rebuild everything.  (One pass: range
    // check and comparison.)
    bool same_shapes = ctx->have_state && ctx->shape_host.size() == n;
    for (size_t i = 0; i < n; ++i) {
        const int v = ids[i];
        if (v < 0 || v >= ctx->n_shapes)
            return set_err(ctx, DEM_ERR_ARG, "shape_id[%zu] out of range", i);
        same_shapes = same_shapes && v == ctx->shape_host[i];
    }
    int rc = DEM_OK;
    if (!same_shapes) {
        ctx->shape_host.assign(ids, ids + n);
        CK(cudaMemcpyAsync(ctx->shape, ctx->shape_host.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
        rc = setup_replicas(ctx);
        if (rc) return rc;
    }
    const int odim = dim == 3 ? 4 : 1, adim = dim == 3 ? 3 : 1;
    // the import kernels record a non-finite value or a zero quaternion here
    CK(cudaMemsetAsync(&ctx->status->bad_input, 0, sizeof(int), ctx->stream));
    ctx->have_state = false;
    const double *src[4] = {pos, orient, vel, angmom};
    const int widths[4] = {dim, odim, dim, adim};
    const double *dsrc[4];
    if (device_ptrs) {
        for (int k = 0; k < 4; ++k) dsrc[k] = src[k];
        CK(launch_import_state((int)n, dim, dsrc[0], dsrc[1], dsrc[2], dsrc[3], ctx->pos, ctx->quat,
                               ctx->vel, ctx->angmom, ctx->status, ctx->stream));
    } else {
        // the four arrays go through the staging buffer one at a time
        double *stage = ctx->staging;
        for (int k = 0; k < 4; ++k) {
            CK(cudaMemcpyAsync(stage, src[k], sizeof(double) * widths[k] * n, cudaMemcpyHostToDevice, ctx->stream));
            const double *p[4] = {nullptr, nullptr, nullptr, nullptr};
            p[k] = stage;
            // import only the array just staged: the others keep their values
            CK(launch_import_state((int)n, dim, k == 0 ? stage : nullptr, k == 1 ? stage : nullptr,
                                   k == 2 ? stage : nullptr, k == 3 ? stage : nullptr, ctx->pos,
                                   ctx->quat, ctx->vel, ctx->angmom, ctx->status, ctx->stream));
        }
    }
    CK(launch_prepare_state((int)n, dim, ctx->pos, ctx->quat, ctx->quatf, ctx->quatf_lo,
                            ctx->xff, ctx->angmom, ctx->rep,
                            ctx->d_reps, 1, ctx->stream));
    CK(cudaMemsetAsync(ctx->thermo, 0, sizeof(Thermo) * ctx->R, ctx->stream));
    if (same_shapes) {
        StepArgs da = step_args(ctx, 0.0, DEM_NVE, 1.0, 1.0);
        CK(launch_displacement(da, ctx->stream));
    } else {
        rc = force_rebuild(ctx);
        if (rc) return rc;
    }
    ctx->have_state = true;
    rc = compute_forces(ctx);
    if (rc) {
        // a rejected input or non-finite forces leave no usable state: steps
        // return DEM_ERR_STATE until a valid dem_set_state, which rebuilds
        ctx->have_state = false;
        return rc;
    }
    StepArgs sa = step_args(ctx, 0.0, DEM_NVE, 1.0, 1.0);
    CK(launch_kinetic(sa, ctx->stream));
    if (!sa.direct_sums) CK(launch_chunk_sums(sa, ctx->stream));
    CK(launch_thermo_end(sa, ctx->stream));   // NVE branch: stores K per replica
    CK(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

int dem_get_state(dem_ctx *ctx, double *pos, double *orient, double *vel, double *angmom,
                  double *thermostat, int device_ptrs) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    const size_t n = ctx->N;
    const int dim = ctx->dim, odim = dim == 3 ? 4 : 1, adim = dim == 3 ? 3 : 1;
    double *dst[4] = {pos, orient, vel, angmom};
    const int widths[4] = {dim, odim, dim, adim};
    for (int k = 0; k < 4; ++k) {
        if (!dst[k]) continue;
        double *target = device_ptrs ? dst[k] : ctx->staging;
        CK(launch_export_state((int)n, dim, ctx->pos, ctx->quat, ctx->vel, ctx->angmom,
                               k == 0 ? target : nullptr, k == 1 ? target : nullptr,
                               k == 2 ? target : nullptr, k == 3 ? target : nullptr, ctx->stream));
        if (!device_ptrs)
            CK(cudaMemcpyAsync(dst[k], ctx->staging, sizeof(double) * widths[k] * n, cudaMemcpyDeviceToHost, ctx->stream));
    }
    if (thermostat) {
        std::vector<Thermo> th(ctx->R);
        CK(cudaMemcpyAsync(th.data(), ctx->thermo, sizeof(Thermo) * ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int r = 0; r < ctx->R; ++r) {
            thermostat[3 * r] = th[r].xi;
            thermostat[3 * r + 1] = th[r].eta;
            thermostat[3 * r + 2] = th[r].pe;
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

int dem_set_thermostat(dem_ctx *ctx, const double *thermostat) {
    if (!valid(ctx) || !thermostat) return DEM_ERR_ARG;
    std::vector<Thermo> th(ctx->R);
    CK(cudaMemcpyAsync(th.data(), ctx->thermo, sizeof(Thermo) * ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < ctx->R; ++r) {
        th[r].xi = thermostat[3 * r];
        th[r].eta = thermostat[3 * r + 1];
        th[r].pe = thermostat[3 * r + 2];
    }
    CK(cudaMemcpyAsync(ctx->thermo, th.data(), sizeof(Thermo) * ctx->R, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

int dem_compute(dem_ctx *ctx) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    return compute_forces(ctx);
}

}  // extern "C"

namespace {

// n steps with no host work in between (graph replays or launches), with the
// overflow retry: the state is snapshotted, and after a list or cell overflow
// the capacities grow and the steps are replayed from the snapshot.
// ---- cooperative multi-step kernel ----
constexpr int COOP_AUTO_MAX_N = 2048;    // before dem_autotune has timed both
constexpr int COOP_TUNE_MAX_N = 65536;   // dem_autotune times it up to this size

// Whether dem_step runs the cooperative kernel (NVE and NVT, one-word
// feature masks, no pair-kernel profiling), and its grid (0: it cannot run).
int coop_plan(dem_ctx *ctx, int ensemble) {
    if (ctx->persistent == 0 || ensemble == DEM_NPT || ctx->mask_words != 1 || ctx->profile)
        return 0;
    if (ctx->persistent < 0 &&
        (ctx->coop_auto == 0 || (ctx->coop_auto < 0 && ctx->N > COOP_AUTO_MAX_N)))
        return 0;
    PairArgs pa = pair_args(ctx);
    return coop_grid(ctx->precision, ctx->dim, ctx->N, ctx->cap, pair_smem_bytes(pa, ctx->precision));
}

int ensure_coop(dem_ctx *ctx) {
    if (!ctx->coop_ctl) CK(dalloc(&ctx->coop_ctl, 1));
    const size_t pb = coop_partial_bytes(ctx->precision, ctx->N, ctx->cap);
    if (pb > ctx->coop_part_bytes) {
        cudaFree(ctx->coop_part);
        ctx->coop_part = nullptr;
        ctx->coop_part_bytes = 0;
        CK(cudaMalloc(&ctx->coop_part, pb));
        ctx->coop_part_bytes = pb;
    }
    const size_t ab = (size_t)ctx->cap * ctx->N;
    if (ab > ctx->coop_act_bytes) {
        cudaFree(ctx->coop_act);
        ctx->coop_act = nullptr;
        ctx->coop_act_bytes = 0;
        CK(cudaMalloc((void **)&ctx->coop_act, ab));
        ctx->coop_act_bytes = ab;
    }
    return DEM_OK;
}

// n steps in cooperative launches.  A launch runs until its steps are done
// or a list rebuild is due after some step's first half; then the list is
// rebuilt here and the next launch starts at that step's pair phase.
int coop_run(dem_ctx *ctx, int grid, int n, double dt, int ensemble, double kT, double tau_T) {
    int rc = ensure_coop(ctx);
    if (rc) return rc;
    const PairArgs pa = pair_args(ctx);
    const NlistArgs na = nlist_args(ctx);
    const size_t smem = pair_smem_bytes(pa, ctx->precision);
    int remaining = n, resume = 0;
    while (remaining > 0) {
        CK(cudaMemsetAsync(ctx->coop_ctl, 0, sizeof(CoopCtl), ctx->stream));
        CoopArgs c = {};
        c.p = pa;
        c.s = step_args(ctx, dt, ensemble, kT, tau_T);
        c.ctl = ctx->coop_ctl;
        c.part = ctx->coop_part;
        c.act = ctx->coop_act;
        c.n_steps = remaining;
        c.resume = resume;
        c.half_skin2 = na.half_skin2;
        c.limit_ns = (long long)(ctx->coop_wait_ms * 1e6);
        c.test_stall = ctx->coop_test_stall;
        ctx->coop_test_stall = 0;
        CK(launch_coop_steps(c, ctx->precision, ctx->dim, grid, smem, ctx->stream));
        ctx->launches += 1;
        CoopCtl h;
        CK(cudaMemcpyAsync(&h, ctx->coop_ctl, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (h.timeout || h.abort)
            return set_err(ctx, DEM_ERR_TIMEOUT, "a barrier of the cooperative step kernel waited "
                           "more than %.0f ms", ctx->coop_wait_ms);
        if (h.stop != 1) {
            if (h.steps_done != remaining)
                return set_err(ctx, DEM_ERR_CUDA, "the cooperative step kernel ended after %d of "
                               "%d steps", h.steps_done, remaining);
            break;
        }
        // the list build of the step whose first half just ran
        CK(launch_cells(na, ctx->n_cells, ctx->stream));
        CK(launch_nlist(na, ctx->stream));
        ctx->launches += 2;
        remaining -= h.steps_done;
        resume = 1;
    }
    return DEM_OK;
}

int step_run(dem_ctx *ctx, int n, double dt, int ensemble, double kT, double tau_T) {
    int rc;
    for (int attempt = 0; attempt < 4; ++attempt) {
        rc = ensure_recs(ctx, ctx->decomp);
        if (rc) return rc;
        rc = snapshot(ctx, false);
        if (rc) return rc;
        rc = clear_flags(ctx);
        if (rc) return rc;
        StepArgs sa = step_args(ctx, dt, ensemble, kT, tau_T);
        if (ensemble == DEM_NPT) {
            CK(launch_kinetic(sa, ctx->stream));
            CK(launch_chunk_sums(sa, ctx->stream));
            ctx->launches += 2;
        }
        if (ensemble != DEM_NVE) {
            CK(launch_thermo_begin(sa, ctx->stream));
            ctx->launches += 1;
        }
        if (ctx->profile) {
            rc = ensure_events(ctx, 2 * (size_t)n);
            if (rc) return rc;
        }
        const int coop = coop_plan(ctx, ensemble);
        ctx->coop_used = coop > 0;
        if (coop > 0) {
            rc = coop_run(ctx, coop, n, dt, ensemble, kT, tau_T);
            if (rc == DEM_ERR_TIMEOUT) {
                // the state from before the call, with its list and forces
                const std::string msg = ctx->err;
                if (snapshot(ctx, true) == DEM_OK && force_rebuild(ctx) == DEM_OK)
                    compute_forces(ctx);
                ctx->err = msg;
                return DEM_ERR_TIMEOUT;
            }
            if (rc) return rc;
        } else if (ctx->use_graph) {
            rc = get_graph(ctx, dt, ensemble, kT, tau_T);
            if (rc) return rc;
            for (int s = 0; s < n; ++s) {
                if (ctx->profile) {
                    CK(cudaGraphExecEventRecordNodeSetEvent(ctx->graph, ctx->ev_node[0], ctx->ev_pool[2 * s]));
                    CK(cudaGraphExecEventRecordNodeSetEvent(ctx->graph, ctx->ev_node[1], ctx->ev_pool[2 * s + 1]));
                }
                CK(cudaGraphLaunch(ctx->graph, ctx->stream));
            }
            ctx->launches += (long long)n * ctx->kernels_per_step;
        } else {
            for (int s = 0; s < n; ++s) {
                rc = ctx->profile ? launch_step(ctx, dt, ensemble, kT, tau_T, ctx->ev_pool[2 * s],
                                                ctx->ev_pool[2 * s + 1])
                                  : launch_step(ctx, dt, ensemble, kT, tau_T);
                if (rc) return rc;
            }
        }
        Status st;
        rc = read_status(ctx, &st);
        if (rc) return rc;
        if (ctx->profile) {
            for (int s = 0; s < n; ++s) {
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, ctx->ev_pool[2 * s], ctx->ev_pool[2 * s + 1]));
                ctx->prof_ms += ms;
            }
            ctx->prof_n += n;
        }
        if (st.nlist_overflow > ctx->cap || st.cell_overflow > ctx->cell_cap ||
            st.term_overflow > ctx->term_capw) {
            int grown;
            rc = grow(ctx, st, &grown);
            if (rc) return rc;
            rc = snapshot(ctx, true);
            if (rc) return rc;
            rc = force_rebuild(ctx);
            if (rc) return rc;
            rc = compute_forces(ctx);
            if (rc) return rc;
            continue;
        }
        if (st.nonfinite) return set_err(ctx, DEM_ERR_NONFINITE, "non-finite force or energy");
        if (st.box_limit)
            return set_err(ctx, DEM_ERR_BOX,
                           "a barostat moved a box beyond its cell grid or below twice the list "
                           "cutoff within %d steps (lower the npt_chunk parameter)", n);
        return DEM_OK;
    }
    return set_err(ctx, DEM_ERR_NLIST_OVERFLOW, "neighbour list kept overflowing");
}

// The per-step kernels (graph replays) against the cooperative multi-step
// kernel: a few NVT steps of each from the same state, timed with CUDA
// events, then the state from before.  The steps are short (dt = 1e-6), so
// neither run rebuilds its list.
int tune_persistent(dem_ctx *ctx, cudaEvent_t e0, cudaEvent_t e1) {
    ctx->tune_step_ms[0] = ctx->tune_step_ms[1] = -1.f;
    if (ctx->N > COOP_TUNE_MAX_N) {
        // a thread per list entry cannot compete at this size (each would
        // take many entries in turn); not worth its partial-sum buffer
        ctx->coop_auto = 0;
        return DEM_OK;
    }
    if (ctx->mask_words != 1 || ctx->profile || coop_grid(ctx->precision, ctx->dim, ctx->N, ctx->cap,
                                                         pair_smem_bytes(pair_args(ctx), ctx->precision)) < 1)
        return DEM_OK;
    const double dt = 1e-6, kT = 1.0, tau = 1.0;
    const int warm = 2, steps = 20;
    int rc = snapshot(ctx, false);
    if (rc) return rc;
    struct KeepPersistent {   // the setting comes back however this returns
        dem_ctx *c;
        int v;
        ~KeepPersistent() { c->persistent = v; }
    } keep{ctx, ctx->persistent};
    float ms[2] = {-1.f, -1.f};
    for (int mode = 0; mode < 2 && rc == DEM_OK; ++mode) {
        ctx->persistent = mode;
        rc = step_run(ctx, warm, dt, DEM_NVT, kT, tau);
        if (rc == DEM_OK) rc = snapshot(ctx, true);   // back to the state before the warm-up
        if (rc != DEM_OK) break;
        CK(cudaEventRecord(e0, ctx->stream));
        rc = step_run(ctx, steps, dt, DEM_NVT, kT, tau);
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        if (rc == DEM_OK) {
            CK(cudaEventElapsedTime(&ms[mode], e0, e1));
            ms[mode] /= steps;
            rc = snapshot(ctx, true);
        }
    }
    ctx->persistent = keep.v;
    if (rc == DEM_ERR_CUDA || rc == DEM_ERR_NOMEM) return rc;
    if (rc != DEM_OK) {
        // these steps could not run here (e.g. a thermostat without degrees
        // of freedom): the state from before them, and the choice by size
        rc = snapshot(ctx, true);
        if (rc) return rc;
        ctx->err.clear();
        rc = force_rebuild(ctx);
        if (rc) return rc;
        return compute_forces(ctx);
    }
    ctx->tune_step_ms[0] = ms[0];
    ctx->tune_step_ms[1] = ms[1];
    ctx->coop_auto = ms[1] < ms[0] ? 1 : 0;
    if (!ctx->coop_auto) {   // its buffers are not needed
        cudaFree(ctx->coop_part);
        cudaFree(ctx->coop_act);
        ctx->coop_part = nullptr;
        ctx->coop_act = nullptr;
        ctx->coop_part_bytes = ctx->coop_act_bytes = 0;
    }
    rc = force_rebuild(ctx);
    if (rc) return rc;
    return compute_forces(ctx);
}

// After NPT steps: the boxes come back to the host, the cell grids and list
// cutoffs follow them, and the list is rebuilt in the new boxes.
int sync_boxes(dem_ctx *ctx) {
    std::vector<Rep> hr(ctx->R);
    CK(cudaMemcpyAsync(hr.data(), ctx->d_reps, sizeof(Rep) * ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < ctx->R; ++r)
        for (int a = 0; a < ctx->dim; ++a) ctx->box[3 * r + a] = hr[r].L[a];
    int rc = setup_replicas(ctx);
    if (rc) return rc;
    return force_rebuild(ctx);
}

}  // namespace

extern "C" {

int dem_step(dem_ctx *ctx, int n, double dt, int ensemble, double kT, double tau_T) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    if (n < 0 || !(dt > 0) || (ensemble != DEM_NVE && ensemble != DEM_NVT && ensemble != DEM_NPT))
        return set_err(ctx, DEM_ERR_ARG, "bad step arguments");
    if (ensemble != DEM_NVE && (!(kT > 0) || !(tau_T > 0)))
        return set_err(ctx, DEM_ERR_ARG, "NVT and NPT need kT > 0 and tau_T > 0");
    if (ensemble == DEM_NPT) {
        if (!(ctx->tau_P > 0))
            return set_err(ctx, DEM_ERR_ARG, "NPT needs dem_set_barostat (tau_P > 0)");
        for (int r = 0; r < ctx->R; ++r)
            if (ctx->sizes[r] < 2)
                return set_err(ctx, DEM_ERR_ARG, "NPT needs at least 2 particles per replica");
    }
    if (n == 0) return DEM_OK;
    int rc;
    if (ensemble == DEM_NPT) {
        for (int done = 0; done < n;) {
            const int m = std::min(ctx->npt_chunk, n - done);
            rc = step_run(ctx, m, dt, ensemble, kT, tau_T);
            if (rc == DEM_OK) rc = sync_boxes(ctx);
            if (rc) return rc;
            done += m;
        }
        ctx->last_P = ctx->P;
        ctx->last_tauP = ctx->tau_P;
    } else {
        rc = step_run(ctx, n, dt, ensemble, kT, tau_T);
        if (rc) return rc;
    }
    if (ensemble != DEM_NVE) { ctx->last_kT = kT; ctx->last_tau = tau_T; }
    ctx->last_ens = ensemble;
    return DEM_OK;
}

int dem_set_barostat(dem_ctx *ctx, double P, double tau_P) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!(P >= 0) || !isfinite(P) || !(tau_P > 0) || !isfinite(tau_P))
        return set_err(ctx, DEM_ERR_ARG, "barostat needs P >= 0 and tau_P > 0");
    ctx->P = P;
    ctx->tau_P = tau_P;
    return DEM_OK;
}

int dem_get_box(dem_ctx *ctx, double *box) {
    if (!valid(ctx) || !box) return DEM_ERR_ARG;
    for (int r = 0; r < ctx->R; ++r)
        for (int a = 0; a < ctx->dim; ++a) box[ctx->dim * r + a] = ctx->box[3 * r + a];
    return DEM_OK;
}

int dem_get_forces(dem_ctx *ctx, double *force, double *torque, int device_ptrs) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    const size_t n = ctx->N;
    const int dim = ctx->dim, tdim = dim == 3 ? 3 : 1;
    if (device_ptrs) {
        CK(launch_export_forces((int)n, dim, ctx->force, ctx->torque, ctx->quat, force, torque, ctx->stream));
    } else {
        if (force) {
            CK(launch_export_forces((int)n, dim, ctx->force, ctx->torque, ctx->quat, ctx->staging, nullptr, ctx->stream));
            CK(cudaMemcpyAsync(force, ctx->staging, sizeof(double) * dim * n, cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (torque) {
            CK(launch_export_forces((int)n, dim, ctx->force, ctx->torque, ctx->quat, nullptr, ctx->staging, ctx->stream));
            CK(cudaMemcpyAsync(torque, ctx->staging, sizeof(double) * tdim * n, cudaMemcpyDeviceToHost, ctx->stream));
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

int dem_get_particle_energy(dem_ctx *ctx, double *energy, int device_ptrs) {
    if (!valid(ctx) || !energy) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    CK(cudaMemcpyAsync(energy, ctx->energy, sizeof(double) * ctx->N,
                       device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

int dem_get_energy(dem_ctx *ctx, double *U, double *K, double *conserved) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    StepArgs sa = step_args(ctx, 0.0, DEM_NVE, 1.0, 1.0);
    CK(launch_kinetic(sa, ctx->stream));
    CK(launch_replica_sums(ctx->R, ctx->d_reps, ctx->energy, 1, 1, ctx->red, ctx->stream));
    CK(launch_replica_sums(ctx->R, ctx->d_reps, ctx->ke, 1, 1, ctx->red + ctx->R, ctx->stream));
    std::vector<double> h(2 * ctx->R);
    std::vector<Thermo> th(ctx->R);
    CK(cudaMemcpyAsync(h.data(), ctx->red, sizeof(double) * 2 * ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(th.data(), ctx->thermo, sizeof(Thermo) * ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int r = 0; r < ctx->R; ++r) {
        if (U) U[r] = h[r];
        if (K) K[r] = h[ctx->R + r];
        if (conserved) {
            double c = h[r] + h[ctx->R + r];
            if (ctx->last_ens == DEM_NVT) {
                double g = ctx->reps[r].g_dof;
                c += g * ctx->last_kT * (0.5 * ctx->last_tau * ctx->last_tau * th[r].xi * th[r].xi + th[r].eta);
            }
            if (ctx->last_ens == DEM_NPT) {
                // K + U + p_e^2/2W + P V + (g + 1) kT (tau^2 xi^2 / 2 + eta)
                const double g1 = ctx->reps[r].g_dof + 1.0, d = ctx->dim;
                const double W = (d * (ctx->sizes[r] - 1.0) + d) * ctx->last_kT * ctx->last_tauP *
                                 ctx->last_tauP;
                double V = 1.0;
                for (int a = 0; a < ctx->dim; ++a) V *= ctx->box[3 * r + a];
                c += 0.5 * th[r].pe * th[r].pe / W + ctx->last_P * V +
                     g1 * ctx->last_kT * (0.5 * ctx->last_tau * ctx->last_tau * th[r].xi * th[r].xi + th[r].eta);
            }
            conserved[r] = c;
        }
    }
    return DEM_OK;
}

int dem_get_virial(dem_ctx *ctx, double *W6) {
    if (!valid(ctx) || !W6) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    CK(launch_replica_sums(ctx->R, ctx->d_reps, ctx->virial, 6, 6, ctx->red, ctx->stream));
    CK(cudaMemcpyAsync(W6, ctx->red, sizeof(double) * 6 * ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return DEM_OK;
}

int dem_set_box(dem_ctx *ctx, const double *box) {
    if (!valid(ctx) || !box) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    std::vector<double> scale(3 * ctx->R, 1.0), old = ctx->box;
    for (int r = 0; r < ctx->R; ++r)
        for (int a = 0; a < ctx->dim; ++a) {
            double L = box[ctx->dim * r + a];
            if (!(L > 0) || !isfinite(L)) return set_err(ctx, DEM_ERR_ARG, "bad box");
            scale[3 * r + a] = L / ctx->box[3 * r + a];
            ctx->box[3 * r + a] = L;
        }
    int rc = setup_replicas(ctx);
    if (rc) { ctx->box = old; setup_replicas(ctx); return rc; }
    CK(cudaMemcpyAsync(ctx->scale3, scale.data(), sizeof(double) * 3 * ctx->R, cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_rescale(ctx->N, ctx->dim, ctx->pos, ctx->x_last, ctx->rep, ctx->scale3, ctx->stream));
    CK(launch_prepare_state(ctx->N, ctx->dim, ctx->pos, ctx->quat, ctx->quatf, ctx->quatf_lo,
                                    ctx->xff, ctx->angmom,
                            ctx->rep, ctx->d_reps, 0, ctx->stream));
    free_graph(ctx);
    rc = force_rebuild(ctx);
    if (rc) return rc;
    return compute_forces(ctx);
}

int dem_get_counters(dem_ctx *ctx, long long *counts) {
    if (!valid(ctx) || !counts) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    // a due rebuild first: the counting launch must read a complete list
    int rc0 = compute_forces(ctx);
    if (rc0) return rc0;
    CK(cudaMemsetAsync(ctx->d_counters, 0, DEM_N_COUNTERS * sizeof(unsigned long long), ctx->stream));
    CK(launch_pair(pair_args(ctx), ctx->precision, ctx->decomp, ctx->block, true, ctx->stream));
    unsigned long long h[DEM_N_COUNTERS];
    CK(cudaMemcpyAsync(h, ctx->d_counters, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    Status st;
    int rc = read_status(ctx, &st);
    if (rc) return rc;
    for (int k = 0; k < DEM_N_COUNTERS; ++k) counts[k] = (long long)h[k];
    counts[13] = st.rebuilds;
    counts[14] = ctx->launches;
    return DEM_OK;
}

int dem_autotune(dem_ctx *ctx) {
    if (!valid(ctx)) return DEM_ERR_ARG;
    if (!ctx->have_state) return set_err(ctx, DEM_ERR_STATE, "no state set");
    int rc = compute_forces(ctx);   // the list is current before timing
    if (rc) return rc;
    // SPLIT at each number of particles per warp, unless the caller fixed it
    struct Cand { int decomp, block, group; };
    const Cand cands[] = {{DEM_DECOMP_THREAD, 64, 0}, {DEM_DECOMP_THREAD, 128, 0},
                          {DEM_DECOMP_WARP, 128, 0},  {DEM_DECOMP_STAGED, 128, 0},
                          {DEM_DECOMP_SPLIT, 128, 32}, {DEM_DECOMP_SPLIT, 128, 16},
                          {DEM_DECOMP_SPLIT, 128, 8},  {DEM_DECOMP_SPLIT, 128, 4}};
    const int G_keep = ctx->split_G;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 3.0e38f;
    Cand pick = cands[0];
    long long kernels = 0;
    ctx->tune_ms.clear();
    for (const Cand &c : cands) {
        if (ctx->mask_words > 1 && c.decomp != DEM_DECOMP_THREAD) {   // wide shapes: THREAD only
            ctx->tune_ms.push_back(-1.f);
            continue;
        }
        if (c.group) {
            if (ctx->split_user && c.group != G_keep) {   // the caller's group only
                ctx->tune_ms.push_back(-1.f);
                continue;
            }
            ctx->split_G = c.group;
        }
        if (ensure_recs(ctx, c.decomp) != DEM_OK) {   // no room for SPLIT's records
            ctx->tune_ms.push_back(-1.f);
            continue;
        }
        kernels += 4 * (c.decomp == DEM_DECOMP_SPLIT                   // warm-up + 3 timed
                            ? (ctx->precision == DEM_FP32_COMP ? 3 : 2) : 1);
        PairArgs pa = pair_args(ctx);
        CK(launch_pair(pa, ctx->precision, c.decomp, c.block, false, ctx->stream));   // warm-up
        CK(cudaEventRecord(e0, ctx->stream));
        const int reps = 3;
        for (int r = 0; r < reps; ++r)
            CK(launch_pair(pa, ctx->precision, c.decomp, c.block, false, ctx->stream));
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        ms /= reps;
        ctx->tune_ms.push_back(ms);
        if (ms < best) { best = ms; pick = c; }
    }
    ctx->launches += kernels;
    ctx->decomp = pick.decomp;
    ctx->block = pick.block;
    ctx->split_G = pick.group ? pick.group : G_keep;
    free_graph(ctx);
    rc = compute_forces(ctx);
    if (rc == DEM_OK && ctx->persistent < 0) rc = tune_persistent(ctx, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // extern "C"
