/*
 * dem_oracle.c -- plain FP64 CPU oracle for the rounded-polytope DEM of
 * Spellings, Marson, Anderson & Glotzer, "GPU Accelerated Discrete Element
 * Method (DEM) Molecular Dynamics for Conservative, Faceted Particle
 * Simulations" (arXiv:1607.02427).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library: it is the slow, obviously
 * correct statement of what that library must compute.
 *
 * What it computes (Section "Model"):
 *   * Each particle is an inner polygon/polyhedron (vertices V, edges E,
 *     faces F) rounded by a disk/sphere of radius sigma/2.
 *   * Eq. DEM (3D): U_ij = sum_{E_i,E_j} U(r*_EE) + sum_{V_i,F_j} U(r*_VF)
 *                          + sum_{V_j,F_i} U(r*_VF).
 *   * Eq. DEM_2D (2D): U_ij = sum_{V_i,E_j} U(r*_VE) + sum_{V_j,E_i} U(r*_VE).
 *   * r* is the distance between the nearest points of the two features,
 *     found with point-segment, segment-segment and point-plane formulae.
 *   * The force of a feature pair acts along the line joining its nearest
 *     points, F = -U'(r) r_hat; torques use the nearest point on each
 *     particle as the point of application.
 *   * U is WCA (Eq. LJ and Eq. WCA): the LJ potential shifted by its value
 *     at r_cut = 2^(1/6) sigma and cut there.
 *   * Nearly parallel edges interact at the midpoint of their overlap
 *     (parallel-edge rule, Section "Model").
 *   * Overcounting of features (Section "Model") is part of the definition:
 *     nothing is de-duplicated.
 * Readings where the paper is silent (each also stated where used):
 *   * sigma_ij = sigma if sigma > 0, else rounding_i + rounding_j.
 *   * Two one-vertex shapes (disks/spheres) interact through one
 *     vertex-vertex term: the central WCA of the sphere limit (Section
 *     "Performance" models spheres with the central WCA).
 *   * "Nearly parallel" means |d1 x d2|^2 <= par_eps |d1|^2 |d2|^2.  Inside
 *     that band the nearest points are: the midpoint of the overlap of the
 *     projection of edge j onto edge i, and its nearest point on edge j;
 *     without overlap, the closest of the four endpoint-to-segment pairs.
 *   * The virial is the centre-of-mass pair virial sum_{i<j} x_ij (x) f_ij
 *     with x_ij = x_i - x_j and f_ij the total force of j on i.
 *
 * Integrator (Section "Energy Conservation" cites a second-order integrator;
 * Section "Assembly" a Nose-Hoover thermostat on translational and
 * rotational degrees of freedom; the paper gives no formulas, so this is the
 * reading the CUDA library implements as well):
 *   * velocity Verlet for translation;
 *   * body-frame angular momentum with the symmetric free-rotor splitting
 *     about the principal axes z(dt/2) y(dt/2) x(dt) y(dt/2) z(dt/2) (the
 *     NO_SQUISH splitting of Miller et al., J. Chem. Phys. 116, 8649 (2002));
 *   * NVT: a symmetric Trotter split T(dt/2) . NVE(dt) . T(dt/2) with one
 *     Nose-Hoover variable xi for all degrees of freedom,
 *     dxi/dt = (2K/(g kT) - 1)/tau^2, g = d(N-1) + rotational DOF, and the
 *     conserved H = K + U + g kT (tau^2 xi^2 / 2 + eta), eta = int xi dt.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXV 128         /* max vertices of one shape */
#define MAXFV 16         /* max vertices of one face */

typedef struct { double x, y, z; } v3;

static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 crs(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(v3 a) { return sqrt(dot(a, a)); }
static double clamp01(double t) { return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }

/* ---------------------------------------------------------------------- */
/* Nearest-point primitives ("standard point-line, line-line and          */
/* point-plane formulae", Section "Model")                               */
/* ---------------------------------------------------------------------- */

/* Nearest point q on segment [a,b] to p; returns |p - q|. */
static double point_segment(v3 p, v3 a, v3 b, v3 *q) {
    v3 d = sub(b, a);
    double dd = dot(d, d);
    double t = dd > 0.0 ? clamp01(dot(sub(p, a), d) / dd) : 0.0;
    *q = add(a, scl(d, t));
    return len(sub(p, *q));
}

/* Nearest point q on the convex planar polygon poly[0..n-1] (counter-
 * clockwise seen from the side its normal points to) to p.  The normal is
 * the polygon's area vector (Newell).  If the orthogonal projection of p
 * lies inside (on the inner side of every edge), q is that projection;
 * otherwise q lies on the boundary and is the nearest of the edge results. */
static double point_face(v3 p, const v3 *poly, int n, v3 *q) {
    v3 nrm = mk(0, 0, 0);
    for (int k = 0; k < n; ++k) nrm = add(nrm, crs(poly[k], poly[(k + 1) % n]));
    nrm = scl(nrm, 1.0 / len(nrm));
    double h = dot(sub(p, poly[0]), nrm);
    v3 proj = sub(p, scl(nrm, h));
    int inside = 1;
    for (int k = 0; k < n; ++k) {
        v3 e = sub(poly[(k + 1) % n], poly[k]);
        if (dot(crs(e, sub(proj, poly[k])), nrm) < 0.0) { inside = 0; break; }
    }
    if (inside) { *q = proj; return fabs(h); }
    double best = INFINITY;
    for (int k = 0; k < n; ++k) {
        v3 c;
        double r = point_segment(p, poly[k], poly[(k + 1) % n], &c);
        if (r < best) { best = r; *q = c; }
    }
    return best;
}

/* Nearest points p1 on [a1,b1] and p2 on [a2,b2]; returns |p1 - p2|.
 * Not nearly parallel: the squared distance is a strictly convex quadratic
 * in the segment parameters (s,t); its stationary point is the answer if it
 * lies in [0,1]^2, otherwise the minimum lies on the boundary of the square,
 * i.e. is one of the four endpoint-to-segment problems.
 * Nearly parallel: the parallel-edge rule (midpoint of overlap). */
static double segment_segment(v3 a1, v3 b1, v3 a2, v3 b2, double par_eps,
                              v3 *p1, v3 *p2, int *parallel) {
    v3 d1 = sub(b1, a1), d2 = sub(b2, a2), w = sub(a1, a2);
    double A = dot(d1, d1), B = dot(d1, d2), C = dot(d2, d2);
    double D = dot(d1, w), E = dot(d2, w);
    v3 cr = crs(d1, d2);
    double cr2 = dot(cr, cr);
    *parallel = !(cr2 > par_eps * A * C);
    if (!*parallel) {
        double den = A * C - B * B;
        double s = (B * E - C * D) / den;
        double t = (A * E - B * D) / den;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
            *p1 = add(a1, scl(d1, s));
            *p2 = add(a2, scl(d2, t));
            return len(sub(*p1, *p2));
        }
    } else {
        double t0 = dot(sub(a2, a1), d1) / A;
        double t1 = dot(sub(b2, a1), d1) / A;
        double lo = fmax(0.0, fmin(t0, t1));
        double hi = fmin(1.0, fmax(t0, t1));
        if (lo <= hi) {
            *p1 = add(a1, scl(d1, 0.5 * (lo + hi)));
            return point_segment(*p1, a2, b2, p2);
        }
    }
    /* the four endpoint-to-segment candidates, in a fixed order */
    double best = INFINITY;
    v3 c;
    double r;
    r = point_segment(a1, a2, b2, &c);
    if (r < best) { best = r; *p1 = a1; *p2 = c; }
    r = point_segment(b1, a2, b2, &c);
    if (r < best) { best = r; *p1 = b1; *p2 = c; }
    r = point_segment(a2, a1, b1, &c);
    if (r < best) { best = r; *p1 = c; *p2 = a2; }
    r = point_segment(b2, a1, b1, &c);
    if (r < best) { best = r; *p1 = c; *p2 = b2; }
    return best;
}

/* ---------------------------------------------------------------------- */
/* WCA potential (Eq. LJ, Eq. WCA)                                        */
/* ---------------------------------------------------------------------- */

/* Returns U(r); *fmag = -dU/dr; *dfdr = d(fmag)/dr.  Zero beyond r_cut. */
static double wca(double r, double eps, double sigma, double *fmag, double *dfdr) {
    double rcut = pow(2.0, 1.0 / 6.0) * sigma;
    if (!(r < rcut)) { *fmag = 0.0; if (dfdr) *dfdr = 0.0; return 0.0; }
    double s6 = pow(sigma / r, 6.0), s12 = s6 * s6;
    double s6c = pow(sigma / rcut, 6.0), s12c = s6c * s6c;
    double u_lj = 4.0 * eps * (s12 - s6);
    double u_lj_cut = 4.0 * eps * (s12c - s6c);
    *fmag = 24.0 * eps * (2.0 * s12 - s6) / r;
    if (dfdr) *dfdr = 24.0 * eps * (-26.0 * s12 + 7.0 * s6) / (r * r);
    return u_lj - u_lj_cut;
}

/* ---------------------------------------------------------------------- */
/* Shapes                                                                 */
/* ---------------------------------------------------------------------- */

typedef struct {
    int nv, ne, nf;
    v3 v[MAXV];               /* body-frame vertices (2D: z = 0)          */
    int e[3 * MAXV][2];       /* edges as vertex index pairs              */
    int fo[2 * MAXV + 1];     /* face k = fidx[fo[k] .. fo[k+1])           */
    int fidx[8 * MAXV];
    double rounding, R;       /* rounding radius, inner circumradius      */
} shape_t;

/* 2D: edges join consecutive vertices of the counter-clockwise polygon
 * ("the edge beginning at that vertex, travelling counterclockwise",
 * Section "Algorithm"); a 2-vertex shape has a single edge.
 * 3D: edges are the distinct vertex pairs adjacent on some face loop. */
static int build_shapes(int dim, int n_shapes, const int *vert_off, const double *verts,
                        const int *shape_face_off, const int *face_vert_off,
                        const int *face_idx, const double *rounding, shape_t *out) {
    for (int s = 0; s < n_shapes; ++s) {
        shape_t *sh = &out[s];
        memset(sh, 0, sizeof(*sh));
        sh->nv = vert_off[s + 1] - vert_off[s];
        if (sh->nv < 1 || sh->nv > MAXV) return -1;
        sh->rounding = rounding[s];
        sh->R = 0.0;
        for (int k = 0; k < sh->nv; ++k) {
            const double *p = verts + 3 * (vert_off[s] + k);
            sh->v[k] = mk(p[0], p[1], dim == 3 ? p[2] : 0.0);
            if (len(sh->v[k]) > sh->R) sh->R = len(sh->v[k]);
        }
        if (dim == 2) {
            sh->nf = 0;
            if (sh->nv == 2) { sh->ne = 1; sh->e[0][0] = 0; sh->e[0][1] = 1; }
            else if (sh->nv >= 3) {
                sh->ne = sh->nv;
                for (int k = 0; k < sh->nv; ++k) { sh->e[k][0] = k; sh->e[k][1] = (k + 1) % sh->nv; }
            }
        } else {
            sh->nf = shape_face_off[s + 1] - shape_face_off[s];
            if (sh->nf > 2 * MAXV) return -1;
            int m = 0;
            sh->fo[0] = 0;
            for (int f = 0; f < sh->nf; ++f) {
                int g = shape_face_off[s] + f;
                int a = face_vert_off[g], b = face_vert_off[g + 1];
                if (b - a < 3 || b - a > MAXFV) return -1;
                for (int k = a; k < b; ++k) sh->fidx[m++] = face_idx[k];
                sh->fo[f + 1] = m;
                for (int k = a; k < b; ++k) {
                    int u = face_idx[k], w = face_idx[k + 1 < b ? k + 1 : a];
                    int lo = u < w ? u : w, hi = u < w ? w : u, seen = 0;
                    for (int q = 0; q < sh->ne; ++q)
                        if (sh->e[q][0] == lo && sh->e[q][1] == hi) { seen = 1; break; }
                    if (!seen) { sh->e[sh->ne][0] = lo; sh->e[sh->ne][1] = hi; sh->ne++; }
                }
            }
        }
    }
    return 0;
}

/* Rotation matrix of the unit quaternion q = (w, x, y, z): v_world = R v_body. */
static void quat_to_mat(const double *q, double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

static void orientation_matrix(int dim, const double *orient, int i, double R[3][3]) {
    if (dim == 3) { quat_to_mat(orient + 4 * i, R); return; }
    double c = cos(orient[i]), s = sin(orient[i]);
    R[0][0] = c; R[0][1] = -s; R[0][2] = 0;
    R[1][0] = s; R[1][1] = c;  R[1][2] = 0;
    R[2][0] = 0; R[2][1] = 0;  R[2][2] = 1;
}

static v3 mat_vec(double R[3][3], v3 v) {
    return mk(R[0][0] * v.x + R[0][1] * v.y + R[0][2] * v.z,
              R[1][0] * v.x + R[1][1] * v.y + R[1][2] * v.z,
              R[2][0] * v.x + R[2][1] * v.y + R[2][2] * v.z);
}
static v3 mat_t_vec(double R[3][3], v3 v) {
    return mk(R[0][0] * v.x + R[1][0] * v.y + R[2][0] * v.z,
              R[0][1] * v.x + R[1][1] * v.y + R[2][1] * v.z,
              R[0][2] * v.x + R[1][2] * v.y + R[2][2] * v.z);
}

/* ---------------------------------------------------------------------- */
/* Forces                                                                 */
/* ---------------------------------------------------------------------- */

typedef struct {
    double eps, sigma, par_eps;
    int dim;
    /* outputs */
    double *force, *torque, *energy, *virial, *fscale, *tscale;
    int *flags;
    long long *counts;
} acc_t;

/* One feature-pair term with nearest points pi (on particle i) and pj (on
 * j), both relative to x_i; d = x_j - x_i (minimum image). */
static void term(acc_t *A, int i, int j, v3 d, v3 pi, v3 pj, double sigma_ij) {
    A->counts[1]++;
    v3 rv = sub(pi, pj);
    double r = len(rv);
    if (!(r < pow(2.0, 1.0 / 6.0) * sigma_ij)) return;   /* beyond r_cut: U = 0 */
    A->counts[2]++;
    double fm, dfdr;
    double U = wca(r, A->eps, sigma_ij, &fm, &dfdr);
    v3 f = scl(rv, fm / r);                 /* force on i */
    int dim = A->dim;
    A->force[dim * i + 0] += f.x; A->force[dim * i + 1] += f.y;
    A->force[dim * j + 0] -= f.x; A->force[dim * j + 1] -= f.y;
    if (dim == 3) { A->force[3 * i + 2] += f.z; A->force[3 * j + 2] -= f.z; }
    v3 ti = crs(pi, f);                     /* lever arm pi - x_i = pi */
    v3 tj = crs(sub(pj, d), scl(f, -1.0));  /* lever arm pj - x_j      */
    if (dim == 3) {
        A->torque[3 * i + 0] += ti.x; A->torque[3 * i + 1] += ti.y; A->torque[3 * i + 2] += ti.z;
        A->torque[3 * j + 0] += tj.x; A->torque[3 * j + 1] += tj.y; A->torque[3 * j + 2] += tj.z;
    } else {
        A->torque[i] += ti.z;
        A->torque[j] += tj.z;
    }
    A->energy[i] += 0.5 * U;
    A->energy[j] += 0.5 * U;
    /* x_i - x_j = -d */
    double xij[3] = {-d.x, -d.y, -d.z}, fv[3] = {f.x, f.y, f.z};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) A->virial[3 * a + b] += xij[a] * fv[b];
    if (A->fscale) {
        double sk = fabs(fm) + sigma_ij * fabs(dfdr);
        A->fscale[i] += sk; A->fscale[j] += sk;
        A->tscale[i] += len(pi) * sk + sigma_ij * fabs(fm);
        A->tscale[j] += len(sub(pj, d)) * sk + sigma_ij * fabs(fm);
    }
}

/* All feature-pair terms of particles i and j (Eq. DEM / Eq. DEM_2D). */
static void pair_terms(acc_t *A, int i, int j, const shape_t *si, const shape_t *sj,
                       double Ri[3][3], double Rj[3][3], v3 d, double sigma_ij) {
    v3 wi[MAXV], wj[MAXV];
    for (int k = 0; k < si->nv; ++k) wi[k] = mat_vec(Ri, si->v[k]);
    for (int k = 0; k < sj->nv; ++k) wj[k] = add(d, mat_vec(Rj, sj->v[k]));
    v3 q;

    if (si->nv == 1 && sj->nv == 1) {        /* sphere / disk limit */
        term(A, i, j, d, wi[0], wj[0], sigma_ij);
        return;
    }
    if (A->dim == 2) {
        for (int a = 0; a < si->nv; ++a)           /* V_i x E_j */
            for (int e = 0; e < sj->ne; ++e) {
                point_segment(wi[a], wj[sj->e[e][0]], wj[sj->e[e][1]], &q);
                term(A, i, j, d, wi[a], q, sigma_ij);
            }
        for (int b = 0; b < sj->nv; ++b)           /* V_j x E_i */
            for (int e = 0; e < si->ne; ++e) {
                point_segment(wj[b], wi[si->e[e][0]], wi[si->e[e][1]], &q);
                term(A, i, j, d, q, wj[b], sigma_ij);
            }
        return;
    }
    /* E_i x E_j.  Segment 1 of every edge pair is i's edge: the lower-
     * indexed particle's edge is the parallel-edge rule's reference (inside
     * the band, and not exactly parallel, the midpoint of the overlap of the
     * other edge's projection on the reference depends on that choice). */
    for (int ea = 0; ea < si->ne; ++ea)
        for (int eb = 0; eb < sj->ne; ++eb) {
            v3 p1, p2;
            int par;
            segment_segment(wi[si->e[ea][0]], wi[si->e[ea][1]],
                            wj[sj->e[eb][0]], wj[sj->e[eb][1]], A->par_eps, &p1, &p2, &par);
            (void)par;
            if (A->flags) {
                /* mark particles with an in-range EE term whose squared sine
                 * lies within a decade of the parallel threshold: there the
                 * rule switches branch, and a lower-precision evaluation may
                 * take the other one */
                v3 d1 = sub(wi[si->e[ea][1]], wi[si->e[ea][0]]);
                v3 d2 = sub(wj[sj->e[eb][1]], wj[sj->e[eb][0]]);
                double s2 = dot(crs(d1, d2), crs(d1, d2)) / (dot(d1, d1) * dot(d2, d2));
                if (s2 > 0.1 * A->par_eps && s2 < 10.0 * A->par_eps &&
                    len(sub(p1, p2)) < pow(2.0, 1.0 / 6.0) * sigma_ij) {
                    A->flags[i] |= 1; A->flags[j] |= 1;
                }
            }
            term(A, i, j, d, p1, p2, sigma_ij);
        }
    v3 poly[MAXFV];
    for (int a = 0; a < si->nv; ++a)               /* V_i x F_j */
        for (int f = 0; f < sj->nf; ++f) {
            int n = sj->fo[f + 1] - sj->fo[f];
            for (int k = 0; k < n; ++k) poly[k] = wj[sj->fidx[sj->fo[f] + k]];
            point_face(wi[a], poly, n, &q);
            term(A, i, j, d, wi[a], q, sigma_ij);
        }
    for (int b = 0; b < sj->nv; ++b)               /* V_j x F_i */
        for (int f = 0; f < si->nf; ++f) {
            int n = si->fo[f + 1] - si->fo[f];
            for (int k = 0; k < n; ++k) poly[k] = wi[si->fidx[si->fo[f] + k]];
            point_face(wj[b], poly, n, &q);
            term(A, i, j, d, q, wj[b], sigma_ij);
        }
}

static v3 min_image(int dim, v3 d, const double *box) {
    double dd[3] = {d.x, d.y, d.z};
    for (int a = 0; a < dim; ++a) dd[a] -= box[a] * nearbyint(dd[a] / box[a]);
    return mk(dd[0], dd[1], dim == 3 ? dd[2] : 0.0);
}

static v3 position(int dim, const double *pos, int i) {
    return mk(pos[dim * i], pos[dim * i + 1], dim == 3 ? pos[dim * i + 2] : 0.0);
}

static int forces_all_pairs(int dim, const shape_t *shapes, double eps, double sigma,
                              double par_eps, int n, const int *shape_id, const double *pos,
                              const double *orient, const double *box, double *force,
                              double *torque, double *energy, double *virial, double *fscale,
                              double *tscale, int *flags, long long *counts) {
    int tdim = dim == 3 ? 3 : 1;
    memset(force, 0, sizeof(double) * dim * n);
    memset(torque, 0, sizeof(double) * tdim * n);
    memset(energy, 0, sizeof(double) * n);
    memset(virial, 0, sizeof(double) * 9);
    if (fscale) { memset(fscale, 0, sizeof(double) * n); memset(tscale, 0, sizeof(double) * n); }
    if (flags) memset(flags, 0, sizeof(int) * n);
    long long local_counts[3] = {0, 0, 0};
    acc_t A = {eps, sigma, par_eps, dim, force, torque, energy, virial, fscale, tscale, flags,
               counts ? counts : local_counts};
    if (counts) counts[0] = counts[1] = counts[2] = 0;
    for (int i = 0; i < n; ++i) {
        double Ri[3][3];
        orientation_matrix(dim, orient, i, Ri);
        const shape_t *si = &shapes[shape_id[i]];
        for (int j = i + 1; j < n; ++j) {
            const shape_t *sj = &shapes[shape_id[j]];
            double sigma_ij = sigma > 0.0 ? sigma : si->rounding + sj->rounding;
            double rcut = pow(2.0, 1.0 / 6.0) * sigma_ij;
            v3 d = min_image(dim, sub(position(dim, pos, j), position(dim, pos, i)), box);
            /* exact skip: every feature lies within R of its centre */
            if (!(len(d) < si->R + sj->R + rcut)) continue;
            A.counts[0]++;
            double Rj[3][3];
            orientation_matrix(dim, orient, j, Rj);
            pair_terms(&A, i, j, si, sj, Ri, Rj, d, sigma_ij);
        }
    }
    return 0;
}


/* ---------------------------------------------------------------------- */
/* Timed CPU baseline only: cell-list pair search, OpenMP over particles  */
/* ---------------------------------------------------------------------- */
/* The benchmark times the oracle on the host cores in two forms: as it
 * stands (all pairs, one thread), and with the pair search restricted to a
 * cell list and the particles shared among OpenMP threads.  The second form
 * evaluates exactly the same pairs and terms (every pair the cell list
 * skips is beyond R_i + R_j + r_cut, the exact skip above; every pair is
 * taken with its lower index first, so the parallel-edge rule keeps its
 * reference) and differs only in the order of the floating-point sums.
 * The tests use the first form; oracle_set_parallel selects the second. */
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_threads = 1, g_cells = 0;

void oracle_set_parallel(int threads, int use_cells) {
    g_threads = threads > 0 ? threads : 1;
    g_cells = use_cells != 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int forces_parallel(int dim, const shape_t *shapes, double eps, double sigma,
                           double par_eps, int n, const int *shape_id, const double *pos,
                           const double *orient, const double *box, double *force,
                           double *torque, double *energy, double *virial, long long *counts) {
    int tdim = dim == 3 ? 3 : 1;
    int nth = g_threads;
#ifndef _OPENMP
    nth = 1;
#endif
    /* cells of width >= the largest interaction range, >= 3 per axis, else
     * every pair */
    double Rmax = 0.0, rnd_max = 0.0;
    for (int i = 0; i < n; ++i) {
        const shape_t *sh = &shapes[shape_id[i]];
        if (sh->R > Rmax) Rmax = sh->R;
        if (sh->rounding > rnd_max) rnd_max = sh->rounding;
    }
    double range = 2.0 * Rmax + pow(2.0, 1.0 / 6.0) * (sigma > 0.0 ? sigma : 2.0 * rnd_max);
    int nc[3] = {1, 1, 1}, use_cells = g_cells;
    for (int a = 0; a < dim; ++a) {
        nc[a] = (int)floor(box[a] / (range * (1.0 + 1e-9)));
        if (nc[a] < 3) use_cells = 0;
    }
    int ncell = nc[0] * nc[1] * nc[2];
    int *head = NULL, *next = NULL, *cell = NULL;
    if (use_cells) {
        head = (int *)malloc(sizeof(int) * ncell);
        next = (int *)malloc(sizeof(int) * n);
        cell = (int *)malloc(sizeof(int) * n);
        if (!head || !next || !cell) { free(head); free(next); free(cell); return -2; }
        for (int c = 0; c < ncell; ++c) head[c] = -1;
        for (int i = n - 1; i >= 0; --i) {
            int cc[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) {
                double x = pos[dim * i + a];
                x -= box[a] * floor(x / box[a]);
                int k = (int)(x / box[a] * nc[a]);
                cc[a] = k < 0 ? 0 : (k >= nc[a] ? nc[a] - 1 : k);
            }
            cell[i] = (cc[2] * nc[1] + cc[1]) * nc[0] + cc[0];
            next[i] = head[cell[i]];
            head[cell[i]] = i;
        }
    }
    /* per-thread accumulators, summed at the end */
    size_t per = (size_t)dim * n + (size_t)tdim * n + n + 9;
    double *buf = (double *)calloc((size_t)nth * per, sizeof(double));
    long long *cnt = (long long *)calloc((size_t)nth * 3, sizeof(long long));
    if (!buf || !cnt) { free(buf); free(cnt); free(head); free(next); free(cell); return -2; }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nth) schedule(dynamic, 8)
#endif
    for (int i = 0; i < n; ++i) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *b = buf + (size_t)t * per;
        acc_t A = {eps, sigma, par_eps, dim, b, b + (size_t)dim * n,
                   b + (size_t)dim * n + (size_t)tdim * n, b + (size_t)dim * n + (size_t)tdim * n + n,
                   NULL, NULL, NULL, cnt + 3 * t};
        double Ri[3][3];
        orientation_matrix(dim, orient, i, Ri);
        const shape_t *si = &shapes[shape_id[i]];
        /* candidate j > i: every particle, or those of the 27 (9) cells
         * around i's cell */
        int cand_cells[27], ncand = 0;
        if (use_cells) {
            int ci = cell[i], cx = ci % nc[0], cy = (ci / nc[0]) % nc[1], cz = ci / (nc[0] * nc[1]);
            for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int x = (cx + dx + nc[0]) % nc[0], y = (cy + dy + nc[1]) % nc[1];
                        int z = dim == 3 ? (cz + dz + nc[2]) % nc[2] : 0;
                        cand_cells[ncand++] = (z * nc[1] + y) * nc[0] + x;
                    }
        }
        int kc = 0, j = use_cells ? -1 : i;
        for (;;) {
            if (use_cells) {
                j = j < 0 ? -1 : next[j];
                while (j < 0 && kc < ncand) j = head[cand_cells[kc++]];
                if (j < 0) break;
                if (j <= i) continue;
            } else {
                if (++j >= n) break;
            }
            const shape_t *sj = &shapes[shape_id[j]];
            double sigma_ij = sigma > 0.0 ? sigma : si->rounding + sj->rounding;
            double rcut = pow(2.0, 1.0 / 6.0) * sigma_ij;
            v3 d = min_image(dim, sub(position(dim, pos, j), position(dim, pos, i)), box);
            if (!(len(d) < si->R + sj->R + rcut)) continue;
            A.counts[0]++;
            double Rj[3][3];
            orientation_matrix(dim, orient, j, Rj);
            pair_terms(&A, i, j, si, sj, Ri, Rj, d, sigma_ij);
        }
    }
    memset(force, 0, sizeof(double) * dim * n);
    memset(torque, 0, sizeof(double) * tdim * n);
    memset(energy, 0, sizeof(double) * n);
    memset(virial, 0, sizeof(double) * 9);
    if (counts) counts[0] = counts[1] = counts[2] = 0;
    for (int t = 0; t < nth; ++t) {
        const double *b = buf + (size_t)t * per;
        for (size_t k = 0; k < (size_t)dim * n; ++k) force[k] += b[k];
        for (size_t k = 0; k < (size_t)tdim * n; ++k) torque[k] += b[(size_t)dim * n + k];
        for (int k = 0; k < n; ++k) energy[k] += b[(size_t)dim * n + (size_t)tdim * n + k];
        for (int k = 0; k < 9; ++k) virial[k] += b[(size_t)dim * n + (size_t)tdim * n + n + k];
        if (counts)
            for (int k = 0; k < 3; ++k) counts[k] += cnt[3 * t + k];
    }
    free(buf); free(cnt); free(head); free(next); free(cell);
    return 0;
}

/* The plain all-pairs evaluation (tests, scales, flags), or the timed
 * baseline's cell-list / OpenMP form when oracle_set_parallel chose it. */
static int forces_with_shapes(int dim, const shape_t *shapes, double eps, double sigma,
                              double par_eps, int n, const int *shape_id, const double *pos,
                              const double *orient, const double *box, double *force,
                              double *torque, double *energy, double *virial, double *fscale,
                              double *tscale, int *flags, long long *counts) {
    if ((g_threads > 1 || g_cells) && !fscale && !tscale && !flags)
        return forces_parallel(dim, shapes, eps, sigma, par_eps, n, shape_id, pos, orient, box,
                               force, torque, energy, virial, counts);
    return forces_all_pairs(dim, shapes, eps, sigma, par_eps, n, shape_id, pos, orient, box,
                            force, torque, energy, virial, fscale, tscale, flags, counts);
}

/* ---------------------------------------------------------------------- */
/* Exported API (ctypes)                                                  */
/* ---------------------------------------------------------------------- */

/* Shapes are passed packed: shape s has vertices verts[3*vert_off[s] ..
 * 3*vert_off[s+1]) (z ignored in 2D), faces shape_face_off[s] ..
 * shape_face_off[s+1]) into face_vert_off, face g with vertex indices
 * face_idx[face_vert_off[g] .. face_vert_off[g+1]).  orient is n*4
 * quaternions (w,x,y,z) in 3D and n angles in 2D; pos is n*dim; box is dim
 * lengths (orthorhombic, periodic).  Outputs: force n*dim, torque n*3 (3D)
 * or n (2D), energy n (half of each term to each particle), virial 9
 * (row-major), fscale/tscale n (per-particle sums of term scales, may be
 * NULL), flags n (may be NULL), counts[3] = pairs within the bounding
 * range, feature pairs evaluated, feature pairs with r < r_cut. */
int oracle_forces(int dim, int n_shapes, const int *vert_off, const double *verts,
                  const int *shape_face_off, const int *face_vert_off, const int *face_idx,
                  const double *rounding, double eps, double sigma, double par_eps, int n,
                  const int *shape_id, const double *pos, const double *orient,
                  const double *box, double *force, double *torque, double *energy,
                  double *virial, double *fscale, double *tscale, int *flags,
                  long long *counts) {
    shape_t *shapes = (shape_t *)malloc(sizeof(shape_t) * (n_shapes > 0 ? n_shapes : 1));
    if (!shapes) return -2;
    if (build_shapes(dim, n_shapes, vert_off, verts, shape_face_off, face_vert_off, face_idx,
                     rounding, shapes)) { free(shapes); return -1; }
    int rc = forces_with_shapes(dim, shapes, eps, sigma, par_eps, n, shape_id, pos, orient, box,
                                force, torque, energy, virial, fscale, tscale, flags, counts);
    free(shapes);
    return rc;
}

/* Primitive access for the brute-force tests. */
double oracle_point_segment(const double *p, const double *a, const double *b, double *q) {
    v3 r;
    double dist = point_segment(mk(p[0], p[1], p[2]), mk(a[0], a[1], a[2]), mk(b[0], b[1], b[2]), &r);
    q[0] = r.x; q[1] = r.y; q[2] = r.z;
    return dist;
}

double oracle_point_face(const double *p, int n, const double *poly, double *q) {
    v3 pl[MAXFV], r;
    if (n < 3 || n > MAXFV) return -1.0;
    for (int k = 0; k < n; ++k) pl[k] = mk(poly[3 * k], poly[3 * k + 1], poly[3 * k + 2]);
    double dist = point_face(mk(p[0], p[1], p[2]), pl, n, &r);
    q[0] = r.x; q[1] = r.y; q[2] = r.z;
    return dist;
}

double oracle_segment_segment(const double *a1, const double *b1, const double *a2,
                              const double *b2, double par_eps, double *p1, double *p2,
                              int *parallel) {
    v3 r1, r2;
    double dist = segment_segment(mk(a1[0], a1[1], a1[2]), mk(b1[0], b1[1], b1[2]),
                                  mk(a2[0], a2[1], a2[2]), mk(b2[0], b2[1], b2[2]), par_eps,
                                  &r1, &r2, parallel);
    p1[0] = r1.x; p1[1] = r1.y; p1[2] = r1.z;
    p2[0] = r2.x; p2[1] = r2.y; p2[2] = r2.z;
    return dist;
}

double oracle_wca(double r, double eps, double sigma, double *fmag) {
    return wca(r, eps, sigma, fmag, NULL);
}

/* ---------------------------------------------------------------------- */
/* Integrator                                                             */
/* ---------------------------------------------------------------------- */

/* q <- q (x) (cos(phi/2), sin(phi/2) e_k): a rotation by phi about body axis k. */
static void quat_rotate_body(double *q, int k, double phi) {
    double c = cos(0.5 * phi), s = sin(0.5 * phi);
    double r[4] = {c, 0, 0, 0};
    r[1 + k] = s;
    double w1 = q[0], x1 = q[1], y1 = q[2], z1 = q[3];
    double w2 = r[0], x2 = r[1], y2 = r[2], z2 = r[3];
    q[0] = w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2;
    q[1] = w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2;
    q[2] = w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2;
    q[3] = w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2;
}

/* Free rotation about body axis k for time dt: the body turns by
 * phi = L_k / I_k dt; the body-frame angular momentum turns by -phi. */
static void free_rotor_axis(double *q, double *Lb, const double *I, int k, double dt) {
    if (!(I[k] > 0.0)) return;
    double phi = Lb[k] / I[k] * dt;
    quat_rotate_body(q, k, phi);
    int a = (k + 1) % 3, b = (k + 2) % 3;
    double c = cos(phi), s = sin(phi);
    double La = Lb[a], Lb_ = Lb[b];
    Lb[a] = c * La + s * Lb_;
    Lb[b] = -s * La + c * Lb_;
}

typedef struct {
    int dim, n;
    const shape_t *shapes;
    const int *shape_id;
    const double *mass, *inertia;   /* per shape; inertia 3 per shape (2D: I_z first) */
    double eps, sigma, par_eps;
    const double *box;
    double *force, *torque, *energy, virial[9];
} sys_t;

static double compute_forces(sys_t *S, const double *pos, const double *orient) {
    forces_with_shapes(S->dim, S->shapes, S->eps, S->sigma, S->par_eps, S->n, S->shape_id,
                       pos, orient, S->box, S->force, S->torque, S->energy, S->virial,
                       NULL, NULL, NULL, NULL);
    double U = 0.0;
    for (int i = 0; i < S->n; ++i) U += S->energy[i];
    return U;
}

/* kinetic energies; Lb is body-frame angular momentum (n*3, 2D: n), or NULL
 * for the translational part only */
static void kinetic(sys_t *S, const double *vel, const double *Lb, double *Kt, double *Kr) {
    *Kt = 0.0; *Kr = 0.0;
    for (int i = 0; i < S->n; ++i) {
        int s = S->shape_id[i];
        double v2 = 0.0;
        for (int a = 0; a < S->dim; ++a) v2 += vel[S->dim * i + a] * vel[S->dim * i + a];
        *Kt += 0.5 * S->mass[s] * v2;
        const double *I = S->inertia + 3 * s;
        if (!Lb) continue;
        if (S->dim == 3) {
            for (int k = 0; k < 3; ++k)
                if (I[k] > 0.0) *Kr += 0.5 * Lb[3 * i + k] * Lb[3 * i + k] / I[k];
        } else if (I[0] > 0.0) {
            *Kr += 0.5 * Lb[i] * Lb[i] / I[0];
        }
    }
}

/* The Nose-Hoover propagator over a time delta (one Trotter half step). */
static void thermostat(sys_t *S, double *vel, double *Lb, double *xi, double *eta, double g,
                       double kT, double tau, double delta) {
    double Kt, Kr;
    kinetic(S, vel, Lb, &Kt, &Kr);
    double K = Kt + Kr;
    *xi += 0.5 * delta * (2.0 * K / (g * kT) - 1.0) / (tau * tau);
    double s = exp(-(*xi) * delta);
    int tdim = S->dim == 3 ? 3 : 1;
    for (int i = 0; i < S->n * S->dim; ++i) vel[i] *= s;
    for (int i = 0; i < S->n * tdim; ++i) Lb[i] *= s;
    *eta += (*xi) * delta;
    K *= s * s;
    *xi += 0.5 * delta * (2.0 * K / (g * kT) - 1.0) / (tau * tau);
}

/* sinh(x)/x (Maclaurin series below |x| = 1e-2, remainder < 1e-17) */
static double sinhc(double x) {
    if (fabs(x) < 1e-2) {
        double x2 = x * x;
        return 1.0 + x2 / 6.0 * (1.0 + x2 / 20.0 * (1.0 + x2 / 42.0));
    }
    return sinh(x) / x;
}

/* Translational kinetic energy sum m v^2 / 2 */
static double kinetic_trans(sys_t *S, const double *vel) {
    double Kt, Kr;
    kinetic(S, vel, NULL, &Kt, &Kr);
    return Kt;
}

/* Isotropic barostat (ensemble 2), the MTK equations integrated as in
 * Tuckerman et al., J. Phys. A 39, 5629 (2006), which Section "Assembly"
 * cites for its NPT runs (the paper gives no formulas; this reading:
 * isotropic scaling of the orthorhombic box, one Nose-Hoover thermostat
 * shared by the particles and the barostat):
 *   dx/dt = v + v_e x,   dv/dt = F/m - alpha v_e v - xi v,   alpha = 1 + d/N_f,
 *   dL_b/dt = tau_b - xi L_b (+ the free rotor),
 *   dV/dt = d V v_e,     v_e = p_e / W,
 *   dp_e/dt = alpha sum m v^2 + Tr(Wvir) - d V P - xi p_e,
 *   dxi/dt = (2K + p_e^2/W - (g + 1) kT) / Q,   Q = (g + 1) kT tau^2,
 * N_f = d (N - 1), W = (N_f + d) kT tau_P^2, Wvir = sum_{i<j} x_ij (x) f_ij.
 * Conserved: K + U + p_e^2/(2W) + P V + (g + 1) kT (tau^2 xi^2 / 2 + eta).
 * One step: T(dt/2) B(dt/2) V(dt/2) X(dt) [forces] V(dt/2) B(dt/2) T(dt/2),
 * each factor solved exactly:
 *   T: the thermostat (as for NVT, also scaling p_e);
 *   B: p_e += delta (alpha 2 K_t + Tr(Wvir) - d V P);
 *   V: v <- v exp(-alpha v_e delta) + (F/m) delta exp(-alpha v_e delta/2)
 *        sinhc(alpha v_e delta/2), L_b += delta tau_b;
 *   X: x <- x exp(v_e dt) + v dt exp(v_e dt/2) sinhc(v_e dt/2), box <- box
 *        exp(v_e dt), then the free rotor over dt. */
static void thermostat_npt(sys_t *S, double *vel, double *Lb, double *pe, double W,
                           double *xi, double *eta, double g1, double kT, double tau,
                           double delta) {
    double Kt, Kr;
    kinetic(S, vel, Lb, &Kt, &Kr);
    double K = Kt + Kr + 0.5 * (*pe) * (*pe) / W;
    *xi += 0.5 * delta * (2.0 * K / (g1 * kT) - 1.0) / (tau * tau);
    double s = exp(-(*xi) * delta);
    int tdim = S->dim == 3 ? 3 : 1;
    for (int i = 0; i < S->n * S->dim; ++i) vel[i] *= s;
    for (int i = 0; i < S->n * tdim; ++i) Lb[i] *= s;
    *pe *= s;
    *eta += (*xi) * delta;
    K *= s * s;
    *xi += 0.5 * delta * (2.0 * K / (g1 * kT) - 1.0) / (tau * tau);
}

static double volume(int dim, const double *box) {
    double V = 1.0;
    for (int a = 0; a < dim; ++a) V *= box[a];
    return V;
}

static double virial_trace(sys_t *S) {
    return S->virial[0] + S->virial[4] + (S->dim == 3 ? S->virial[8] : 0.0);
}

/* Run nsteps of NVE (ensemble 0), NVT (ensemble 1) or NPT (ensemble 2) from
 * the given state.  angmom is world-frame (3D n*3, 2D n); thermo = {xi, eta,
 * p_e} (p_e only for NPT); box (dim lengths) is updated by NPT; P and tau_P
 * are the NPT pressure and barostat time.  trace, if not NULL, receives per
 * step {K_trans, K_rot, U, H, V} after the step, where H is the conserved
 * quantity (K + U for NVE).  Returns 0, or -1 on bad input. */
int oracle_run(int dim, int n_shapes, const int *vert_off, const double *verts,
               const int *shape_face_off, const int *face_vert_off, const int *face_idx,
               const double *rounding, const double *mass, const double *inertia, double eps,
               double sigma, double par_eps, int n, const int *shape_id, double *pos,
               double *orient, double *vel, double *angmom, double *box, double *thermo,
               int nsteps, double dt, int ensemble, double kT, double tau, double P,
               double tau_P, double *trace) {
    shape_t *shapes = (shape_t *)malloc(sizeof(shape_t) * (n_shapes > 0 ? n_shapes : 1));
    int tdim = dim == 3 ? 3 : 1;
    double *force = (double *)malloc(sizeof(double) * dim * n);
    double *torque = (double *)malloc(sizeof(double) * tdim * n);
    double *energy = (double *)malloc(sizeof(double) * n);
    double *Lb = (double *)malloc(sizeof(double) * tdim * n);
    double *tb = (double *)malloc(sizeof(double) * tdim * n);
    if (!shapes || !force || !torque || !energy || !Lb || !tb) return -2;
    if (build_shapes(dim, n_shapes, vert_off, verts, shape_face_off, face_vert_off, face_idx,
                     rounding, shapes)) return -1;
    sys_t S = {dim, n, shapes, shape_id, mass, inertia, eps, sigma, par_eps, box,
               force, torque, energy, {0}};

    /* degrees of freedom: translational d(N-1), one rotational per I_k > 0 */
    double g = dim * (n - 1.0);
    for (int i = 0; i < n; ++i) {
        const double *I = inertia + 3 * shape_id[i];
        if (dim == 3) { for (int k = 0; k < 3; ++k) g += I[k] > 0.0; }
        else g += I[0] > 0.0;
    }

    /* world -> body angular momentum */
    for (int i = 0; i < n; ++i) {
        if (dim == 3) {
            double R[3][3];
            quat_to_mat(orient + 4 * i, R);
            v3 lb = mat_t_vec(R, mk(angmom[3 * i], angmom[3 * i + 1], angmom[3 * i + 2]));
            Lb[3 * i] = lb.x; Lb[3 * i + 1] = lb.y; Lb[3 * i + 2] = lb.z;
        } else {
            Lb[i] = angmom[i];
        }
    }
    double xi = thermo ? thermo[0] : 0.0, eta = thermo ? thermo[1] : 0.0;
    double pe = (thermo && ensemble == 2) ? thermo[2] : 0.0;
    const double Nf = dim * (n - 1.0), alpha = 1.0 + dim / Nf;
    const double W = (Nf + dim) * kT * tau_P * tau_P;
    if (ensemble == 2 && !(n >= 2 && tau_P > 0.0)) return -1;
    double U = compute_forces(&S, pos, orient);

    for (int step = 0; step < nsteps; ++step) {
        if (ensemble == 1) thermostat(&S, vel, Lb, &xi, &eta, g, kT, tau, 0.5 * dt);
        if (ensemble == 2) {
            thermostat_npt(&S, vel, Lb, &pe, W, &xi, &eta, g + 1.0, kT, tau, 0.5 * dt);
            pe += 0.5 * dt * (alpha * 2.0 * kinetic_trans(&S, vel) + virial_trace(&S) -
                              dim * volume(dim, box) * P);
        }
        const double ve = ensemble == 2 ? pe / W : 0.0;
        /* velocity factors of the V(dt/2) step (1 and dt/2 without a barostat) */
        const double av = exp(-alpha * ve * 0.5 * dt);
        const double bv = 0.5 * dt * exp(-alpha * ve * 0.25 * dt) * sinhc(alpha * ve * 0.25 * dt);
        for (int half = 0; half < 2; ++half) {
            /* half kick with the force and the body-frame torque */
            for (int i = 0; i < n; ++i) {
                double m = mass[shape_id[i]];
                for (int a = 0; a < dim; ++a)
                    vel[dim * i + a] = vel[dim * i + a] * av + bv * force[dim * i + a] / m;
                if (dim == 3) {
                    double R[3][3];
                    quat_to_mat(orient + 4 * i, R);
                    v3 t = mat_t_vec(R, mk(torque[3 * i], torque[3 * i + 1], torque[3 * i + 2]));
                    Lb[3 * i] += 0.5 * dt * t.x; Lb[3 * i + 1] += 0.5 * dt * t.y;
                    Lb[3 * i + 2] += 0.5 * dt * t.z;
                } else {
                    Lb[i] += 0.5 * dt * torque[i];
                }
            }
            if (half == 1) break;
            /* drift (with the box dilation under NPT), free rotation, wrap */
            const double ax = exp(ve * dt), bx = dt * exp(0.5 * ve * dt) * sinhc(0.5 * ve * dt);
            if (ensemble == 2)
                for (int a = 0; a < dim; ++a) box[a] *= ax;
            for (int i = 0; i < n; ++i) {
                for (int a = 0; a < dim; ++a) {
                    double x = pos[dim * i + a] * ax + bx * vel[dim * i + a];
                    x -= box[a] * floor(x / box[a]);
                    if (x >= box[a]) x -= box[a];
                    pos[dim * i + a] = x;
                }
                const double *I = inertia + 3 * shape_id[i];
                if (dim == 3) {
                    double *q = orient + 4 * i, *L = Lb + 3 * i;
                    free_rotor_axis(q, L, I, 2, 0.5 * dt);
                    free_rotor_axis(q, L, I, 1, 0.5 * dt);
                    free_rotor_axis(q, L, I, 0, dt);
                    free_rotor_axis(q, L, I, 1, 0.5 * dt);
                    free_rotor_axis(q, L, I, 2, 0.5 * dt);
                    double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
                    for (int k = 0; k < 4; ++k) q[k] /= nq;
                } else if (I[0] > 0.0) {
                    orient[i] += Lb[i] / I[0] * dt;
                }
            }
            U = compute_forces(&S, pos, orient);
        }
        if (ensemble == 1) thermostat(&S, vel, Lb, &xi, &eta, g, kT, tau, 0.5 * dt);
        if (ensemble == 2) {
            pe += 0.5 * dt * (alpha * 2.0 * kinetic_trans(&S, vel) + virial_trace(&S) -
                              dim * volume(dim, box) * P);
            thermostat_npt(&S, vel, Lb, &pe, W, &xi, &eta, g + 1.0, kT, tau, 0.5 * dt);
        }
        if (trace) {
            double Kt, Kr;
            kinetic(&S, vel, Lb, &Kt, &Kr);
            double H = Kt + Kr + U;
            if (ensemble == 1) H += g * kT * (0.5 * tau * tau * xi * xi + eta);
            if (ensemble == 2)
                H += 0.5 * pe * pe / W + P * volume(dim, box) +
                     (g + 1.0) * kT * (0.5 * tau * tau * xi * xi + eta);
            trace[5 * step + 0] = Kt; trace[5 * step + 1] = Kr;
            trace[5 * step + 2] = U;  trace[5 * step + 3] = H;
            trace[5 * step + 4] = volume(dim, box);
        }
    }
    /* body -> world angular momentum */
    for (int i = 0; i < n; ++i) {
        if (dim == 3) {
            double R[3][3];
            quat_to_mat(orient + 4 * i, R);
            v3 lw = mat_vec(R, mk(Lb[3 * i], Lb[3 * i + 1], Lb[3 * i + 2]));
            angmom[3 * i] = lw.x; angmom[3 * i + 1] = lw.y; angmom[3 * i + 2] = lw.z;
        } else {
            angmom[i] = Lb[i];
        }
    }
    if (thermo) { thermo[0] = xi; thermo[1] = eta; if (ensemble == 2) thermo[2] = pe; }
    free(shapes); free(force); free(torque); free(energy); free(Lb); free(tb);
    return 0;
}
