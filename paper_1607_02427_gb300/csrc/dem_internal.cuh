// dem_internal.cuh -- device data layout and launch wrappers shared by the
// translation units of libdem (not part of the public ABI).
//
// Layout in HBM (N particles over all replicas, R replicas):
//   pos, vel, quat, angmom_b, force, torque_b, x_last : double4_32a[N]
//       (w unused; 32-byte records so a neighbour gather is one sector)
//   quatf        : float4[N]  FP32 copy of quat read by the FP32 pair kernels
//   shape, rep   : int[N]     shape index and replica index of each particle
//   energy, ke   : double[N]  per-particle potential / kinetic energy
//   virial       : double[6N] symmetric per-particle virial
//   nlist        : float4[cap * N], column-major (slot k of particle i at
//                  k*N+i): x, y, z = x_j - x_i (minimum image, FP32) when the
//                  list was built, w = the bits of the int j
//   delta        : float4[N]  x_i - x_i(list build) (minimum image, FP32), so
//                  that x_j - x_i = d0 + delta_j - delta_i between builds
//   nn           : int[N]     neighbour count
//   cell_count   : int[C]     particles per cell (C cells over all replicas)
//   cell_slots   : int[C * cell_cap]
//   reps         : Rep[R]     box, particle range and cell grid per replica
//   geometry table: Real4 records per distinct shape geometry (see Geom)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dem.h"

namespace dem {

constexpr int MAX_VERTS = 128;      // vertices of one shape
constexpr int MAX_EDGES = 128;      // edges of one shape
constexpr int MAX_FACES = 128;      // faces of one shape
constexpr int NARROW_FEATURES = 32; // up to this many of each: one-word feature masks;
                                    // more: WIDE_WORDS words (THREAD decomposition)
constexpr int WIDE_WORDS = 4;
constexpr int MAX_FACE_VERTS = 12;  // vertices of one face
constexpr int MAX_GEOMS = 64;       // distinct geometries per context
constexpr int THREADS = 128;

// One distinct geometry.  Offsets count Real4 records in the geometry table.
//   verts:  nv records  (x, y, z, 0)
//   edges:  2 ne records: a = (start, half length), d = (vector, 1/|d|^2)
//   faces:  nf records  n = (unit outward normal, n . a0)
//   fedges: 3 nfe records per face edge: a = (start, 0),
//           e = (vector, 1/|e|^2), m = (inward in-plane normal, m . a)
//   face k uses fedges [fe_begin[k], fe_begin[k] + fe_count[k]) (ints table)
//   int table also: a 32-bit mask of the vertices of each edge and each face
struct Geom {
    int nv, ne, nf, nfe;
    int v_off, e_off, f_off, fe_off;
    int fi_off;          // offset of this geometry's faces in the int table
    float R;             // circumradius of the inner shape
    int vem_off;         // int table: per vertex, the mask of its edges
    int vfm_off;         // int table: per vertex, the mask of its faces
};

struct ShapeDev {
    int geom;
    float R;             // circumradius (copy of the geometry's)
    double rounding;
    double mass;
    double inertia[3];   // principal moments (2D: inertia[2] = I_z)
    double inv_inertia[3];  // 1 / inertia[k], 0 where inertia[k] = 0
    double inv_mass;
    float rounding_f;    // FP32 copy of rounding for the FP32 kernels
    float rounding_lo;   // rounding - rounding_f (FP32 + two-sum refinement)
};

// An FP64 value as the unevaluated sum of two floats hi + lo.
__host__ __device__ inline void split_ff(double x, float *h, float *l) {
    const float hi = (float)x;
    *h = hi;
    *l = (float)(x - (double)hi);
}

struct Rep {
    double L[3];
    double inv_L[3];     // 1 / L[k]
    int off, n;          // particle range
    int cell_off;        // first cell of this replica in the global cell arrays
    int nc[3];           // cells per axis
    int allpairs;        // 1: neighbour search over all particles of the replica
    int g_dof;           // degrees of freedom for the thermostat (as int)
    double r_list;       // neighbour-list cutoff (largest pair range + skin)
    double L_build0;     // L[0] when the list was last built
    double sc_d;         // L[0] / L_build0: list separations scale with the box (NPT)
    float sc;            // FP32 copy of sc_d for the FP32 pair kernels
    float disp_pad;      // 0.5 max(0, 1 - sc) r_list, added to displacements in the
                         // rebuild test so that a shrinking box cannot hide a pair
    int chunk_off, n_chunk;   // this replica's reduction chunks (see SUM_CHUNK)
    float Lf[3], Lf_lo[3];    // L as hi + lo floats (FP32 + two-sum refinement)
};

// Fill the float-float copies of a replica's box lengths.
__host__ __device__ inline void rep_box_ff(Rep &rp) {
    for (int k = 0; k < 3; ++k) split_ff(rp.L[k], &rp.Lf[k], &rp.Lf_lo[k]);
}

// Per-step replica sums run over fixed chunks of SUM_CHUNK particles (one
// block each), then over each replica's chunk partials: a fixed order, and
// a large replica is not summed by a single block.
constexpr int SUM_CHUNK = 1024;

// Device status word block.
struct Status {
    unsigned int maxdisp2;   // max squared displacement since last build (float bits)
    int rebuild;             // forced rebuild request
    int nlist_overflow;      // needed capacity if the list overflowed (else 0)
    int cell_overflow;       // needed cell capacity if a cell overflowed
    int nonfinite;           // 1 if a non-finite force/energy was produced
    int rebuilds;            // rebuild counter
    int built;               // set by the list build when it ran this step
    int box_limit;           // NPT: a box fell below what its cell grid or minimum
                             // image allows within the call
    int bad_input;           // 1 + index of a particle whose imported state was not
                             // finite or whose quaternion had zero norm (else 0)
    int term_overflow;       // SPLIT, FP32 + two-sum: terms a warp needed beyond its
                             // region of the term buffer (the largest count), else 0
};

// Per-replica thermostat state (FP64): canonical end-of-step values and the
// values after the first Trotter half step of the step in progress.
struct Thermo {
    double xi, eta, K;       // canonical (end of the last completed step)
    double xi_h, eta_h;      // after this step's first half step
    double s1;               // velocity scale of this step's first half step
    double s2;               // velocity scale of this step's second half step
    double pe;               // NPT: barostat momentum (canonical)
    double pe_h;             // NPT: after this step's first half step
    double av, bv;           // NPT: v <- av v + bv F/m (half kick with dilation)
    double ax, bx;           // NPT: x <- ax x + bx v, box <- ax box (drift)
    double pad;
};

struct PairArgs {
    int n, dim, cap;
    const double4_32a *pos;
    const double4_32a *quat;
    const float4 *quatf;
    const int *shape, *rep;
    const Rep *reps;
    const ShapeDev *shapes;
    const Geom *geoms;
    int n_geoms;
    const void *table;       // float4 or double4_32a records
    int table_len;           // records
    const int *itable;       // face -> (fe_begin, fe_count) pairs
    int itable_len;
    const float4 *nlist;
    const int *nn;
    const float4 *delta;
    double4_32a *force, *torque;
    double *energy, *virial;
    double eps, sigma, par_eps;
    Status *status;
    unsigned long long *counters;  // counting launches only
    // SPLIT decomposition: active-pair records of each group of `group`
    // particles (32, 16, 8 or 4; group g at recs + g * group * cap records)
    // and their counts
    void *recs;
    int *rec_count;
    int group;
    // FP32 + two-sum refinement of the terms (NULL in the other modes): the
    // FP64 state split into hi + lo floats
    const float4 *quatf_lo;  // q - quatf
    const float4 *xff;       // per particle: (x, y, z) hi, then (x, y, z) lo
    const float4 *table_lo;  // geometry records minus their FP32 copies
    float sigma_f, sigma_lo; // the one sigma of all pairs (when sigma > 0)
    // SPLIT in the FP32 + two-sum mode: the feature kernel writes every term
    // it finds (features, parameters, pair data) to its warp's region of
    // term_capw records; a term kernel refines them.  Per group of particles:
    // the first record and the count.
    float4 *term_a, *term_b;  // (s, t, r_cut^2, spec code), (dl, j)
    int *term_info;           // owner | gi << 8 | gj << 16 | jref << 24
    int *term_start, *term_cnt;
    int term_capw;
    int term_ppw;             // the term kernel's particles per warp (set at its launch)
    // SPLIT: particles per slice (0: all at once).  The three kernels run
    // slice after slice, so that a slice's active-pair and term records are
    // read back while they are still in L2; [p_lo, p_hi) is the slice of a
    // launch (set at the launch)
    int slice;
    int p_lo, p_hi;
    int mask_words;           // words per feature mask and incidence row: 1, or
                              // WIDE_WORDS when a shape has more than 32 features
};
// Upper bound of the warps of SPLIT's feature kernel (regions of the term
// buffer), and the launch of its term kernel (FP32 + two-sum).
int split_apply_max_warps();

// Bytes of one active-pair record of the SPLIT decomposition.
size_t pair_record_bytes(int precision);
// Particles per warp group of the SPLIT kernels for n particles.
int split_group(int n);

struct NlistArgs {
    int n, dim, cap, cell_cap;
    const double4_32a *pos;
    const int *shape, *rep;
    const Rep *reps;
    const ShapeDev *shapes;
    double sigma, skin;
    int *cell_count, *cell_slots;
    float4 *nlist;
    int *nn;
    double4_32a *x_last;
    float4 *delta;
    Status *status;
    float half_skin2;        // rebuild threshold (skin/2)^2
    Rep *reps_rw;            // a rebuild records the box it was built in
    float4 *posf;            // FP32 positions for the candidate test (w: shape index)
};

struct StepArgs {
    int n, dim, n_reps;
    double dt;
    int nvt;
    double kT, tau;
    double4_32a *pos, *vel, *quat, *angmom, *x_last;
    float4 *quatf, *delta;
    const double4_32a *force, *torque;
    const int *shape, *rep;
    const Rep *reps;
    const ShapeDev *shapes;
    double *ke;
    Thermo *thermo;
    Status *status;
    int rotor32;             // FP32 modes: free-rotor increments in FP32
    int npt;                 // isotropic barostat (ensemble DEM_NPT)
    double P, tau_P;         // NPT pressure and barostat time
    double *ket;             // NPT: translational kinetic energy per particle
    const double *virial;    // per-particle virial (xx, xy, xz, yy, yz, zz)
    Rep *reps_rw;            // the replica records (NPT moves the box)
    int n_chunks;            // reduction chunks over all replicas
    const int *chunk_rep;    // replica of each chunk
    double *partial;         // n_chunks * 3 chunk sums: K, K_trans (NPT), Tr W (NPT)
    int direct_sums;         // NVE/NVT, every replica small: k_thermo_end sums the kinetic
                             // energies itself and, under NVT, applies the second scaling
    float4 *quatf_lo, *xff;  // FP32 + two-sum: hi + lo state (NULL otherwise)
    int int_conv;            // the first half step converts double <-> float by integer
                             // operations (large systems) or by the instructions
};

// Cooperative multi-step kernel (persistent.cu): control block in device
// memory, cleared by the host before each launch.
struct CoopCtl {
    unsigned bar_count, bar_gen;   // grid barrier: arrivals, generation
    int abort;                     // a block gave up waiting: every block returns
    int timeout;                   // the reason was a wait past the time limit
    int steps_done;                // steps completed (a stop: its first half done)
    int stop;                      // 1: stopped for a list rebuild after a first half step
    int kmax;                      // longest neighbour list of the launch
    unsigned maxd[2];              // per-step maximum squared displacement (float bits),
                                   // by step parity
};

struct CoopArgs {
    PairArgs p;
    StepArgs s;
    CoopCtl *ctl;
    void *part;                    // partial sums per list entry: component c of entry
                                   // (i, k) at [(c * cap + k) * n + i] (float or double)
    unsigned char *act;            // entry (i, k) is an active pair: act[k * n + i]
    int n_steps;
    int resume;                    // 1: the first step starts at the pair phase
    float half_skin2;              // rebuild threshold (skin/2)^2
    long long limit_ns;            // barrier wait limit
    int test_stall;                // test hook: block 0 never reaches a barrier
};
size_t coop_partial_bytes(int precision, int n, int cap);
// Blocks of the cooperative launch (0 when the kernel cannot run).
int coop_grid(int precision, int dim, int n, int cap, size_t smem);
cudaError_t launch_coop_steps(const CoopArgs &c, int precision, int dim, int grid, size_t smem,
                              cudaStream_t s);

// ---- launch wrappers (pair.cu, nlist.cu, integrate.cu) ----
cudaError_t launch_pair(const PairArgs &a, int precision, int decomp, int block, bool count,
                        cudaStream_t s);
size_t pair_smem_bytes(const PairArgs &a, int precision);
// STAGED decomposition (pair_staged.cu); smem_tables = pair_smem_bytes().
cudaError_t launch_pair_staged(const PairArgs &a, int precision, bool count, size_t smem_tables,
                               cudaStream_t s);
// SPLIT decomposition (pair_staged.cu): a scan kernel writes the active pairs,
// a feature kernel evaluates them.
cudaError_t launch_pair_split(const PairArgs &a, int precision, bool count, size_t smem_tables,
                              cudaStream_t s);
cudaError_t launch_cells(const NlistArgs &a, int n_cells, cudaStream_t s);
cudaError_t launch_nlist(const NlistArgs &a, cudaStream_t s);
cudaError_t launch_first_half(const StepArgs &a, cudaStream_t s);
// the rebuild test and the FP32 deltas for positions set from outside
cudaError_t launch_displacement(const StepArgs &a, cudaStream_t s);
cudaError_t launch_second_half(const StepArgs &a, cudaStream_t s);
cudaError_t launch_thermo_begin(const StepArgs &a, cudaStream_t s);
cudaError_t launch_thermo_end(const StepArgs &a, cudaStream_t s);
cudaError_t launch_box(const StepArgs &a, cudaStream_t s);
cudaError_t launch_chunk_sums(const StepArgs &a, cudaStream_t s);
cudaError_t launch_scale(const StepArgs &a, cudaStream_t s);
cudaError_t launch_kinetic(const StepArgs &a, cudaStream_t s);
cudaError_t launch_replica_sums(int n_reps, const Rep *reps, const double *per_particle,
                                int stride, int comps, double *out, cudaStream_t s);
cudaError_t launch_prepare_state(int n, int dim, double4_32a *pos, double4_32a *quat, float4 *quatf,
                                 float4 *quatf_lo, float4 *xff,
                                 double4_32a *angmom, const int *rep, const Rep *reps,
                                 int world_to_body, cudaStream_t s);
cudaError_t launch_check_conversions(unsigned long long n, unsigned long long seed,
                                    unsigned long long *bad, cudaStream_t s);
// FP32 / float-float copies of an FP64 state restored unchanged (snapshots).
cudaError_t launch_refresh_copies(int n, const double4_32a *pos, const double4_32a *quat,
                                  float4 *quatf, float4 *quatf_lo, float4 *xff, cudaStream_t s);
cudaError_t launch_export_state(int n, int dim, const double4_32a *pos, const double4_32a *quat,
                                const double4_32a *vel, const double4_32a *angmom, double *pos_out,
                                double *orient_out, double *vel_out, double *angmom_out,
                                cudaStream_t s);
cudaError_t launch_import_state(int n, int dim, const double *pos_in, const double *orient_in,
                                const double *vel_in, const double *angmom_in, double4_32a *pos,
                                double4_32a *quat, double4_32a *vel, double4_32a *angmom,
                                Status *status, cudaStream_t s);
cudaError_t launch_export_forces(int n, int dim, const double4_32a *force, const double4_32a *torque_b,
                                 const double4_32a *quat, double *force_out, double *torque_out,
                                 cudaStream_t s);
cudaError_t launch_rescale(int n, int dim, double4_32a *pos, double4_32a *x_last, const int *rep,
                           const double *scale3, cudaStream_t s);

// Geometry tables of a shape set built on the host, in the layout the pair
// kernels read (api.cu).
struct HostTables {
    std::vector<float4> tf_lo;    // td - tf per component (FP32 + two-sum refinement)
    int mask_words = 1;           // 1, or WIDE_WORDS for shapes beyond 32 features
    int dim = 3;
    std::vector<float4> tf;
    std::vector<double4_32a> td;
    std::vector<int> itab;
    std::vector<Geom> geoms;
    std::vector<ShapeDev> shapes;
    double Rmax = 0, rnd_max = 0;
};
int make_host_tables(const dem_shape *shapes, int n_shapes, HostTables *t, std::string *err);

// Centre distance within which two particles of bounding radii up to Rmax
// (the padded FP32 radii of the geometry records) can interact, plus the
// list skin: 2 Rmax + r_cut(sigma_max) + skin, the radii enlarged by 1e-6
// relative so that no rounding can bring an interacting pair beyond it.
inline double pair_range(double Rmax, double sig_max, double skin) {
    return 2.0 * Rmax * (1.0 + 1e-6) + 1.122462048309373 * sig_max + skin;
}
void set_global_error(const std::string &msg);

}  // namespace dem
