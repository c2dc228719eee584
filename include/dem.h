/*
 * dem.h -- C ABI of libdem, a GB300 (sm_103a) implementation of the
 * discrete element method for conservative, faceted (rounded polygon and
 * polyhedron) particles of Spellings, Marson, Anderson & Glotzer,
 * arXiv:1607.02427.
 *
 * What the library computes (Section "Model"):
 *   Each particle is an inner polygon (2D) or polyhedron (3D), convex or
 *   concave, rounded by a disk/sphere of radius sigma/2.  Particles i and j interact through
 *   the WCA potential (Eq. LJ, Eq. WCA; r_cut = 2^(1/6) sigma) evaluated at
 *   the nearest-point distance of every feature pair:
 *     3D (Eq. DEM):    all edge-edge pairs, all vertex(i)-face(j) pairs and
 *                      all vertex(j)-face(i) pairs;
 *     2D (Eq. DEM_2D): all vertex(i)-edge(j) and vertex(j)-edge(i) pairs.
 *   Each term's force acts along the line joining its nearest points, and
 *   its torque about each particle's centre uses that particle's nearest
 *   point.  Nearly parallel edges interact at the midpoint of their overlap
 *   (parallel-edge rule, Section "Model").  Feature overcounting is kept
 *   (Section "Model").  Two one-vertex shapes (disks/spheres) interact
 *   through one central WCA term (the sphere limit).
 *   The particles move with velocity Verlet and a symmetric body-axis
 *   free-rotor splitting (a second-order integrator, Section "Energy
 *   Conservation"), optionally coupled to a Nose-Hoover thermostat acting
 *   on translational and rotational degrees of freedom (Section
 *   "Assembly").
 *
 * Conventions for every call:
 *   * Returns DEM_OK (0) or a negative DEM_ERR_* code; dem_last_error()
 *     gives a one-line reason.  Nothing throws across the ABI.
 *   * "host" arrays are read or written during the call and never kept.
 *     When a call takes device_ptrs = 1 the same arrays are CUDA device
 *     pointers (for example torch tensors) instead; they are used on the
 *     context's stream and must stay valid until the call returns.
 *   * The library owns all of its device memory; dem_destroy frees it.
 *   * N is the total particle count over all replicas; particles of replica
 *     r are the contiguous block after those of replicas 0..r-1.
 *   * dim is 2 or 3 and is the same for every shape of a context.
 *   * Positions are periodic in each replica's orthorhombic box [0, L_a).
 *   * Orientation: 3D unit quaternion (w, x, y, z) rotating body to world;
 *     2D angle theta (radians).
 *   * Angular momentum: 3D world-frame vector; 2D scalar L_z.
 *   * Mass and inertia: per shape; shapes must be given in their principal
 *     axes (the inertia tensor of the body frame is diagonal).
 *   * All floating-point values cross the ABI as double.
 */
#ifndef DEM_H
#define DEM_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define DEM_OK 0
#define DEM_ERR_ARG (-1)             /* invalid argument or shape             */
#define DEM_ERR_CUDA (-2)            /* a CUDA call failed                     */
#define DEM_ERR_NONFINITE (-3)       /* a force, torque or energy is not finite */
#define DEM_ERR_NLIST_OVERFLOW (-4)  /* neighbour list still overflowing after
                                        growing it and retrying the call       */
#define DEM_ERR_TIMEOUT (-5)         /* a bounded device wait gave up          */
#define DEM_ERR_BOX (-6)             /* box below twice the neighbour cutoff   */
#define DEM_ERR_STATE (-7)           /* no state set yet                       */
#define DEM_ERR_NOMEM (-8)           /* device allocation failed               */

/* ---- precision modes of the pair kernel ---- */
#define DEM_FP64 0        /* geometry, force and accumulation in FP64            */
#define DEM_FP32 1        /* geometry and force in FP32, plain FP32 sums        */
#define DEM_FP32_COMP 2   /* culls and nearest-point searches in FP32; every term
                             found (r < r_cut) re-evaluated in float-float (pairs
                             of floats, about 48 bits) from the FP64 state: its
                             nearest points, WCA force and torque; compensated
                             (two-sum) sums of force and torque                 */
/* In every mode positions, velocities, orientations, angular momenta,
 * per-particle energies and virials are held in FP64.  In the FP32 modes the
 * neighbour list keeps each pair's separation d0 = x_j - x_i of the last
 * list build (taken in FP64, rounded to FP32) and each particle keeps its
 * displacement delta since that build (FP64, rounded to FP32); the pair
 * kernels' searches form x_j - x_i = d0 + delta_j - delta_i in FP32.
 * DEM_FP32_COMP re-evaluates each term from the positions, quaternions and
 * geometry split into hi + lo floats, so its forces and torques follow the
 * FP64 definition to about 1e-7 of each particle's own force (DEM_FP32:
 * about 1e-4 where a particle's terms cancel). */

/* ---- ensembles ---- */
#define DEM_NVE 0
#define DEM_NVT 1
#define DEM_NPT 2   /* NVT plus an isotropic barostat (dem_set_barostat)      */

/* ---- pair-kernel decompositions (parameter "decomp") ---- */
#define DEM_DECOMP_AUTO 0    /* chosen by dem_autotune (default: THREAD)        */
#define DEM_DECOMP_THREAD 1  /* one thread walks all neighbours of particle i   */
#define DEM_DECOMP_WARP 2    /* one warp per 32 particles: the lanes scan their
                                list entries, queue the pairs that pass the
                                culls, and evaluate 32 queued pairs at a time,
                                one per lane; each particle's lane sums its
                                pairs in queue order                           */
#define DEM_DECOMP_STAGED 3  /* one warp per 32 particles streams their work
                                through shared-memory queues: (pair, vertex)
                                and (pair, edge) items with the cheap tests,
                                then the queued survivors (face nearest point,
                                segment-segment, WCA terms) 32 at a time       */
#define DEM_DECOMP_SPLIT 4   /* STAGED in two kernels: a list scan writes the
                                active pairs of each group of G particles
                                ("split_group") to device memory (N *
                                nlist_cap records), a feature kernel runs the
                                queues on them; with DEM_FP32_COMP a third
                                kernel refines the terms the feature kernel
                                found                                          */

typedef struct dem_ctx dem_ctx;   /* opaque; owned by the library */

/* A shape (Section "Model": features V, E, F of the inner shape, rounded by
 * radius sigma/2).
 *   dim            2 or 3
 *   n_verts        number of vertices, >= 1 (1 = disk / sphere)
 *   verts          n_verts * dim body-frame coordinates, centred on the
 *                  centre of mass, in principal axes
 *   n_faces        3D: number of faces (0 for a sphere, else >= 4);
 *                  2D: ignored (the polygon is the vertex loop: simple and
 *                  counter-clockwise, convex or not; 2 vertices make one edge)
 *   face_offsets   3D: n_faces + 1 offsets into face_verts
 *   face_verts     3D: vertex indices of each face, counter-clockwise seen
 *                  from outside; each face must be convex and planar, and
 *                  the faces must close the surface (every edge bounds two
 *                  faces, traversed in opposite directions)
 *   rounding_radius  sigma/2 of the shape (> 0)
 *   mass           > 0
 *   inertia        3D: 3 principal moments, 2D: 1 (I_z); NULL derives them
 *                  for a uniform-density inner solid of the given mass.
 * The inner shape may be concave (Section "Model"); only its faces must be
 * convex, because the nearest point on a face is found by its edge tests.
 * A self-intersecting 3D surface is not detected and is the caller's
 * responsibility.  3D edges are derived from the faces.  A shape has at
 * most 128 vertices, 128 edges, 128 faces and 12 vertices per face.  Up to
 * 32 of each, the pair kernels cull features with one 32-bit mask per kind;
 * a context holding a larger shape uses two-level masks (four words, empty
 * words skipped) and runs the THREAD decomposition only ("decomp" refuses
 * the others, dem_autotune times THREAD alone).
 * Rejected with DEM_ERR_ARG: a 2D polygon with clockwise order, meeting
 * non-neighbour edges or a fold; a 3D face that is not planar or convex; an
 * open or inconsistently oriented surface; a non-positive enclosed volume. */
typedef struct dem_shape {
    int dim;
    int n_verts;
    const double *verts;
    int n_faces;
    const int *face_offsets;
    const int *face_verts;
    double rounding_radius;
    double mass;
    const double *inertia;
} dem_shape;

/* Create a context for n_replicas independent periodic systems.
 *   shapes/n_shapes  shape table (copied)
 *   epsilon          WCA energy scale (Eq. LJ)
 *   sigma            > 0: one sigma for all pairs; <= 0: sigma_ij =
 *                    rounding_i + rounding_j (Eq. WCA's rounding radius
 *                    sigma_ij / 2 per particle)
 *   box              n_replicas * dim box lengths
 *   replica_sizes    n_replicas particle counts (>= 1 each)
 *   precision        DEM_FP64, DEM_FP32 or DEM_FP32_COMP
 * Errors: DEM_ERR_ARG (bad shape, sizes, precision, box), DEM_ERR_CUDA,
 * DEM_ERR_NOMEM.  On error *out is NULL.  Whether each box is large enough
 * is checked by dem_set_state, once the shape of every particle is known. */
int dem_create(dem_ctx **out, const dem_shape *shapes, int n_shapes, double epsilon,
               double sigma, const double *box, int n_replicas, const int *replica_sizes,
               int precision);

/* Set the state of all N particles (host or device arrays):
 *   shape_id  N ints in [0, n_shapes)
 *   pos       N * dim (wrapped into the box by the library)
 *   orient    3D: N * 4 quaternions (w,x,y,z), normalised by the library;
 *             2D: N angles
 *   vel       N * dim
 *   angmom    3D: N * 3 world-frame angular momenta; 2D: N values of L_z
 * Evaluates forces and resets the thermostat variables to zero.  The
 * neighbour list is rebuilt when any shape id differs from the previous
 * call's, or when a particle lies more than skin/2 from its position at the
 * last build (the test a step makes); otherwise the list is kept, which is
 * exact: it holds every pair within the interaction range.
 * Errors: DEM_ERR_ARG (a shape id out of range; a non-finite position,
 * orientation, velocity or angular momentum, or a quaternion of zero norm:
 * checked on the device as the arrays are imported, host or device alike),
 * DEM_ERR_BOX (a box edge below twice the neighbour-list cutoff
 * R_i + R_j + r_cut + skin of the replica's largest shapes), DEM_ERR_CUDA,
 * DEM_ERR_NONFINITE (the forces of the state are not finite, e.g. two
 * particles that coincide).  After an error the context has no state
 * (dem_step returns DEM_ERR_STATE) until a dem_set_state succeeds. */
int dem_set_state(dem_ctx *ctx, const int *shape_id, const double *pos, const double *orient,
                  const double *vel, const double *angmom, int device_ptrs);

/* Read the state (host or device arrays; any pointer may be NULL):
 * pos N*dim, orient N*4 (3D) or N (2D), vel N*dim, angmom N*3 (3D, world
 * frame) or N (2D), thermostat n_replicas * 3 (xi, eta, p_e). */
int dem_get_state(dem_ctx *ctx, double *pos, double *orient, double *vel, double *angmom,
                  double *thermostat, int device_ptrs);

/* Set the extended variables of each replica (host array, n_replicas * 3):
 * the Nose-Hoover friction xi, its time integral eta, and the barostat
 * momentum p_e (used by DEM_NPT; 0 otherwise). */
int dem_set_thermostat(dem_ctx *ctx, const double *thermostat);

/* Barostat of DEM_NPT steps: pressure P >= 0 and time constant tau_P > 0.
 * Section "Assembly" runs NPT with a Nose-Hoover thermostat on translation
 * and rotation and a barostat that takes the pressure from the virial
 * tensor as in MD, citing Tuckerman et al. (J. Phys. A 39, 5629 (2006)); the
 * paper gives no formulas.  This library integrates the MTK equations for an
 * isotropically scaled box (each replica its own), with one thermostat
 * shared by the particles and the barostat:
 *   dx/dt = v + v_e x, dv/dt = F/m - alpha v_e v - xi v, alpha = 1 + d/N_f,
 *   dV/dt = d V v_e, v_e = p_e / W, dp_e/dt = alpha sum m v^2 + Tr W_vir
 *   - d V P - xi p_e, dxi/dt = (2K + p_e^2/W - (g + 1) kT) / Q,
 * N_f = d (N_r - 1), W = (N_f + d) kT tau_P^2, Q = (g + 1) kT tau_T^2, by
 * the symmetric factorisation T B V X V B T of that paper, each factor
 * solved exactly.  Errors: DEM_ERR_ARG. */
int dem_set_barostat(dem_ctx *ctx, double P, double tau_P);

/* Current box lengths of every replica (host array, n_replicas * dim);
 * DEM_NPT steps change them. */
int dem_get_box(dem_ctx *ctx, double *box);

/* Advance all replicas n steps of size dt.
 *   ensemble  DEM_NVE, DEM_NVT (Nose-Hoover at temperature kT with
 *             time constant tau_T: dxi/dt = (2K/(g kT) - 1) / tau_T^2,
 *             g = dim (N_r - 1) + rotational degrees of freedom), or DEM_NPT
 *             (see dem_set_barostat; every replica needs N_r >= 2)
 * One step: thermostat half step (NVT, NPT), barostat half step (NPT), half
 * kick of v and L, drift (with the box dilation under NPT) and free
 * rotation, neighbour-list rebuild if some particle moved more than skin/2
 * since the last build (under NPT less the distance a shrinking box can
 * close), pair forces, half kick, barostat and thermostat half steps.  NPT
 * calls run in chunks of "npt_chunk" steps; between chunks the boxes come
 * back to the host and the cell grids follow them.
 * Execution: NVE and NVT calls on small systems (parameter "persistent")
 * run as cooperative launches of one kernel that does many whole steps,
 * with grid-wide barriers between the phases of a step; a list rebuild ends
 * a launch, the list is rebuilt and the next launch continues.  In the FP32
 * modes the result is bit-identical to the per-step kernels with the WARP
 * decomposition; in FP64 it agrees with them to rounding.
 * Other calls replay one captured CUDA graph per step ("graph").
 * Errors: DEM_ERR_ARG, DEM_ERR_STATE, DEM_ERR_NONFINITE,
 * DEM_ERR_NLIST_OVERFLOW (after an internal grow-and-retry from the state at
 * the start of the call), DEM_ERR_BOX (NPT: a box shrank by more than 5%
 * within a chunk or below twice the list cutoff), DEM_ERR_TIMEOUT (a barrier
 * of the cooperative kernel waited longer than "persistent_wait_ms"; the
 * state is restored to the start of the call and the context stays
 * usable), DEM_ERR_CUDA. */
int dem_step(dem_ctx *ctx, int n, double dt, int ensemble, double kT, double tau_T);

/* Evaluate forces, torques, energies and virials at the current state. */
int dem_compute(dem_ctx *ctx);

/* Forces (N*dim, world frame) and torques about each centre (3D N*3 world
 * frame; 2D N) of the last force evaluation. */
int dem_get_forces(dem_ctx *ctx, double *force, double *torque, int device_ptrs);

/* Per-replica totals (host arrays of n_replicas, any may be NULL):
 * potential energy U (sum over pairs of Eq. DEM / Eq. DEM_2D), kinetic
 * energy K (translational + rotational) and the conserved quantity
 * (K + U in NVE; K + U + g kT (tau_T^2 xi^2 / 2 + eta) after an NVT call;
 * K + U + p_e^2/(2W) + P V + (g + 1) kT (tau_T^2 xi^2 / 2 + eta) after an
 * NPT call).
 * Per-particle energies (N, half of each pair's energy to each particle)
 * may be read with dem_get_particle_energy. */
int dem_get_energy(dem_ctx *ctx, double *per_replica_U, double *per_replica_K,
                   double *conserved);
int dem_get_particle_energy(dem_ctx *ctx, double *energy, int device_ptrs);

/* Per-replica centre-of-mass pair virial W = sum_{i<j} x_ij (x) f_ij
 * (x_ij = x_i - x_j, f_ij the force of j on i), symmetric part as 6 values
 * xx, xy, xz, yy, yz, zz (2D: xx, xy, 0, yy, 0, 0).  Host array of
 * n_replicas * 6.  The pressure of an MD barostat follows from it
 * (Section "Assembly"). */
int dem_get_virial(dem_ctx *ctx, double *per_replica_W6);

/* Change the boxes (host array n_replicas * dim), scaling centre positions
 * affinely; rebuilds the neighbour list and re-evaluates forces.
 * Errors: DEM_ERR_ARG, DEM_ERR_BOX. */
int dem_set_box(dem_ctx *ctx, const double *box);

/* Named numeric parameters:
 *   "skin"        neighbour-list skin (default: the largest sigma_ij, at most 0.4)
 *   "split_group" SPLIT decomposition: particles per warp, 4, 8, 16 or 32; 0
 *                 (default) takes 32, or fewer while N leaves the GPU
 *                 underfilled; get_param returns the size in use
 *   "split_slice" SPLIT decomposition: particles per slice (0, the default: all
 *                 at once).  The scan, feature and term kernels then run slice
 *                 after slice, so that a slice's active-pair and term records
 *                 are read back while they are still in L2
 *   "par_eps"     squared-sine threshold of the parallel-edge rule (1e-6)
 *   "decomp"      DEM_DECOMP_* of the pair kernel
 *   "block"       threads per block of the pair kernel (0 = default)
 *   "graph"       1 = replay each step as a captured CUDA graph (default 1)
 *   "nlist_cap"   neighbour slots per particle (grown automatically, at most 768)
 *   "persistent"  cooperative multi-step kernel for dem_step: -1 (default) as
 *                 dem_autotune timed it, and before any dem_autotune for NVE
 *                 and NVT calls on systems of at most 2048 particles; 1 for
 *                 every NVE and NVT call; 0 never.  Not with "profile" on, nor
 *                 for shapes of more than 32 vertices, edges or faces
 *   "persistent_wait_ms"  limit of one barrier wait of that kernel (1000)
 *   "persistent_test_stall"  testing: 1 = in the next cooperative launch one
 *                 block never reaches the barriers, so the others' waits run
 *                 out and dem_step returns DEM_ERR_TIMEOUT
 *   "term_cap"    DEM_FP32_COMP in the SPLIT decomposition: term records per
 *                 warp of the feature kernel (0 until first needed; default
 *                 sixteen per particle on average, at least 512; grown
 *                 automatically, the evaluation redone)
 *   "npt_chunk"   DEM_NPT steps between host updates of the cell grids (100)
 *   "profile"     1 = time every pair-kernel launch of dem_step with a pair
 *                 of CUDA events on the context's stream (inside the
 *                 captured graph too); setting it resets the totals
 * Read-only (dem_get_param):
 *   "pair_ms_total"  summed pair-kernel time of the profiled steps (ms)
 *   "pair_launches"  number of profiled pair-kernel launches
 *   "launches"       kernel launches issued by this context so far
 *   "persistent_used"  1 if the last dem_step ran the cooperative kernel
 *   "persistent_auto"  dem_autotune's choice: 1 cooperative, 0 per-step
 *                    kernels, -1 not timed
 *   "autotune_step_ms_graph", "autotune_step_ms_persistent"  its step times
 *   "n_cells", "allpairs_replicas"  cell-list layout
 * Setting an unknown name or an invalid value returns DEM_ERR_ARG. */
int dem_set_param(dem_ctx *ctx, const char *name, double value);
int dem_get_param(dem_ctx *ctx, const char *name, double *value);

/* Run every pair-kernel decomposition and block size on the current state
 * and keep the fastest (timed with CUDA events on the context's stream).
 * Candidates, in order: THREAD with 64 and 128 threads per block, WARP,
 * STAGED, and SPLIT with 32, 16, 8 and 4 particles per warp (-1 when its
 * records do not fit in device memory, or for the group sizes other than
 * one fixed with "split_group"); their mean times are readable as
 * parameters "autotune_ms_0" ... "autotune_ms_7".  Results are identical for
 * every choice up to floating-point summation order; the chosen one is the
 * "decomp", "block" and "split_group" parameters.
 * With "persistent" at -1 and at most 65,536 particles it then times a few
 * NVT steps (dt = 1e-6, too short to rebuild the list) with the per-step
 * kernels and with the cooperative multi-step kernel from the same state,
 * keeps the faster for dem_step, and puts the state back as it was; larger
 * systems keep the per-step kernels. */
int dem_autotune(dem_ctx *ctx);

/* Work counters of one force evaluation at the current state (host array of
 * DEM_N_COUNTERS long longs).  The pair kernel evaluates every ordered pair
 * (i, j) of the full neighbour list in i's body frame and skips, exactly,
 * feature pairs whose bounding spheres are farther apart than r_cut:
 *  [0] ordered particle pairs within the bounding-sphere range
 *  [1] feature pairs Eq. DEM / Eq. DEM_2D assigns to those pairs
 *  [2] feature pairs with r < r_cut (WCA terms evaluated)
 *  [3] vertex transforms into the other particle's frame (+ reach test)
 *  [4] vertex-face plane tests      [5] in-plane edge tests of faces
 *  [6] point-segment nearest points [7] edge transforms (+ reach test)
 *  [8] edge bounding-sphere tests   [9] segment-segment nearest points
 *  [10] neighbour-list entries scanned
 *  [11] vertex-face projections inside the face
 *  [12] terms evaluated in j's frame (vertex(i)-face(j), vertex(i)-edge(j))
 *  [13] neighbour-list rebuilds so far  [14] kernel launches so far
 *  [15] pairs that pass the separating-axis test along the centre line
 *  [16] vertex projections of that test  [17] carrier-line distance tests
 *  [18], [19] 0
 * Entries other than [13] and [14] come from a separate instrumented
 * evaluation at the current state (the evaluation used by dem_step is not
 * instrumented). */
#define DEM_N_COUNTERS 20
int dem_get_counters(dem_ctx *ctx, long long *counts);

/* Use this CUDA stream (a cudaStream_t, e.g. torch.cuda.current_stream()).
 * NULL selects the library's own stream. */
int dem_set_stream(dem_ctx *ctx, void *stream);

/* Host-only helper, no GPU needed: derived properties of a shape:
 * out[0] circumradius of the inner shape, out[1] number of edges,
 * out[2..4] principal moments of the uniform inner solid of the shape's
 * mass (2D: out[2] = I_z), out[5] inner volume (3D) or area (2D),
 * out[6] largest off-diagonal inertia element (0 in principal axes). */
int dem_shape_info(const dem_shape *shape, double *out);

/* Forces without any device allocation.  The paper has no counterpart: this
 * is a library convenience for callers that cannot call cudaMalloc, such as
 * code inside a framework whose pool allocator owns all device memory, a
 * process already at its device-memory limit, or a real-time loop that must
 * not take the device-wide synchronisation cudaMalloc and cudaFree can cause.
 * It computes, for ONE periodic system, the forces, torques and per-particle
 * energies dem_compute would, holding every intermediate array (packed
 * state, geometry tables, neighbour list, status) in one static device array
 * of the library: about 21 MiB, reserved on every GPU that loads libdem until
 * the process exits.
 *   shapes, n_shapes, epsilon, sigma, precision   as for dem_create (host)
 *   box        dim box lengths (host); each edge at least twice the
 *              interaction range 2 R_max + r_cut, else DEM_ERR_BOX
 *   n          1 <= n <= DEM_NOALLOC_MAX_N, else DEM_ERR_ARG
 *   shape_id   device, n ints;  pos device, n*dim;  orient device, n*4
 *              quaternions (3D) or n angles (2D)
 *   force      device, n*dim (world frame), written
 *   torque     device, 3D n*3 (world frame) or 2D n, written
 *   energy     device, n (half of each pair's energy per particle) or NULL
 *   stream     cudaStream_t to run on; NULL is the default stream
 * Neighbours are searched over all pairs (cost ~ n^2: meant for small
 * systems); a particle with more than DEM_NOALLOC_MAX_NEIGHBOURS partners in
 * range gives DEM_ERR_NLIST_OVERFLOW, since no memory can be added.  A
 * non-finite position or orientation, or a zero quaternion, gives
 * DEM_ERR_ARG.  The call returns after its stream has finished the work.
 * The first call in each CUDA context (on a device: its primary context, and
 * the new one after a cudaDeviceReset) looks up the static array's address
 * in that context, which is then current; make that first call before any
 * stream capture.  Every call on a device shares
 * the one array, which keeps the last call's contents (each call clears what
 * must start at zero); calls that overlap on the GPU (from other threads or
 * streams) race, so the caller must serialise them.  Errors are reported by
 * dem_last_error(NULL). */
#define DEM_NOALLOC_MAX_N 16384
#define DEM_NOALLOC_MAX_NEIGHBOURS 64
int dem_forces_noalloc(const dem_shape *shapes, int n_shapes, double epsilon, double sigma,
                       const double *box, int n, const int *shape_id, const double *pos,
                       const double *orient, int precision, double *force, double *torque,
                       double *energy, void *stream);

/* Measured fused multiply-add throughput of the current device: every
 * thread of a full-occupancy grid runs 8 independent chains a <- a b + c of
 * iters turns (iters >= 4) in FP32 (precision DEM_FP32) or FP64 (DEM_FP64);
 * *tflops = 2 flops per FMA over the best of three timed launches (CUDA
 * events, after one warm-up launch), *ms that launch's duration.  The paper
 * has no counterpart: the pair kernels do plain ALU arithmetic, and this is
 * the peak their roofline fraction is taken against.  Allocates a small
 * device buffer and a stream for the measurement.  Errors: DEM_ERR_ARG,
 * DEM_ERR_CUDA (dem_last_error(NULL) gives the reason). */
int dem_fma_peak(int precision, int iters, double *tflops, double *ms);

/* Self-check of the conversions between double and float that the
 * integrator makes with integer operations on the IEEE-754 fields (to keep
 * them off the FP64 pipe): n inputs, each a double (a quarter of them on a
 * rounding tie, a quarter with exponents around the float range) and a
 * float drawn by a counter-based hash (splitmix64) of seed + index, are
 * converted both ways and compared with the conversion instructions (round
 * to nearest even).  mismatches[0] counts double-to-float, mismatches[1]
 * float-to-double differences (host array of 2).  The paper has no
 * counterpart.  Allocates 16 bytes of device memory and a stream.  Errors:
 * DEM_ERR_ARG, DEM_ERR_CUDA (dem_last_error(NULL) gives the reason). */
int dem_check_conversions(unsigned long long n, unsigned long long seed,
                          unsigned long long *mismatches);

/* One-line description of the last error of ctx (or of the last failed
 * dem_create, dem_forces_noalloc, dem_fma_peak or dem_check_conversions
 * when ctx is NULL). */
const char *dem_last_error(const dem_ctx *ctx);

void dem_destroy(dem_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DEM_H */
