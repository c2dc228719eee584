// noalloc.cu -- dem_forces_noalloc: the force evaluation of dem_compute for
// one periodic system, with no device allocation.  Every intermediate array
// (packed state, geometry tables, neighbour list, status word) lives in one
// file-scope static device array; the caller supplies inputs and outputs.
//
// Some callers cannot call cudaMalloc: a framework whose pool allocator owns
// all device memory, a process running under a device-memory limit that is
// already reached, or a real-time loop that must not take the device-wide
// synchronisation cudaMalloc and cudaFree can cause.  They can still get
// forces from this entry point.
//
// The static array is about 21 MiB and is reserved on every GPU that loads
// the library, until the process exits.  All calls on a device share it and
// it keeps the last call's contents, so each call clears what must start at
// zero (the status word, the replica index of every particle), and calls
// that overlap on the GPU race: the caller must serialise them.
#include <cuda.h>   // CUcontext / CUresult types only; the entry points are looked up

#include <mutex>

#include "dem_internal.cuh"

using namespace dem;

namespace {

constexpr int MAX_N = DEM_NOALLOC_MAX_N;
constexpr int CAP = DEM_NOALLOC_MAX_NEIGHBOURS;
constexpr size_t TABLE_BYTES = 128 * 1024;      // geometry records
constexpr int MAX_ITAB = 8192;                  // face-edge ranges
constexpr int MAX_SHAPES = 256;

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Byte offsets of the regions of the static array.
constexpr size_t OFF_POS = 0;
constexpr size_t OFF_QUAT = OFF_POS + align256(sizeof(double4_32a) * MAX_N);
constexpr size_t OFF_FORCE = OFF_QUAT + align256(sizeof(double4_32a) * MAX_N);
constexpr size_t OFF_TORQUE = OFF_FORCE + align256(sizeof(double4_32a) * MAX_N);
constexpr size_t OFF_XLAST = OFF_TORQUE + align256(sizeof(double4_32a) * MAX_N);
constexpr size_t OFF_QUATF = OFF_XLAST + align256(sizeof(double4_32a) * MAX_N);
constexpr size_t OFF_ENERGY = OFF_QUATF + align256(sizeof(float4) * MAX_N);
constexpr size_t OFF_VIRIAL = OFF_ENERGY + align256(sizeof(double) * MAX_N);
constexpr size_t OFF_SHAPE = OFF_VIRIAL + align256(6 * sizeof(double) * MAX_N);
constexpr size_t OFF_REP = OFF_SHAPE + align256(sizeof(int) * MAX_N);
constexpr size_t OFF_NN = OFF_REP + align256(sizeof(int) * MAX_N);
constexpr size_t OFF_DELTA = OFF_NN + align256(sizeof(int) * MAX_N);
constexpr size_t OFF_POSF = OFF_DELTA + align256(sizeof(float4) * MAX_N);
constexpr size_t OFF_NLIST = OFF_POSF + align256(sizeof(float4) * MAX_N);
constexpr size_t OFF_TABLE = OFF_NLIST + align256(sizeof(float4) * (size_t)MAX_N * CAP);
constexpr size_t OFF_GEOMS = OFF_TABLE + align256(TABLE_BYTES);
constexpr size_t OFF_ITAB = OFF_GEOMS + align256(sizeof(Geom) * MAX_GEOMS);
constexpr size_t OFF_SHAPES = OFF_ITAB + align256(sizeof(int) * MAX_ITAB);
constexpr size_t OFF_REPREC = OFF_SHAPES + align256(sizeof(ShapeDev) * MAX_SHAPES);
constexpr size_t OFF_STATUS = OFF_REPREC + align256(sizeof(Rep));
// FP32 + two-sum: the state and the geometry records as hi + lo floats
constexpr size_t OFF_QUATF_LO = OFF_STATUS + align256(sizeof(Status));
constexpr size_t OFF_XFF = OFF_QUATF_LO + align256(sizeof(float4) * MAX_N);
constexpr size_t OFF_TABLE_LO = OFF_XFF + align256(2 * sizeof(float4) * MAX_N);
constexpr size_t SCRATCH_BYTES = OFF_TABLE_LO + align256(TABLE_BYTES);

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Device address of the static array in the CUDA context current on the
// calling thread.  The address belongs to a context, not to a device
// ordinal: after cudaDeviceReset the module is loaded again into a new
// primary context, and a caller may make a context of its own current.  So
// the address is looked up (cudaGetSymbolAddress, with that context current)
// once per context, keyed by the driver's unique context id, and cached.
// The context queries come from the driver through the runtime's
// entry-point lookup, so the library does not link libcuda.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext *);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long *);

std::mutex g_mu;
struct ScratchEntry {
    unsigned long long ctx_id;
    void *base;
};
ScratchEntry g_cache[64];
int g_cached = 0;
PfnCtxGetCurrent g_ctx_current = nullptr;
PfnCtxGetId g_ctx_id = nullptr;

int current_context_id(unsigned long long *id, std::string *err) {
    if (!g_ctx_current || !g_ctx_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            *err = "driver context queries unavailable";
            return DEM_ERR_CUDA;
        }
        g_ctx_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
        g_ctx_id = reinterpret_cast<PfnCtxGetId>(f2);
    }
    CUcontext c = nullptr;
    if (g_ctx_current(&c) != CUDA_SUCCESS) { *err = "cuCtxGetCurrent failed"; return DEM_ERR_CUDA; }
    if (!c) {
        // no context yet on this thread: make the current device's primary
        // context current (cudaSetDevice initialises it)
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaSetDevice(dev);
        if (e != cudaSuccess) { *err = cudaGetErrorString(e); return DEM_ERR_CUDA; }
        if (g_ctx_current(&c) != CUDA_SUCCESS || !c) { *err = "no CUDA context"; return DEM_ERR_CUDA; }
    }
    if (g_ctx_id(c, id) != CUDA_SUCCESS) { *err = "cuCtxGetId failed"; return DEM_ERR_CUDA; }
    return DEM_OK;
}

int scratch_base(void **out, std::string *err) {
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    int rc = current_context_id(&id, err);
    if (rc) return rc;
    for (int k = 0; k < g_cached; ++k)
        if (g_cache[k].ctx_id == id) { *out = g_cache[k].base; return DEM_OK; }
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        *err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return DEM_ERR_CUDA;
    }
    // a full cache drops its oldest entry (contexts of a finished reset)
    if (g_cached == 64) {
        for (int k = 1; k < 64; ++k) g_cache[k - 1] = g_cache[k];
        --g_cached;
    }
    g_cache[g_cached++] = {id, p};
    *out = p;
    return DEM_OK;
}

int fail(int code, const std::string &msg) {
    set_global_error(msg);
    return code;
}

#define NA_CK(call)                                                                     \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return fail(DEM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" int dem_forces_noalloc(const dem_shape *shapes, int n_shapes, double epsilon,
                                  double sigma, const double *box, int n, const int *shape_id,
                                  const double *pos, const double *orient, int precision,
                                  double *force, double *torque, double *energy, void *stream) {
    if (!shapes || n_shapes < 1 || !box || !shape_id || !pos || !orient || !force || !torque)
        return fail(DEM_ERR_ARG, "dem_forces_noalloc: missing argument");
    if (n < 1 || n > MAX_N)
        return fail(DEM_ERR_ARG, "dem_forces_noalloc: n must be in [1, " + std::to_string(MAX_N) +
                                     "], got " + std::to_string(n));
    if (n_shapes > MAX_SHAPES)
        return fail(DEM_ERR_ARG, "dem_forces_noalloc: at most " + std::to_string(MAX_SHAPES) + " shapes");
    if (precision != DEM_FP64 && precision != DEM_FP32 && precision != DEM_FP32_COMP)
        return fail(DEM_ERR_ARG, "dem_forces_noalloc: unknown precision");
    if (!(epsilon > 0.0)) return fail(DEM_ERR_ARG, "dem_forces_noalloc: epsilon must be > 0");
    HostTables t;
    std::string err;
    int rc = make_host_tables(shapes, n_shapes, &t, &err);
    if (rc) return fail(rc, "dem_forces_noalloc: " + err);
    const int dim = t.dim;
    const size_t rec = precision == DEM_FP64 ? sizeof(double4_32a) : sizeof(float4);
    if (t.td.size() * rec > TABLE_BYTES || t.itab.size() > (size_t)MAX_ITAB)
        return fail(DEM_ERR_ARG, "dem_forces_noalloc: shape tables exceed the static limit");
    // minimum image is exact when every box edge is at least twice the range
    const double sig_max = sigma > 0 ? sigma : 2.0 * t.rnd_max;
    const double range = pair_range(t.Rmax, sig_max, 0.0);
    Rep rp = {};
    for (int a = 0; a < 3; ++a) {
        rp.L[a] = a < dim ? box[a] : 1.0;
        rp.inv_L[a] = 1.0 / rp.L[a];
        rp.nc[a] = 1;
        if (a < dim && !(rp.L[a] >= 2.0 * range))
            return fail(DEM_ERR_BOX, "dem_forces_noalloc: box edge below twice the interaction range");
    }
    rp.off = 0;
    rp.n = n;
    rp.allpairs = 1;
    rp.g_dof = 0;
    rp.r_list = range;
    rep_box_ff(rp);
    rp.L_build0 = rp.L[0];
    rp.sc_d = 1.0;
    rp.sc = 1.f;
    rp.disp_pad = 0.f;

    void *base = nullptr;
    rc = scratch_base(&base, &err);
    if (rc) return fail(rc, "dem_forces_noalloc: " + err);
    unsigned char *b = static_cast<unsigned char *>(base);
    double4_32a *pos4 = reinterpret_cast<double4_32a *>(b + OFF_POS);
    double4_32a *quat4 = reinterpret_cast<double4_32a *>(b + OFF_QUAT);
    double4_32a *force4 = reinterpret_cast<double4_32a *>(b + OFF_FORCE);
    double4_32a *torque4 = reinterpret_cast<double4_32a *>(b + OFF_TORQUE);
    double4_32a *xlast = reinterpret_cast<double4_32a *>(b + OFF_XLAST);
    float4 *quatf = reinterpret_cast<float4 *>(b + OFF_QUATF);
    double *en = reinterpret_cast<double *>(b + OFF_ENERGY);
    double *vir = reinterpret_cast<double *>(b + OFF_VIRIAL);
    int *shp = reinterpret_cast<int *>(b + OFF_SHAPE);
    int *rep = reinterpret_cast<int *>(b + OFF_REP);
    int *nn = reinterpret_cast<int *>(b + OFF_NN);
    float4 *delta = reinterpret_cast<float4 *>(b + OFF_DELTA);
    float4 *nlist = reinterpret_cast<float4 *>(b + OFF_NLIST);
    float4 *posf = reinterpret_cast<float4 *>(b + OFF_POSF);
    void *table = b + OFF_TABLE;
    Geom *geoms = reinterpret_cast<Geom *>(b + OFF_GEOMS);
    int *itab = reinterpret_cast<int *>(b + OFF_ITAB);
    ShapeDev *sdev = reinterpret_cast<ShapeDev *>(b + OFF_SHAPES);
    Rep *reprec = reinterpret_cast<Rep *>(b + OFF_REPREC);
    Status *status = reinterpret_cast<Status *>(b + OFF_STATUS);
    const bool ffm = precision == DEM_FP32_COMP;
    float4 *quatf_lo = ffm ? reinterpret_cast<float4 *>(b + OFF_QUATF_LO) : nullptr;
    float4 *xff = ffm ? reinterpret_cast<float4 *>(b + OFF_XFF) : nullptr;
    float4 *table_lo = ffm ? reinterpret_cast<float4 *>(b + OFF_TABLE_LO) : nullptr;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // shape indices are checked on the host
    std::vector<int> sid(n);
    NA_CK(cudaMemcpyAsync(sid.data(), shape_id, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    for (int i = 0; i < n; ++i)
        if (sid[i] < 0 || sid[i] >= n_shapes)
            return fail(DEM_ERR_ARG, "dem_forces_noalloc: shape_id out of range");

    // tables and the replica record; the status word and the replica index of
    // every particle start at zero; a list build is requested
    if (precision == DEM_FP64)
        NA_CK(cudaMemcpyAsync(table, t.td.data(), sizeof(double4_32a) * t.td.size(), cudaMemcpyHostToDevice, st));
    else
        NA_CK(cudaMemcpyAsync(table, t.tf.data(), sizeof(float4) * t.tf.size(), cudaMemcpyHostToDevice, st));
    if (ffm)
        NA_CK(cudaMemcpyAsync(table_lo, t.tf_lo.data(), sizeof(float4) * t.tf_lo.size(),
                              cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(geoms, t.geoms.data(), sizeof(Geom) * t.geoms.size(), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(itab, t.itab.data(), sizeof(int) * t.itab.size(), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(sdev, t.shapes.data(), sizeof(ShapeDev) * t.shapes.size(), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemcpyAsync(reprec, &rp, sizeof(Rep), cudaMemcpyHostToDevice, st));
    Status s0 = {};
    s0.rebuild = 1;
    NA_CK(cudaMemcpyAsync(status, &s0, sizeof(Status), cudaMemcpyHostToDevice, st));
    NA_CK(cudaMemsetAsync(rep, 0, sizeof(int) * n, st));
    NA_CK(cudaMemcpyAsync(shp, shape_id, sizeof(int) * n, cudaMemcpyDeviceToDevice, st));

    // pack the state, all-pairs list, pair kernel, world-frame outputs
    NA_CK(launch_import_state(n, dim, pos, orient, nullptr, nullptr, pos4, quat4, nullptr, nullptr,
                              status, st));
    NA_CK(launch_prepare_state(n, dim, pos4, quat4, quatf, quatf_lo, xff, nullptr, rep, reprec, 0, st));
    NlistArgs na = {};
    na.n = n; na.dim = dim; na.cap = CAP; na.cell_cap = 0;
    na.pos = pos4; na.shape = shp; na.rep = rep; na.reps = reprec; na.shapes = sdev;
    na.sigma = sigma > 0 ? sigma : 0.0; na.skin = 0.0;
    na.cell_count = nullptr; na.cell_slots = nullptr;
    na.nlist = nlist; na.nn = nn; na.x_last = xlast; na.status = status; na.half_skin2 = 0.f;
    na.delta = delta;
    na.posf = posf;
    NA_CK(launch_cells(na, 0, st));
    NA_CK(launch_nlist(na, st));
    PairArgs pa = {};
    pa.n = n; pa.dim = dim; pa.cap = CAP;
    pa.pos = pos4; pa.quat = quat4; pa.quatf = quatf;
    pa.shape = shp; pa.rep = rep; pa.reps = reprec; pa.shapes = sdev;
    pa.geoms = geoms; pa.n_geoms = (int)t.geoms.size();
    pa.table = table; pa.table_len = (int)t.td.size();
    pa.itable = itab; pa.itable_len = (int)t.itab.size();
    pa.nlist = nlist; pa.nn = nn; pa.delta = delta;
    pa.force = force4; pa.torque = torque4; pa.energy = en; pa.virial = vir;
    pa.eps = epsilon; pa.sigma = sigma > 0 ? sigma : 0.0; pa.par_eps = 1e-6;
    pa.status = status; pa.counters = nullptr;
    pa.mask_words = t.mask_words;
    if (ffm) {
        pa.quatf_lo = quatf_lo;
        pa.xff = xff;
        pa.table_lo = table_lo;
        split_ff(sigma > 0 ? sigma : 0.0, &pa.sigma_f, &pa.sigma_lo);
    }
    NA_CK(launch_pair(pa, precision, DEM_DECOMP_THREAD, 0, false, st));
    NA_CK(launch_export_forces(n, dim, force4, torque4, quat4, force, torque, st));
    if (energy) NA_CK(cudaMemcpyAsync(energy, en, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    Status hs;
    NA_CK(cudaMemcpyAsync(&hs, status, sizeof(Status), cudaMemcpyDeviceToHost, st));
    NA_CK(cudaStreamSynchronize(st));
    if (hs.bad_input)
        return fail(DEM_ERR_ARG, "dem_forces_noalloc: particle " + std::to_string(hs.bad_input - 1) +
                                     ": non-finite position or orientation, or a zero quaternion");
    if (hs.nlist_overflow)
        return fail(DEM_ERR_NLIST_OVERFLOW, "dem_forces_noalloc: a particle has more than " +
                                                std::to_string(CAP) + " neighbours in range");
    if (hs.nonfinite) return fail(DEM_ERR_NONFINITE, "dem_forces_noalloc: non-finite force or energy");
    return DEM_OK;
}
