// nlist.cu -- cell list and Verlet neighbour list over particle bounding
// spheres.  The paper only says that each particle sums over its
// "neighbors" (Section "Algorithm") and names cell lists as a data
// structure for contact search (Section "Summary"); this is the standard
// MD construction:
//   * cells of width >= R_max + R_max + r_cut,max + skin per replica;
//   * the Verlet list of i holds every j (any image within the minimum-image
//     convention) with |x_ij| < R_i + R_j + r_cut,ij + skin;
//   * the list is rebuilt when some particle has moved more than skin/2
//     since the last build.  Rotation never invalidates it: bounding spheres
//     are rotation invariant.
// Replicas whose box has fewer than 3 cells along some axis search all
// particles of the replica instead of the 27-cell (9 in 2D) stencil.
// Neighbour indices are sorted so that the pair kernels sum in a fixed
// order regardless of the order in which atomics filled the cells: each
// thread collects its indices in a shared-memory column, sorts them there
// and writes its entries once (a column-major list is strided per thread,
// so sorting it in place in global memory would be slow).
// Each entry also carries x_j - x_i at build time (minimum image taken here in
// FP64, then rounded to FP32); the integrator keeps each particle's FP32
// displacement since the build, so the FP32 pair kernels form
// x_j - x_i = d0 + delta_j - delta_i without FP64 arithmetic.
#include "dem_internal.cuh"

namespace dem {
namespace {

constexpr double WCA_CUT = 1.122462048309373;

__device__ __forceinline__ bool rebuild_due(const NlistArgs &a) {
    const Status *st = a.status;
    return st->rebuild != 0 || __uint_as_float(st->maxdisp2) > a.half_skin2;
}

__device__ __forceinline__ int cell_coord(double x, double L, int nc) {
    int c = (int)floor(x / L * nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_assign(const NlistArgs a) {
    if (!rebuild_due(a)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const Rep &rp = a.reps[a.rep[i]];
        double4_32a x = a.pos[i];
        a.posf[i] = make_float4((float)x.x, (float)x.y, (float)x.z, __int_as_float(a.shape[i]));
        if (rp.allpairs) continue;
        int cx = cell_coord(x.x, rp.L[0], rp.nc[0]);
        int cy = cell_coord(x.y, rp.L[1], rp.nc[1]);
        int cz = a.dim == 3 ? cell_coord(x.z, rp.L[2], rp.nc[2]) : 0;
        int c = rp.cell_off + (cz * rp.nc[1] + cy) * rp.nc[0] + cx;
        int slot = atomicAdd(a.cell_count + c, 1);
        if (slot < a.cell_cap) a.cell_slots[(size_t)c * a.cell_cap + slot] = i;
        else atomicMax(&a.status->cell_overflow, slot + 1);
    }
}

constexpr int NL_BLOCK = 64;   // threads per block of the list build

// Minimum-image separation x_j - x_i (FP64).
__device__ __forceinline__ void separation(const NlistArgs &a, int j, double4_32a xi, const Rep &rp,
                                           double *dx, double *dy, double *dz) {
    const double4_32a xj = a.pos[j];
    double x = xj.x - xi.x, y = xj.y - xi.y, z = xj.z - xi.z;
    x -= rp.L[0] * rint(x * rp.inv_L[0]);
    y -= rp.L[1] * rint(y * rp.inv_L[1]);
    if (a.dim == 3) z -= rp.L[2] * rint(z * rp.inv_L[2]); else z = 0.0;
    *dx = x; *dy = y; *dz = z;
}

// FP32 view of particle i and of its replica for the candidate test.
struct CandI {
    float x, y, z;
    float R, rnd;
    float L[3], inv_L[3];
    float slack;         // covers the FP32 rounding of positions and images
};

// Candidate j of particle i: kept (in the thread's shared-memory column
// keys[k * NL_BLOCK]) when its bounding sphere is within the list cutoff.
// The test runs in FP32 on rounded positions with a slack of 1e-6 (L + 1),
// well above their rounding error (~4e-7 L): the kept set contains every j
// the FP64 test keeps, plus possibly a few just beyond the cutoff, whose
// terms the pair kernels' own range test rejects.  FP64 throughput is a
// small fraction of FP32 on this part, and the build tests ~27 cells of
// candidates per particle.
__device__ __forceinline__ void consider(const NlistArgs &a, int i, int j, const CandI &c,
                                         int *keys, int *count) {
    if (j == i) return;
    const float4 pj = a.posf[j];
    float dx = pj.x - c.x, dy = pj.y - c.y, dz = pj.z - c.z;
    dx -= c.L[0] * rintf(dx * c.inv_L[0]);
    dy -= c.L[1] * rintf(dy * c.inv_L[1]);
    if (a.dim == 3) dz -= c.L[2] * rintf(dz * c.inv_L[2]); else dz = 0.f;
    const ShapeDev &sj = a.shapes[__float_as_int(pj.w)];
    const float sig = a.sigma > 0.0 ? (float)a.sigma : c.rnd + sj.rounding_f;
    const float lim = c.R + sj.R + (float)WCA_CUT * sig + (float)a.skin + c.slack;
    if (dx * dx + dy * dy + dz * dz < lim * lim) {
        if (*count < a.cap) keys[(*count) * NL_BLOCK] = j;
        (*count)++;
    }
}

__global__ void k_nlist(const NlistArgs a) {
    if (!rebuild_due(a)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(&a.status->rebuilds, 1);
        a.status->built = 1;
    }
    extern __shared__ int nl_keys[];
    int *keys = nl_keys + threadIdx.x;    // this thread's column, stride NL_BLOCK
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const Rep &rp = a.reps[a.rep[i]];
        const double4_32a xi = a.pos[i];
        const ShapeDev &si = a.shapes[a.shape[i]];
        CandI c;
        c.x = (float)xi.x; c.y = (float)xi.y; c.z = (float)xi.z;
        c.R = si.R; c.rnd = si.rounding_f;
        double Lmax = 0.0;
        for (int k = 0; k < 3; ++k) {
            c.L[k] = (float)rp.L[k];
            c.inv_L[k] = (float)rp.inv_L[k];
            if (k < a.dim) Lmax = fmax(Lmax, rp.L[k]);
        }
        c.slack = (float)(1e-6 * (Lmax + 1.0));
        int count = 0;
        if (rp.allpairs) {
            for (int j = rp.off; j < rp.off + rp.n; ++j) consider(a, i, j, c, keys, &count);
        } else {
            int c0[3] = {cell_coord(xi.x, rp.L[0], rp.nc[0]), cell_coord(xi.y, rp.L[1], rp.nc[1]),
                         a.dim == 3 ? cell_coord(xi.z, rp.L[2], rp.nc[2]) : 0};
            int zr = a.dim == 3 ? 1 : 0;
            for (int oz = -zr; oz <= zr; ++oz) {
                int cz = a.dim == 3 ? (c0[2] + oz + rp.nc[2]) % rp.nc[2] : 0;
                for (int oy = -1; oy <= 1; ++oy) {
                    int cy = (c0[1] + oy + rp.nc[1]) % rp.nc[1];
                    for (int ox = -1; ox <= 1; ++ox) {
                        int cx = (c0[0] + ox + rp.nc[0]) % rp.nc[0];
                        int cl = rp.cell_off + (cz * rp.nc[1] + cy) * rp.nc[0] + cx;
                        int m = a.cell_count[cl];
                        if (m > a.cell_cap) m = a.cell_cap;
                        for (int s = 0; s < m; ++s)
                            consider(a, i, a.cell_slots[(size_t)cl * a.cell_cap + s], c, keys,
                                     &count);
                    }
                }
            }
        }
        if (count > a.cap) {
            atomicMax(&a.status->nlist_overflow, count);
            count = a.cap;
        }
        // insertion sort of the column (ascending j), then one write per entry
        for (int p = 1; p < count; ++p) {
            const int v = keys[p * NL_BLOCK];
            int q = p - 1;
            while (q >= 0 && keys[q * NL_BLOCK] > v) {
                keys[(q + 1) * NL_BLOCK] = keys[q * NL_BLOCK];
                --q;
            }
            keys[(q + 1) * NL_BLOCK] = v;
        }
        for (int p = 0; p < count; ++p) {
            const int j = keys[p * NL_BLOCK];
            double dx, dy, dz;
            separation(a, j, xi, rp, &dx, &dy, &dz);
            a.nlist[(size_t)p * a.n + i] = make_float4((float)dx, (float)dy, (float)dz, __int_as_float(j));
        }
        a.nn[i] = count;
        a.x_last[i] = xi;
        a.delta[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(a.shape[i]));   // w: shape index
        if (i == rp.off && a.reps_rw) {
            // the list of this replica is now in its current box
            Rep &w = a.reps_rw[a.rep[i]];
            const double L0 = rp.L[0];
            w.L_build0 = L0;
            w.sc_d = 1.0;
            w.sc = 1.f;
            w.disp_pad = 0.f;
        }
    }
}

}  // namespace

// Cell binning (when a rebuild is due) and the FP32 position copy of every
// particle; with no cell arrays (all replicas search all pairs) only the copy.
cudaError_t launch_cells(const NlistArgs &a, int n_cells, cudaStream_t s) {
    if (a.cell_count) {
        cudaError_t e = cudaMemsetAsync(a.cell_count, 0, sizeof(int) * (size_t)(n_cells > 0 ? n_cells : 1), s);
        if (e != cudaSuccess) return e;
    }
    int grid = (a.n + 255) / 256;
    k_cell_assign<<<grid > 0 ? grid : 1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

size_t nlist_smem_bytes(int cap) { return sizeof(int) * (size_t)NL_BLOCK * (size_t)cap; }

cudaError_t launch_nlist(const NlistArgs &a, cudaStream_t s) {
    const size_t smem = nlist_smem_bytes(a.cap);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_nlist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int grid = (a.n + NL_BLOCK - 1) / NL_BLOCK;
    k_nlist<<<grid > 0 ? grid : 1, NL_BLOCK, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dem
