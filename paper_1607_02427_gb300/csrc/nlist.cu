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
// order regardless of the order in which atomics filled the cells.
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
        if (rp.allpairs) continue;
        double4_32a x = a.pos[i];
        int cx = cell_coord(x.x, rp.L[0], rp.nc[0]);
        int cy = cell_coord(x.y, rp.L[1], rp.nc[1]);
        int cz = a.dim == 3 ? cell_coord(x.z, rp.L[2], rp.nc[2]) : 0;
        int c = rp.cell_off + (cz * rp.nc[1] + cy) * rp.nc[0] + cx;
        int slot = atomicAdd(a.cell_count + c, 1);
        if (slot < a.cell_cap) a.cell_slots[(size_t)c * a.cell_cap + slot] = i;
        else atomicMax(&a.status->cell_overflow, slot + 1);
    }
}

__device__ __forceinline__ void consider(const NlistArgs &a, int i, int j, double4_32a xi,
                                         double Ri, double rnd_i, const Rep &rp, int *count) {
    if (j == i) return;
    double4_32a xj = a.pos[j];
    double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
    dx -= rp.L[0] * rint(dx * rp.inv_L[0]);
    dy -= rp.L[1] * rint(dy * rp.inv_L[1]);
    if (a.dim == 3) dz -= rp.L[2] * rint(dz * rp.inv_L[2]); else dz = 0.0;
    const ShapeDev &sj = a.shapes[a.shape[j]];
    double sig = a.sigma > 0.0 ? a.sigma : rnd_i + sj.rounding;
    double lim = Ri + (double)sj.R + WCA_CUT * sig + a.skin;
    if (dx * dx + dy * dy + dz * dz < lim * lim) {
        if (*count < a.cap)
            a.nlist[(size_t)(*count) * a.n + i] =
                make_float4((float)dx, (float)dy, (float)dz, __int_as_float(j));
        (*count)++;
    }
}

__global__ void k_nlist(const NlistArgs a) {
    if (!rebuild_due(a)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(&a.status->rebuilds, 1);
        a.status->built = 1;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const Rep &rp = a.reps[a.rep[i]];
        const double4_32a xi = a.pos[i];
        const ShapeDev &si = a.shapes[a.shape[i]];
        const double Ri = si.R, rnd_i = si.rounding;
        int count = 0;
        if (rp.allpairs) {
            for (int j = rp.off; j < rp.off + rp.n; ++j) consider(a, i, j, xi, Ri, rnd_i, rp, &count);
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
                        int c = rp.cell_off + (cz * rp.nc[1] + cy) * rp.nc[0] + cx;
                        int m = a.cell_count[c];
                        if (m > a.cell_cap) m = a.cell_cap;
                        for (int s = 0; s < m; ++s)
                            consider(a, i, a.cell_slots[(size_t)c * a.cell_cap + s], xi, Ri, rnd_i,
                                     rp, &count);
                    }
                }
            }
        }
        if (count > a.cap) {
            atomicMax(&a.status->nlist_overflow, count);
            count = a.cap;
        }
        // insertion sort of the column (ascending j)
        for (int p = 1; p < count; ++p) {
            float4 v = a.nlist[(size_t)p * a.n + i];
            int q = p - 1;
            while (q >= 0 && __float_as_int(a.nlist[(size_t)q * a.n + i].w) > __float_as_int(v.w)) {
                a.nlist[(size_t)(q + 1) * a.n + i] = a.nlist[(size_t)q * a.n + i];
                --q;
            }
            a.nlist[(size_t)(q + 1) * a.n + i] = v;
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

cudaError_t launch_cells(const NlistArgs &a, int n_cells, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.cell_count, 0, sizeof(int) * (size_t)(n_cells > 0 ? n_cells : 1), s);
    if (e != cudaSuccess) return e;
    int grid = (a.n + 255) / 256;
    k_cell_assign<<<grid > 0 ? grid : 1, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_nlist(const NlistArgs &a, cudaStream_t s) {
    int grid = (a.n + 127) / 128;
    k_nlist<<<grid > 0 ? grid : 1, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dem
