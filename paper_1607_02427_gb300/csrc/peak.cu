// peak.cu -- dem_fma_peak: the FP32 and FP64 fused multiply-add throughput
// of the device, measured by independent FMA chains.  The pair kernels are
// bound by plain FP32 (or, in the FP64 mode, FP64) ALU arithmetic, not by
// tensor cores or memory, so their roofline is this rate.  It has no
// counterpart in the paper; the bench reports the pair kernels' achieved
// flop rate as a fraction of it.
#include "dem_internal.cuh"

namespace {

constexpr int CHAINS = 8;        // independent accumulators per thread
constexpr int PBLOCK = 256;

// Every thread runs CHAINS independent chains a <- a * b + c for `iters`
// turns (unrolled by 4): 2 * CHAINS * iters flops per thread, no memory
// traffic inside the loop.  b < 1 keeps every chain bounded.
template <class T>
__global__ void __launch_bounds__(PBLOCK) k_fma_chain(int iters, T b, T c, T *sink) {
    T a[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; it += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < CHAINS; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += a[k];
    // one store per block keeps the chains live
    if (s == T(-1.2345e30)) sink[blockIdx.x] = s;
    if (threadIdx.x == 0 && blockIdx.x == 0) sink[0] = s;
}

template <class T>
int measure(int iters, double *tflops, double *ms_out, std::string *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chain<T>, PBLOCK, 0);
    if (e != cudaSuccess) { *err = cudaGetErrorString(e); return DEM_ERR_CUDA; }
    if (per_sm < 1) per_sm = 1;
    const int grid = sms * per_sm;
    T *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st = nullptr;
    float best = 0.f;
    e = cudaMalloc(&sink, sizeof(T) * grid);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    // one warm-up launch, then the best of three timed ones
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) {
            k_fma_chain<T><<<grid, PBLOCK, 0, st>>>(iters, T(0.999999), T(1e-6), sink);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess) { *err = cudaGetErrorString(e); return DEM_ERR_CUDA; }
    const double flops = 2.0 * CHAINS * (double)((iters + 3) / 4 * 4) * PBLOCK * (double)grid;
    *tflops = flops / (best * 1e-3) / 1e12;
    *ms_out = best;
    return DEM_OK;
}

}  // namespace

extern "C" int dem_fma_peak(int precision, int iters, double *tflops, double *ms) {
    if (!tflops || !ms || iters < 4 || (precision != DEM_FP64 && precision != DEM_FP32)) {
        dem::set_global_error("dem_fma_peak: precision must be DEM_FP32 or DEM_FP64, iters >= 4");
        return DEM_ERR_ARG;
    }
    std::string err;
    const int rc = precision == DEM_FP32 ? measure<float>(iters, tflops, ms, &err)
                                         : measure<double>(iters, tflops, ms, &err);
    if (rc) dem::set_global_error("dem_fma_peak: " + err);
    return rc;
}
