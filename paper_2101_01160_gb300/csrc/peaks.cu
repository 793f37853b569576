// Fused multiply-add throughput of the GPU in FP32 and FP64: the ALU
// denominators of the MD kernels' rooflines (the FP64 path and the
// shared-memory-resident FP32 path are bound by arithmetic, not by HBM).
//
// Every thread runs CHAINS independent multiply-add chains a = a * b + c
// (one FFMA / DFMA each, two flops) for `iters` rounds; the grid is the
// full resident grid of the device, so every scheduler of every SM has
// independent work each cycle.  The values stay finite and are stored once
// behind a data-dependent test, so nothing is removed by the compiler.
#include "common.cuh"

namespace mdlg {

constexpr int PEAK_CHAINS = 8;
constexpr int PEAK_BLOCK = 256;

template <typename T>
__global__ void __launch_bounds__(PEAK_BLOCK) k_fma_peak(T b, T c, long long iters, T *sink) {
    T a[PEAK_CHAINS];
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PEAK_CHAINS; ++k) a[k] = a[k] * b + c;
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < PEAK_CHAINS; ++k) s += a[k];
    if (s == T(-1.2345)) *sink = s;   // never true for these inputs
}

}  // namespace mdlg

using namespace mdlg;

extern "C" int mdlg_fma_peak(int32_t f64, int64_t iters, double *flops_per_s, double *ms_out,
                             void *stream) {
    if (!flops_per_s || iters < 1 || iters > (1ll << 32)) return fail(MD_E_ARG, "mdlg_fma_peak: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0, per_sm = 0;
    MD_CUDA_TRY(cudaGetDevice(&dev));
    MD_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const void *fn = f64 ? (const void *)k_fma_peak<double> : (const void *)k_fma_peak<float>;
    MD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PEAK_BLOCK, 0));
    const int grid = nsm * (per_sm > 0 ? per_sm : 1);
    void *sink = nullptr;
    MD_CUDA_TRY(cudaMallocAsync(&sink, 16, st));
    cudaEvent_t e0, e1;
    MD_CUDA_TRY(cudaEventCreate(&e0));
    MD_CUDA_TRY(cudaEventCreate(&e1));
    auto launch = [&](long long n) {
        if (f64)
            k_fma_peak<double><<<grid, PEAK_BLOCK, 0, st>>>(0.999999, 1e-7, n, (double *)sink);
        else
            k_fma_peak<float><<<grid, PEAK_BLOCK, 0, st>>>(0.9999f, 1e-4f, n, (float *)sink);
    };
    launch(iters / 8 + 1);   // warm-up (clocks ramp, module loaded)
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (e != cudaSuccess) return fail(MD_E_CUDA, "mdlg_fma_peak: %s", cudaGetErrorString(e));
    MD_CUDA_TRY(cudaGetLastError());
    const double flops = 2.0 * PEAK_CHAINS * (double)iters * (double)grid * PEAK_BLOCK;
    *flops_per_s = flops / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return MD_OK;
}
