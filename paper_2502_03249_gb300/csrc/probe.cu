// probe.cu -- measurement support: the FMA throughput of the FP64 and FP32
// pipes of the current GPU, the ALU roofline of the IEEE-double operator (an
// FP64-FMA-bound kernel on GB300) and of the float operators.
//
// Every thread runs NCHAIN independent FMA chains (enough to cover the
// pipeline latency) for iters steps; the grid holds BLOCKS_PER_SM blocks per
// SM so every scheduler has warps to issue.  The chains' results are summed
// into one output so that the compiler keeps every FMA.
#include "ctx.h"

namespace stag {

constexpr int PROBE_BS = 256;
constexpr int PROBE_CHAINS = 16;
constexpr int PROBE_BLOCKS_PER_SM = 8;

template <typename T>
__global__ void __launch_bounds__(PROBE_BS) k_fma_probe(int iters, T b, T c, T* out)
{
    T a[PROBE_CHAINS];
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = (T)(threadIdx.x + j);
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < PROBE_CHAINS; ++j) a[j] = fma(a[j], b, c);
    }
    T s = 0;
#pragma unroll
    for (int j = 0; j < PROBE_CHAINS; ++j) s += a[j];
    if (s == (T)12345.678) out[blockIdx.x] = s;   // practically never taken; keeps the chains live
}

}  // namespace stag

using namespace stag;

extern "C" int stag_fma_probe(int prec, int iters, double* tflops)
{
    if ((prec != STAG_F64 && prec != STAG_F32) || iters < 1 || !tflops) {
        set_error("stag_fma_probe: prec STAG_F64 or STAG_F32, iters >= 1, tflops non-NULL");
        return STAG_EINVAL;
    }
    int dev = 0, sms = 0;
    STAG_CUDA_TRY(cudaGetDevice(&dev));
    STAG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * PROBE_BLOCKS_PER_SM;
    void* out = nullptr;
    STAG_CUDA_TRY(cudaMalloc(&out, (size_t)blocks * sizeof(double)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        auto launch = [&]() {
            if (prec == STAG_F64)
                k_fma_probe<double><<<blocks, PROBE_BS>>>(iters, 0.999999, 1e-7, (double*)out);
            else
                k_fma_probe<float><<<blocks, PROBE_BS>>>(iters, 0.999999f, 1e-7f, (float*)out);
        };
        launch();   // warm-up
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    STAG_CUDA_TRY(e);
    const double fmas = (double)blocks * PROBE_BS * PROBE_CHAINS * (double)iters;
    *tflops = 2.0 * fmas / ((double)ms * 1e-3) * 1e-12;
    return STAG_OK;
}
