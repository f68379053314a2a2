// smol_probe.cu - smol_fma_rate: the arithmetic ceiling that the right-hand-side
// kernels are measured against. The FP64 form's transforms are bound by the FP64 pipe,
// whose rate on this part is a small fraction of its FP32 rate, so its roofline needs a
// measured FP64 peak rather than a datasheet figure; the FP32 rate serves the FP32 and
// double-float forms. Measurement aid only: nothing on the solver's path calls it.
#include <cuda_runtime.h>

#include "../../include/smol.h"

namespace {

constexpr int CHAINS = 8;      // independent fused multiply-add chains per thread
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 4;

// Each thread runs CHAINS dependent chains x <- x * a + b for `iters` steps (values
// stay near the fixed point b / (1 - a)); the sum is stored only if it equals a value
// the chains cannot reach (and the sink is non-NULL), so the compiler keeps every step
// and nothing is written.
template <typename T>
__global__ void __launch_bounds__(THREADS) k_fma_chains(T a, T b, long long iters, T never, T* sink) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    if (s == never && sink != nullptr) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run(long long iters, cudaStream_t st, double* tflops, double* ms_out) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return SMOL_ECUDA;
    const int grid = sms * CTAS_PER_SM;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SMOL_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SMOL_ECUDA;
    }
    const T a = (T)0.999, b = (T)1e-3, never = (T)-1.0;  // chains stay positive: never is never reached
    k_fma_chains<T><<<grid, THREADS, 0, st>>>(a, b, iters / 8 + 1, never, (T*)nullptr);  // warm-up
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<grid, THREADS, 0, st>>>(a, b, iters, never, (T*)nullptr);
    cudaEventRecord(e1, st);
    int rc = SMOL_OK;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess || !(ms > 0.f))
        rc = SMOL_ECUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SMOL_OK) return rc;
    const double flops = 2.0 * CHAINS * (double)iters * (double)grid * THREADS;
    *tflops = flops / ((double)ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return SMOL_OK;
}

}  // namespace

extern "C" int smol_fma_rate(int32_t precision, int64_t iters, void* stream, double* tflops, double* ms) {
    if (!tflops || iters < 1) return SMOL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == SMOL_FP64) return run<double>(iters, st, tflops, ms);
    if (precision == SMOL_FP32CONV) return run<float>(iters, st, tflops, ms);
    return SMOL_EINVAL;
}
