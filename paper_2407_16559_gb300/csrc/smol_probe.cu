// smol_probe.cu - smol_fma_rate: the arithmetic ceiling that the right-hand-side
// kernels are measured against. The FP64 form's transforms are bound by the FP64 pipe,
// whose rate on this part is a small fraction of its FP32 rate, so its roofline needs a
// measured FP64 peak rather than a datasheet figure; the FP32 rate serves the FP32 and
// double-float forms. smol_op_latency gives the dependent-chain latencies behind the
// kernels' FP64 costs. Measurement aids only: nothing on the solver's path calls them.
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

// Dependent-chain latency: `warps` warps of one CTA each run one chain of `iters`
// dependent operations OP (0: FP64 fused multiply-add, 1: FP64 add, 2: FP32 fused
// multiply-add, 3: FP32 -> FP64 conversion followed by an FP64 multiply); warp 0 lane 0
// times its chain with clock64 and writes cycles per operation to *out. Stored only if
// the chain ends on a value it cannot reach, so the compiler keeps every step.
template <int OP>
__global__ void k_chain(double a, double b, int iters, double never, double* sink, double* out) {
    double x = a + (double)threadIdx.x * 1e-9;
    float xf = (float)a;
    __syncwarp();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
        if (OP == 0) x = fma(x, b, 1e-3);
        else if (OP == 1) x = x + b;
        else if (OP == 2) xf = fmaf(xf, (float)b, 1e-3f);
        else x = (double)(float)x * b;
    }
    const long long t1 = clock64();
    if (threadIdx.x == 0) *out = (double)(t1 - t0) / (double)iters;
    if (x + (double)xf == never && sink != nullptr) sink[threadIdx.x] = x;
}

template <int OP>
int chain(int warps, cudaStream_t st, double* cycles) {
    double* d = nullptr;
    if (cudaMalloc(&d, sizeof(double)) != cudaSuccess) return SMOL_ECUDA;
    const double b = OP == 1 ? 1e-9 : (OP == 3 ? 1.0000001 : 0.999);
    k_chain<OP><<<1, 32 * warps, 0, st>>>(0.5, b, 64, -1.0, nullptr, d);  // warm-up
    k_chain<OP><<<1, 32 * warps, 0, st>>>(0.5, b, 4096, -1.0, nullptr, d);
    int rc = SMOL_OK;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(cycles, d, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = SMOL_ECUDA;
    cudaFree(d);
    return rc;
}

}  // namespace

extern "C" int smol_op_latency(int32_t op, int32_t warps, void* stream, double* cycles) {
    if (!cycles || warps < 1 || warps > 32) return SMOL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    switch (op) {
        case 0: return chain<0>(warps, st, cycles);
        case 1: return chain<1>(warps, st, cycles);
        case 2: return chain<2>(warps, st, cycles);
        case 3: return chain<3>(warps, st, cycles);
        default: return SMOL_EINVAL;
    }
}

extern "C" int smol_fma_rate(int32_t precision, int64_t iters, void* stream, double* tflops, double* ms) {
    if (!tflops || iters < 1) return SMOL_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == SMOL_FP64) return run<double>(iters, st, tflops, ms);
    if (precision == SMOL_FP32CONV) return run<float>(iters, st, tflops, ms);
    return SMOL_EINVAL;
}
