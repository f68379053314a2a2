// smol_fft.cuh - complex arithmetic, twiddle lookup and the shared-memory Stockham
// FFT tile used by the right-hand-side kernels.
//
// The birth term of Eq. (4) is a linear convolution (Sec. 1: K = U V turns the
// double sum into R convolutions). It is evaluated with real FFTs of length 2*Mp
// (Mp = FFT size, a power of two >= M), each computed as a complex FFT of length Mp
// on the even/odd-packed sequence. A length-Mp transform is split Mp = N1 * N2
// ("four-step"): N2 column transforms of length N1, a twiddle W_Mp^{n2 k1}, then N1
// row transforms of length N2. Each column / row transform runs inside one CTA in
// shared memory as an autosorting Stockham FFT with radix-4 passes (and one radix-2
// pass when log2 of the length is odd).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace smol {

template <typename R>
struct cx {
    R x, y;
};

template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) {
    cx<R> r;
    r.x = a;
    r.y = b;
    return r;
}
template <typename R>
__device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename R>
__device__ __forceinline__ cx<R> operator-(cx<R> a) { return mk(-a.x, -a.y); }
template <typename R>
__device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__device__ __forceinline__ cx<R> scl(cx<R> a, R s) { return mk(a.x * s, a.y * s); }
template <typename R>
__device__ __forceinline__ cx<R> conj(cx<R> a) { return mk(a.x, -a.y); }
// multiply by -i and by +i
template <typename R>
__device__ __forceinline__ cx<R> mul_mi(cx<R> a) { return mk(a.y, -a.x); }
template <typename R>
__device__ __forceinline__ cx<R> mul_pi(cx<R> a) { return mk(-a.y, a.x); }

// Read-only cached load of one complex value.
__device__ __forceinline__ cx<double> ldg(const cx<double>* p) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
}
__device__ __forceinline__ cx<float> ldg(const cx<float>* p) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return mk(v.x, v.y);
}

// Twiddle table: tw[e] = exp(-2 pi i e / (2 Mp)) for e in [0, Mp). Returns W_{2Mp}^e
// for any e in [0, 2 Mp) using W^{e + Mp} = -W^e.
template <typename R>
__device__ __forceinline__ cx<R> twl(const cx<R>* __restrict__ tw, uint32_t e, uint32_t Mp) {
    cx<R> w = ldg(tw + (e & (Mp - 1)));
    return (e & Mp) ? -w : w;
}

// Stockham autosort FFT of length P = 2^lgP on G interleaved sequences held in shared
// memory as buf[p * G + g] (g fastest). Ping-pongs between a and b and returns the
// buffer holding the result, in natural order. INV selects the sign +i (unnormalised
// inverse). Every thread of the block must call it; the caller synchronises before.
//
// Pass with radix r on sub-transform length p (product of the radices so far): for
// butterfly i in [0, P/r), k = i mod p, inputs in[i + m P/r] (m < r) are multiplied
// by W_{r p}^{m k}, transformed by a length-r DFT and stored at out[(i-k) r + k + m p].
template <typename R, bool INV>
__device__ cx<R>* tile_fft(cx<R>* a, cx<R>* b, int lgP, int G, const cx<R>* __restrict__ tw, int lgMp) {
    const int P = 1 << lgP;
    const uint32_t Mp = 1u << lgMp;
    int lgp = 0;
    while (lgp < lgP) {
        const int p = 1 << lgp;
        if (lgP - lgp >= 2) {
            const int q = P >> 2;
            const int nb = q * G;
            const int sh = (lgMp + 1) - 2 - lgp;   // W_{4p}^{e} = W_{2Mp}^{e << sh}
            for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
                const int g = idx % G;
                const int i = idx / G;
                const int k = i & (p - 1);
                cx<R> u0 = a[i * G + g];
                cx<R> u1 = a[(i + q) * G + g];
                cx<R> u2 = a[(i + 2 * q) * G + g];
                cx<R> u3 = a[(i + 3 * q) * G + g];
                if (k) {
                    cx<R> w1 = twl(tw, (uint32_t)k << sh, Mp);
                    cx<R> w2 = twl(tw, (uint32_t)(2 * k) << sh, Mp);
                    cx<R> w3 = twl(tw, (uint32_t)(3 * k) << sh, Mp);
                    if (INV) {
                        w1 = conj(w1);
                        w2 = conj(w2);
                        w3 = conj(w3);
                    }
                    u1 = u1 * w1;
                    u2 = u2 * w2;
                    u3 = u3 * w3;
                }
                cx<R> a0 = u0 + u2, a1 = u0 - u2, a2 = u1 + u3, a3 = u1 - u3;
                a3 = INV ? mul_pi(a3) : mul_mi(a3);
                const int j = ((i - k) << 2) + k;
                b[j * G + g] = a0 + a2;
                b[(j + p) * G + g] = a1 + a3;
                b[(j + 2 * p) * G + g] = a0 - a2;
                b[(j + 3 * p) * G + g] = a1 - a3;
            }
            lgp += 2;
        } else {
            const int q = P >> 1;
            const int nb = q * G;
            const int sh = (lgMp + 1) - 1 - lgp;
            for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
                const int g = idx % G;
                const int i = idx / G;
                const int k = i & (p - 1);
                cx<R> u0 = a[i * G + g];
                cx<R> u1 = a[(i + q) * G + g];
                if (k) {
                    cx<R> w = twl(tw, (uint32_t)k << sh, Mp);
                    if (INV) w = conj(w);
                    u1 = u1 * w;
                }
                const int j = ((i - k) << 1) + k;
                b[j * G + g] = u0 + u1;
                b[(j + p) * G + g] = u0 - u1;
            }
            lgp += 1;
        }
        __syncthreads();
        cx<R>* t = a;
        a = b;
        b = t;
    }
    return a;
}

// Deterministic block-wide sum (fixed reduction order). sh: >= 32 doubles of shared
// memory. The result is valid in every thread. Ends with a barrier.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < nw) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    return sh[32];
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < nw) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    return sh[32];
}

}  // namespace smol
