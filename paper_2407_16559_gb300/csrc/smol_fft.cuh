// smol_fft.cuh - complex arithmetic, twiddle lookup and the shared-memory Stockham
// FFT tile used by the right-hand-side kernels.
//
// The birth term of Eq. (4) is a linear convolution (Sec. 1: K = U V turns the
// double sum into R convolutions). It is evaluated with real FFTs of length 2*Mp
// (Mp = FFT size, a power of two >= M), each computed as a complex FFT of length Mp
// on the even/odd-packed sequence. A length-Mp transform is split Mp = N1 * N2
// ("four-step"): N2 column transforms of length N1, a twiddle W_Mp^{n2 k1}, then N1
// row transforms of length N2. Each column / row transform runs inside one CTA in
// shared memory as an autosorting Stockham FFT with radix-8 passes (and one radix-4
// or radix-2 pass for the remaining factor).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "smol_dd.cuh"

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
__device__ __forceinline__ cx<dd> ldg(const cx<dd>* p) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return mk(dd(v.x, v.y), dd(v.z, v.w));
}

// 1/sqrt(2) in type R (the radix-8 butterfly's rotation by W_8).
template <typename R>
__device__ __forceinline__ R sqrt_half() { return (R)0.70710678118654752440; }
template <>
__device__ __forceinline__ dd sqrt_half<dd>() {
    return dd(0.70710677f, 1.21016175e-08f);  // 0.7071067811865475244 split into two floats
}

// Twiddle table: tw[e] = exp(-2 pi i e / (2 Mp)) for e in [0, Mp). Returns W_{2Mp}^e
// for any e in [0, 2 Mp) using W^{e + Mp} = -W^e.
template <typename R>
__device__ __forceinline__ cx<R> twl(const cx<R>* __restrict__ tw, uint32_t e, uint32_t Mp) {
    cx<R> w = ldg(tw + (e & (Mp - 1)));
    return (e & Mp) ? -w : w;
}

// Quotient and remainder by a runtime divisor: shifts for powers of two (the usual
// case: FFT lengths, column groups, T = 1, 2, 4), a division otherwise.
struct Div {
    int d, sh;
    bool p2;
};
__device__ __forceinline__ Div mkdiv(int d) {
    Div r;
    r.d = d;
    r.p2 = (d & (d - 1)) == 0;
    r.sh = __ffs(d) - 1;
    return r;
}
__device__ __forceinline__ void divmod(const Div& D, int x, int& q, int& r) {
    if (D.p2) {
        q = x >> D.sh;
        r = x & (D.d - 1);
    } else {
        q = x / D.d;
        r = x - q * D.d;
    }
}

// The transform direction is a run-time argument (inv: the sign +i, the unnormalised
// inverse). Both directions compute the same sums and products (the rotations differ
// only in signs and in which of them goes to the real part).

// Length-4 DFT in place (forward: W_4 = -i; inverse: +i).
template <typename R>
__device__ __forceinline__ void dft4(cx<R>& x0, cx<R>& x1, cx<R>& x2, cx<R>& x3, bool inv) {
    const cx<R> s0 = x0 + x2, d0 = x0 - x2, s1 = x1 + x3;
    const cx<R> t = x1 - x3;
    const cx<R> d1 = inv ? mul_pi(t) : mul_mi(t);
    x0 = s0 + s1;
    x2 = s0 - s1;
    x1 = d0 + d1;
    x3 = d0 - d1;
}

// Length-8 DFT in place: a radix-2 split (u_m +- u_{m+4}, the difference rotated by
// W_8^m), then two length-4 DFTs giving the even and the odd outputs.
template <typename R>
__device__ __forceinline__ void dft8(cx<R>* u, bool inv) {
    const R h = sqrt_half<R>();
    cx<R> a0 = u[0] + u[4], a1 = u[1] + u[5], a2 = u[2] + u[6], a3 = u[3] + u[7];
    cx<R> b0 = u[0] - u[4], b1 = u[1] - u[5], b2 = u[2] - u[6], b3 = u[3] - u[7];
    // b1 * (1 -+ i)/sqrt 2, b2 * (-+ i), b3 * (-1 -+ i)/sqrt 2 (upper sign: forward)
    const R s1 = (b1.x + b1.y) * h, d1 = (b1.x - b1.y) * h;
    const R s3 = (b3.x + b3.y) * h, d3 = (b3.x - b3.y) * h;
    b1 = inv ? mk<R>(d1, s1) : mk<R>(s1, -d1);
    b2 = inv ? mul_pi(b2) : mul_mi(b2);
    b3 = inv ? mk<R>(-s3, d3) : mk<R>(-d3, -s3);
    dft4<R>(a0, a1, a2, a3, inv);
    dft4<R>(b0, b1, b2, b3, inv);
    u[0] = a0;
    u[1] = b0;
    u[2] = a1;
    u[3] = b1;
    u[4] = a2;
    u[5] = b2;
    u[6] = a3;
    u[7] = b3;
}

// Length-8 DFT of u[0..3] with u[4..7] = 0 (the first pass of a zero-padded input):
// the radix-2 split is then a copy, a_m = b_m = u_m.
template <typename R>
__device__ __forceinline__ void dft8_lower(cx<R>* u, bool inv) {
    const R h = sqrt_half<R>();
    cx<R> a0 = u[0], a1 = u[1], a2 = u[2], a3 = u[3];
    cx<R> b0 = u[0], b1 = u[1], b2 = u[2], b3 = u[3];
    const R s1 = (b1.x + b1.y) * h, d1 = (b1.x - b1.y) * h;
    const R s3 = (b3.x + b3.y) * h, d3 = (b3.x - b3.y) * h;
    b1 = inv ? mk<R>(d1, s1) : mk<R>(s1, -d1);
    b2 = inv ? mul_pi(b2) : mul_mi(b2);
    b3 = inv ? mk<R>(-s3, d3) : mk<R>(-d3, -s3);
    dft4<R>(a0, a1, a2, a3, inv);
    dft4<R>(b0, b1, b2, b3, inv);
    u[0] = a0;
    u[1] = b0;
    u[2] = a1;
    u[3] = b1;
    u[4] = a2;
    u[5] = b2;
    u[6] = a3;
    u[7] = b3;
}

// Which half of a tile transform is known or wanted (zero-padded convolution inputs
// and the linear part of the inverse): HALF_IN, the upper half of the input is zero and
// not read (first pass); HALF_OUT, only the lower half of the output is written (last
// pass: outputs m < RAD / 2 of each butterfly).
enum { HALF_NONE = 0, HALF_IN = 1, HALF_OUT = 2 };

// One Stockham pass of radix RAD (8, 4 or 2) on sub-transform length p = 2^lgp of a
// length-P transform over G interleaved sequences: for butterfly i in [0, P/RAD),
// k = i mod p, inputs in[i + m P/RAD] (m < RAD) are multiplied by W_{RAD p}^{m k},
// transformed by a length-RAD DFT and stored at out[(i-k) RAD + k + m p].
// twP is a shared-memory table twP[e] = W_P^e, e < P (conjugated for the inverse).
template <typename R, int RAD, int HALF = HALF_NONE>
__device__ __forceinline__ void stockham_pass(const cx<R>* __restrict__ a, cx<R>* __restrict__ b, int lgP, int lgp,
                                              int G, const cx<R>* __restrict__ twP, bool inv) {
    constexpr int LGR = RAD == 8 ? 3 : (RAD == 4 ? 2 : 1);
    const int P = 1 << lgP;
    const int p = 1 << lgp;
    const int q = P >> LGR;
    const int nb = q * G;
    const int sh = lgP - LGR - lgp;  // W_{RAD p}^{e} = W_P^{e << sh}
    const Div DG = mkdiv(G);
    for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
        int g, i;
        divmod(DG, idx, i, g);
        const int k = i & (p - 1);
        cx<R> u[RAD];
#pragma unroll
        for (int m = 0; m < RAD; ++m)
            u[m] = (HALF == HALF_IN && m >= RAD / 2) ? mk<R>((R)0, (R)0) : a[(i + m * q) * G + g];
        if (HALF == HALF_IN && RAD == 8) {
            dft8_lower<R>(u, inv);  // a first pass (p = 1): k = 0, no twiddles
        } else {
            if (k) {
#pragma unroll
                for (int m = 1; m < RAD; ++m) {
                    cx<R> w = twP[(m * k) << sh];
                    if (inv) w = conj(w);
                    u[m] = u[m] * w;
                }
            }
            if (RAD == 8) {
                dft8<R>(u, inv);
            } else if (RAD == 4) {
                dft4<R>(u[0], u[1], u[2], u[3], inv);
            } else {
                const cx<R> t = u[0] - u[1];
                u[0] = u[0] + u[1];
                u[1] = t;
            }
        }
        const int j = ((i - k) << LGR) + k;
#pragma unroll
        for (int m = 0; m < (HALF == HALF_OUT ? RAD / 2 : RAD); ++m) b[(j + m * p) * G + g] = u[m];
    }
}

template <typename R, int HALF>
__device__ __forceinline__ void pass_sel(const cx<R>* a, cx<R>* b, int lgP, int lgp, int G,
                                         const cx<R>* __restrict__ twP, bool inv, int rad) {
    if (rad == 8) stockham_pass<R, 8, HALF>(a, b, lgP, lgp, G, twP, inv);
    else if (rad == 4) stockham_pass<R, 4, HALF>(a, b, lgP, lgp, G, twP, inv);
    else stockham_pass<R, 2, HALF>(a, b, lgP, lgp, G, twP, inv);
}

// Stockham autosort FFT of length P = 2^lgP on G interleaved sequences held in shared
// memory as buf[p * G + g] (g fastest), radix-8 passes first, then one radix-4 or
// radix-2 pass for the remaining factor. Ping-pongs between a and b and returns the
// buffer holding the result, in natural order. inv selects the sign +i (unnormalised
// inverse). twP: shared table W_P^e, e < P. HALF_IN: the upper half of the input is zero
// and is not read; HALF_OUT: only the lower half of the result is written. Every thread
// of the block must call it; the caller synchronises before.
template <typename R, int HALF = HALF_NONE>
__device__ __forceinline__ cx<R>* tile_fft_body(cx<R>* a, cx<R>* b, int lgP, int G, const cx<R>* __restrict__ twP,
                                                bool inv) {
    int lgp = 0;
    while (lgp < lgP) {
        const int rem = lgP - lgp;
        const int rad = rem >= 3 ? 8 : (rem == 2 ? 4 : 2);
        const int lgr = rem >= 3 ? 3 : rem;
        if (HALF == HALF_IN && lgp == 0) pass_sel<R, HALF_IN>(a, b, lgP, lgp, G, twP, inv, rad);
        else if (HALF == HALF_OUT && lgp + lgr == lgP) pass_sel<R, HALF_OUT>(a, b, lgP, lgp, G, twP, inv, rad);
        else pass_sel<R, HALF_NONE>(a, b, lgP, lgp, G, twP, inv, rad);
        lgp += lgr;
        __syncthreads();
        cx<R>* t = a;
        a = b;
        b = t;
    }
    return a;
}
template <typename R, int HALF = HALF_NONE>
__device__ __forceinline__ cx<R>* tile_fft(cx<R>* a, cx<R>* b, int lgP, int G, const cx<R>* __restrict__ twP,
                                           bool inv) {
    return tile_fft_body<R, HALF>(a, b, lgP, G, twP, inv);
}

// Asynchronous global -> shared copies of one element (4, 8 or 16 bytes; both addresses
// aligned to the size): every copy a thread issues is in flight at once, and
// cp_async_wait() waits for all of the calling thread's copies (a barrier then makes
// them visible to the CTA).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
template <typename T>
__device__ __forceinline__ void cp_async_el(T* smem, const T* gmem) {
    cp_async<(int)sizeof(T)>(smem, gmem);
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Gather of data that other CTAs wrote earlier in the same kernel (the persistent
// attempt kernel): through L2 only, since an SM's L1 may still hold the lines of an
// earlier phase. 16-byte elements keep the asynchronous copy (cp.async.cg); smaller ones
// are loaded with ld.global.cg and stored. CG = false: the ordinary cached copy.
template <bool CG, typename T>
__device__ __forceinline__ void gather_el(T* smem, const T* gmem) {
    if constexpr (!CG) {
        cp_async_el(smem, gmem);
    } else if constexpr (sizeof(T) == 16) {
        const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
    } else {
        static_assert(sizeof(T) == 8, "8- or 16-byte elements");
        *reinterpret_cast<float2*>(smem) = __ldcg(reinterpret_cast<const float2*>(gmem));
    }
}

// Stages the table W_P^e (e < P) of a length-P tile transform into shared memory from
// the global table of W_{2Mp}^e (e < Mp; W^{e + Mp} = -W^e): stage_tw issues the
// copies, stage_tw_fix (after cp_async_wait, by the same threads) negates the entries
// taken from the second half-period.
template <typename R>
__device__ __forceinline__ void stage_tw(cx<R>* twP, int lgP, const cx<R>* __restrict__ tw, int lgMp) {
    const int P = 1 << lgP;
    const int sh = lgMp + 1 - lgP;
    const uint32_t Mp = 1u << lgMp;
    for (int e = threadIdx.x; e < P; e += blockDim.x) cp_async_el(twP + e, tw + (((uint32_t)e << sh) & (Mp - 1)));
}
template <typename R>
__device__ __forceinline__ void stage_tw_fix(cx<R>* twP, int lgP, int lgMp) {
    const int P = 1 << lgP;
    const int sh = lgMp + 1 - lgP;
    const uint32_t Mp = 1u << lgMp;
    for (int e = threadIdx.x; e < P; e += blockDim.x)
        if (((uint32_t)e << sh) & Mp) twP[e] = -twP[e];
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

// Block-wide minimum (inactive lanes contribute +inf). The result is valid in every
// thread; ends with a barrier.
__device__ __forceinline__ double block_min(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < nw) ? sh[lane] : INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
        if (lane == 0) sh[32] = v;
    }
    __syncthreads();
    return sh[32];
}

// Block-wide maximum of non-negative values (inactive lanes contribute 0).
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
