// smol_rhs.cuh - device data structures and the three kernels of one evaluation of
// the right-hand side S(y) of Eq. (4) (aggregation-shattering, truncated at M) for a
// low-rank kernel K = U V (Sec. 1).
//
// Notation. Sizes s = 1..M are stored 0-based (y[s-1] = y_s). The distinct vectors
// among the columns U_alpha and rows V_alpha are W_t (t < T); U_alpha = cu W_{u(alpha)},
// V_alpha = cv W_{v(alpha)}, coef_alpha = cu cv. With x_t = W_t . y (elementwise):
//   birth_s  = 1/2 sum_alpha coef_alpha (x_u * x_v)[s-2]        (linear convolution)
//   D_s      = sum_j K_{s,j} y_j = sum_alpha coef_alpha W_u[s] mu_v,  mu_t = sum_i W_t[i] y_i
//   S_s      = birth_s - (1 + lambda [s>=2]) y_s D_s             (s >= 2: Eq. (4), 2nd line)
//   S_1      = -y_1 D_1 + (lambda/2) sum_{i,j>=2} (i+j) K_ij y_i y_j + lambda y_1 sum_{j>=2} j K_1j y_j
// with the two shattering sums written through rank-R moments:
//   sum_{i,j>=2} (i+j) K_ij y_i y_j = sum_alpha coef_alpha (rho_u sigma_v + sigma_u rho_v),
//   sum_{j>=2} j K_1j y_j          = sum_alpha coef_alpha W_u[1] rho_v,
//   sigma_t = sum_{i>=2} W_t[i] y_i,   rho_t = sum_{i>=2} i W_t[i] y_i.
//
// FFT route (per evaluation): x_t has length M; it is zero-padded to the real length
// L = 2 Mp and packed as z_t[j] = x_t[2j] + i x_t[2j+1] (j < Mp/2; zero above). With
// Z_t = FFT_Mp(z_t):  X_t[k] = E + W_L^k O and X_t[Mp-k] = conj(E - W_L^k O), where
// E = (Z[k] + conj Z[Mp-k]) / 2, O = -i (Z[k] - conj Z[Mp-k]) / 2. The product sum
// C = sum_pairs coef X_u X_v is delayed by one sample (C'[k] = W_L^k C[k]) so that the
// inverse yields c'[i] = c[i-1] and birth at 0-based index i is c'[i] / 2 directly.
// The real inverse of length L is again done at length Mp on the packed form
//   Y[k] = 1/2 [ W_L^k (C[k] - conj C[Mp-k]) + i (C[k] + conj C[Mp-k]) ],
// whose inverse FFT gives y[j] = c'[2j] + i c'[2j+1] (times Mp; the 1/Mp and the 1/2 of
// the birth term are applied in FP64 in the epilogue).
#pragma once
#include "smol_fft.cuh"

namespace smol {

constexpr int MAXR = 8;         // largest rank R
constexpr int MAXT = 2 * MAXR;  // largest number of distinct transforms
constexpr int MAXV = 10;        // terms of a stage-input linear combination

// Device-resident control block of one integration (and of standalone evaluations).
struct Ctl {
    double t, tau, h, t1, tol;  // time, proposed step, step of the current attempt, end, tolerance
    double err_last;            // error estimate of the last attempt
    double nrm2;                // ||n||_2^2 of the current state
    double ymax;                // max_i |n_i| of the current state (FP32 input scaling)
    double steady;              // ||S(n)||_2^2 of the current attempt's first stage (unscaled)
    int32_t done, status, cur, clamped;
    int64_t attempts, accepted, rejected, rhs_evals, rhs_paper;
    double* state[2];           // double-buffered state; state[cur] is n^k
    uint32_t arrive;            // arrival counter of the last-block-done reductions
    int32_t pad;
};

// Static description of a system, passed by value to every kernel.
struct SysDev {
    int M, Mp, lgMp, N1, N2, lgN1, lgN2, T, R, npairs, nbxA;
    double lambda;
    const double* W;             // T x Mp weights (zero beyond M)
    const void* tw;              // twiddles W_{2Mp}^e, e < Mp, as cx<R>
    void* Y;                     // T x Mp spectra after the column pass, [t][k1][n2]
    void* G2;                    // Mp values after the row pass, [k1][n2]
    double* ybuf;                // stage input y (Mp doubles)
    double* mpart;               // moment partials [t][bx][2]
    int au[MAXR], av[MAXR];      // ordered pairs (u(alpha), v(alpha))
    double acoef[MAXR];
    int pu[MAXR], pv[MAXR];      // unordered pairs for the spectral product
    double pcoef[MAXR];
    int wexp[MAXT];              // ilogb(max_i |W_t[i]|)
};

// Stage input y = sum_j c_j v_j. sel[j] < 0: v[j] as given; sel[j] = 0 / 1: the
// current / other state buffer of the control block.
struct StageIn {
    int nv, direct;              // direct: y is v[0] itself (nv == 1, c == 1)
    int sel[MAXV];
    const double* v[MAXV];
    double c[MAXV];
};

// Epilogue outputs of an evaluation.
struct EpiOut {
    double* out;                 // out = scale * S(y); scale = h * hfac (use_h) or 1
    double* birth;               // optional term outputs
    double* loss;
    double* source;
    double* sqpart;              // optional per-CTA partials of ||S(y)||_2^2
    double hfac;
    int use_h;
};

__device__ __forceinline__ const double* resolve(const StageIn& in, const Ctl* ctl, int j) {
    return in.sel[j] < 0 ? in.v[j] : ctl->state[ctl->cur ^ in.sel[j]];
}

// The term pointers of a stage input with the state buffers resolved once (the control
// block is read a single time per thread).
struct StagePtrs {
    const double* p[MAXV];
};

__device__ __forceinline__ StagePtrs resolve_all(const StageIn& in, const Ctl* ctl) {
    StagePtrs r;
    const int cur = ctl->cur;
    const double* s0 = ctl->state[0];
    const double* s1 = ctl->state[1];
#pragma unroll
    for (int j = 0; j < MAXV; ++j) r.p[j] = in.sel[j] < 0 ? in.v[j] : (((cur ^ in.sel[j]) & 1) ? s1 : s0);
    return r;
}

// y at indices i and i+1 (i even); zero at and beyond M. All term loads are issued
// before the first multiply-add (unrolled over MAXV, predicated on nv) so that their
// latencies overlap.
__device__ __forceinline__ void stage_pair(const StageIn& in, const StagePtrs& P, int M, int i, double& y0,
                                           double& y1) {
    y0 = 0.0;
    y1 = 0.0;
    if (i + 1 < M) {
        double2 v[MAXV];
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) v[j] = __ldg(reinterpret_cast<const double2*>(P.p[j] + i));
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) {
                y0 += in.c[j] * v[j].x;
                y1 += in.c[j] * v[j].y;
            }
    } else if (i < M) {
        double v[MAXV];
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) v[j] = __ldg(P.p[j] + i);
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) y0 += in.c[j] * v[j];
    }
}

template <typename R>
__device__ __forceinline__ R to_r(double v, int e) {
    return (R)(e ? ldexp(v, -e) : v);
}

// Exponent of the input scaling of transform t: FP64 runs unscaled; FP32 divides
// x_t by 2^(ilogb(max|W_t|) + ilogb(max|y|)) so that its largest entry is near 1.
template <typename R>
__device__ __forceinline__ int xexp(const SysDev& S, const Ctl* ctl, int t) {
    if (sizeof(R) == sizeof(double)) return 0;
    const double ym = ctl->ymax;
    return (ym > 0.0 && isfinite(ym)) ? S.wexp[t] + ilogb(ym) : S.wexp[t];
}

// ---------------------------------------------------------------------------
// Kernel A: stage input, moments, column transforms of length N1.
// grid (N2 / G, T); one transform t and G adjacent columns n2 per CTA.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_fwd_cols(const SysDev S, const StageIn in, const Ctl* __restrict__ ctl, int G) {
    if (ctl->done) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[33];
    cx<R>* a = reinterpret_cast<cx<R>*>(smraw);
    cx<R>* b = a + (S.N1 * G);
    const int t = blockIdx.y;
    const int n2b = blockIdx.x * G;
    const int e = xexp<R>(S, ctl, t);
    const double* Wt = S.W + (size_t)t * S.Mp;
    const int half = (S.N1 >> 1) * G;
    double mu = 0.0, nu = 0.0;
    const bool store_y = (t == 0) && !in.direct;
    const StagePtrs sp = resolve_all(in, ctl);
    for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
        const int g = idx % G;
        const int n1 = idx / G;
        const int j = (n1 << S.lgN2) + n2b + g;
        const int i = 2 * j;
        double y0, y1;
        stage_pair(in, sp, S.M, i, y0, y1);
        const double2 w = __ldg(reinterpret_cast<const double2*>(Wt + i));
        const double x0 = w.x * y0, x1 = w.y * y1;
        mu += x0 + x1;
        nu += (double)(i + 1) * x0 + (double)(i + 2) * x1;
        if (store_y) *reinterpret_cast<double2*>(S.ybuf + i) = make_double2(y0, y1);
        a[idx] = mk<R>(to_r<R>(x0, e), to_r<R>(x1, e));
    }
    for (int idx = half + threadIdx.x; idx < S.N1 * G; idx += blockDim.x) a[idx] = mk<R>((R)0, (R)0);
    mu = block_sum(mu, red);
    nu = block_sum(nu, red);
    if (threadIdx.x == 0) {
        double* p = S.mpart + 2 * ((size_t)t * gridDim.x + blockIdx.x);
        p[0] = mu;
        p[1] = nu;
    }
    const cx<R>* tw = reinterpret_cast<const cx<R>*>(S.tw);
    cx<R>* res = tile_fft<R, false>(a, b, S.lgN1, G, tw, S.lgMp);
    cx<R>* Y = reinterpret_cast<cx<R>*>(S.Y) + (size_t)t * S.Mp;
    const uint32_t mask2 = 2u * (uint32_t)S.Mp - 1u;
    for (int idx = threadIdx.x; idx < S.N1 * G; idx += blockDim.x) {
        const int g = idx % G;
        const int k1 = idx / G;
        const int n2 = n2b + g;
        const cx<R> w = twl(tw, (2u * (uint32_t)n2 * (uint32_t)k1) & mask2, (uint32_t)S.Mp);
        Y[(size_t)k1 * S.N2 + n2] = res[idx] * w;
    }
}

// ---------------------------------------------------------------------------
// Kernel B: row transforms of length N2 for a pair of rows (k1, N1 - k1), the
// real-FFT split, the product sum over kernel terms, the packed inverse spectrum,
// inverse row transforms and the inverse twiddle.
// grid N1 / 2. CTA b owns rows (b, N1 - b); CTA 0 owns rows (0, N1 / 2).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void spectral_pair(const SysDev& S, const cx<R>* Z, int G, int ia, int ib, uint32_t ka,
                                              const cx<R>* tw, const R* pc, cx<R>& Ya, cx<R>& Yb) {
    // Z holds the row spectra as Z[k2 * G + col], col = 2 t + rho; ia / ib are the
    // offsets k2 * G + rho of the pair's two frequencies (ka and Mp - ka).
    const cx<R> w = ldg(tw + ka);  // W_L^ka, ka < Mp
    cx<R> Ca = mk<R>((R)0, (R)0), Cb = Ca;
    for (int p = 0; p < S.npairs; ++p) {
        const int u = S.pu[p], v = S.pv[p];
        cx<R> Xa[2], Xb[2];
        const int tt[2] = {u, v};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const cx<R> za = Z[ia + 2 * tt[q]];
            const cx<R> zb = conj(Z[ib + 2 * tt[q]]);
            const cx<R> E = scl(za + zb, (R)0.5);
            const cx<R> O = scl(mul_mi(za - zb), (R)0.5);
            const cx<R> wO = w * O;
            Xa[q] = E + wO;
            Xb[q] = conj(E - wO);
        }
        Ca = Ca + scl(Xa[0] * Xa[1], pc[p]);
        Cb = Cb + scl(Xb[0] * Xb[1], pc[p]);
    }
    const cx<R> wb = -conj(w);  // W_L^(Mp - ka)
    Ya = scl(w * (Ca - conj(Cb)) + mul_pi(Ca + conj(Cb)), (R)0.5);
    Yb = scl(wb * (Cb - conj(Ca)) + mul_pi(Cb + conj(Ca)), (R)0.5);
}

template <typename R>
__global__ void __launch_bounds__(256) k_rows(const SysDev S, const Ctl* __restrict__ ctl) {
    if (ctl->done) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ R pc[MAXR];
    const int G = 2 * S.T;
    cx<R>* a = reinterpret_cast<cx<R>*>(smraw);
    cx<R>* b = a + S.N2 * G;
    const int blk = blockIdx.x;
    const int r0 = blk ? blk : 0;
    const int r1 = blk ? S.N1 - blk : (S.N1 >> 1);
    const int N2 = S.N2;
    if (threadIdx.x < S.npairs) {
        // FP32: pair p carries 2^(e_u + e_v - e_max) so that the sum stays in range.
        double c = S.pcoef[threadIdx.x];
        if (sizeof(R) == sizeof(float)) {
            int emax = -100000;
            for (int p = 0; p < S.npairs; ++p)
                emax = max(emax, xexp<R>(S, ctl, S.pu[p]) + xexp<R>(S, ctl, S.pv[p]));
            c = ldexp(c, xexp<R>(S, ctl, S.pu[threadIdx.x]) + xexp<R>(S, ctl, S.pv[threadIdx.x]) - emax);
        }
        pc[threadIdx.x] = (R)c;
    }
    const cx<R>* Yin = reinterpret_cast<const cx<R>*>(S.Y);
    for (int idx = threadIdx.x; idx < N2 * G; idx += blockDim.x) {
        const int k2 = idx % N2;      // consecutive threads read consecutive k2 (coalesced)
        const int col = idx / N2;
        const int t = col >> 1, rho = col & 1;
        const int r = rho ? r1 : r0;
        a[k2 * G + col] = Yin[(size_t)t * S.Mp + (size_t)r * N2 + k2];
    }
    __syncthreads();
    const cx<R>* tw = reinterpret_cast<const cx<R>*>(S.tw);
    cx<R>* Z = tile_fft<R, false>(a, b, S.lgN2, G, tw, S.lgMp);
    cx<R>* Yo = (Z == a) ? b : a;  // packed inverse spectrum, [k2 * 2 + rho]
    const int ntask = blk ? N2 : N2 + 1;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int k2a, rhoa, k2b, rhob;
        if (blk) {
            k2a = task; rhoa = 0; k2b = N2 - 1 - task; rhob = 1;
        } else if (task <= (N2 >> 1)) {
            k2a = task; rhoa = 0; k2b = (N2 - task) & (N2 - 1); rhob = 0;
        } else {
            k2a = task - (N2 >> 1) - 1; rhoa = 1; k2b = N2 - 1 - k2a; rhob = 1;
        }
        const uint32_t ka = (uint32_t)(rhoa ? r1 : r0) + (uint32_t)S.N1 * (uint32_t)k2a;
        cx<R> Ya, Yb;
        spectral_pair<R>(S, Z, G, k2a * G + rhoa, k2b * G + rhob, ka, tw, pc, Ya, Yb);
        Yo[k2a * 2 + rhoa] = Ya;
        if (k2a != k2b || rhoa != rhob) Yo[k2b * 2 + rhob] = Yb;
    }
    __syncthreads();
    cx<R>* res = tile_fft<R, true>(Yo, Z, S.lgN2, 2, tw, S.lgMp);
    cx<R>* G2 = reinterpret_cast<cx<R>*>(S.G2);
    const uint32_t mask2 = 2u * (uint32_t)S.Mp - 1u;
    for (int idx = threadIdx.x; idx < 2 * N2; idx += blockDim.x) {
        const int n2 = idx % N2;
        const int rho = idx / N2;
        const int r = rho ? r1 : r0;
        const cx<R> w = conj(twl(tw, (2u * (uint32_t)n2 * (uint32_t)r) & mask2, (uint32_t)S.Mp));
        G2[(size_t)r * N2 + n2] = res[n2 * 2 + rho] * w;
    }
}

// ---------------------------------------------------------------------------
// Kernel C: inverse column transforms of length N1 (only the first half of the
// outputs is needed), then the epilogue: birth, death, shattering, monomer source,
// scaled output. grid N2 / G.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_inv_cols(const SysDev S, const StageIn in, const Ctl* __restrict__ ctl,
                                                  const EpiOut eo, int G) {
    if (ctl->done) return;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double red[33];
    __shared__ double mom[2 * MAXT];
    __shared__ double delta[MAXT];
    __shared__ double w1s[MAXT];
    __shared__ double src_s, bscale_s;
    cx<R>* a = reinterpret_cast<cx<R>*>(smraw);
    cx<R>* b = a + (S.N1 * G);
    const int n2b = blockIdx.x * G;
    const cx<R>* G2 = reinterpret_cast<const cx<R>*>(S.G2);
    for (int idx = threadIdx.x; idx < S.N1 * G; idx += blockDim.x) {
        const int g = idx % G;
        const int k1 = idx / G;
        a[idx] = G2[(size_t)k1 * S.N2 + n2b + g];
    }
    // Moments mu_t, nu_t from the column-pass partials: one warp per quantity, fixed order.
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int q = warp; q < 2 * S.T; q += nw) {
            const int t = q >> 1, which = q & 1;
            double s = 0.0;
            for (int bx = lane; bx < S.nbxA; bx += 32) s += S.mpart[2 * ((size_t)t * S.nbxA + bx) + which];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) mom[q] = s;
        }
    }
    __syncthreads();
    const double* ysrc = in.direct ? resolve_all(in, ctl).p[0] : S.ybuf;
    if (threadIdx.x == 0) {
        const double y1 = (S.M > 0) ? ysrc[0] : 0.0;
        double sig[MAXT], rho[MAXT];
        for (int t = 0; t < S.T; ++t) {
            const double w1 = S.W[(size_t)t * S.Mp];
            w1s[t] = w1;
            sig[t] = mom[2 * t] - w1 * y1;        // sum_{i>=2} W_t[i] y_i
            rho[t] = mom[2 * t + 1] - w1 * y1;    // sum_{i>=2} i W_t[i] y_i
            delta[t] = 0.0;
        }
        double shat = 0.0, mono = 0.0;
        for (int al = 0; al < S.R; ++al) {
            const int u = S.au[al], v = S.av[al];
            const double c = S.acoef[al];
            delta[u] += c * mom[2 * v];
            shat += c * (rho[u] * sig[v] + sig[u] * rho[v]);
            mono += c * w1s[u] * rho[v];
        }
        src_s = 0.5 * S.lambda * shat + S.lambda * y1 * mono;
        int emax = 0;
        if (sizeof(R) == sizeof(float)) {
            emax = -100000;
            for (int p = 0; p < S.npairs; ++p)
                emax = max(emax, xexp<R>(S, ctl, S.pu[p]) + xexp<R>(S, ctl, S.pv[p]));
        }
        bscale_s = ldexp(0.5 / (double)S.Mp, emax);
    }
    __syncthreads();
    const cx<R>* tw = reinterpret_cast<const cx<R>*>(S.tw);
    cx<R>* res = tile_fft<R, true>(a, b, S.lgN1, G, tw, S.lgMp);
    const double scale = eo.use_h ? ctl->h * eo.hfac : 1.0;
    const double bscale = bscale_s, lam = S.lambda, src = src_s;
    const int half = (S.N1 >> 1) * G;
    double sq = 0.0;
    for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
        const int g = idx % G;
        const int n1 = idx / G;
        const int j = (n1 << S.lgN2) + n2b + g;
        const int i = 2 * j;
        if (i >= S.M) continue;
        const cx<R> z = res[idx];
        double D0 = 0.0, D1 = 0.0;
        for (int t = 0; t < S.T; ++t) {
            const double2 w = __ldg(reinterpret_cast<const double2*>(S.W + (size_t)t * S.Mp + i));
            D0 += delta[t] * w.x;
            D1 += delta[t] * w.y;
        }
        double y0, y1;
        if (i + 1 < S.M) {
            const double2 yy = *reinterpret_cast<const double2*>(ysrc + i);
            y0 = yy.x;
            y1 = yy.y;
        } else {
            y0 = ysrc[i];
            y1 = 0.0;
        }
        const double b0 = (i == 0) ? 0.0 : (double)z.x * bscale;
        const double b1 = (double)z.y * bscale;
        const double l0 = (1.0 + (i == 0 ? 0.0 : lam)) * y0 * D0;
        const double l1 = (1.0 + lam) * y1 * D1;
        const double s0 = b0 - l0 + (i == 0 ? src : 0.0);
        const double s1 = b1 - l1;
        if (i + 1 < S.M) {
            if (eo.out) *reinterpret_cast<double2*>(eo.out + i) = make_double2(scale * s0, scale * s1);
            if (eo.birth) *reinterpret_cast<double2*>(eo.birth + i) = make_double2(b0, b1);
            if (eo.loss) *reinterpret_cast<double2*>(eo.loss + i) = make_double2(l0, l1);
            sq += s0 * s0 + s1 * s1;
        } else {
            if (eo.out) eo.out[i] = scale * s0;
            if (eo.birth) eo.birth[i] = b0;
            if (eo.loss) eo.loss[i] = l0;
            sq += s0 * s0;
        }
    }
    if (eo.source && blockIdx.x == 0 && threadIdx.x == 0) eo.source[0] = src;
    if (eo.sqpart) {
        sq = block_sum(sq, red);
        if (threadIdx.x == 0) eo.sqpart[blockIdx.x] = sq;
    }
}

}  // namespace smol
