// smol_rhs.cuh - device data structures and the kernels of one evaluation of the
// right-hand side S(y) of Eq. (4) (aggregation-shattering, truncated at M; with the
// point sources of Eq. (3)) for a low-rank kernel K = U V (Sec. 1), for one system or a
// ragged batch of systems: the forward column pass, the row kernel (with the scalar
// CTA), the inverse column pass, and the fused inverse + forward column kernel.
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
// the birth term are applied in the epilogue).
//
// Precision. R is the arithmetic type of everything inside S(y) and of the stage
// vectors k_j = h S(y_j): double for the plain FP64 solver, float for the FP32 form,
// dd (double-float, smol_dd.cuh) for the FP64-accurate form on the FP32 pipes.
// The state n and its update, the error estimate, the step control and the mass
// moment are always FP64 (they are handled in smol_int.cuh); the moment sums are
// accumulated per thread in R and reduced across threads in FP64.
//
// Batching. Every kernel takes a device array of system descriptors and a map from
// blockIdx.x to (system, block of that system); one system is a batch of one.
#pragma once
#include <type_traits>

#include "smol_fft.cuh"

namespace smol {

constexpr int MAXR = 16;        // largest rank R (SMOL_MAX_R)
constexpr int MAXT = 2 * MAXR;  // largest number of distinct transforms
constexpr int MAXV = 10;        // terms of a stage-input linear combination
constexpr int NVEC = 12;        // stage / work vectors per system
constexpr int FPW = MAXT + 8;   // doubles per block of the finish / preparation partials
// Threads of a column CTA: at most 256 by default, up to 512 for a single FP64 or
// double-float system with SMOL_FLAG_WIDE_COLS (one thread per element pair of a
// column tile).
constexpr int COL_THREADS_MAX = 512;
// Launch bounds of the column kernels: the FP32 instances keep to 256 threads (a bound
// of 512 caps registers at 128 and changes their allocation: one register more than 80
// leaves the batch two CTAs per SM instead of three); the FP64 and double-float ones
// allow 512 threads (128 registers a thread).
template <typename R>
struct ColBounds {
    static constexpr int threads = COL_THREADS_MAX;
};
template <>
struct ColBounds<float> {
    static constexpr int threads = 256;
};
constexpr int MAXSRC = 8;       // point sources P_k of Eq. (3) per system
constexpr int TILT_T = 4;       // FP32 form: input tilt for systems of at most this many transforms

// Device-resident control block of one system's integration (and of standalone
// evaluations).
struct Ctl {
    double t, tau, h, t1, tol;  // time, proposed step, step of the current attempt, end, tolerance
    double err_last;            // error estimate of the last attempt
    double nrm2;                // ||n||_2^2 of the current state
    double ymax;                // max_i |n_i| of the current state (FP32 input scaling)
    double steady;              // ||S(n)||_2^2 of the last attempt's first stage (unscaled)
    double mass;                // sum_s s n_s of the current state
    double itol2;               // 1 / tol^2 (0 for constant steps without a tolerance)
    double hf;                  // when reuse: h / (the step work vector 0 is scaled with)
    int32_t done, status, cur, clamped;
    int64_t attempts, accepted, rejected, rhs_evals, rhs_paper;
    double* state[2];           // double-buffered state; state[cur] is n^k
    uint32_t arrive;            // arrival counter of the last-block-done reductions
    int32_t reuse;              // the last attempt was rejected: work vector 0 holds
                                // (h / hf) S(n^k) of the current state, and the next
                                // attempt rescales it instead of evaluating S(n^k) again
    int32_t xe[MAXT];           // FP32 form: input scale exponents of the transforms
    int32_t tilt;               // FP32 form: exponential tilt 2^(tilt i / Mp) of the inputs
    int32_t pad_;
    float tlog[TILT_T];         // FP32 form: log2 max_i |W_t[i] n_i| of the current state, t < TILT_T
};

// One system, as the kernels see it (device memory; 256-byte aligned array).
struct SysDev {
    int M, Mp, lgMp, N1, N2, lgN1, lgN2, G, T, R, npairs, nbx;  // nbx = N2 / G column CTAs
    double lambda;
    const void* W;   // R-typed T x Mp weights (zero beyond M)
    const void* tw;  // cx<R> twiddles W_{2Mp}^e, e < Mp
    const void* twc; // cx<R> four-step twiddles W_Mp^{n2 k1} as [n2][k1] (column kernels)
    const void* twr; // cx<R> their conjugates as [k1][n2] (row kernel, inverse)
    const void* tws; // cx<R> spectral twiddles W_{2Mp}^{k1 + N1 k2} as [k1][k2] (row kernel)
    void* Y;         // cx<R> T x Mp spectra after the column pass, [t][k1][n2]
    void* G2;        // cx<R> Mp values after the row pass, [k1][n2]
    void* ybuf;      // R-typed stage input y of the current evaluation (Mp)
    void* vec;       // R-typed work vectors, vec + j * vstride (Mp each)
    double* half;    // FP64 half-step state of step doubling (Mp)
    double* mpart;   // moment partials [t][bx][2]
    double* fpart;   // partials of the finish / preparation kernels [block][FPW]
    double* sqpart;  // ||S||^2 partials [bx]
    double* aux;     // MAXT + 1 doubles: collision-rate coefficients of the preparation
    double* rsc;     // RHS scalars of the current evaluation: death coefficients delta_t
                     // [0, MAXT), monomer source [MAXT], S_1 [MAXT + 1]; then delta_t
                     // rounded to FP32 (MAXT floats, rsc_f)
    void* shadow0;   // FP32 form: R-typed copies of the two state buffers (stage inputs)
    void* shadow1;
    double* log_t;   // step log ring (log_cap entries each, shared capacity)
    double* log_h;
    double* log_e;
    int32_t* log_a;
    Ctl* ctl;
    int64_t vstride;
    int nfin;        // blocks of the finish / lincomb / preparation kernels
    int au[MAXR], av[MAXR];  // ordered pairs (u(alpha), v(alpha))
    double acoef[MAXR];
    int pu[MAXR], pv[MAXR];  // unordered pairs for the spectral product
    double pcoef[MAXR];
    int wexp[MAXT];          // ilogb(max_i |W_t[i]|)
    double bnorm;            // 1 / (2 Mp): the 1/Mp of the inverse and the 1/2 of the birth term
    int nsrc;                // point sources of Eq. (3): S_s += P_s at 0-based sizes src_i
    int src_i[MAXSRC];
    double src_v[MAXSRC];
    int pad[3];
};

// Stage input y = sum_j c_j v_j. slot >= 0: work vector (type R); slot -1 / -2: the
// current / other state buffer; -3: the caller's vector `ext` (single system); -4: the
// half-step state. Slots < 0 are FP64 vectors.
enum { SLOT_CUR = -1, SLOT_OTHER = -2, SLOT_EXT = -3, SLOT_HALF = -4, SLOT_CURF = -5 };
// SLOT_CURF: the current state's R-typed shadow (FP32 form), read by stage inputs of
// the right-hand side; resolves to the FP64 state where no shadow exists or where the
// FP64 value is needed.
struct StageIn {
    int nv, direct;  // direct: y is the single FP64 term itself (c == 1)
    int first;       // the attempt's evaluation of S(n^k), reused on a retry (Ctl::reuse)
    int slot[MAXV];
    double c[MAXV];
    float cf[MAXV];  // c rounded to FP32 and the remainder c - cf rounded to FP32 (set on
    float cl[MAXV];  // the host; the FP32 and double-float forms' stage inputs)
    const double* ext;
};

// Epilogue outputs of an evaluation.
struct EpiOut {
    int out_slot;     // >= 0: k written to work vector out_slot (type R), scaled by h * hfac
    double* out;      // or (out_slot < 0): S(y) written as FP64 to this caller vector
    double* birth;    // optional term outputs (FP64, caller vectors)
    double* loss;
    double* source;
    int sq;           // write ||S(y)||^2 partials (steady test)
    double hfac;
};

// The fields of a system's control block that every kernel reads, fetched once per CTA
// into shared memory.
struct CtlView {
    int done, cur;
    int reuse;  // Ctl::reuse
    double hf;  // Ctl::hf: the rescaling of a reused k_1
    const double* s0;
    const double* s1;
    double h, ymax;
    int tilt;  // Ctl::tilt
    float tlog[TILT_T];
    int xe[MAXT];
};

// Resolved term pointers of a stage input: bit j of dmask set = term j is FP64.
template <typename R>
struct Terms {
    const void* p[MAXV];
    unsigned dmask;
};

template <typename R>
__device__ __forceinline__ Terms<R> resolve_terms(const StageIn& in, const SysDev& S, const CtlView& cv,
                                                  bool shadow_ok = true) {
    Terms<R> tr;
    const int cur = cv.cur;
    const double* s0 = cv.s0;
    const double* s1 = cv.s1;
    tr.dmask = 0u;
#pragma unroll
    for (int j = 0; j < MAXV; ++j) {
        int sl = in.slot[j];
        if (sl == SLOT_CURF) {
            if (shadow_ok && S.shadow0) {
                tr.p[j] = cur ? S.shadow1 : S.shadow0;
                continue;
            }
            sl = SLOT_CUR;
        }
        if (sl >= 0) {
            tr.p[j] = reinterpret_cast<const R*>(S.vec) + (int64_t)sl * S.vstride;
        } else {
            tr.dmask |= 1u << j;
            if (sl == SLOT_CUR) tr.p[j] = cur ? s1 : s0;
            else if (sl == SLOT_OTHER) tr.p[j] = cur ? s0 : s1;
            else if (sl == SLOT_EXT) tr.p[j] = in.ext;
            else tr.p[j] = S.half;
        }
    }
    return tr;
}

template <typename R>
struct vec2 {};
template <>
struct vec2<double> {
    typedef double2 T;
};
template <>
struct vec2<float> {
    typedef float2 T;
};
template <>
struct vec2<dd> {
    typedef dd2 T;
};

// What the right-hand side's arithmetic type R implies: inputs scaled per transform
// (FP32 exponent range), an R-typed shadow of the FP64 state for stage inputs, the
// FP64 form's folded spectral constants.
template <typename R>
struct Tr {
    static constexpr bool scaled = true, shadowed = true, fp64 = false, tilted = false;
};
template <>
struct Tr<float> {
    static constexpr bool scaled = true, shadowed = true, fp64 = false, tilted = true;
};
template <>
struct Tr<double> {
    static constexpr bool scaled = false, shadowed = false, fp64 = true, tilted = false;
};
// Column transforms pruned to the zero padding (HALF_IN) and to the sizes up to M
// (HALF_OUT): FP64 and FP32; not double-float, whose kernels are bound by instruction
// fetch, where the extra pass variants cost more than the work they save.
template <typename R>
constexpr bool PRUNE = !std::is_same<R, dd>::value;

// Loads of one R value and of the R pair at 2 * pair, 2 * pair + 1: read-only path
// (ldg) or coherent L2 path (ldcg).
template <typename R>
__device__ __forceinline__ typename vec2<R>::T ld2g(const R* p, int pair) {
    return __ldg(reinterpret_cast<const typename vec2<R>::T*>(p) + pair);
}
template <>
__device__ __forceinline__ dd2 ld2g<dd>(const dd* p, int pair) {
    return as_dd2(__ldg(reinterpret_cast<const float4*>(p) + pair));
}
template <typename R>
__device__ __forceinline__ typename vec2<R>::T ld2cg(const R* p, int pair) {
    return __ldcg(reinterpret_cast<const typename vec2<R>::T*>(p) + pair);
}
template <>
__device__ __forceinline__ dd2 ld2cg<dd>(const dd* p, int pair) {
    return as_dd2(__ldcg(reinterpret_cast<const float4*>(p) + pair));
}
template <typename R>
__device__ __forceinline__ R ld1cg(const R* p) {
    return __ldcg(p);
}
template <>
__device__ __forceinline__ dd ld1cg<dd>(const dd* p) {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return dd(v.x, v.y);
}
template <typename R>
__device__ __forceinline__ R ld1g(const R* p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ dd ld1g<dd>(const dd* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dd(v.x, v.y);
}

// Stage-input coefficient c_j in type A (from the host's FP32 split for the FP32 and
// double-float forms, so that no FP64 conversion runs per element).
template <typename A>
__device__ __forceinline__ A coef(const StageIn& in, int j) {
    return (A)in.c[j];
}
template <>
__device__ __forceinline__ float coef<float>(const StageIn& in, int j) {
    return in.cf[j];
}
template <>
__device__ __forceinline__ dd coef<dd>(const StageIn& in, int j) {
    return dd(in.cf[j], in.cl[j]);
}

// Stage input at indices i, i+1 (i even), accumulated in type A: zero at and beyond M.
// All term loads are issued before the first multiply-add so that their latencies
// overlap. The loads go to L2 (coherent): a fused kernel reads stage vectors that it
// wrote itself.
template <typename A, typename R>
__device__ __forceinline__ void stage_pair(const StageIn& in, const Terms<R>& P, int M, int i, A& y0, A& y1) {
    y0 = (A)0;
    y1 = (A)0;
    if (i + 1 < M) {
        A v0[MAXV], v1[MAXV];
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) {
                if ((P.dmask >> j) & 1u) {
                    const double2 v = __ldcg(reinterpret_cast<const double2*>(P.p[j]) + (i >> 1));
                    v0[j] = (A)v.x;
                    v1[j] = (A)v.y;
                } else {
                    const typename vec2<R>::T v = ld2cg<R>(reinterpret_cast<const R*>(P.p[j]), i >> 1);
                    v0[j] = (A)v.x;
                    v1[j] = (A)v.y;
                }
            }
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) {
                const A c = coef<A>(in, j);
                y0 += c * v0[j];
                y1 += c * v1[j];
            }
    } else if (i < M) {
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) {
                const A v = ((P.dmask >> j) & 1u) ? (A)__ldcg(reinterpret_cast<const double*>(P.p[j]) + i)
                                                  : (A)ld1cg<R>(reinterpret_cast<const R*>(P.p[j]) + i);
                y0 += coef<A>(in, j) * v;
            }
    }
}

// Transforms whose weights a column CTA loads ahead of the wait for the previous
// kernel (all of them for T <= WPRE), and a register-array lookup by a runtime index.
constexpr int WPRE = 4;
template <typename V>
__device__ __forceinline__ V pick(const V (&v)[WPRE], int t) {
    return t == 0 ? v[0] : (t == 1 ? v[1] : (t == 2 ? v[2] : v[3]));
}

// Exponent of the input scaling of transform t: FP64 runs unscaled; FP32 divides
// x_t by 2^(ilogb(max|W_t|) + ilogb(max|y|)) so that its largest entry is near 1.
template <typename R>
__device__ __forceinline__ int xexp(const SysDev& S, const CtlView& cv, int t) {
    return Tr<R>::scaled ? cv.xe[t] : 0;
}

// Sets the input scale exponents of the FP32 form from max|n| (once per accepted
// step, by one thread): 2^(ilogb(max|W_t|) + ilogb(max|n|)).
__device__ __forceinline__ void set_xe(Ctl* c, const SysDev& S, double ymax) {
    const int ey = (ymax > 0.0 && isfinite(ymax)) ? ilogb(ymax) : 0;
    for (int t = 0; t < S.T; ++t) c->xe[t] = S.wexp[t] + ey;
}

// An integer 0 <= k < 2^23 as a float without a conversion instruction (conversions
// issue on a slower pipe than the FP32 arithmetic of these kernels): the bits of
// 2^23 + k, minus 2^23, both exact.
__device__ __forceinline__ float exact_float(int k) { return __int_as_float(0x4B000000 | k) - 8388608.0f; }
template <typename R>
__device__ __forceinline__ R index_r(int k) {
    return (R)k;
}
template <>
__device__ __forceinline__ float index_r<float>(int k) {
    return exact_float(k);
}
template <>
__device__ __forceinline__ dd index_r<dd>(int k) {
    return dd(exact_float(k));
}

// Exponential tilt of the FP32 form (exponential tilting of a convolution: if x'_i =
// x_i theta^i and y'_j = y_j theta^j then (x' * y')_m = theta^m (x * y)_m). A transform
// rounds every output to about eps ||x'|| ||y'||; after the output is multiplied back by
// theta^-m that floor falls off as theta^-m, so the tail of the size distribution, where
// the true birth terms are tiny but the shattering source weights them by powers of the
// size, no longer carries the FP32 rounding of the whole transform. theta = 2^(p / Mp)
// with an integer p in [0, TILT_PMAX], chosen from the state so that |n_i| theta^i <=
// max |n| (the inputs keep their largest entry at the head, and their norm).
constexpr int TILT_PMAX = 48;
// 2^(p i / Mp) and 2^(-p i / Mp) in FP32: p i is an exact integer (p <= TILT_PMAX,
// i < 2^25), its fraction over Mp goes through exp2f, the integer part is a power of two.
__device__ __forceinline__ float pow2f_int(int e) {
    e = max(-126, min(127, e));
    return __int_as_float((127 + e) << 23);
}
__device__ __forceinline__ float tilt_up(int p, int i, int lgMp) {
    const int E = p * i;
    return exp2f(exact_float(E & ((1 << lgMp) - 1)) * pow2f_int(-lgMp)) * pow2f_int(E >> lgMp);
}
__device__ __forceinline__ float tilt_down(int p, int i, int lgMp) {
    const int E = p * i;
    return exp2f(-exact_float(E & ((1 << lgMp) - 1)) * pow2f_int(-lgMp)) * pow2f_int(-(E >> lgMp));
}
// The tilt must keep every transform's input below its own largest entry: with
// x_t[i] = W_t[i] n_i, b = min_t min_i (log2 max_j |x_t[j]| - log2 |x_t[i]|) / i over the
// nonzero entries i >= 1 (+inf when there are none), and p = floor(b Mp), clamped. The
// bound of an accepted state sets the tilt of the next attempt's evaluations (all of
// them: an evaluation's forward and inverse passes must use the same tilt). Systems
// with more than TILT_T transforms are not tilted.
__device__ __forceinline__ int tilt_from_bound(double b, int Mp, int T) {
    if (T > TILT_T || !(b > 0.0)) return 0;
    const double p = floor(b * (double)Mp);
    return p >= (double)TILT_PMAX ? TILT_PMAX : (int)p;
}
// One input entry's contribution to that bound (ltop: log2 of its transform's max).
__device__ __forceinline__ float tilt_bound_el(float ltop, float v, int i) {
    const float a = fabsf(v);
    if (i < 1 || !(a > 0.f) || !isfinite(a)) return INFINITY;
    return __fdividef(ltop - __log2f(a), exact_float(i));  // floored to p / Mp: approximate is enough
}
// The reference log2 of a transform input's maximum, stored in tlog, with one bit of
// slack: the bound is taken against the previous state's maxima (or maxima computed in
// another rounding), and an entry at or just above such a maximum would otherwise
// give a negative bound and no tilt at all. The tilted inputs may then reach twice the
// maximum, which leaves the rounding floor of the transform unchanged to a factor 2.
__device__ __forceinline__ float tilt_log(float mx) { return mx > 0.f && isfinite(mx) ? __log2f(mx) + 1.0f : 0.f; }

// 2^e as R, exactly, without a double-precision ldexp (e within the normal range).
template <typename R>
__device__ __forceinline__ R pow2(int e) {
    e = max(-1022, min(1023, e));
    return (R)__longlong_as_double((long long)(1023 + e) << 52);
}
template <>
__device__ __forceinline__ float pow2<float>(int e) {
    e = max(-126, min(127, e));
    return __int_as_float((127 + e) << 23);
}
template <>
__device__ __forceinline__ dd pow2<dd>(int e) {
    return dd(pow2<float>(e));
}

// Last-CTA-done pattern: every CTA of a system writes its partials, then one atomic
// per CTA; the CTA that arrives last sees all partials and returns true (all threads).
__device__ __forceinline__ bool arrive_last(Ctl* ctl, int nblk, bool* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->arrive, 1u);
        *flag = (prev == (unsigned)nblk - 1);
    }
    __syncthreads();
    if (*flag) __threadfence();
    return *flag;
}

// GPU-scope acquire-release atomic add (PTX memory model): releases the writes ordered
// before it (those of the whole CTA, through the preceding block barrier) and acquires
// those released by earlier arrivals, in one operation.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// arrive_last with the arrival as one acquire-release atomic and no fences: for callers
// that read the other CTAs' partials through L2 only (ld.cg), which the acquire orders.
__device__ __forceinline__ bool arrive_last_ar(Ctl* ctl, int nblk, bool* flag) {
    __syncthreads();
    if (threadIdx.x == 0) *flag = atom_add_acq_rel(&ctl->arrive, 1u) == (unsigned)nblk - 1;
    __syncthreads();
    return *flag;
}

// FP32 copies of delta_t behind the FP64 scalars: [0, MAXT) rounded, [MAXT, 2 MAXT) the
// remainders (the double-float form's low parts).
__device__ __forceinline__ float* rsc_f(const SysDev& S) { return reinterpret_cast<float*>(S.rsc + MAXT + 2); }
template <typename R>
__device__ __forceinline__ R delta_r(const SysDev& S, int t) {
    return (R)__ldcg(S.rsc + t);
}
template <>
__device__ __forceinline__ float delta_r<float>(const SysDev& S, int t) {
    return __ldcg(rsc_f(S) + t);
}
template <>
__device__ __forceinline__ dd delta_r<dd>(const SysDev& S, int t) {
    return dd(__ldcg(rsc_f(S) + t), __ldcg(rsc_f(S) + MAXT + t));
}

// Scalars of one evaluation (the scalar CTA of the row kernel): y_1 in FP64, the
// moments mu_t, nu_t summed over the column CTAs' partials in a fixed order, then
//   delta_t = sum_{alpha: u=t} coef_alpha mu_{v(alpha)}   (death: D_s = sum_t delta_t W_t[s])
//   source  = lambda/2 sum coef (rho_u sigma_v + sigma_u rho_v) + lambda y_1 sum coef W_u[1] rho_v
//   S_1     = -y_1 D_1 + source  (FP64: its two terms nearly cancel)
// with sigma_t = mu_t - W_t[1] y_1, rho_t = nu_t - W_t[1] y_1. All loads (partials and
// the stage-input terms at s = 1) are issued together; sh: >= 4 MAXT + 1 doubles of
// shared memory, sh[3 MAXT + t] = W_t[1] staged by the caller before its wait.
template <typename R>
__device__ void finalize_scalars(const SysDev& S, const CtlView& cv, const StageIn& in, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double* mom = sh;                  // [2 MAXT]
    double* w1s = sh + 3 * MAXT;       // [MAXT]
    double* y1p = sh + 4 * MAXT;       // [1]
    // y_1 in FP64 (from the FP64 state, not an FP32 shadow): lane j of warp 0 loads term j
    if (warp == 0) {
        const Terms<R> P = resolve_terms<R>(in, S, cv, false);
        double v = 0.0;
        if (lane < in.nv)
            v = ((P.dmask >> lane) & 1u) ? __ldcg(reinterpret_cast<const double*>(P.p[lane]))
                                         : (double)ld1cg<R>(reinterpret_cast<const R*>(P.p[lane]));
        double y1 = 0.0;
        for (int j = 0; j < in.nv; ++j) y1 += in.c[j] * __shfl_sync(0xffffffffu, v, j);
        if (lane == 0) *y1p = y1;
    }
    for (int q = warp; q < 2 * S.T; q += nw) {
        const int t = q >> 1, which = q & 1;
        double v = 0.0;
        for (int c = lane; c < S.nbx; c += 32) v += __ldcg(S.mpart + 2 * ((size_t)t * S.nbx + c) + which);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) mom[q] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double y1 = *y1p;
    double shat = 0.0, mono = 0.0;
    for (int al = 0; al < S.R; ++al) {
        const int u = S.au[al], v = S.av[al];
        const double c = S.acoef[al];
        const double su = mom[2 * u] - w1s[u] * y1, ru = mom[2 * u + 1] - w1s[u] * y1;
        const double sv = mom[2 * v] - w1s[v] * y1, rv = mom[2 * v + 1] - w1s[v] * y1;
        shat += c * (ru * sv + su * rv);
        mono += c * w1s[u] * rv;
    }
    double D1 = 0.0;
    for (int t = 0; t < S.T; ++t) {
        double del = 0.0;
        for (int al = 0; al < S.R; ++al)
            if (S.au[al] == t) del += S.acoef[al] * mom[2 * S.av[al]];
        S.rsc[t] = del;
        const float dh = (float)del;
        rsc_f(S)[t] = dh;
        rsc_f(S)[MAXT + t] = (float)(del - (double)dh);
        D1 += del * w1s[t];
    }
    const double src = 0.5 * S.lambda * shat + S.lambda * y1 * mono;
    double p1 = 0.0;  // a point source at s = 1 (Eq. (3))
    for (int q = 0; q < S.nsrc; ++q)
        if (S.src_i[q] == 0) p1 += S.src_v[q];
    S.rsc[MAXT] = src;
    S.rsc[MAXT + 1] = -y1 * D1 + src + p1;
}

// Programmatic dependent launch. The kernels of an evaluation sequence are launched
// with programmatic stream serialisation, so that a kernel's CTAs may be scheduled
// while its predecessor in the stream is still running. griddep_wait() returns once
// every predecessor grid has completed and its writes are visible (at once for a
// kernel launched without the attribute); griddep_release() then lets the next kernel
// of the stream start its own prologue. Before griddep_wait() a kernel reads only what
// no kernel of the sequence writes (descriptors, block maps, weights, twiddle tables)
// and writes only its own shared memory.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Copies the descriptor of this CTA's system into shared memory and returns the block
// index within the system. A launch over a single system passes map == nullptr and the
// descriptor itself as a kernel argument (no global round trip); a batch passes the
// device array and the block map. Ends with a barrier.
__device__ __forceinline__ int load_desc(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                         const SysDev& one, SysDev& sh) {
    int blk;
    const int* src;
    if (map == nullptr) {
        blk = blockIdx.x;
        src = reinterpret_cast<const int*>(&one);
    } else {
        const int2 m = map[blockIdx.x];
        blk = m.y;
        src = reinterpret_cast<const int*>(sysv + m.x);
    }
    int* dst = reinterpret_cast<int*>(&sh);
    for (int q = threadIdx.x; q < (int)(sizeof(SysDev) / 4); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
    return blk;
}

// Waits for the predecessor kernels (griddep_wait), releases the next one, and fetches
// the fields of the system's control block that every kernel reads. Ends with a barrier.
// The control block is read through L2 (ld.cg): in the persistent attempt kernel
// another CTA's controller wrote it earlier in the same kernel.
__device__ __forceinline__ void load_ctl_fields(const SysDev& sh, CtlView& cv) {
    const Ctl* c = sh.ctl;
    if (threadIdx.x < MAXT) cv.xe[threadIdx.x] = __ldcg(c->xe + threadIdx.x);
    if (threadIdx.x == 0) {
        cv.done = __ldcg(&c->done);
        cv.cur = __ldcg(&c->cur);
        cv.s0 = reinterpret_cast<const double*>(__ldcg(reinterpret_cast<const long long*>(&c->state[0])));
        cv.s1 = reinterpret_cast<const double*>(__ldcg(reinterpret_cast<const long long*>(&c->state[1])));
        cv.h = __ldcg(&c->h);
        cv.ymax = __ldcg(&c->ymax);
        cv.reuse = __ldcg(&c->reuse);
        cv.hf = __ldcg(&c->hf);
        cv.tilt = __ldcg(&c->tilt);
    }
    if (threadIdx.x < TILT_T) cv.tlog[threadIdx.x] = __ldcg(c->tlog + threadIdx.x);
    __syncthreads();
}
__device__ __forceinline__ void load_ctl(const SysDev& sh, CtlView& cv) {
    griddep_wait();
    griddep_release();
    load_ctl_fields(sh, cv);
}

// A retry after a rejected attempt starts from the same state n^k (Sec. 2: the step
// is repeated from n^k with a smaller tau), so its first evaluation S(n^k) is the one
// the rejected attempt made: the forward and row kernels of that evaluation return at
// once, and its inverse pass rescales the stored k_1 = h' S(n^k) to the new step h.
__device__ __forceinline__ bool reused(const StageIn& in, const CtlView& cv) { return in.first && cv.reuse; }

// Both steps, for kernels with no prologue of their own.
__device__ __forceinline__ int load_sys(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                        const SysDev& one, SysDev& sh, CtlView& cv) {
    const int blk = load_desc(sysv, map, one, sh);
    load_ctl(sh, cv);
    return blk;
}

// ---------------------------------------------------------------------------
// Column CTAs. One CTA per G adjacent columns n2 of one system; the forward pass
// (stage input, moments, column transforms of length N1) and the inverse pass (inverse
// column transforms and the right-hand-side epilogue) touch the same elements
// i = 2 (n1 N2 + n2), n1 < N1 / 2, with the same thread per element pair, so the
// inverse pass of one stage and the forward pass of the next can run in one kernel.
// Shared memory (forward layout; the inverse pass uses the first N1 G entries of a and
// b): a, b (N1 G T complex each), the tile twiddles W_N1^e (N1), the four-step
// twiddles W_Mp^{n2 k1} of the CTA's columns (N1 G), y (N1 G reals).
// ---------------------------------------------------------------------------
template <typename R>
struct ColSm {
    cx<R>* a;
    cx<R>* b;
    cx<R>* twP;
    cx<R>* tw4;
    R* ys;
};
template <typename R>
__device__ __forceinline__ ColSm<R> col_sm(const SysDev& S, unsigned char* raw) {
    ColSm<R> m;
    const int n = S.N1 * S.G * S.T;
    m.a = reinterpret_cast<cx<R>*>(raw);
    m.b = m.a + n;
    m.twP = m.b + n;
    m.tw4 = m.twP + S.N1;
    m.ys = reinterpret_cast<R*>(m.tw4 + S.N1 * S.G);
    return m;
}

// Element index of pair idx of column CTA bx.
__device__ __forceinline__ int col_elem(const SysDev& S, const Div& DG, int bx, int idx) {
    int g, n1;
    divmod(DG, idx, n1, g);
    return 2 * ((n1 << S.lgN2) + bx * S.G + g);
}

// Forward prologue (constant data, before the wait for the previous kernel): the
// four-step twiddles of the CTA's columns (asynchronous copies) and the weights of
// the thread's first element pair for the first WPRE transforms.
template <typename R>
__device__ __forceinline__ void fwd_prologue(const SysDev& S, int bx, const ColSm<R>& m,
                                             typename vec2<R>::T (&wpre)[WPRE]) {
    const int G = S.G, N1 = S.N1;
    const cx<R>* twc = reinterpret_cast<const cx<R>*>(S.twc);
    for (int idx = threadIdx.x; idx < N1 * G; idx += blockDim.x) {
        const int k1 = idx & (N1 - 1), g = idx >> S.lgN1;  // contiguous reads along k1
        cp_async_el(m.tw4 + k1 * G + g, twc + (size_t)(bx * G + g) * N1 + k1);
    }
    const R* Wall = reinterpret_cast<const R*>(S.W);
    if ((int)threadIdx.x < (N1 >> 1) * G) {
        const int i = col_elem(S, mkdiv(G), bx, threadIdx.x);
#pragma unroll
        for (int t = 0; t < WPRE; ++t)
            if (t < S.T) wpre[t] = ld2g<R>(Wall + (size_t)t * S.Mp, i >> 1);
    }
}

// Forward pass after the wait: stage input y (computed once per element), moments, and
// the column transforms of all T inputs x_t = W_t . y, interleaved in one tile
// transform over T G sequences. fix_tw: the tile twiddles still need stage_tw_fix.
// red: 2 MAXT x 8 doubles of shared memory.
template <typename R>
__device__ __forceinline__ void fwd_body(const SysDev& S, const CtlView& cv, const StageIn& in, int bx,
                                         const ColSm<R>& m, const typename vec2<R>::T (&wpre)[WPRE], bool fix_tw,
                                         double (*red)[8]) {
    const int G = S.G, T = S.T, GT = G * T, N1 = S.N1;
    const int half = (N1 >> 1) * G;
    const int n2b = bx * G;
    cx<R>* a = m.a;
    cx<R>* b = m.b;
    R* ys = m.ys;
    const Div DG = mkdiv(G);
    const R* Wall = reinterpret_cast<const R*>(S.W);
    const Terms<R> P = resolve_terms<R>(in, S, cv);
    R* yb = reinterpret_cast<R*>(S.ybuf);
    for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
        const int i = col_elem(S, DG, bx, idx);
        R y0, y1;
        stage_pair<R, R>(in, P, S.M, i, y0, y1);
        ys[2 * idx] = y0;
        ys[2 * idx + 1] = y1;
        if (!in.direct) *reinterpret_cast<typename vec2<R>::T*>(yb + i) = {y0, y1};
    }
    // rows n1 >= N1 / 2 of the columns are the zero padding: the FP64 and FP32 transforms
    // do not read them (HALF_IN); the double-float one takes them as zeros (its variant
    // with the pruned first pass costs more in instruction fetch than it saves)
    if (!PRUNE<R>)
        for (int q = half * T + threadIdx.x; q < N1 * GT; q += blockDim.x) a[q] = mk<R>((R)0, (R)0);
    cp_async_wait();
    if (fix_tw) stage_tw_fix(m.twP, S.lgN1, S.lgMp);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    // FP64 form: the per-thread moments go through shared memory (the second tile
    // buffer, unused until the transform) and each is summed by one warp, which takes
    // far fewer FP64 instructions than a shuffle tree in every warp; the FP32 form sums
    // in FP32 shuffles and then in FP64 across warps.
    const bool viasm = Tr<R>::fp64 && N1 * G >= (int)blockDim.x;
    // the per-warp partials of the shuffle path: red for up to 8 warps, else the second
    // tile buffer (a CTA of more than 256 threads has N1 G >= 1024 points there)
    const bool wbuf = ColBounds<R>::threads > 256 && !viasm && nw > 8;
    double* rb = reinterpret_cast<double*>(b);
    for (int t = 0; t < T; ++t) {
        const R sc = pow2<R>(-xexp<R>(S, cv, t));
        const R* Wt = Wall + (size_t)t * S.Mp;
        R mu = (R)0, nu = (R)0;
        for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
            int g, n1;
            divmod(DG, idx, n1, g);
            const int i = 2 * ((n1 << S.lgN2) + n2b + g);
            const typename vec2<R>::T w = (idx == (int)threadIdx.x && t < WPRE) ? pick(wpre, t) : ld2g<R>(Wt, i >> 1);
            const R x0 = w.x * ys[2 * idx], x1 = w.y * ys[2 * idx + 1];
            mu += x0 + x1;
            nu += index_r<R>(i + 1) * x0 + index_r<R>(i + 2) * x1;
            if constexpr (Tr<R>::tilted) {
                if (cv.tilt) {  // the transform's input is tilted; the moments are not
                    a[n1 * GT + t * G + g] =
                        mk<R>(x0 * (sc * tilt_up(cv.tilt, i, S.lgMp)), x1 * (sc * tilt_up(cv.tilt, i + 1, S.lgMp)));
                    continue;
                }
            }
            a[n1 * GT + t * G + g] = mk<R>(x0 * sc, x1 * sc);
        }
        if (viasm) {
            rb[(2 * t) * blockDim.x + threadIdx.x] = (double)mu;
            rb[(2 * t + 1) * blockDim.x + threadIdx.x] = (double)nu;
            continue;
        }
        for (int o = 16; o > 0; o >>= 1) {
            mu += shfl_down(mu, o);
            nu += shfl_down(nu, o);
        }
        if (lane == 0) {
            double* rp = wbuf ? rb + 64 * t : red[2 * t];
            const int st = wbuf ? 32 : 8;
            rp[warp] = (double)mu;
            rp[st + warp] = (double)nu;
        }
    }
    __syncthreads();
    if (viasm) {
        for (int q = warp; q < 2 * T; q += nw) {
            double v = 0.0;
            for (int k = lane; k < (int)blockDim.x; k += 32) v += rb[q * blockDim.x + k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) S.mpart[2 * ((size_t)(q >> 1) * S.nbx + bx) + (q & 1)] = v;
        }
        __syncthreads();  // the transform overwrites the second tile buffer
    } else {
        if (threadIdx.x < 2 * T) {
            const double* rp = wbuf ? rb + 32 * threadIdx.x : red[threadIdx.x];
            double v = 0.0;
            for (int w = 0; w < nw; ++w) v += rp[w];
            const int t = threadIdx.x >> 1;
            S.mpart[2 * ((size_t)t * S.nbx + bx) + (threadIdx.x & 1)] = v;
        }
        if (wbuf) __syncthreads();  // the transform overwrites the second tile buffer
    }
    cx<R>* res = tile_fft<R, PRUNE<R> ? HALF_IN : HALF_NONE>(a, b, S.lgN1, GT, m.twP, false);
    cx<R>* Yall = reinterpret_cast<cx<R>*>(S.Y);
    const Div DGT = mkdiv(GT);
    for (int idx = threadIdx.x; idx < N1 * GT; idx += blockDim.x) {
        int c, k1, t, g;
        divmod(DGT, idx, k1, c);
        divmod(DG, c, t, g);
        Yall[(size_t)t * S.Mp + (size_t)k1 * S.N2 + n2b + g] = res[idx] * m.tw4[k1 * G + g];
    }
}

// Kernel A: the forward pass of one evaluation.
template <typename R>
__global__ void __launch_bounds__(ColBounds<R>::threads) k_fwd_cols(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                  const __grid_constant__ SysDev one, const StageIn in) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ double red[2 * MAXT][8];
    extern __shared__ __align__(16) unsigned char smraw[];
    const int bx = load_desc(sysv, map, one, S);
    const ColSm<R> m = col_sm<R>(S, smraw);
    // twiddle tables and weights first (constant): their loads overlap the wait
    stage_tw(m.twP, S.lgN1, reinterpret_cast<const cx<R>*>(S.tw), S.lgMp);
    typename vec2<R>::T wpre[WPRE];
    fwd_prologue<R>(S, bx, m, wpre);
    load_ctl(S, cv);
    if (cv.done || reused(in, cv)) {
        cp_async_wait();  // no copy into this CTA's shared memory outlives it
        return;
    }
    fwd_body<R>(S, cv, in, bx, m, wpre, true, red);
}

// ---------------------------------------------------------------------------
// Kernel B: row transforms of length N2 for a pair of rows (k1, N1 - k1), the
// real-FFT split, the product sum over kernel terms, the packed inverse spectrum,
// inverse row transforms and the inverse twiddle. CTA 0 of a system is its scalar CTA;
// CTA b + 1 owns rows (b, N1 - b), CTA 1 rows (0, N1 / 2).
// ---------------------------------------------------------------------------
// Whether a pair coefficient must be applied (the FP64 form skips an exact 1).
__device__ __forceinline__ bool pc_not_one(double c) { return c != 1.0; }
template <typename R>
__device__ __forceinline__ bool pc_not_one(R) { return true; }

// FP64 form (FOLD): the factors 1/2 of E, O and of the packed inverse and the first
// pair's coefficient are taken out of the per-frequency arithmetic (it then forms 2 X,
// sums pc[p] / pc[0] (2X_u)(2X_v) and returns 2 Y / pc[0] * 4) and applied once in the
// birth scale of the inverse column kernel (fold_scale); the FP64 pipe is what bounds
// this kernel. The FP32 form keeps them in place, where they keep the values in range.
template <typename R>
__device__ __forceinline__ void spectral_pair(const SysDev& S, const cx<R>* Z, int G, int ia, int ib, cx<R> w,
                                              const R* pc, cx<R>& Ya, cx<R>& Yb) {
    // Z holds the row spectra as Z[k2 * G + col], col = 2 t + rho; ia / ib are the
    // offsets k2 * G + rho of the pair's two frequencies ka and Mp - ka; w = W_L^ka.
    constexpr bool FOLD = Tr<R>::fp64;
    cx<R> Ca, Cb;
    for (int p = 0; p < S.npairs; ++p) {
        const int u = S.pu[p], v = S.pv[p];
        cx<R> Xa[2], Xb[2];
        const int tt[2] = {u, v};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const cx<R> za = Z[ia + 2 * tt[q]];
            const cx<R> zb = conj(Z[ib + 2 * tt[q]]);
            cx<R> E = za + zb, O = mul_mi(za - zb);
            if (!FOLD) {
                E = scl(E, (R)0.5);
                O = scl(O, (R)0.5);
            }
            const cx<R> wO = w * O;
            Xa[q] = E + wO;
            Xb[q] = conj(E - wO);
        }
        cx<R> pa = Xa[0] * Xa[1], pb = Xb[0] * Xb[1];
        if (!FOLD || pc_not_one(pc[p])) {
            pa = scl(pa, pc[p]);
            pb = scl(pb, pc[p]);
        }
        Ca = p ? Ca + pa : pa;  // npairs >= 1
        Cb = p ? Cb + pb : pb;
    }
    // Packed inverse spectrum at ka and Mp - ka:
    //   Ya = w (Ca - conj Cb) + i (Ca + conj Cb),
    //   Yb = wb (Cb - conj Ca) + i (Cb + conj Ca) with wb = W_L^(Mp - ka) = -conj w.
    // With D = Ca - conj Cb, G = Ca + conj Cb and P = w D: Cb - conj Ca = -conj D and
    // Cb + conj Ca = conj G, so Yb = conj P + i conj G; one complex product serves both.
    const cx<R> D = Ca - conj(Cb), Gs = Ca + conj(Cb);
    const cx<R> P = w * D;
    Ya = mk<R>(P.x - Gs.y, P.y + Gs.x);
    Yb = mk<R>(P.x + Gs.y, Gs.x - P.y);
    if (!FOLD) {
        Ya = scl(Ya, (R)0.5);
        Yb = scl(Yb, (R)0.5);
    }
}

// First pair coefficient taken out of the FP64 spectral product (1 if it is zero).
__device__ __forceinline__ double fold_coef(const SysDev& S) { return S.pcoef[0] != 0.0 ? S.pcoef[0] : 1.0; }

// Shared memory of a row unit: a, b (N2 x 2T complex each), the tile twiddles W_N2^e,
// the spectral twiddles of the two rows and their inverse four-step twiddles.
template <typename R>
struct RowSm {
    cx<R>* a;
    cx<R>* b;
    cx<R>* twP;  // W_N2^e
    cx<R>* tws;  // W_L^{r + N1 k2} of the two rows, [rho][k2]
    cx<R>* twi;  // conj W_Mp^{n2 r} of the two rows, [rho][n2]
};
template <typename R>
__device__ __forceinline__ RowSm<R> row_sm(const SysDev& S, unsigned char* raw) {
    RowSm<R> m;
    const int n = S.N2 * 2 * S.T;
    m.a = reinterpret_cast<cx<R>*>(raw);
    m.b = m.a + n;
    m.twP = m.b + n;
    m.tws = m.twP + S.N2;
    m.twi = m.tws + 2 * S.N2;
    return m;
}
// The rows (r0, r1) of row unit blk: (blk, N1 - blk), and (0, N1 / 2) for blk = 0.
__device__ __forceinline__ void row_pair_of(const SysDev& S, int blk, int& r0, int& r1) {
    r0 = blk ? blk : 0;
    r1 = blk ? S.N1 - blk : (S.N1 >> 1);
}
// Row prologue (constant data, before the wait for the previous kernel): the twiddles.
template <typename R>
__device__ __forceinline__ void row_prologue(const SysDev& S, int blk, const RowSm<R>& m) {
    const int N2 = S.N2;
    int r0, r1;
    row_pair_of(S, blk, r0, r1);
    stage_tw(m.twP, S.lgN2, reinterpret_cast<const cx<R>*>(S.tw), S.lgMp);
    for (int idx = threadIdx.x; idx < 2 * N2; idx += blockDim.x) {
        const int rho = idx >> S.lgN2, k2 = idx & (N2 - 1);
        const uint32_t r = (uint32_t)(rho ? r1 : r0);
        cp_async_el(m.tws + idx, reinterpret_cast<const cx<R>*>(S.tws) + (size_t)r * N2 + k2);
        cp_async_el(m.twi + idx, reinterpret_cast<const cx<R>*>(S.twr) + (size_t)r * N2 + k2);
    }
}
// Row unit after the wait: gather of the 2T rows, row FFTs, real-FFT split, product sum,
// packed inverse spectrum, inverse row FFTs and the inverse four-step twiddle. pc: MAXR
// values of shared memory. CG: gather through L2 (persistent kernel).
template <typename R, bool CG = false>
__device__ __forceinline__ void row_body(const SysDev& S, const CtlView& cv, int blk, const RowSm<R>& m, R* pc) {
    const int G = 2 * S.T;
    const int N2 = S.N2;
    cx<R>* a = m.a;
    cx<R>* b = m.b;
    cx<R>* twP = m.twP;
    const cx<R>* tws = m.tws;
    const cx<R>* twi = m.twi;
    int r0, r1;
    row_pair_of(S, blk, r0, r1);
    if (threadIdx.x < S.npairs) {
        // FP32: pair p carries 2^(e_u + e_v - e_max) so that the sum stays in range.
        // FP64: pc[0] is folded into the birth scale (spectral_pair).
        R c = (R)S.pcoef[threadIdx.x];
        if (Tr<R>::fp64) c = (R)(S.pcoef[threadIdx.x] / fold_coef(S));
        if (Tr<R>::scaled) {
            int emax = -100000;
            for (int p = 0; p < S.npairs; ++p) emax = max(emax, xexp<R>(S, cv, S.pu[p]) + xexp<R>(S, cv, S.pv[p]));
            c = c * pow2<R>(xexp<R>(S, cv, S.pu[threadIdx.x]) + xexp<R>(S, cv, S.pv[threadIdx.x]) - emax);
        }
        pc[threadIdx.x] = c;
    }
    const cx<R>* Yin = reinterpret_cast<const cx<R>*>(S.Y);
    for (int idx = threadIdx.x; idx < N2 * G; idx += blockDim.x) {
        const int k2 = idx & (N2 - 1);  // consecutive threads read consecutive k2 (coalesced)
        const int col = idx >> S.lgN2;
        const int t = col >> 1, rho = col & 1;
        const int r = rho ? r1 : r0;
        gather_el<CG>(a + k2 * G + col, Yin + (size_t)t * S.Mp + (size_t)r * N2 + k2);
    }
    cp_async_wait();
    stage_tw_fix(twP, S.lgN2, S.lgMp);
    __syncthreads();
    cx<R>* Z = tile_fft<R>(a, b, S.lgN2, G, twP, false);
    cx<R>* Yo = (Z == a) ? b : a;  // packed inverse spectrum, [k2 * 2 + rho]
    const int ntask = blk ? N2 : N2 + 1;
    for (int task = threadIdx.x; task < ntask; task += blockDim.x) {
        int k2a, rhoa, k2b, rhob;
        if (blk) {
            k2a = task;
            rhoa = 0;
            k2b = N2 - 1 - task;
            rhob = 1;
        } else if (task <= (N2 >> 1)) {
            k2a = task;
            rhoa = 0;
            k2b = (N2 - task) & (N2 - 1);
            rhob = 0;
        } else {
            k2a = task - (N2 >> 1) - 1;
            rhoa = 1;
            k2b = N2 - 1 - k2a;
            rhob = 1;
        }
        cx<R> Ya, Yb;
        spectral_pair<R>(S, Z, G, k2a * G + rhoa, k2b * G + rhob, tws[rhoa * N2 + k2a], pc, Ya, Yb);
        Yo[k2a * 2 + rhoa] = Ya;
        if (k2a != k2b || rhoa != rhob) Yo[k2b * 2 + rhob] = Yb;
    }
    __syncthreads();
    cx<R>* res = tile_fft<R>(Yo, Z, S.lgN2, 2, twP, true);
    cx<R>* G2 = reinterpret_cast<cx<R>*>(S.G2);
    for (int idx = threadIdx.x; idx < 2 * N2; idx += blockDim.x) {
        const int n2 = idx & (N2 - 1);
        const int rho = idx >> S.lgN2;
        const int r = rho ? r1 : r0;
        G2[(size_t)r * N2 + n2] = res[n2 * 2 + rho] * twi[idx];
    }
}

// The scalar unit's prologue: W_t[1] of every transform into sh[3 MAXT + t].
template <typename R>
__device__ __forceinline__ void scalar_prologue(const SysDev& S, double* sh) {
    if ((int)threadIdx.x < S.T) sh[3 * MAXT + threadIdx.x] = (double)reinterpret_cast<const R*>(S.W)[(size_t)threadIdx.x * S.Mp];
}

template <typename R>
__global__ void __launch_bounds__(256) k_rows(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                              const __grid_constant__ SysDev one, const StageIn in) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ R pc[MAXR];
    extern __shared__ __align__(16) unsigned char smraw[];
    const int cta = load_desc(sysv, map, one, S);
    if (cta == 0) {
        // The scalar CTA of the system, beside the row CTAs: the evaluation's scalars,
        // which only the inverse column kernel reads (y_1 from the FP64 state, not its
        // FP32 shadow: the two large terms of the monomer equation nearly cancel).
        double* sh = reinterpret_cast<double*>(smraw);
        scalar_prologue<R>(S, sh);
        load_ctl(S, cv);
        if (cv.done || reused(in, cv)) return;
        finalize_scalars<R>(S, cv, in, sh);
        return;
    }
    const int blk = cta - 1;  // row pair
    const RowSm<R> m = row_sm<R>(S, smraw);
    row_prologue<R>(S, blk, m);
    load_ctl(S, cv);
    if (cv.done || reused(in, cv)) {
        cp_async_wait();  // no copy into this CTA's shared memory outlives it
        return;
    }
    row_body<R>(S, cv, blk, m, pc);
}

// Epilogue inputs of the element pair (i, i + 1): the collision rates D_s = sum_t
// delta_t W_t[s] (delta_t from the evaluation's scalars) and the stage input y_s.
template <typename R>
__device__ __forceinline__ void epi_inputs(const SysDev& S, const R* Wr, const R* yr, const double* yd, int i, R& D0,
                                           R& D1, R& y0, R& y1) {
    D0 = (R)0;
    D1 = (R)0;
    for (int t = 0; t < S.T; ++t) {
        const R d = delta_r<R>(S, t);
        const typename vec2<R>::T w = ld2g<R>(Wr + (size_t)t * S.Mp, i >> 1);
        D0 += d * w.x;
        D1 += d * w.y;
    }
    if (yd) {
        y0 = (R)yd[i];
        y1 = (i + 1 < S.M) ? (R)yd[i + 1] : (R)0;
    } else {
        const typename vec2<R>::T yy = *reinterpret_cast<const typename vec2<R>::T*>(yr + i);
        y0 = yy.x;
        y1 = yy.y;
    }
}

// Inverse pass after the wait: inverse column transforms of length N1 (only the first
// half of the outputs is needed), then the epilogue: birth, death, shattering, monomer
// source, the scaled output k = h S(y) (or S(y) to a caller vector). The tile twiddles
// were issued by stage_tw and are fixed here. sm: the CTA's shared scalars.
template <typename R>
struct InvSm {
    double red[33];
    double src_s, bscale_s, s1_s;
    R rs[5];  // scale, birth scale, 1 + lambda, S_1, loss_1 in type R
};

template <typename R, bool CG = false>
__device__ __forceinline__ void inv_body(const SysDev& S, const CtlView& cv, const StageIn& in, const EpiOut& eo,
                                         int bx, const ColSm<R>& m, InvSm<R>& sm) {
    const int G = S.G;
    cx<R>* a = m.a;
    cx<R>* b = a + (S.N1 * G);
    double* red = sm.red;
    double& src_s = sm.src_s;
    double& bscale_s = sm.bscale_s;
    double& s1_s = sm.s1_s;
    R* rs = sm.rs;
    const int n2b = bx * G;
    const cx<R>* G2 = reinterpret_cast<const cx<R>*>(S.G2);
    const Div DG = mkdiv(G);
    for (int idx = threadIdx.x; idx < S.N1 * G; idx += blockDim.x) {
        int g, k1;
        divmod(DG, idx, k1, g);
        gather_el<CG>(a + idx, G2 + (size_t)k1 * S.N2 + n2b + g);
    }
    const R* yr = reinterpret_cast<const R*>(S.ybuf);
    const double* yd = in.direct ? reinterpret_cast<const double*>(resolve_terms<R>(in, S, cv).p[0]) : nullptr;
    const R* Wr = reinterpret_cast<const R*>(S.W);
    const int half = (S.N1 >> 1) * G;
    // The epilogue inputs of this thread's first element pair (idx = threadIdx.x) are
    // loaded before the transform, so that their latency overlaps it.
    R pD0 = (R)0, pD1 = (R)0, py0 = (R)0, py1 = (R)0;
    if (threadIdx.x < half) {
        const int i = col_elem(S, DG, bx, threadIdx.x);
        if (i < S.M) epi_inputs<R>(S, Wr, yr, yd, i, pD0, pD1, py0, py1);
    }
    if (threadIdx.x == 0) {
        src_s = __ldcg(S.rsc + MAXT);
        s1_s = __ldcg(S.rsc + MAXT + 1);
        int emax = 0;
        if (Tr<R>::scaled) {
            emax = -100000;
            for (int p = 0; p < S.npairs; ++p) emax = max(emax, xexp<R>(S, cv, S.pu[p]) + xexp<R>(S, cv, S.pv[p]));
        }
        bscale_s = S.bnorm * (double)pow2<float>(emax);
        // FP64: the factors the spectral product left out, (1/2)^3 pc[0]
        if (Tr<R>::fp64) bscale_s *= 0.125 * fold_coef(S);
        // the epilogue's scalars, converted once per CTA
        rs[0] = (R)(eo.out_slot >= 0 ? cv.h * eo.hfac : 1.0);
        rs[1] = (R)bscale_s;
        rs[2] = (R)(1.0 + S.lambda);
        rs[3] = (R)s1_s;
        rs[4] = (R)(-(s1_s - src_s));
    }
    cp_async_wait();
    stage_tw_fix(m.twP, S.lgN1, S.lgMp);
    __syncthreads();
    // only rows n1 < N1 / 2 (sizes up to M) are needed: the pruned transform writes no others
    cx<R>* res = tile_fft<R, PRUNE<R> ? HALF_OUT : HALF_NONE>(a, b, S.lgN1, G, m.twP, true);
    const R scale = rs[0], bscale = rs[1], lam1 = rs[2], s1r = rs[3], l1r = rs[4];
    const int tilt = cv.tilt;
    const double src = src_s;
    R* kout = eo.out_slot >= 0 ? reinterpret_cast<R*>(S.vec) + (int64_t)eo.out_slot * S.vstride : nullptr;
    double sq = 0.0;
    for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
        const int i = col_elem(S, DG, bx, idx);
        if (i >= S.M) continue;
        const cx<R> z = res[idx];
        R D0 = pD0, D1 = pD1, y0 = py0, y1 = py1;
        if (idx != (int)threadIdx.x) epi_inputs<R>(S, Wr, yr, yd, i, D0, D1, y0, y1);
        R b0 = (i == 0) ? (R)0 : z.x * bscale;
        R b1 = z.y * bscale;
        if constexpr (Tr<R>::tilted) {
            // birth at index i is c[i - 1], tilted by theta^(i - 1)
            if (tilt) {
                if (i > 0) b0 *= tilt_down(tilt, i - 1, S.lgMp);
                b1 *= tilt_down(tilt, i, S.lgMp);
            }
        }
        const R l0 = (i == 0) ? l1r : lam1 * y0 * D0;
        const R l1 = lam1 * y1 * D1;
        R s0 = b0 - l0;
        R s1 = b1 - l1;
        if (i == 0) s0 = s1r;
        for (int q = 0; q < S.nsrc; ++q) {  // point sources of Eq. (3) (s = 1 is in S_1)
            const int si = S.src_i[q];
            if (si == i && i != 0) s0 += (R)S.src_v[q];
            if (si == i + 1) s1 += (R)S.src_v[q];
        }
        const bool two = i + 1 < S.M;
        if (kout) {
            if (two) *reinterpret_cast<typename vec2<R>::T*>(kout + i) = {scale * s0, scale * s1};
            else kout[i] = scale * s0;
        }
        if (eo.out) {
            if (two) *reinterpret_cast<double2*>(eo.out + i) = make_double2((double)s0, (double)s1);
            else eo.out[i] = (double)s0;
        }
        if (eo.birth) {
            eo.birth[i] = (double)b0;
            if (two) eo.birth[i + 1] = (double)b1;
        }
        if (eo.loss) {
            eo.loss[i] = (double)l0;
            if (two) eo.loss[i + 1] = (double)l1;
        }
        if (eo.sq) sq += (double)(s0 * s0 + (two ? s1 * s1 : (R)0));
    }
    if (eo.source && bx == 0 && threadIdx.x == 0) eo.source[0] = src;
    if (eo.sq) {
        sq = block_sum(sq, red);
        if (threadIdx.x == 0) S.sqpart[bx] = sq;
    }
}

// The inverse pass of a reused first evaluation: k_1 <- (h / h') k_1 at the CTA's
// elements (the same thread per element pair as inv_body and fwd_body).
template <typename R>
__device__ __forceinline__ void rescale_k1(const SysDev& S, const CtlView& cv, const EpiOut& eo, int bx) {
    if (eo.out_slot < 0) return;
    R* k = reinterpret_cast<R*>(S.vec) + (int64_t)eo.out_slot * S.vstride;
    const R f = (R)cv.hf;
    const Div DG = mkdiv(S.G);
    const int half = (S.N1 >> 1) * S.G;
    for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
        const int i = col_elem(S, DG, bx, idx);
        if (i >= S.M) continue;
        k[i] = f * k[i];
        if (i + 1 < S.M) k[i + 1] = f * k[i + 1];
    }
}

// ---------------------------------------------------------------------------
// Kernel C: the inverse pass of one evaluation.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(ColBounds<R>::threads) k_inv_cols(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                  const __grid_constant__ SysDev one, const StageIn in,
                                                  const EpiOut eo) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ InvSm<R> sm;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int bx = load_desc(sysv, map, one, S);
    const ColSm<R> m = col_sm<R>(S, smraw);
    stage_tw(m.twP, S.lgN1, reinterpret_cast<const cx<R>*>(S.tw), S.lgMp);
    load_ctl(S, cv);
    if (cv.done || reused(in, cv)) {
        cp_async_wait();  // no copy into this CTA's shared memory outlives it
        if (!cv.done) rescale_k1<R>(S, cv, eo, bx);
        return;
    }
    inv_body<R>(S, cv, in, eo, bx, m, sm);
}

// ---------------------------------------------------------------------------
// Kernel C+A: the inverse pass of one evaluation (stage input `in`, output eo) and the
// forward pass of the next (stage input nx) in one kernel: the column CTA that forms
// k of this stage at its elements goes on to form the next stage input there.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(ColBounds<R>::threads) k_inv_fwd(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                 const __grid_constant__ SysDev one, const StageIn in,
                                                 const EpiOut eo, const StageIn nx) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ InvSm<R> sm;
    __shared__ double red[2 * MAXT][8];
    extern __shared__ __align__(16) unsigned char smraw[];
    const int bx = load_desc(sysv, map, one, S);
    const ColSm<R> m = col_sm<R>(S, smraw);
    stage_tw(m.twP, S.lgN1, reinterpret_cast<const cx<R>*>(S.tw), S.lgMp);
    typename vec2<R>::T wpre[WPRE];
    fwd_prologue<R>(S, bx, m, wpre);
    load_ctl(S, cv);
    if (cv.done) {
        cp_async_wait();  // no copy into this CTA's shared memory outlives it
        return;
    }
    if (reused(in, cv)) {
        cp_async_wait();
        stage_tw_fix(m.twP, S.lgN1, S.lgMp);  // as inv_body does
        rescale_k1<R>(S, cv, eo, bx);
    } else {
        inv_body<R>(S, cv, in, eo, bx, m, sm);
    }
    __syncthreads();  // the forward pass reuses the tile buffers
    fwd_body<R>(S, cv, nx, bx, m, wpre, false, red);
}

}  // namespace smol
