// smol_int.cuh - device side of the adaptive integrators of Sec. 2: the RK stage
// combination, the embedded / step-doubling error norm and the step-size controller,
// all kept on the device (per system) so that no host synchronisation happens per
// step. The state, its update, the error estimate, the controller and the mass moment
// sum_s s n_s are FP64 whatever the precision of the right-hand side.
#pragma once
#include <type_traits>

#include "smol_rhs.cuh"

namespace smol {

enum { SCHEME_RK2 = 0, SCHEME_RK4 = 1, SCHEME_RKF45 = 2 };
enum { CTRL_DOUBLE_HALVE = 0, CTRL_FORMULA = 1 };
enum { ST_OK = 0, ST_STEADY = 1, ST_ENONFINITE = -3, ST_EUNDERFLOW = -4, ST_EMAXATT = -5 };

// Controller settings of one integration (passed by value; the same for every system).
struct CtlParams {
    int scheme, ctrl, rel_norm, fixed, order;
    int evals, evals_paper;  // S evaluations per attempt: actual and stages x steps
    double tau_min_rel, steady_rtol, fac_min, fac_max;
    int64_t max_attempts;
    int log_cap;
    int steady;              // the first stage wrote ||S(n)||^2 partials
};

// Square root and n-th roots for the controller, in FP64 accuracy without the
// double-precision library routines (whose long dependent chains are slow on this
// part's narrow FP64 path): an FP32 estimate refined by Newton steps in FP64.
//   r = 1/sqrt(x):  r <- r (3 - x r^2) / 2          (Newton on r^-2 - x = 0)
//   z = x^(-1/n):   z <- z (1 + (1 - x z^n) / n)   (Newton on z^-n - x = 0)
// Each step doubles the number of correct bits: two steps take the FP32 estimate
// (~1e-7) to below 1e-16.
__device__ __forceinline__ double rsqrt_d(double x) {
    double r = (double)rsqrtf((float)x);
    r = r * (1.5 - 0.5 * x * r * r);
    r = r * (1.5 - 0.5 * x * r * r);
    return r;
}
__device__ __forceinline__ double sqrt_d(double x) {
    if (!(x > 0.0)) return x == 0.0 ? 0.0 : sqrt(x);  // zero, negative or NaN: exact path
    if (x < 1e-30 || x > 1e30 || !isfinite(x)) return sqrt(x);
    return x * rsqrt_d(x);
}
// Step factor of Sec. 2 from a = (err / tol)^2: s (tol / err)^(1/p) = s a^(-1/q), q = 2p,
// clamped to [fac_min, fac_max]. y = a^(-1/q) from an FP32 estimate refined by one
// Newton step in FP64 on y^-q - a = 0, y <- y (1 + (1 - a y^q) / q), which takes the
// ~1e-7 estimate below 1e-13; a is first clamped to [1e-36, 1e36] (the factor sits at
// a clamp bound well inside that range). err = 0 gives fac_max.
__device__ __forceinline__ double step_factor(const CtlParams& P, double a, double s, int q) {
    if (!(a > 0.0)) return P.fac_max;
    a = fmin(fmax(a, 1e-36), 1e36);
    double y = (double)exp2f(-log2f((float)a) / (float)q);
    const double y2 = y * y, y4 = y2 * y2, y8 = y4 * y4;
    const double yq = q == 10 ? y8 * y2 : (q == 8 ? y8 : (q == 4 ? y4 : y2));
    y = y * (1.0 + (1.0 - a * yq) * (1.0 / (double)q));
    return fmin(fmax(s * y, P.fac_min), P.fac_max);
}

// Step-size rules of Sec. 2 from a = (err / tol)^2. Returns the proposed step; *acc the
// decision (err <= tol, i.e. a <= 1).
__device__ __forceinline__ double propose(const CtlParams& P, double h, double tau, double a, int* acc) {
    if (P.fixed) {
        *acc = 1;
        return tau;
    }
    *acc = a <= 1.0;
    if (P.scheme == SCHEME_RKF45) return h * step_factor(P, a, 0.9, 10);      // 0.9 tau (tol/err)^(1/5)
    if (P.ctrl == CTRL_FORMULA) return h * step_factor(P, a, 0.25, 2 * P.order);  // Eq. (6)
    // halve on reject, double on accept
    return *acc ? 2.0 * h : 0.5 * h;
}

// The steady stop: ||S(n)|| / ||n|| < rtol, i.e. Q < rtol^2 nrm2 (both non-negative).
__device__ __forceinline__ bool steady_stop(const CtlParams& P, double nrm2, double Q) {
    return P.steady && nrm2 > 0.0 && Q < P.steady_rtol * P.steady_rtol * nrm2;
}

__device__ __forceinline__ void set_next_step(Ctl* c) {
    c->clamped = c->tau >= c->t1 - c->t;
    c->h = c->clamped ? c->t1 - c->t : c->tau;
}

// Double-float (FP32 pair) accumulation of sum c_j k_j over FP32 stage vectors, used by
// the FP32 form so that its increments and error vectors keep ~2^-44 relative accuracy
// without the narrow FP64 path. Built on the error-free transformations of Dekker
// (1971) and Knuth (TAOCP vol. 2): the exact product of two floats as p + e with a fused
// multiply-add, and the exact sum of two floats as s + t. Coefficients are split on the
// host into c = ch + cl (both floats).
struct DF {
    float hi, lo;
};
__device__ __forceinline__ void df_fma(DF& acc, float ch, float cl, float k) {
    const float p = ch * k;
    const float e = fmaf(ch, k, -p) + cl * k;  // ch*k - p exactly, plus the low part
    const float s = acc.hi + p;
    const float bb = s - acc.hi;
    const float t = (acc.hi - (s - bb)) + (p - bb);  // acc.hi + p - s exactly
    acc.hi = s;
    acc.lo += t + e;
}
__device__ __forceinline__ double df_value(const DF& a) { return (double)a.hi + (double)a.lo; }

// Half-step state of step doubling (FP64): half = sum c_j v_j over [0, M).
template <typename R>
__global__ void __launch_bounds__(128) k_lincomb(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                 const __grid_constant__ SysDev one, const StageIn in) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    const int blk = load_sys(sysv, map, one, S, cv);
    if (cv.done) return;
    const int np = (S.M + 1) >> 1;
    const Terms<R> tr = resolve_terms<R>(in, S, cv, false);
    for (int p = blk * blockDim.x + threadIdx.x; p < np; p += S.nfin * blockDim.x) {
        double y0, y1;
        stage_pair<double, R>(in, tr, S.M, 2 * p, y0, y1);
        if (2 * p + 1 < S.M) *reinterpret_cast<double2*>(S.half + 2 * p) = make_double2(y0, y1);
        else S.half[2 * p] = y0;
    }
}

// Controller of one system after an attempt (one thread, on a shared-memory copy c of
// the control block). E = ||error||^2, C = ||candidate||^2, X = max|candidate|, bad:
// the candidate is not finite, MS = sum_s s candidate_s, Q = ||S(n)||^2. The accept
// decision and the step factor use a = E / tol^2 (divided by nrm2 for the relative
// norm) and need no square root; err itself (stats and log) is formed by another
// thread at the same time (error_norm).
__device__ __forceinline__ void controller(const CtlParams& P, const SysDev& S, Ctl& cref, double E, double C,
                                           double X, bool bad, double MS, double Q, double TB, const float* TMX) {
    Ctl* c = &cref;
    c->arrive = 0;
    if (!c->reuse) c->rhs_evals += 1;  // S(n^k) of the first stage (reused on a retry)
    if (P.steady) {
        c->steady = Q;
        if (steady_stop(P, c->nrm2, Q)) {
            c->status = ST_STEADY;
            c->done = 1;
            return;
        }
    }
    c->rhs_evals += P.evals - 1;
    c->rhs_paper += P.evals_paper;
    c->attempts += 1;
    double a = (P.fixed && P.scheme != SCHEME_RKF45) ? 0.0 : E * c->itol2;
    if (P.rel_norm && c->nrm2 > 0.0) a /= c->nrm2;
    if (bad || !(E <= 1.7e308)) {
        c->status = ST_ENONFINITE;
        c->done = 1;
        return;
    }
    int acc;
    const double h = c->h;
    const double tau_new = propose(P, h, c->tau, a, &acc);
    if (P.log_cap > 0) {
        const int64_t slot = (c->attempts - 1) % P.log_cap;
        S.log_t[slot] = c->t;
        S.log_h[slot] = h;
        S.log_a[slot] = acc;
    }
    if (acc) {
        c->cur ^= 1;
        c->t = c->clamped ? c->t1 : c->t + h;
        c->accepted += 1;
        c->nrm2 = C;
        c->ymax = X;
        c->mass = MS;
        set_xe(c, S, X);
        c->tilt = tilt_from_bound(TB, S.Mp, S.T);  // FP32 form (the other forms ignore it)
        for (int t = 0; t < TILT_T; ++t) c->tlog[t] = tilt_log(TMX[t]);
        if (!c->clamped) c->tau = tau_new;
        c->reuse = 0;
    } else {
        c->rejected += 1;
        c->tau = tau_new;
        c->reuse = 1;  // the retry starts from the same n^k: work vector 0 holds h S(n^k)
    }
    if (c->t < c->t1 && c->tau < P.tau_min_rel * fmax(1.0, fabs(c->t))) {
        c->status = ST_EUNDERFLOW;
        c->done = 1;
    } else if (c->t >= c->t1) {
        c->done = 1;
    } else if (c->attempts >= P.max_attempts) {
        c->status = ST_EMAXATT;
        c->done = 1;
    }
    if (!c->done) {
        set_next_step(c);
        if (c->reuse) c->hf = c->h / h;  // rescales the kept k_1 = h S(n^k) to the new step
    }
}

// err of an attempt for the stats and the step log (beside the controller, on another
// warp): sqrt(E), over ||n|| for the relative norm. nrm2_0 and att0 are ||n||^2 and
// the attempt count read before the controller runs; of c only err_last is written.
__device__ __forceinline__ void error_norm(const CtlParams& P, const SysDev& S, Ctl& c, double nrm2_0, int64_t att0,
                                           double E, bool bad, double Q) {
    if (steady_stop(P, nrm2_0, Q)) return;
    double err = (P.fixed && P.scheme != SCHEME_RKF45) ? 0.0 : sqrt_d(E);
    if (P.rel_norm) {
        const double nn = sqrt_d(nrm2_0);
        if (nn > 0.0) err /= nn;
    }
    c.err_last = err;
    if (bad || !(E <= 1.7e308)) return;
    if (P.log_cap > 0) S.log_e[att0 % P.log_cap] = err;
}

// |x| as the bit pattern of a double (an unsigned integer order that agrees with the
// order of the non-negative doubles; NaN and infinity patterns are >= INF_BITS).
constexpr unsigned long long INF_BITS = 0x7ff0000000000000ull;
__device__ __forceinline__ unsigned long long absbits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Candidate and error combinations of the final kernel over one set of terms: each
// term is loaded once; cand = sum c_j v_j and err = sum d_j v_j.
struct Comb2 {
    StageIn in;  // slots and candidate coefficients c_j
    double d[MAXV];
    float ch[MAXV], cl[MAXV], dh[MAXV], dl[MAXV];  // c and d split into float pairs
};

// Per-thread accumulators of the final combination: ||error||^2, ||candidate||^2 and
// sum_s s candidate_s (FP64), max |candidate| as the bit pattern of a non-negative
// double (integer max is monotone on those, and a NaN or infinity pattern is at least
// INF_BITS, which marks a non-finite candidate); the FP32 form keeps its per-thread
// norms, max and finite test in FP32.
struct FinAcc {
    double se, sc, ms;
    unsigned long long mxb;
    float fse, fsc, fmx;
    float tb;              // FP32 form: the candidate's tilt bound (against the current state's
    float tmx[TILT_T];     // input maxima) and its own input maxima max_i |W_t[i] n_i|
    bool fbad;
};
__device__ __forceinline__ FinAcc fin_acc() {
    FinAcc a;
    a.se = a.sc = a.ms = 0.0;
    a.mxb = 0ull;
    a.fse = a.fsc = a.fmx = 0.f;
    a.tb = INFINITY;
#pragma unroll
    for (int t = 0; t < TILT_T; ++t) a.tmx[t] = 0.f;
    a.fbad = false;
    return a;
}

// Final combination at the element pair (i, i + 1) (i even): candidate = sum c_j v_j
// (FP64) written to the other state buffer (and, FP32 form, its FP32 shadow), error
// vector sum d_j v_j reduced into the accumulators. Terms are read from L2 (a fused
// kernel reads the stage vector it has just written).
template <typename R>
__device__ __forceinline__ void fin_pair(const SysDev& S, const Comb2& cd, const Terms<R>& tp, double* outp,
                                         void* shadv, int i, FinAcc& a, const float* tlog) {
    const StageIn& in = cd.in;
    const int p = i >> 1;
    const bool two = i + 1 < S.M;
    if constexpr (std::is_same<R, float>::value) {
        float* shad = reinterpret_cast<float*>(shadv);
        // FP32 form: the FP32 stage terms are combined in double-float arithmetic, the FP64
        // terms (state, half-step state) in FP64; FP64 is used only for those terms, the
        // candidate's final sum and the mass moment. Norms, max and the finite test work
        // on the FP32 image of the candidate, which also becomes the next state's shadow.
        DF c0 = {0.f, 0.f}, c1 = {0.f, 0.f}, d0 = {0.f, 0.f}, d1 = {0.f, 0.f};
        double b0 = 0.0, b1 = 0.0, e0 = 0.0, e1 = 0.0;
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) {
                if ((tp.dmask >> j) & 1u) {
                    const double* v = reinterpret_cast<const double*>(tp.p[j]);
                    const double v0 = __ldcg(v + i), v1 = two ? __ldcg(v + i + 1) : 0.0;
                    b0 += in.c[j] * v0;
                    b1 += in.c[j] * v1;
                    if (cd.d[j] != 0.0) {
                        e0 += cd.d[j] * v0;
                        e1 += cd.d[j] * v1;
                    }
                } else {
                    const float* v = reinterpret_cast<const float*>(tp.p[j]);
                    float v0, v1;
                    if (two) {
                        const float2 w = __ldcg(reinterpret_cast<const float2*>(v) + p);
                        v0 = w.x;
                        v1 = w.y;
                    } else {
                        v0 = __ldcg(v + i);
                        v1 = 0.f;
                    }
                    df_fma(c0, cd.ch[j], cd.cl[j], v0);
                    df_fma(c1, cd.ch[j], cd.cl[j], v1);
                    df_fma(d0, cd.dh[j], cd.dl[j], v0);
                    df_fma(d1, cd.dh[j], cd.dl[j], v1);
                }
            }
        const double y0 = b0 + df_value(c0), y1 = b1 + df_value(c1);
        // error: the FP64 part only where FP64 terms enter it (step doubling)
        float q0, q1;
        if (e0 != 0.0 || e1 != 0.0) {
            q0 = (float)(e0 + df_value(d0));
            q1 = (float)(e1 + df_value(d1));
        } else {
            q0 = d0.hi + d0.lo;
            q1 = d1.hi + d1.lo;
        }
        a.fse += q0 * q0 + q1 * q1;
        const float f0 = (float)y0, f1 = (float)y1;
        if (two) {
            *reinterpret_cast<double2*>(outp + i) = make_double2(y0, y1);
            *reinterpret_cast<float2*>(shad + i) = make_float2(f0, f1);
            a.ms += (double)(i + 1) * y0 + (double)(i + 2) * y1;
        } else {
            outp[i] = y0;
            shad[i] = f0;
            a.ms += (double)(i + 1) * y0;
        }
        a.fsc += f0 * f0 + f1 * f1;
        a.fmx = fmaxf(a.fmx, fmaxf(fabsf(f0), fabsf(f1)));
        a.fbad = a.fbad || !isfinite(f0) || !isfinite(f1);
        if (S.T <= TILT_T) {
            // the next attempt's tilt: the transform inputs W_t n of the candidate
            const float* Wf = reinterpret_cast<const float*>(S.W);
#pragma unroll
            for (int t = 0; t < TILT_T; ++t)
                if (t < S.T) {
                    const float w0 = __ldg(Wf + (size_t)t * S.Mp + i), w1 = two ? __ldg(Wf + (size_t)t * S.Mp + i + 1) : 0.f;
                    const float v0 = w0 * f0, v1 = w1 * f1;
                    a.tmx[t] = fmaxf(a.tmx[t], fmaxf(fabsf(v0), fabsf(v1)));
                    a.tb = fminf(a.tb, fminf(tilt_bound_el(tlog[t], v0, i), tilt_bound_el(tlog[t], v1, i + 1)));
                }
        }
    } else if constexpr (std::is_same<R, dd>::value) {
        // Double-float form: the stage terms (double-float) are combined in double-float
        // arithmetic (high and low parts each through df_fma), the FP64 terms in FP64;
        // the candidate, its error vector, norms and mass in FP64, and the candidate's
        // double-float image becomes the next state's shadow.
        dd* shad = reinterpret_cast<dd*>(shadv);
        DF c0 = {0.f, 0.f}, c1 = {0.f, 0.f}, d0 = {0.f, 0.f}, d1 = {0.f, 0.f};
        double b0 = 0.0, b1 = 0.0, e0 = 0.0, e1 = 0.0;
#pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < in.nv) {
                if ((tp.dmask >> j) & 1u) {
                    const double* v = reinterpret_cast<const double*>(tp.p[j]);
                    const double v0 = __ldcg(v + i), v1 = two ? __ldcg(v + i + 1) : 0.0;
                    b0 += in.c[j] * v0;
                    b1 += in.c[j] * v1;
                    if (cd.d[j] != 0.0) {
                        e0 += cd.d[j] * v0;
                        e1 += cd.d[j] * v1;
                    }
                } else {
                    const dd* v = reinterpret_cast<const dd*>(tp.p[j]);
                    dd v0, v1;
                    if (two) {
                        const dd2 w = ld2cg<dd>(v, p);
                        v0 = w.x;
                        v1 = w.y;
                    } else {
                        v0 = ld1cg<dd>(v + i);
                        v1 = dd(0.f, 0.f);
                    }
                    df_fma(c0, cd.ch[j], cd.cl[j], v0.hi);
                    df_fma(c0, cd.ch[j], cd.cl[j], v0.lo);
                    df_fma(c1, cd.ch[j], cd.cl[j], v1.hi);
                    df_fma(c1, cd.ch[j], cd.cl[j], v1.lo);
                    df_fma(d0, cd.dh[j], cd.dl[j], v0.hi);
                    df_fma(d0, cd.dh[j], cd.dl[j], v0.lo);
                    df_fma(d1, cd.dh[j], cd.dl[j], v1.hi);
                    df_fma(d1, cd.dh[j], cd.dl[j], v1.lo);
                }
            }
        const double y0 = b0 + df_value(c0), y1 = b1 + df_value(c1);
        const double q0 = e0 + df_value(d0), q1 = e1 + df_value(d1);
        if (two) {
            *reinterpret_cast<double2*>(outp + i) = make_double2(y0, y1);
            dd2 sh;
            sh.x = dd(y0);
            sh.y = dd(y1);
            *reinterpret_cast<dd2*>(shad + i) = sh;
        } else {
            outp[i] = y0;
            shad[i] = dd(y0);
        }
        a.se += q0 * q0 + q1 * q1;
        a.sc += y0 * y0 + y1 * y1;
        a.ms += (double)(i + 1) * y0 + (double)(i + 2) * y1;
        a.mxb = max(a.mxb, max(absbits(y0), absbits(y1)));
    } else {
        double y0 = 0.0, y1 = 0.0, d0 = 0.0, d1 = 0.0;
        if (two) {
            double v0[MAXV], v1[MAXV];
#pragma unroll
            for (int j = 0; j < MAXV; ++j)
                if (j < in.nv) {
                    if ((tp.dmask >> j) & 1u) {
                        const double2 v = __ldcg(reinterpret_cast<const double2*>(tp.p[j]) + p);
                        v0[j] = v.x;
                        v1[j] = v.y;
                    } else {
                        const typename vec2<R>::T v = ld2cg<R>(reinterpret_cast<const R*>(tp.p[j]), p);
                        v0[j] = (double)v.x;
                        v1[j] = (double)v.y;
                    }
                }
#pragma unroll
            for (int j = 0; j < MAXV; ++j)
                if (j < in.nv) {
                    y0 += in.c[j] * v0[j];
                    y1 += in.c[j] * v1[j];
                    d0 += cd.d[j] * v0[j];
                    d1 += cd.d[j] * v1[j];
                }
            *reinterpret_cast<double2*>(outp + i) = make_double2(y0, y1);
        } else {
#pragma unroll
            for (int j = 0; j < MAXV; ++j)
                if (j < in.nv) {
                    const double v = ((tp.dmask >> j) & 1u) ? __ldcg(reinterpret_cast<const double*>(tp.p[j]) + i)
                                                            : (double)ld1cg<R>(reinterpret_cast<const R*>(tp.p[j]) + i);
                    y0 += in.c[j] * v;
                    d0 += cd.d[j] * v;
                }
            outp[i] = y0;
        }
        a.se += d0 * d0 + d1 * d1;
        a.sc += y0 * y0 + y1 * y1;
        a.ms += (double)(i + 1) * y0 + (double)(i + 2) * y1;
        a.mxb = max(a.mxb, max(absbits(y0), absbits(y1)));
    }
}

// Shared memory of fin_tail: per-warp partials (up to 32 warps) and the last CTA's
// reduced values.
struct FinSm {
    double wred[3][32];
    unsigned long long xred[32];
    float tred[32];
    float tmred[TILT_T][32];
    double res[5];            // last CTA: E, C, sum s n_s, tilt bound, Q
    unsigned long long resx;  // last CTA: max |candidate| bits
    float restm[TILT_T];      // last CTA: the tilt's input maxima
    bool last;
};

// End of an attempt, after every thread of the CTA has accumulated its elements: the
// CTA's partials are written to slot blk of nblk; the last CTA of the system reduces
// them and runs the controller (thread 0) and the error norm (thread 32) on the shared
// copy cs of the control block, which it then writes back.
//
// The reductions are short: the FP64 pipe of this part takes about 64 cycles per
// dependent operation, so the last CTA gives each quantity its own warp (E, C, the mass
// moment, Q, and the max / min / tilt values), whose lanes stride over the partials and
// then meet in a shuffle tree; every order is fixed. The FP32 form's per-thread norms
// are FP32 sums; from there on they are summed in FP64 (an FP32 warp sum would make the
// error norm depend on the launch shape at 1e-7, enough to move the step sequence).
template <typename R>
__device__ __forceinline__ void fin_tail(const SysDev& S, const CtlParams& P, Ctl* ctl, Ctl& cs, int blk, int nblk,
                                         FinAcc acc, FinSm& f) {
    constexpr int CW = (int)(sizeof(Ctl) / 4);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double se, sc;
    unsigned long long mxb;
    if constexpr (std::is_same<R, float>::value) {
        se = (double)acc.fse;
        sc = (double)acc.fsc;
        mxb = acc.fbad ? INF_BITS : absbits((double)acc.fmx);
    } else {
        se = acc.se;
        sc = acc.sc;
        mxb = acc.mxb;
    }
    for (int o = 16; o > 0; o >>= 1) {
        se += __shfl_down_sync(0xffffffffu, se, o);
        sc += __shfl_down_sync(0xffffffffu, sc, o);
        mxb = max(mxb, __shfl_down_sync(0xffffffffu, mxb, o));
    }
    double ms = acc.ms;
    float tb = acc.tb;
    float tmx[TILT_T];
#pragma unroll
    for (int t = 0; t < TILT_T; ++t) tmx[t] = acc.tmx[t];
    for (int o = 16; o > 0; o >>= 1) {
        ms += __shfl_down_sync(0xffffffffu, ms, o);
        tb = fminf(tb, __shfl_down_sync(0xffffffffu, tb, o));
#pragma unroll
        for (int t = 0; t < TILT_T; ++t) tmx[t] = fmaxf(tmx[t], __shfl_down_sync(0xffffffffu, tmx[t], o));
    }
    if (lane == 0) {
        f.wred[0][warp] = se;
        f.wred[1][warp] = sc;
        f.wred[2][warp] = ms;
        f.xred[warp] = mxb;
        f.tred[warp] = tb;
#pragma unroll
        for (int t = 0; t < TILT_T; ++t) f.tmred[t][warp] = tmx[t];
    }
    __syncthreads();
    if (threadIdx.x >= 5 && threadIdx.x < 5 + TILT_T) {
        const int t = threadIdx.x - 5;
        float x = f.tmred[t][0];
        for (int w = 1; w < nw; ++w) x = fmaxf(x, f.tmred[t][w]);
        S.fpart[FPW * blk + 5 + t] = (double)x;  // slots 5..: input maxima of the tilt
    }
    if (threadIdx.x < 5) {
        const int q = threadIdx.x;
        double v = 0.0;
        if (q == 2) {
            unsigned long long x = f.xred[0];
            for (int w = 1; w < nw; ++w) x = max(x, f.xred[w]);
            v = __longlong_as_double((long long)x);
        } else if (q == 4) {
            float x = f.tred[0];
            for (int w = 1; w < nw; ++w) x = fminf(x, f.tred[w]);
            v = (double)x;
        } else {
            const int r = q < 2 ? q : 2;
            v = f.wred[r][0];
            for (int w = 1; w < nw; ++w) v += f.wred[r][w];
        }
        // slots: E, C, max bits, tilt bound, mass moment
        S.fpart[FPW * blk + (q == 3 ? 4 : (q == 4 ? 3 : q))] = v;
    }
    if (!arrive_last_ar(ctl, nblk, &f.last)) return;
    for (int qi = warp; qi < 5; qi += nw) {
        if (qi == 4 && !P.steady) continue;
        if (qi != 3) {
            // sums: E (slot 0), C (slot 1), mass moment (slot 4); Q over the forward CTAs
            double v = 0.0;
            if (qi == 4) {
                for (int b = lane; b < S.nbx; b += 32) v += __ldcg(S.sqpart + b);
            } else {
                const int slot = qi == 2 ? 4 : qi;
                for (int b = lane; b < nblk; b += 32) v += __ldcg(S.fpart + FPW * b + slot);
            }
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) f.res[qi == 2 ? 2 : (qi == 4 ? 4 : qi)] = v;
        } else {
            // max |candidate| bits (slot 2), tilt bound (slot 3, min), input maxima (5..)
            unsigned long long x = 0ull;
            double b3 = INFINITY;
            float tm[TILT_T];
#pragma unroll
            for (int t = 0; t < TILT_T; ++t) tm[t] = 0.f;
            for (int b = lane; b < nblk; b += 32) {
                const double* q = S.fpart + FPW * b;
                x = max(x, (unsigned long long)__double_as_longlong(__ldcg(q + 2)));
                b3 = fmin(b3, __ldcg(q + 3));
#pragma unroll
                for (int t = 0; t < TILT_T; ++t) tm[t] = fmaxf(tm[t], (float)__ldcg(q + 5 + t));
            }
            for (int o = 16; o > 0; o >>= 1) {
                x = max(x, __shfl_down_sync(0xffffffffu, x, o));
                b3 = fmin(b3, __shfl_down_sync(0xffffffffu, b3, o));
#pragma unroll
                for (int t = 0; t < TILT_T; ++t) tm[t] = fmaxf(tm[t], __shfl_down_sync(0xffffffffu, tm[t], o));
            }
            if (lane == 0) {
                f.resx = x;
                f.res[3] = b3;
#pragma unroll
                for (int t = 0; t < TILT_T; ++t) f.restm[t] = tm[t];
            }
        }
    }
    const double nrm2_0 = cs.nrm2;  // read before the controller may overwrite them
    const int64_t att0 = cs.attempts;
    __syncthreads();
    const int t2 = blockDim.x > 32 ? 32 : 0;
    if (threadIdx.x == 0 || threadIdx.x == t2) {
        const double E = f.res[0], Q = P.steady ? f.res[4] : 0.0;
        const bool bad = f.resx >= INF_BITS;
        if (threadIdx.x == t2) error_norm(P, S, cs, nrm2_0, att0, E, bad, Q);
        if (threadIdx.x == 0)
            controller(P, S, cs, E, f.res[1], __longlong_as_double((long long)f.resx), bad, f.res[2], Q, f.res[3],
                       f.restm);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < CW; q += blockDim.x)
        reinterpret_cast<int*>(ctl)[q] = reinterpret_cast<const int*>(&cs)[q];
}

// Copies the control block into shared memory (no kernel writes it while an attempt's
// final kernel runs): the last CTA runs the controller on that copy, off global memory.
__device__ __forceinline__ void copy_ctl(const Ctl* ctl, Ctl& cs) {
    constexpr int CW = (int)(sizeof(Ctl) / 4);
    for (int q = threadIdx.x; q < CW; q += blockDim.x)
        reinterpret_cast<int*>(&cs)[q] = __ldcg(reinterpret_cast<const int*>(ctl) + q);
}

// Final kernel of an attempt: the combination over all element pairs of each system
// (CTA blk of nfin takes pairs blk * blockDim + tid, + nfin * blockDim, ...), then
// fin_tail (error norm, candidate norms, controller).
template <typename R>
__global__ void __launch_bounds__(128, 4) k_finish(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                   const __grid_constant__ SysDev one, const Comb2 cd,
                                                   const CtlParams P) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ FinSm f;
    __shared__ __align__(16) Ctl cs;
    const int blk = load_sys(sysv, map, one, S, cv);
    if (cv.done) return;
    copy_ctl(S.ctl, cs);
    double* outp = const_cast<double*>(cv.cur ? cv.s0 : cv.s1);
    void* shad = cv.cur ? S.shadow0 : S.shadow1;
    const Terms<R> tp = resolve_terms<R>(cd.in, S, cv, false);
    FinAcc acc = fin_acc();
    const int np = (S.M + 1) >> 1;
    for (int p = blk * blockDim.x + threadIdx.x; p < np; p += S.nfin * blockDim.x)
        fin_pair<R>(S, cd, tp, outp, shad, 2 * p, acc, cv.tlog);
    fin_tail<R>(S, P, S.ctl, cs, blk, S.nfin, acc, f);
}

// The last inverse pass of an attempt fused with the final combination: each column
// CTA combines the element pairs whose stage vector it has just formed, then fin_tail
// over the nbx column CTAs of the system.
template <typename R>
__global__ void __launch_bounds__(ColBounds<R>::threads) k_inv_finish(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                    const __grid_constant__ SysDev one, const StageIn in,
                                                    const EpiOut eo, const Comb2 cd, const CtlParams P) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ InvSm<R> sm;
    __shared__ FinSm f;
    __shared__ __align__(16) Ctl cs;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int bx = load_desc(sysv, map, one, S);
    const ColSm<R> m = col_sm<R>(S, smraw);
    stage_tw(m.twP, S.lgN1, reinterpret_cast<const cx<R>*>(S.tw), S.lgMp);
    load_ctl(S, cv);
    if (cv.done) {
        cp_async_wait();  // no copy into this CTA's shared memory outlives it
        return;
    }
    copy_ctl(S.ctl, cs);
    inv_body<R>(S, cv, in, eo, bx, m, sm);
    double* outp = const_cast<double*>(cv.cur ? cv.s0 : cv.s1);
    void* shad = cv.cur ? S.shadow0 : S.shadow1;
    const Terms<R> tp = resolve_terms<R>(cd.in, S, cv, false);
    FinAcc acc = fin_acc();
    const Div DG = mkdiv(S.G);
    const int half = (S.N1 >> 1) * S.G;
    for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
        const int i = col_elem(S, DG, bx, idx);
        if (i < S.M) fin_pair<R>(S, cd, tp, outp, shad, i, acc, cv.tlog);
    }
    fin_tail<R>(S, P, S.ctl, cs, bx, S.nbx, acc, f);
}

// End of an integration: where the current state is the engine's second buffer, copy it
// and its R-typed shadow to the caller's buffer and make that buffer current (the last
// CTA of the system, after all copies), so that the caller's vector holds the result
// and later attempts continue from it. Runs on the device: the host learns the outcome
// with the statistics, after a single synchronisation.
template <typename R>
__global__ void __launch_bounds__(128) k_restore(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                 const __grid_constant__ SysDev one) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ bool last;
    const int blk = load_sys(sysv, map, one, S, cv);
    if (!cv.cur) return;
    double* dst = const_cast<double*>(cv.s0);
    const double* src = cv.s1;
    for (int i = blk * blockDim.x + threadIdx.x; i < S.M; i += S.nfin * blockDim.x) dst[i] = __ldcg(src + i);
    if (S.shadow0) {
        R* sd = reinterpret_cast<R*>(S.shadow0);
        const R* ss = reinterpret_cast<const R*>(S.shadow1);
        for (int i = blk * blockDim.x + threadIdx.x; i < S.M; i += S.nfin * blockDim.x) sd[i] = ss[i];
    }
    if (!arrive_last(S.ctl, S.nfin, &last)) return;
    if (threadIdx.x == 0) {
        S.ctl->arrive = 0;
        S.ctl->cur = 0;
    }
}

// Preparation of an integration, pass 1: moments mu_t of n0, ||n0||^2, max|n0| and
// sum_s s n0_s, in FP64 (the weights are read in type R). The last CTA of each system
// stores nrm2, ymax and mass in the control block and delta_t = sum_{alpha: u=t} coef
// mu_v (collision-rate coefficients) in aux.
template <typename R>
__global__ void __launch_bounds__(128) k_prep1(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                               const __grid_constant__ SysDev one) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ double red[33];
    __shared__ double fin[MAXT + 3 + TILT_T];
    __shared__ bool last;
    const int blk = load_sys(sysv, map, one, S, cv);
    Ctl* ctl = S.ctl;
    const double* n = cv.cur ? cv.s1 : cv.s0;
    const R* Wr = reinterpret_cast<const R*>(S.W);
    const int W = S.T + 3;  // mu_t..., n2, max, mass
    double acc[MAXT + 3];
    for (int q = 0; q < W; ++q) acc[q] = 0.0;
    double tmx[TILT_T];  // max_i |W_t[i] n_i| (the FP32 form's input tilt)
    for (int t = 0; t < TILT_T; ++t) tmx[t] = 0.0;
    R* shad = S.shadow0 ? reinterpret_cast<R*>(cv.cur ? S.shadow1 : S.shadow0) : nullptr;
    for (int i = blk * blockDim.x + threadIdx.x; i < S.M; i += S.nfin * blockDim.x) {
        const double y = n[i];
        if (shad) shad[i] = (R)y;
        for (int t = 0; t < S.T; ++t) {
            const double x = (double)Wr[(size_t)t * S.Mp + i] * y;
            acc[t] += x;
            if (t < TILT_T) tmx[t] = fmax(tmx[t], fabs(x));
        }
        acc[S.T] += y * y;
        acc[S.T + 1] = fmax(acc[S.T + 1], fabs(y));
        acc[S.T + 2] += (double)(i + 1) * y;
    }
    for (int q = 0; q < W; ++q) {
        const double v = (q == S.T + 1) ? block_max(acc[q], red) : block_sum(acc[q], red);
        if (threadIdx.x == 0) S.fpart[(size_t)FPW * blk + q] = v;
    }
    for (int t = 0; t < TILT_T; ++t) {  // slots W.. (FPW >= MAXT + 4 >= W + TILT_T)
        const double v = block_max(tmx[t], red);
        if (threadIdx.x == 0) S.fpart[(size_t)FPW * blk + W + t] = v;
    }
    if (!arrive_last(ctl, S.nfin, &last)) return;
    for (int q = 0; q < W + TILT_T; ++q) {
        const bool mx = q == S.T + 1 || q >= W;
        double v = 0.0;
        for (int b = threadIdx.x; b < S.nfin; b += blockDim.x) {
            const double x = __ldcg(S.fpart + (size_t)FPW * b + q);
            v = mx ? fmax(v, x) : v + x;
        }
        v = mx ? block_max(v, red) : block_sum(v, red);
        if (threadIdx.x == 0) fin[q] = v;
    }
    if (threadIdx.x != 0) return;
    for (int t = 0; t < TILT_T; ++t) ctl->tlog[t] = tilt_log((float)fin[W + t]);
    ctl->arrive = 0;
    ctl->nrm2 = fin[S.T];
    ctl->ymax = fin[S.T + 1];
    ctl->mass = fin[S.T + 2];
    set_xe(ctl, S, fin[S.T + 1]);
    for (int t = 0; t < S.T; ++t) S.aux[t] = 0.0;
    for (int al = 0; al < S.R; ++al) S.aux[S.au[al]] += S.acoef[al] * fin[S.av[al]];
}

// Pass 2: collision rate D_i = sum_j K_ij n_j = sum_t delta_t W_t[i]; its maximum
// gives the first step by the Euler criterion of Sec. 1, tau0 = a / max_i D_i, when
// the caller gave none (ctl->tau <= 0). Then the first attempt's step h is set, and
// (FP32 form) the input tilt from max |n| of pass 1.
template <typename R>
__global__ void __launch_bounds__(128) k_prep2(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                               const __grid_constant__ SysDev one, double euler_a) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ double red[33];
    __shared__ bool last;
    const int blk = load_sys(sysv, map, one, S, cv);
    Ctl* ctl = S.ctl;
    const R* Wr = reinterpret_cast<const R*>(S.W);
    const double* n = cv.cur ? cv.s1 : cv.s0;
    double mx = -INFINITY, tb = INFINITY;
    for (int i = blk * blockDim.x + threadIdx.x; i < S.M; i += S.nfin * blockDim.x) {
        double d = 0.0;
        for (int t = 0; t < S.T; ++t) {
            const double w = (double)Wr[(size_t)t * S.Mp + i];
            d += __ldcg(S.aux + t) * w;
            if (t < TILT_T) tb = fmin(tb, (double)tilt_bound_el(cv.tlog[t], (float)(w * n[i]), i));
        }
        mx = fmax(mx, d);
    }
    mx = block_max(mx, red);
    tb = block_min(tb, red);
    if (threadIdx.x == 0) {
        S.fpart[(size_t)FPW * blk] = mx;
        S.fpart[(size_t)FPW * blk + 1] = tb;
    }
    if (!arrive_last(ctl, S.nfin, &last)) return;
    double rate = -INFINITY, tbm = INFINITY;
    for (int b = threadIdx.x; b < S.nfin; b += blockDim.x) {
        rate = fmax(rate, __ldcg(S.fpart + (size_t)FPW * b));
        tbm = fmin(tbm, __ldcg(S.fpart + (size_t)FPW * b + 1));
    }
    rate = block_max(rate, red);
    tbm = block_min(tbm, red);
    if (threadIdx.x != 0) return;
    ctl->arrive = 0;
    ctl->tilt = tilt_from_bound(tbm, S.Mp, S.T);  // FP32 form: the first attempt's input tilt
    if (!(ctl->tau > 0.0)) ctl->tau = (rate > 0.0) ? euler_a / rate : 1.0;
    if (ctl->t >= ctl->t1) ctl->done = 1;
    else set_next_step(ctl);
}

// max_i |n_i| of the caller's vector into ctl->ymax (input scaling of a standalone
// FP32 evaluation; single system).
__global__ void __launch_bounds__(128) k_absmax(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                                const __grid_constant__ SysDev one, const double* __restrict__ n,
                                                int tilt) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ double red[33];
    __shared__ bool last;
    const int blk = load_sys(sysv, map, one, S, cv);
    Ctl* ctl = S.ctl;
    // with tilt (FP32 weights): also max_i |W_t[i] n_i| per transform t < TILT_T
    const float* Wf = tilt ? reinterpret_cast<const float*>(S.W) : nullptr;
    double mx = 0.0, tmx[TILT_T];
    for (int t = 0; t < TILT_T; ++t) tmx[t] = 0.0;
    for (int i = blk * blockDim.x + threadIdx.x; i < S.M; i += S.nfin * blockDim.x) {
        mx = fmax(mx, fabs(n[i]));
        if (Wf)
            for (int t = 0; t < S.T && t < TILT_T; ++t) tmx[t] = fmax(tmx[t], fabs((double)Wf[(size_t)t * S.Mp + i] * n[i]));
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) S.fpart[(size_t)FPW * blk] = mx;
    for (int t = 0; t < TILT_T; ++t) {
        const double v = block_max(tmx[t], red);
        if (threadIdx.x == 0) S.fpart[(size_t)FPW * blk + 1 + t] = v;
    }
    if (!arrive_last(ctl, S.nfin, &last)) return;
    for (int q = 0; q <= TILT_T; ++q) {
        double m = 0.0;
        for (int b = threadIdx.x; b < S.nfin; b += blockDim.x) m = fmax(m, __ldcg(S.fpart + (size_t)FPW * b + q));
        m = block_max(m, red);
        if (threadIdx.x != 0) continue;
        if (q == 0) {
            ctl->ymax = m;
            set_xe(ctl, S, m);
        } else {
            ctl->tlog[q - 1] = tilt_log((float)m);
        }
    }
    if (threadIdx.x == 0) ctl->arrive = 0;
}

// The input tilt of a standalone FP32 evaluation of the caller's vector n (after
// k_absmax has stored the transform inputs' maxima; single system).
__global__ void __launch_bounds__(128) k_tilt(const SysDev* __restrict__ sysv, const int2* __restrict__ map,
                                              const __grid_constant__ SysDev one, const double* __restrict__ n) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ double red[33];
    __shared__ bool last;
    const int blk = load_sys(sysv, map, one, S, cv);
    Ctl* ctl = S.ctl;
    const float* Wf = reinterpret_cast<const float*>(S.W);
    double tb = INFINITY;
    if (S.T <= TILT_T)
        for (int i = blk * blockDim.x + threadIdx.x; i < S.M; i += S.nfin * blockDim.x)
            for (int t = 0; t < S.T; ++t)
                tb = fmin(tb, (double)tilt_bound_el(cv.tlog[t], Wf[(size_t)t * S.Mp + i] * (float)n[i], i));
    tb = block_min(tb, red);
    if (threadIdx.x == 0) S.fpart[(size_t)FPW * blk] = tb;
    if (!arrive_last(ctl, S.nfin, &last)) return;
    double m = INFINITY;
    for (int b = threadIdx.x; b < S.nfin; b += blockDim.x) m = fmin(m, __ldcg(S.fpart + (size_t)FPW * b));
    m = block_min(m, red);
    if (threadIdx.x != 0) return;
    ctl->arrive = 0;
    ctl->tilt = tilt_from_bound(m, S.Mp, S.T);
}

// Keeps the stream busy for about `cycles` SM clocks (a bounded loop on the clock
// counter, no wait on memory) so that the host can enqueue a profiled sequence of
// kernels ahead of the device; measurement aid only.
__global__ void k_delay(long long cycles) {
    const long long t0 = clock64();
    while (clock64() - t0 < cycles) {
    }
}

}  // namespace smol
