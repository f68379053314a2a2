// smol_int.cuh - device side of the adaptive integrators of Sec. 2: the RK stage
// combination, the embedded / step-doubling error norm and the step-size controller,
// all kept on the device so that no host synchronisation happens per step.
#pragma once
#include "smol_rhs.cuh"

namespace smol {

enum { SCHEME_RK2 = 0, SCHEME_RK4 = 1, SCHEME_RKF45 = 2 };
enum { CTRL_DOUBLE_HALVE = 0, CTRL_FORMULA = 1 };
enum { ST_OK = 0, ST_STEADY = 1, ST_ENONFINITE = -3, ST_EUNDERFLOW = -4, ST_EMAXATT = -5 };

// Controller settings of one integration (passed by value).
struct CtlParams {
    int scheme, ctrl, rel_norm, fixed, order;
    int evals, evals_paper;        // S evaluations per attempt: actual and stages x steps
    double tau_min_rel, steady_rtol, fac_min, fac_max;
    int64_t max_attempts;
    int log_cap;
    double* log_t;
    double* log_h;
    double* log_err;
    int32_t* log_acc;
    const double* sqpart;          // ||S(n)||^2 partials of stage 1 (steady test), or null
    int nsq;
};

// Step-size rules of Sec. 2. Returns the proposed step; *acc the decision.
__device__ __forceinline__ double propose(const CtlParams& P, double h, double tau, double err, double tol, int* acc) {
    if (P.fixed) {
        *acc = 1;
        return tau;
    }
    *acc = err <= tol;
    if (P.scheme == SCHEME_RKF45 || P.ctrl == CTRL_FORMULA) {
        // RKF45: tau <- 0.9 tau (tol/err)^(1/5); Eq. (6): tau <- 1/4 tau (tol/err)^(1/p).
        const double s = (P.scheme == SCHEME_RKF45) ? 0.9 : 0.25;
        const double ex = (P.scheme == SCHEME_RKF45) ? 0.2 : 1.0 / (double)P.order;
        double fac;
        if (err == 0.0) fac = P.fac_max;
        else fac = fmin(fmax(s * pow(tol / err, ex), P.fac_min), P.fac_max);
        return h * fac;
    }
    // halve on reject, double on accept
    return *acc ? 2.0 * h : 0.5 * h;
}

__device__ __forceinline__ void set_next_step(Ctl* c) {
    c->clamped = c->tau >= c->t1 - c->t;
    c->h = c->clamped ? c->t1 - c->t : c->tau;
}

// out = sum c_j v_j over [0, M), elementwise (intermediate states, e.g. the
// half-step state of step doubling).
__global__ void __launch_bounds__(256) k_lincomb(const StageIn in, const Ctl* __restrict__ ctl, double* out, int M) {
    if (ctl->done) return;
    const int np = (M + 1) >> 1;
    const StagePtrs sp = resolve_all(in, ctl);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        double y0, y1;
        stage_pair(in, sp, M, 2 * p, y0, y1);
        if (2 * p + 1 < M) *reinterpret_cast<double2*>(out + 2 * p) = make_double2(y0, y1);
        else out[2 * p] = y0;
    }
}

// Final kernel of an attempt: candidate = sum c_j v_j written to the other state
// buffer, error vector sum d_j w_j reduced to ||.||_2^2, ||candidate||^2 and
// max|candidate|; the last CTA to finish reduces the partials in a fixed order and
// runs the controller (accept / reject, t, tau, counters, log, termination).
__global__ void __launch_bounds__(256) k_finish(const StageIn cand, const StageIn del, Ctl* __restrict__ ctl,
                                                const CtlParams P, double* part, int M) {
    if (ctl->done) return;
    __shared__ double red[33];
    __shared__ bool last;
    double* outp = ctl->state[ctl->cur ^ 1];
    double se = 0.0, sc = 0.0, mx = 0.0, bad = 0.0;
    const int np = (M + 1) >> 1;
    const StagePtrs cp = resolve_all(cand, ctl);
    const StagePtrs dp = resolve_all(del, ctl);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        const int i = 2 * p;
        double y0, y1, d0, d1;
        stage_pair(cand, cp, M, i, y0, y1);
        stage_pair(del, dp, M, i, d0, d1);
        if (i + 1 < M) *reinterpret_cast<double2*>(outp + i) = make_double2(y0, y1);
        else outp[i] = y0;
        se += d0 * d0 + d1 * d1;
        sc += y0 * y0 + y1 * y1;
        mx = fmax(mx, fmax(fabs(y0), fabs(y1)));
        if (!isfinite(y0) || !isfinite(y1)) bad = 1.0;
    }
    se = block_sum(se, red);
    sc = block_sum(sc, red);
    mx = block_max(mx, red);
    bad = block_max(bad, red);
    if (threadIdx.x == 0) {
        double* q = part + 4 * blockIdx.x;
        q[0] = se;
        q[1] = sc;
        q[2] = mx;
        q[3] = bad;
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->arrive, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // The last CTA reduces the per-CTA partials with all its threads (fixed order:
    // thread j takes partials j, j + blockDim, ...; then the block-wide tree).
    double E = 0.0, C = 0.0, X = 0.0, B = 0.0, Q = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
        E += __ldcg(part + 4 * b);
        C += __ldcg(part + 4 * b + 1);
        X = fmax(X, __ldcg(part + 4 * b + 2));
        B = fmax(B, __ldcg(part + 4 * b + 3));
    }
    if (P.steady_rtol > 0.0 && P.sqpart)
        for (int b = threadIdx.x; b < P.nsq; b += blockDim.x) Q += __ldcg(P.sqpart + b);
    E = block_sum(E, red);
    C = block_sum(C, red);
    Q = block_sum(Q, red);
    X = block_max(X, red);
    B = block_max(B, red);
    if (threadIdx.x != 0) return;
    Ctl* c = ctl;
    c->arrive = 0;
    c->rhs_evals += 1;  // S(n^k) of the first stage
    if (P.steady_rtol > 0.0 && P.sqpart) {
        const double s2 = Q;
        const double nn = sqrt(c->nrm2);
        c->steady = s2;
        if (nn > 0.0 && sqrt(s2) / nn < P.steady_rtol) {
            c->status = ST_STEADY;
            c->done = 1;
            return;
        }
    }
    c->rhs_evals += P.evals - 1;
    c->rhs_paper += P.evals_paper;
    c->attempts += 1;
    double err = (P.fixed && P.scheme != SCHEME_RKF45) ? 0.0 : sqrt(E);
    if (P.rel_norm) {
        const double nn = sqrt(c->nrm2);
        if (nn > 0.0) err /= nn;
    }
    c->err_last = err;
    if (!isfinite(err) || B != 0.0) {
        c->status = ST_ENONFINITE;
        c->done = 1;
        return;
    }
    int acc;
    const double h = c->h;
    const double tau_new = propose(P, h, c->tau, err, c->tol, &acc);
    if (P.log_cap > 0) {
        const int64_t slot = (c->attempts - 1) % P.log_cap;
        P.log_t[slot] = c->t;
        P.log_h[slot] = h;
        P.log_err[slot] = err;
        P.log_acc[slot] = acc;
    }
    if (acc) {
        c->cur ^= 1;
        c->t = c->clamped ? c->t1 : c->t + h;
        c->accepted += 1;
        c->nrm2 = C;
        c->ymax = X;
        if (!c->clamped) c->tau = tau_new;
    } else {
        c->rejected += 1;
        c->tau = tau_new;
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
    if (!c->done) set_next_step(c);
}

// Preparation of an integration, pass 1: moments mu_t of n0, ||n0||^2, max|n0|.
// Partials [blk][T + 2]; the last CTA reduces them, stores nrm2 and ymax in the control
// block and delta_t = sum_{alpha: u=t} coef mu_v (for the collision rate) in dout.
__global__ void __launch_bounds__(256) k_prep1(const SysDev S, Ctl* __restrict__ ctl, double* part, double* dout) {
    __shared__ double red[33];
    __shared__ bool last;
    const double* n = ctl->state[ctl->cur];
    const int W = S.T + 2;
    double acc[MAXT + 2];
    for (int q = 0; q < W; ++q) acc[q] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.M; i += gridDim.x * blockDim.x) {
        const double y = n[i];
        for (int t = 0; t < S.T; ++t) acc[t] += S.W[(size_t)t * S.Mp + i] * y;
        acc[S.T] += y * y;
        acc[S.T + 1] = fmax(acc[S.T + 1], fabs(y));
    }
    for (int q = 0; q < W; ++q) {
        const double v = (q == S.T + 1) ? block_max(acc[q], red) : block_sum(acc[q], red);
        if (threadIdx.x == 0) part[(size_t)blockIdx.x * W + q] = v;
    }
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double fin[MAXT + 2];
    for (int q = 0; q < W; ++q) {
        double v = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
            const double x = __ldcg(part + (size_t)b * W + q);
            v = (q == S.T + 1) ? fmax(v, x) : v + x;
        }
        v = (q == S.T + 1) ? block_max(v, red) : block_sum(v, red);
        if (threadIdx.x == 0) fin[q] = v;
    }
    if (threadIdx.x != 0) return;
    ctl->arrive = 0;
    ctl->nrm2 = fin[S.T];
    ctl->ymax = fin[S.T + 1];
    for (int t = 0; t < S.T; ++t) dout[t] = 0.0;
    for (int al = 0; al < S.R; ++al) dout[S.au[al]] += S.acoef[al] * fin[S.av[al]];
}

// Pass 2: collision rate D_i = sum_j K_ij n_j = sum_t delta_t W_t[i]; its maximum
// gives the first step by the Euler criterion of Sec. 1, tau0 = a / max_i D_i, when
// the caller gave none (ctl->tau <= 0). Then the first attempt's step h is set.
__global__ void __launch_bounds__(256) k_prep2(const SysDev S, Ctl* __restrict__ ctl, const double* delta, double* part,
                                               double euler_a) {
    __shared__ double red[33];
    __shared__ bool last;
    double mx = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.M; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int t = 0; t < S.T; ++t) d += delta[t] * S.W[(size_t)t * S.Mp + i];
        mx = fmax(mx, d);
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = mx;
        __threadfence();
        last = (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double rate = -INFINITY;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) rate = fmax(rate, __ldcg(part + b));
    rate = block_max(rate, red);
    if (threadIdx.x != 0) return;
    ctl->arrive = 0;
    if (!(ctl->tau > 0.0)) ctl->tau = (rate > 0.0) ? euler_a / rate : 1.0;
    if (ctl->t >= ctl->t1) ctl->done = 1;
    else set_next_step(ctl);
}

// max_i |n_i| of a vector into ctl->ymax (input scaling of a standalone FP32 evaluation).
__global__ void __launch_bounds__(256) k_absmax(const double* __restrict__ n, int M, Ctl* __restrict__ ctl, double* part) {
    __shared__ double red[33];
    __shared__ bool last;
    double mx = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < M; i += gridDim.x * blockDim.x) mx = fmax(mx, fabs(n[i]));
    mx = block_max(mx, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = mx;
        __threadfence();
        last = (atomicAdd(&ctl->arrive, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double m = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) m = fmax(m, __ldcg(part + b));
    m = block_max(m, red);
    if (threadIdx.x != 0) return;
    ctl->arrive = 0;
    ctl->ymax = m;
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
