// smol.cu - host side of the C interface declared in include/smol.h: system set-up
// (distinct transforms, weights, twiddles, workspace layout), one evaluation of
// S(n) as three kernel launches, and the device-resident adaptive integrators of
// Sec. 2 driven through captured CUDA graphs.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "../../include/smol.h"
#include "smol_int.cuh"

using namespace smol;

namespace {

constexpr int NVEC = 12;        // stage / work vectors of the integrators
constexpr int FIN_BLOCKS = 608; // 4 x 152 SMs (128-thread CTAs)
constexpr int PREP_BLOCKS = 152;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ilog2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// Largest dynamic shared memory a kernel may use (opt-in limit of sm_100-class parts).
constexpr size_t SMEM_LIMIT = 227 * 1024;

struct Shape {
    int M, Mp, lgMp, N1, N2, lgN1, lgN2, G;
    size_t csz;  // bytes of one complex value
};

Shape make_shape(int64_t M, int precision) {
    Shape s;
    s.M = (int)M;
    s.lgMp = ilog2(M < 4 ? 4 : M);
    s.Mp = 1 << s.lgMp;
    s.lgN1 = (s.lgMp + 1) / 2;
    s.lgN2 = s.lgMp / 2;
    s.N1 = 1 << s.lgN1;
    s.N2 = 1 << s.lgN2;
    // columns per CTA of the column passes: one column of N1 >= 256 points per CTA
    // (many small CTAs spread the latency-bound passes over all SMs), more columns for
    // short columns so that a CTA keeps at least 32 radix-8 butterflies per pass
    int G = 256 / s.N1;
    if (G < 1) G = 1;
    if (G > s.N2) G = s.N2;
    s.G = G;
    s.csz = precision == SMOL_FP32CONV ? 8 : 16;
    return s;
}

size_t smem_cols(const Shape& s) { return 2 * (size_t)s.N1 * s.G * s.csz; }
size_t smem_rows(const Shape& s, int T) { return 2 * (size_t)s.N2 * 2 * T * s.csz; }

struct Layout {
    size_t ctl, rctl, tw, W, Y, G2, ybuf, vec, stateB, mpart, fpart, sqpart, ppart, delta, log_t, log_h, log_e, log_a,
        total;
};

Layout make_layout(const Shape& s, int R, int log_cap) {
    const int Tm = 2 * R;
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += align256(bytes);
        return r;
    };
    L.ctl = take(sizeof(Ctl));
    L.rctl = take(sizeof(Ctl));
    L.tw = take((size_t)s.Mp * s.csz);
    L.W = take((size_t)Tm * s.Mp * 8);
    L.Y = take((size_t)Tm * s.Mp * s.csz);
    L.G2 = take((size_t)s.Mp * s.csz);
    L.ybuf = take((size_t)s.Mp * 8);
    L.vec = take((size_t)NVEC * align256((size_t)s.Mp * 8));
    L.stateB = take((size_t)s.Mp * 8);
    L.mpart = take((size_t)Tm * (s.N2 / s.G) * 2 * 8);
    L.fpart = take((size_t)FIN_BLOCKS * 4 * 8);
    L.sqpart = take((size_t)(s.N2 / s.G) * 8);
    L.ppart = take((size_t)PREP_BLOCKS * (MAXT + 2) * 8);
    L.delta = take((size_t)MAXT * 8);
    L.log_t = take((size_t)log_cap * 8);
    L.log_h = take((size_t)log_cap * 8);
    L.log_e = take((size_t)log_cap * 8);
    L.log_a = take((size_t)log_cap * 4);
    L.total = o;
    return L;
}

void default_opts(smol_opts* o) {
    memset(o, 0, sizeof(*o));
    o->precision = SMOL_FP64;
    o->ctrl = SMOL_CTRL_DOUBLE_HALVE;
    o->norm = SMOL_NORM_ABS;
    o->log_capacity = 0;
    o->tau0 = 0.0;
    o->euler_a = 0.1;
    o->tau_min_rel = 1e-12;
    o->steady_rtol = 0.0;
    o->fixed_tau = 0.0;
    o->fac_min = 0.1;
    o->fac_max = 4.0;
    o->max_attempts = (int64_t)1 << 62;
    o->chunk = 32;
    o->stream = nullptr;
}

bool proportional(const double* x, const double* w, int M, double* c) {
    int i0 = 0;
    double wmax = 0.0;
    for (int i = 0; i < M; ++i)
        if (fabs(w[i]) > wmax) {
            wmax = fabs(w[i]);
            i0 = i;
        }
    if (wmax == 0.0) return false;
    const double r = x[i0] / w[i0];
    for (int i = 0; i < M; ++i) {
        const double d = fabs(x[i] - r * w[i]);
        if (d > 4e-16 * fmax(fabs(x[i]), fabs(r * w[i]))) return false;
    }
    *c = r;
    return true;
}

}  // namespace

struct smol_system {
    Shape s;
    int R, T;
    double lambda;
    smol_opts o;
    cudaStream_t stream;
    cudaStream_t cap;  // private stream used only for graph capture
    char* ws;
    Layout L;
    SysDev dev;
    Ctl* ctl;
    Ctl* rctl;
    Ctl* h_ctl;  // pinned host copy
    double* vec[NVEC];
    double* stateB;
    // cached graph of one chunk, keyed by (scheme, fixed, steady, log)
    cudaGraphExec_t gexec;
    int gkey;
    int64_t last_attempts;
    // current run (smol_integrate_start .. smol_integrate_finish)
    double* run_dn;
    int run_scheme;
    int64_t run_attempts;
};

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
namespace {

template <typename R>
int set_smem_attrs(const smol_system* S) {
    const size_t sc = smem_cols(S->s), sr = smem_rows(S->s, S->T);
    if (cudaFuncSetAttribute(k_fwd_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc) != cudaSuccess)
        return SMOL_ECUDA;
    if (cudaFuncSetAttribute(k_inv_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc) != cudaSuccess)
        return SMOL_ECUDA;
    if (cudaFuncSetAttribute(k_rows<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr) != cudaSuccess)
        return SMOL_ECUDA;
    return SMOL_OK;
}

// Threads of a CTA whose passes have `points` points per sequence-group: one thread per
// radix-8 butterfly, between 32 and 256.
int threads_for(int points) {
    int t = points / 8;
    if (t > 256) t = 256;
    if (t < 32) t = 32;
    return (t + 31) & ~31;
}

// Optional per-kernel timing of eagerly launched attempts (smol_profile_attempts).
constexpr int PROF_MAX = 64;
struct Prof {
    cudaEvent_t ev0[PROF_MAX], ev1[PROF_MAX];
    int kind[PROF_MAX];
    int n;
};
struct ProfScope {
    Prof* p;
    cudaStream_t st;
    int q;
    ProfScope(Prof* p_, cudaStream_t st_, int kind) : p(p_), st(st_), q(-1) {
        if (p && p->n < PROF_MAX) {
            q = p->n++;
            p->kind[q] = kind;
            cudaEventRecord(p->ev0[q], st);
        }
    }
    ~ProfScope() {
        if (q >= 0) cudaEventRecord(p->ev1[q], st);
    }
};

template <typename R>
void launch_eval(const smol_system* S, const StageIn& in, const Ctl* ctl, const EpiOut& eo, cudaStream_t st,
                 Prof* pr) {
    const Shape& s = S->s;
    const int nbx = s.N2 / s.G;
    const size_t sc = smem_cols(s), sr = smem_rows(s, S->T);
    {
        ProfScope ps(pr, st, SMOL_PROF_FWD_COLS);
        k_fwd_cols<R><<<dim3(nbx, S->T), threads_for(s.N1 * s.G), sc, st>>>(S->dev, in, ctl, s.G);
    }
    {
        ProfScope ps(pr, st, SMOL_PROF_ROWS);
        k_rows<R><<<s.N1 / 2, threads_for(s.N2 * 2 * S->T), sr, st>>>(S->dev, ctl);
    }
    {
        ProfScope ps(pr, st, SMOL_PROF_INV_COLS);
        k_inv_cols<R><<<nbx, threads_for(s.N1 * s.G), sc, st>>>(S->dev, in, ctl, eo, s.G);
    }
}

void eval(const smol_system* S, const StageIn& in, const Ctl* ctl, const EpiOut& eo, cudaStream_t st,
          Prof* pr = nullptr) {
    if (S->o.precision == SMOL_FP32CONV) launch_eval<float>(S, in, ctl, eo, st, pr);
    else launch_eval<double>(S, in, ctl, eo, st, pr);
}

StageIn stage(std::initializer_list<std::pair<int, double>> terms, const smol_system* S) {
    // term index: -1 = current state, -2 = other state, k >= 0 = work vector k
    StageIn in;
    memset(&in, 0, sizeof(in));
    in.nv = 0;
    for (auto& tc : terms) {
        const int j = in.nv++;
        if (tc.first == -1) {
            in.sel[j] = 0;
            in.v[j] = nullptr;
        } else if (tc.first == -2) {
            in.sel[j] = 1;
            in.v[j] = nullptr;
        } else {
            in.sel[j] = -1;
            in.v[j] = S->vec[tc.first];
        }
        in.c[j] = tc.second;
    }
    in.direct = 0;
    return in;
}

StageIn from_ptr(const double* p) {
    StageIn in;
    memset(&in, 0, sizeof(in));
    in.nv = 1;
    in.direct = 1;
    in.sel[0] = -1;
    in.v[0] = p;
    in.c[0] = 1.0;
    return in;
}

EpiOut epi_k(double* out, double hfac, double* sqpart) {
    EpiOut e;
    memset(&e, 0, sizeof(e));
    e.out = out;
    e.hfac = hfac;
    e.use_h = 1;
    e.sqpart = sqpart;
    return e;
}

constexpr int FIN_THREADS = 128;

int fin_blocks(int M) {
    int b = (M / 2 + FIN_THREADS - 1) / FIN_THREADS;
    if (b < 1) b = 1;
    if (b > FIN_BLOCKS) b = FIN_BLOCKS;
    return b;
}

// Enqueues one step attempt of the given scheme on stream st.
void enqueue_attempt(smol_system* S, int scheme, bool fixed, const CtlParams& P, cudaStream_t st, Prof* pr) {
    double* sq = (double*)(S->ws + S->L.sqpart);
    double* fpart = (double*)(S->ws + S->L.fpart);
    const int M = S->s.M;
    Ctl* c = S->ctl;
    auto E = [&](const StageIn& in, int k, double hfac, bool first) {
        eval(S, in, c, epi_k(S->vec[k], hfac, (first && P.sqpart) ? sq : nullptr), st, pr);
    };
    if (scheme == SCHEME_RKF45) {
        E(stage({{-1, 1.0}}, S), 0, 1.0, true);
        E(stage({{-1, 1.0}, {0, 0.25}}, S), 1, 1.0, false);
        E(stage({{-1, 1.0}, {0, 3.0 / 32.0}, {1, 9.0 / 32.0}}, S), 2, 1.0, false);
        E(stage({{-1, 1.0}, {0, 1932.0 / 2197.0}, {1, -7200.0 / 2197.0}, {2, 7296.0 / 2197.0}}, S), 3, 1.0, false);
        E(stage({{-1, 1.0}, {0, 439.0 / 216.0}, {1, -8.0}, {2, 3680.0 / 513.0}, {3, -845.0 / 4104.0}}, S), 4, 1.0,
          false);
        E(stage({{-1, 1.0},
                 {0, -8.0 / 27.0},
                 {1, 2.0},
                 {2, -3544.0 / 2565.0},
                 {3, 1859.0 / 4104.0},
                 {4, -11.0 / 40.0}},
                S),
          5, 1.0, false);
        StageIn cand = stage({{-1, 1.0}, {0, 25.0 / 216.0}, {2, 1408.0 / 2565.0}, {3, 2197.0 / 4104.0}, {4, -1.0 / 5.0}}, S);
        // n_RK5 - n^{k+1}: differences of the two weight rows of the tableau
        StageIn del = stage({{0, 16.0 / 135.0 - 25.0 / 216.0},
                             {2, 6656.0 / 12825.0 - 1408.0 / 2565.0},
                             {3, 28561.0 / 56430.0 - 2197.0 / 4104.0},
                             {4, -9.0 / 50.0 + 1.0 / 5.0},
                             {5, 2.0 / 55.0}},
                            S);
        { ProfScope ps(pr, st, SMOL_PROF_STEP); k_finish<<<fin_blocks(M), FIN_THREADS, 0, st>>>(cand, del, c, P, fpart, M); }
        return;
    }
    if (scheme == SCHEME_RK2) {
        E(stage({{-1, 1.0}}, S), 0, 1.0, true);                      // k1 = h S(n)
        E(stage({{-1, 1.0}, {0, 1.0}}, S), 1, 1.0, false);           // k2 = h S(n + k1)
        if (fixed) {
            StageIn cand = stage({{-1, 1.0}, {0, 0.5}, {1, 0.5}}, S);
            StageIn del = stage({{0, 0.0}}, S);
            { ProfScope ps(pr, st, SMOL_PROF_STEP); k_finish<<<fin_blocks(M), FIN_THREADS, 0, st>>>(cand, del, c, P, fpart, M); }
            return;
        }
        // half step 1: l1 = k1/2, l2 = (h/2) S(n + k1/2); n_half = n + (l1 + l2)/2
        E(stage({{-1, 1.0}, {0, 0.5}}, S), 2, 0.5, false);
        { ProfScope ps(pr, st, SMOL_PROF_STEP); k_lincomb<<<fin_blocks(M), FIN_THREADS, 0, st>>>(stage({{-1, 1.0}, {0, 0.25}, {2, 0.5}}, S), c, S->vec[3], M); }
        // half step 2 from n_half: m1, m2
        E(stage({{3, 1.0}}, S), 4, 0.5, false);
        E(stage({{3, 1.0}, {4, 1.0}}, S), 5, 0.5, false);
        StageIn cand = stage({{3, 1.0}, {4, 0.5}, {5, 0.5}}, S);
        StageIn del = stage({{3, 1.0}, {4, 0.5}, {5, 0.5}, {-1, -1.0}, {0, -0.5}, {1, -0.5}}, S);
        { ProfScope ps(pr, st, SMOL_PROF_STEP); k_finish<<<fin_blocks(M), FIN_THREADS, 0, st>>>(cand, del, c, P, fpart, M); }
        return;
    }
    // RK4
    E(stage({{-1, 1.0}}, S), 0, 1.0, true);                          // k1
    E(stage({{-1, 1.0}, {0, 0.5}}, S), 1, 1.0, false);               // k2
    E(stage({{-1, 1.0}, {1, 0.5}}, S), 2, 1.0, false);               // k3
    E(stage({{-1, 1.0}, {2, 1.0}}, S), 3, 1.0, false);               // k4
    if (fixed) {
        StageIn cand = stage({{-1, 1.0}, {0, 1.0 / 6.0}, {1, 1.0 / 3.0}, {2, 1.0 / 3.0}, {3, 1.0 / 6.0}}, S);
        StageIn del = stage({{0, 0.0}}, S);
        { ProfScope ps(pr, st, SMOL_PROF_STEP); k_finish<<<fin_blocks(M), FIN_THREADS, 0, st>>>(cand, del, c, P, fpart, M); }
        return;
    }
    // half step 1 with h/2: l1 = k1/2
    E(stage({{-1, 1.0}, {0, 0.25}}, S), 4, 0.5, false);              // l2 = (h/2) S(n + l1/2)
    E(stage({{-1, 1.0}, {4, 0.5}}, S), 5, 0.5, false);               // l3
    E(stage({{-1, 1.0}, {5, 1.0}}, S), 6, 0.5, false);               // l4
    { ProfScope ps(pr, st, SMOL_PROF_STEP); k_lincomb<<<fin_blocks(M), FIN_THREADS, 0, st>>>(
        stage({{-1, 1.0}, {0, 1.0 / 12.0}, {4, 1.0 / 3.0}, {5, 1.0 / 3.0}, {6, 1.0 / 6.0}}, S), c, S->vec[7], M); }
    E(stage({{7, 1.0}}, S), 8, 0.5, false);                          // m1
    E(stage({{7, 1.0}, {8, 0.5}}, S), 9, 0.5, false);                // m2
    E(stage({{7, 1.0}, {9, 0.5}}, S), 10, 0.5, false);               // m3
    E(stage({{7, 1.0}, {10, 1.0}}, S), 11, 0.5, false);              // m4
    StageIn cand = stage({{7, 1.0}, {8, 1.0 / 6.0}, {9, 1.0 / 3.0}, {10, 1.0 / 3.0}, {11, 1.0 / 6.0}}, S);
    // n_hat - n^{k+1} (the full step of length h)
    StageIn del = stage({{7, 1.0},
                         {8, 1.0 / 6.0},
                         {9, 1.0 / 3.0},
                         {10, 1.0 / 3.0},
                         {11, 1.0 / 6.0},
                         {-1, -1.0},
                         {0, -1.0 / 6.0},
                         {1, -1.0 / 3.0},
                         {2, -1.0 / 3.0},
                         {3, -1.0 / 6.0}},
                        S);
    { ProfScope ps(pr, st, SMOL_PROF_STEP); k_finish<<<fin_blocks(M), FIN_THREADS, 0, st>>>(cand, del, c, P, fpart, M); }
}

CtlParams make_params(const smol_system* S, int scheme, bool steady) {
    CtlParams P;
    memset(&P, 0, sizeof(P));
    const bool fixed = S->o.fixed_tau > 0.0;
    P.scheme = scheme;
    P.ctrl = S->o.ctrl;
    P.rel_norm = S->o.norm == SMOL_NORM_REL;
    P.fixed = fixed;
    P.order = scheme == SCHEME_RK2 ? 2 : 4;
    const int stages = scheme == SCHEME_RK2 ? 2 : (scheme == SCHEME_RK4 ? 4 : 6);
    if (scheme == SCHEME_RKF45) {
        P.evals = 6;
        P.evals_paper = 6;
    } else if (fixed) {
        P.evals = stages;
        P.evals_paper = stages;
    } else {
        P.evals = 3 * stages - 1;
        P.evals_paper = 3 * stages;
    }
    P.tau_min_rel = S->o.tau_min_rel;
    P.steady_rtol = steady ? S->o.steady_rtol : 0.0;
    P.fac_min = S->o.fac_min;
    P.fac_max = S->o.fac_max;
    P.max_attempts = S->o.max_attempts;
    P.log_cap = S->o.log_capacity;
    P.log_t = (double*)(S->ws + S->L.log_t);
    P.log_h = (double*)(S->ws + S->L.log_h);
    P.log_err = (double*)(S->ws + S->L.log_e);
    P.log_acc = (int32_t*)(S->ws + S->L.log_a);
    P.sqpart = steady ? (const double*)(S->ws + S->L.sqpart) : nullptr;
    P.nsq = S->s.N2 / S->s.G;
    return P;
}

#define CK(x)                                      \
    do {                                           \
        if ((x) != cudaSuccess) return SMOL_ECUDA; \
    } while (0)

}  // namespace

// ---------------------------------------------------------------------------
// C interface
// ---------------------------------------------------------------------------
extern "C" {

void smol_default_opts(smol_opts* opts) {
    if (opts) default_opts(opts);
}

int64_t smol_max_m(int32_t R, int32_t precision) {
    if (R < 1 || R > MAXR) return 0;
    int64_t best = 0;
    for (int lg = 2; lg <= 22; ++lg) {
        Shape s = make_shape((int64_t)1 << lg, precision);
        if (smem_cols(s) <= SMEM_LIMIT && smem_rows(s, 2 * R) <= SMEM_LIMIT) best = (int64_t)1 << lg;
    }
    return best;
}

size_t smol_workspace_bytes(int64_t M, int32_t R, const smol_opts* opts) {
    smol_opts o;
    if (opts) o = *opts;
    else default_opts(&o);
    if (M < 1 || R < 1 || R > MAXR || M > smol_max_m(R, o.precision)) return 0;
    Shape s = make_shape(M, o.precision);
    return make_layout(s, R, o.log_capacity > 0 ? o.log_capacity : 0).total;
}

int smol_init_system(smol_system** out, int64_t M, int32_t R, const double* h_U, const double* h_V, double lambda,
                     const smol_opts* opts, void* d_workspace, size_t workspace_bytes) {
    if (!out || !h_U || !h_V || !d_workspace || M < 1 || R < 1 || R > MAXR || !(lambda >= 0.0)) return SMOL_EINVAL;
    *out = nullptr;
    smol_opts o;
    if (opts) o = *opts;
    else default_opts(&o);
    if (o.precision != SMOL_FP64 && o.precision != SMOL_FP32CONV) return SMOL_EINVAL;
    if (o.log_capacity < 0 || o.chunk < 0) return SMOL_EINVAL;
    if (o.chunk == 0) o.chunk = 32;
    if (M > smol_max_m(R, o.precision)) return SMOL_EUNSUPPORTED;
    if (((uintptr_t)d_workspace & 255) != 0) return SMOL_EINVAL;
    const size_t need = smol_workspace_bytes(M, R, &o);
    if (workspace_bytes < need) return SMOL_ENOSPACE;

    smol_system* S = new smol_system();
    memset(S, 0, sizeof(*S));
    S->s = make_shape(M, o.precision);
    S->R = R;
    S->lambda = lambda;
    S->o = o;
    S->stream = (cudaStream_t)o.stream;
    S->ws = (char*)d_workspace;
    S->L = make_layout(S->s, R, o.log_capacity);
    const Shape& s = S->s;
    const int Mi = (int)M;

    // Distinct transforms among the columns of U and rows of V.
    std::vector<std::vector<double>> W;
    std::vector<int> au, av;
    std::vector<double> acoef;
    std::vector<double> ucol(Mi), vrow(Mi);
    auto find_or_add = [&](const std::vector<double>& x, double* c) -> int {
        for (size_t t = 0; t < W.size(); ++t)
            if (proportional(x.data(), W[t].data(), Mi, c)) return (int)t;
        W.push_back(x);
        *c = 1.0;
        return (int)W.size() - 1;
    };
    for (int al = 0; al < R; ++al) {
        bool uz = true, vz = true;
        for (int i = 0; i < Mi; ++i) {
            ucol[i] = h_U[(size_t)i * R + al];
            vrow[i] = h_V[(size_t)al * Mi + i];
            uz = uz && ucol[i] == 0.0;
            vz = vz && vrow[i] == 0.0;
            if (!isfinite(ucol[i]) || !isfinite(vrow[i])) {
                delete S;
                return SMOL_EINVAL;
            }
        }
        if (uz || vz) continue;  // the term vanishes
        double cu, cv;
        const int u = find_or_add(ucol, &cu);
        const int v = find_or_add(vrow, &cv);
        au.push_back(u);
        av.push_back(v);
        acoef.push_back(cu * cv);
    }
    if (W.empty()) {  // K == 0: keep one zero transform so that every path is well formed
        W.push_back(std::vector<double>(Mi, 0.0));
        au.push_back(0);
        av.push_back(0);
        acoef.push_back(0.0);
    }
    S->T = (int)W.size();
    SysDev& d = S->dev;
    memset(&d, 0, sizeof(d));
    d.M = Mi;
    d.Mp = s.Mp;
    d.lgMp = s.lgMp;
    d.N1 = s.N1;
    d.N2 = s.N2;
    d.lgN1 = s.lgN1;
    d.lgN2 = s.lgN2;
    d.T = S->T;
    d.R = (int)au.size();
    d.lambda = lambda;
    d.nbxA = s.N2 / s.G;
    for (int al = 0; al < d.R; ++al) {
        d.au[al] = au[al];
        d.av[al] = av[al];
        d.acoef[al] = acoef[al];
    }
    // unordered pairs for the spectral product: (u,v) and (v,u) give the same product
    d.npairs = 0;
    for (int al = 0; al < d.R; ++al) {
        int a = au[al], b = av[al];
        if (a > b) {
            int t = a;
            a = b;
            b = t;
        }
        int p = 0;
        for (; p < d.npairs; ++p)
            if (d.pu[p] == a && d.pv[p] == b) break;
        if (p == d.npairs) {
            d.pu[p] = a;
            d.pv[p] = b;
            d.pcoef[p] = 0.0;
            d.npairs++;
        }
        d.pcoef[p] += acoef[al];
    }
    for (int t = 0; t < S->T; ++t) {
        double mx = 0.0;
        for (int i = 0; i < Mi; ++i) mx = fmax(mx, fabs(W[t][i]));
        d.wexp[t] = mx > 0.0 ? ilogb(mx) : 0;
    }
    if (smem_rows(s, S->T) > SMEM_LIMIT) {
        delete S;
        return SMOL_EUNSUPPORTED;
    }
    char* ws = S->ws;
    S->ctl = (Ctl*)(ws + S->L.ctl);
    S->rctl = (Ctl*)(ws + S->L.rctl);
    d.W = (const double*)(ws + S->L.W);
    d.tw = ws + S->L.tw;
    d.Y = ws + S->L.Y;
    d.G2 = ws + S->L.G2;
    d.ybuf = (double*)(ws + S->L.ybuf);
    d.mpart = (double*)(ws + S->L.mpart);
    for (int k = 0; k < NVEC; ++k) S->vec[k] = (double*)(ws + S->L.vec + (size_t)k * align256((size_t)s.Mp * 8));
    S->stateB = (double*)(ws + S->L.stateB);

    // Host images of the tables.
    std::vector<double> hW((size_t)S->T * s.Mp, 0.0);
    for (int t = 0; t < S->T; ++t)
        for (int i = 0; i < Mi; ++i) hW[(size_t)t * s.Mp + i] = W[t][i];
    // Twiddles W_{2Mp}^e = exp(-i pi e / Mp), e < Mp, in extended precision.
    std::vector<double> tw64(2 * (size_t)s.Mp);
    for (int e = 0; e < s.Mp; ++e) {
        const long double th = 3.141592653589793238462643383279502884L * (long double)e / (long double)s.Mp;
        tw64[2 * e] = (double)cosl(th);
        tw64[2 * e + 1] = (double)-sinl(th);
    }
    cudaStream_t st = S->stream;
    cudaError_t err = cudaSuccess;
    if (o.precision == SMOL_FP32CONV) {
        std::vector<float> tw32(2 * (size_t)s.Mp);
        for (size_t q = 0; q < tw32.size(); ++q) tw32[q] = (float)tw64[q];
        err = cudaMemcpyAsync(ws + S->L.tw, tw32.data(), tw32.size() * 4, cudaMemcpyHostToDevice, st);
    } else {
        err = cudaMemcpyAsync(ws + S->L.tw, tw64.data(), tw64.size() * 8, cudaMemcpyHostToDevice, st);
    }
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(ws + S->L.W, hW.data(), hW.size() * 8, cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(ws + S->L.ctl, 0, 2 * align256(sizeof(Ctl)), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(ws + S->L.vec, 0, (size_t)NVEC * align256((size_t)s.Mp * 8), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(ws + S->L.ybuf, 0, (size_t)s.Mp * 8, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(ws + S->L.stateB, 0, (size_t)s.Mp * 8, st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(st);
    if (err == cudaSuccess) err = cudaHostAlloc((void**)&S->h_ctl, sizeof(Ctl), cudaHostAllocDefault);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&S->cap, cudaStreamNonBlocking);
    int rc = (err == cudaSuccess) ? SMOL_OK : SMOL_ECUDA;
    if (rc == SMOL_OK) rc = (o.precision == SMOL_FP32CONV) ? set_smem_attrs<float>(S) : set_smem_attrs<double>(S);
    if (rc != SMOL_OK) {
        smol_destroy(S);
        return rc;
    }
    S->gkey = -1;
    *out = S;
    return SMOL_OK;
}

int smol_set_stream(smol_system* S, void* stream) {
    if (!S) return SMOL_EINVAL;
    S->stream = (cudaStream_t)stream;
    S->o.stream = stream;
    return SMOL_OK;
}

int smol_num_transforms(const smol_system* S) { return S ? S->T : 0; }

static int rhs_common(smol_system* S, const double* d_n, double* d_out, double* d_birth, double* d_loss, double* d_src) {
    if (!S || !d_n) return SMOL_EINVAL;
    if (((uintptr_t)d_n & 15) || ((uintptr_t)d_out & 15) || ((uintptr_t)d_birth & 15) || ((uintptr_t)d_loss & 15))
        return SMOL_EINVAL;
    cudaStream_t st = S->stream;
    if (S->o.precision == SMOL_FP32CONV) {
        const int nb = fin_blocks(S->s.M) > PREP_BLOCKS ? PREP_BLOCKS : fin_blocks(S->s.M);
        k_absmax<<<nb, 256, 0, st>>>(d_n, S->s.M, S->rctl, (double*)(S->ws + S->L.ppart));
    }
    EpiOut eo;
    memset(&eo, 0, sizeof(eo));
    eo.out = d_out;
    eo.birth = d_birth;
    eo.loss = d_loss;
    eo.source = d_src;
    eo.hfac = 1.0;
    eo.use_h = 0;
    eval(S, from_ptr(d_n), S->rctl, eo, st);
    return cudaGetLastError() == cudaSuccess ? SMOL_OK : SMOL_ECUDA;
}

int smol_rhs(smol_system* S, const double* d_n, double* d_out) {
    if (!d_out) return SMOL_EINVAL;
    return rhs_common(S, d_n, d_out, nullptr, nullptr, nullptr);
}

int smol_rhs_terms(smol_system* S, const double* d_n, double* d_birth, double* d_loss, double* d_source) {
    return rhs_common(S, d_n, nullptr, d_birth, d_loss, d_source);
}

int smol_integrate_start(smol_system* S, double* d_n, double t0, double t1, double tol, int32_t scheme) {
    if (!S || !d_n || ((uintptr_t)d_n & 15)) return SMOL_EINVAL;
    if (!(t1 >= t0) || !isfinite(t0) || !isfinite(t1)) return SMOL_EINVAL;
    if (scheme < SMOL_RK2 || scheme > SMOL_RKF45) return SMOL_EINVAL;
    const bool fixed = S->o.fixed_tau > 0.0;
    if (!fixed && !(tol > 0.0)) return SMOL_EINVAL;
    const bool steady = S->o.steady_rtol > 0.0;
    cudaStream_t st = S->stream;

    Ctl h;
    memset(&h, 0, sizeof(h));
    h.t = t0;
    h.t1 = t1;
    h.tol = tol;
    h.tau = S->o.tau0 > 0.0 ? S->o.tau0 : (fixed ? S->o.fixed_tau : 0.0);
    h.state[0] = d_n;
    h.state[1] = S->stateB;
    // the pinned block may still be the target of an earlier read-back: wait for it
    CK(cudaStreamSynchronize(st));
    *S->h_ctl = h;
    CK(cudaMemcpyAsync(S->ctl, S->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    double* ppart = (double*)(S->ws + S->L.ppart);
    double* delta = (double*)(S->ws + S->L.delta);
    k_prep1<<<PREP_BLOCKS, 256, 0, st>>>(S->dev, S->ctl, ppart, delta);
    k_prep2<<<PREP_BLOCKS, 256, 0, st>>>(S->dev, S->ctl, delta, ppart, S->o.euler_a);
    CK(cudaGetLastError());

    // One CUDA graph holds `chunk` attempts (fewer if max_attempts is smaller); kernels
    // of attempts after termination return at once (they read ctl->done first).
    int64_t na = S->o.chunk;
    if (S->o.max_attempts < na) na = S->o.max_attempts;
    if (na < 1) na = 1;
    const int key = (int)na * 64 + scheme * 16 + (fixed ? 8 : 0) + (steady ? 4 : 0) +
                    (S->o.precision == SMOL_FP32CONV ? 2 : 0);
    if (S->gkey != key) {
        if (S->gexec) {
            cudaGraphExecDestroy(S->gexec);
            S->gexec = nullptr;
        }
        S->gkey = -1;
        CtlParams P = make_params(S, scheme, steady);
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(S->cap, cudaStreamCaptureModeThreadLocal));
        for (int64_t q = 0; q < na; ++q) enqueue_attempt(S, scheme, fixed, P, S->cap, nullptr);
        cudaError_t e1 = cudaStreamEndCapture(S->cap, &g);
        if (e1 != cudaSuccess) return SMOL_ECUDA;
        e1 = cudaGraphInstantiate(&S->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e1 != cudaSuccess) {
            S->gexec = nullptr;
            return SMOL_ECUDA;
        }
        S->gkey = key;
    }
    S->run_dn = d_n;
    S->run_scheme = scheme;
    S->run_attempts = na;
    return SMOL_OK;
}

int smol_integrate_advance(smol_system* S) {
    if (!S || !S->run_dn || !S->gexec) return SMOL_EINVAL;
    CK(cudaGraphLaunch(S->gexec, S->stream));
    return SMOL_OK;
}

int smol_integrate_finish(smol_system* S, smol_stats* stats) {
    if (!S || !S->run_dn) return SMOL_EINVAL;
    cudaStream_t st = S->stream;
    CK(cudaStreamSynchronize(st));
    Ctl fin;
    CK(cudaMemcpy(&fin, S->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    if (fin.cur == 1) {
        CK(cudaMemcpyAsync(S->run_dn, S->stateB, (size_t)S->s.M * 8, cudaMemcpyDeviceToDevice, st));
        CK(cudaStreamSynchronize(st));
        // the caller's buffer holds the state again: keep later advances consistent
        int zero = 0;
        CK(cudaMemcpy(&S->ctl->cur, &zero, sizeof(int), cudaMemcpyHostToDevice));
    }
    S->last_attempts = fin.attempts;
    if (stats) {
        stats->t = fin.t;
        stats->tau_next = fin.tau;
        stats->err_last = fin.err_last;
        stats->rhs_evals = fin.rhs_evals;
        stats->rhs_evals_paper = fin.rhs_paper;
        stats->accepted = fin.accepted;
        stats->rejected = fin.rejected;
        stats->attempts = fin.attempts;
        stats->status = fin.status;
        stats->reserved = 0;
    }
    return fin.status;
}

int smol_integrate(smol_system* S, double* d_n, double t0, double t1, double tol, int32_t scheme, smol_stats* stats) {
    int rc = smol_integrate_start(S, d_n, t0, t1, tol, scheme);
    if (rc != SMOL_OK) return rc;
    if (!(t1 > t0)) return smol_integrate_finish(S, stats);  // nothing to integrate
    cudaStream_t st = S->stream;
    // Launch chunks, keeping one in flight while the status of the previous one is read
    // from a pinned copy of the control block.
    cudaEvent_t ev[2];
    CK(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    Ctl* snap = S->h_ctl;
    const int64_t maxa = S->o.max_attempts;
    int64_t launched = S->run_attempts;  // attempts enqueued so far
    bool done = false;
    int cur = 0;
    if (cudaGraphLaunch(S->gexec, st) != cudaSuccess ||
        cudaMemcpyAsync(snap, S->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(ev[cur], st) != cudaSuccess)
        rc = SMOL_ECUDA;
    while (rc == SMOL_OK && !done && launched < maxa) {
        if (cudaGraphLaunch(S->gexec, st) != cudaSuccess) {
            rc = SMOL_ECUDA;
            break;
        }
        launched += S->run_attempts;
        if (cudaEventSynchronize(ev[cur]) != cudaSuccess) {
            rc = SMOL_ECUDA;
            break;
        }
        done = snap->done != 0;
        if (done) break;
        if (cudaMemcpyAsync(snap, S->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaEventRecord(ev[cur ^ 1], st) != cudaSuccess) {
            rc = SMOL_ECUDA;
            break;
        }
        cur ^= 1;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = SMOL_ECUDA;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc != SMOL_OK) return rc;
    return smol_integrate_finish(S, stats);
}

int smol_profile_attempts(smol_system* S, int32_t reps, double* kernel_ms, int64_t* kernel_launches, int32_t nkinds) {
    if (!S || !S->run_dn || reps < 1 || !kernel_ms || nkinds < SMOL_PROF_KINDS) return SMOL_EINVAL;
    cudaStream_t st = S->stream;
    Prof pr;
    memset(&pr, 0, sizeof(pr));
    for (int q = 0; q < PROF_MAX; ++q) {
        CK(cudaEventCreate(&pr.ev0[q]));
        CK(cudaEventCreate(&pr.ev1[q]));
    }
    const bool fixed = S->o.fixed_tau > 0.0;
    CtlParams P = make_params(S, S->run_scheme, S->o.steady_rtol > 0.0);
    double acc[SMOL_PROF_KINDS] = {0};
    int64_t cnt[SMOL_PROF_KINDS] = {0};
    int rc = SMOL_OK;
    for (int r = 0; r < reps && rc == SMOL_OK; ++r) {
        pr.n = 0;
        // ~0.5 ms of device work first, so that the whole attempt is enqueued before the
        // device reaches it and the events time the kernels, not the host launches
        k_delay<<<1, 32, 0, st>>>(1000000LL);
        enqueue_attempt(S, S->run_scheme, fixed, P, st, &pr);
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            rc = SMOL_ECUDA;
            break;
        }
        for (int q = 0; q < pr.n; ++q) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, pr.ev0[q], pr.ev1[q]) != cudaSuccess) {
                rc = SMOL_ECUDA;
                break;
            }
            acc[pr.kind[q]] += ms;
            cnt[pr.kind[q]] += 1;
        }
    }
    for (int q = 0; q < PROF_MAX; ++q) {
        cudaEventDestroy(pr.ev0[q]);
        cudaEventDestroy(pr.ev1[q]);
    }
    if (rc != SMOL_OK) return rc;
    for (int k = 0; k < SMOL_PROF_KINDS; ++k) {
        kernel_ms[k] = cnt[k] ? acc[k] / (double)cnt[k] : 0.0;
        if (kernel_launches) kernel_launches[k] = cnt[k];
    }
    return SMOL_OK;
}

int smol_get_log(smol_system* S, double* h_t, double* h_tau, double* h_err, int32_t* h_acc, int32_t cap, int64_t* count) {
    if (!S || cap < 0) return SMOL_EINVAL;
    const int64_t n = S->last_attempts;
    if (count) *count = n;
    const int lc = S->o.log_capacity;
    if (lc <= 0 || cap == 0 || n == 0) return SMOL_OK;
    const int64_t keep = n < lc ? n : lc;
    const int64_t take = keep < cap ? keep : cap;
    std::vector<double> t(lc), hh(lc), e(lc);
    std::vector<int32_t> a(lc);
    CK(cudaMemcpy(t.data(), S->ws + S->L.log_t, lc * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hh.data(), S->ws + S->L.log_h, lc * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(e.data(), S->ws + S->L.log_e, lc * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(a.data(), S->ws + S->L.log_a, lc * 4, cudaMemcpyDeviceToHost));
    for (int64_t q = 0; q < take; ++q) {
        const int64_t att = n - take + q;  // 0-based attempt index, oldest first
        const int64_t slot = att % lc;
        if (h_t) h_t[q] = t[slot];
        if (h_tau) h_tau[q] = hh[slot];
        if (h_err) h_err[q] = e[slot];
        if (h_acc) h_acc[q] = a[slot];
    }
    return SMOL_OK;
}

void smol_destroy(smol_system* S) {
    if (!S) return;
    if (S->gexec) cudaGraphExecDestroy(S->gexec);
    if (S->cap) cudaStreamDestroy(S->cap);
    if (S->h_ctl) cudaFreeHost(S->h_ctl);
    delete S;
}

const char* smol_strerror(int code) {
    switch (code) {
        case SMOL_OK: return "ok";
        case SMOL_STEADY: return "stopped at a steady state (||S(n)||/||n|| below steady_rtol)";
        case SMOL_EINVAL: return "invalid argument";
        case SMOL_ECUDA: return "CUDA runtime error";
        case SMOL_ENONFINITE: return "non-finite value in the error estimate or the state";
        case SMOL_ESTEP_UNDERFLOW: return "step size underflow";
        case SMOL_EMAXATTEMPTS: return "maximum number of step attempts reached";
        case SMOL_ETIMEOUT: return "a bounded device wait timed out";
        case SMOL_ENOSPACE: return "workspace too small";
        case SMOL_EUNSUPPORTED: return "shape not supported by the kernels";
        default: return "unknown status";
    }
}

}  // extern "C"
