// smol.cu - host side of the C interface declared in include/smol.h: set-up of one
// system or of a ragged batch of independent systems (distinct transforms, weights,
// twiddles, FFT schedule, workspace layout, block maps), one evaluation of S(n) as three
// kernel launches, and the device-resident adaptive integrators of Sec. 2 driven
// through captured CUDA graphs. A single system is a batch of one: the kernels of a
// launch span every system of the batch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "../../include/smol.h"
#include "smol_attr.h"
#include "smol_persist.cuh"

using namespace smol;

namespace {

constexpr int FIN_THREADS = 128;
constexpr int FIN_MAX_BLOCKS = 608;  // per system (4 x 152 SMs)
constexpr size_t SMEM_LIMIT = 227 * 1024;
constexpr int MAX_BATCH = 1 << 16;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ilog2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// FFT schedule of one system size: the four-step split Mp = N1 x N2 and the number G of
// adjacent columns per CTA of the column passes.
struct Shape {
    int M, Mp, lgMp, N1, N2, lgN1, lgN2, G, nfin;
    size_t csz, rsz;  // bytes of one complex / one real value of the compute type
};

// `wide`: the system is part of a batch large enough to fill the GPU on its own; its
// CTAs then take more work each (fewer, fuller CTAs: the per-CTA set-up is amortised and
// column stores fill whole 32-byte sectors), where a lone system wants many small CTAs.
// FFT schedule of one system. The rule: N1 = 2^ceil(lg Mp / 2) (column length), N2 =
// Mp / N1; one column of N1 >= 256 points per CTA, several short columns per CTA so
// that a CTA keeps at least 32 radix-8 butterflies per pass. lgn1 > 0 / g > 0 replace
// the rule's log2 N1 / columns per CTA (single systems; chosen by the autotuner).
Shape make_shape(int64_t M, int precision, bool wide = false, int lgn1 = 0, int g = 0) {
    Shape s;
    s.M = (int)M;
    s.lgMp = ilog2(M < 4 ? 4 : M);
    s.Mp = 1 << s.lgMp;
    s.lgN1 = (s.lgMp + 1) / 2;
    if (lgn1 > 0 && lgn1 < s.lgMp) s.lgN1 = lgn1;
    s.lgN2 = s.lgMp - s.lgN1;
    s.N1 = 1 << s.lgN1;
    s.N2 = 1 << s.lgN2;
    int G = 256 / s.N1;
    if (G < 1) G = 1;
    if (wide && G < 4) G = 4;
    if (g > 0) G = g;
    if (G > s.N2) G = s.N2;
    s.G = G;
    const int ppt = wide ? 8 : 1;  // element pairs per thread of the finish kernels
    int nf = (s.M / 2 + FIN_THREADS * ppt - 1) / (FIN_THREADS * ppt);
    s.nfin = std::max(1, std::min(nf, FIN_MAX_BLOCKS));
    s.csz = precision == SMOL_FP32CONV ? 8 : 16;
    s.rsz = s.csz / 2;
    return s;
}

// Shape of system q of an engine of `count` systems: a single system takes fft_lgn1 /
// fft_g, a batch its size class's entry of batch_lgn1 / batch_g (0: the rule).
Shape engine_shape(int count, int64_t M, const smol_opts& o, bool wide) {
    if (count == 1) return make_shape(M, o.precision, false, o.fft_lgn1, o.fft_g);
    const int k = ilog2(M < 4 ? 4 : M);
    const int lg = k < SMOL_SIZE_CLASSES ? o.batch_lgn1[k] : 0;
    const int g = k < SMOL_SIZE_CLASSES ? o.batch_g[k] : 0;
    return make_shape(M, o.precision, wide, lg, g);
}

// Dynamic shared memory of the column kernels (the larger of the forward pass: T*G
// interleaved sequences, tile and four-step twiddles, y; and the inverse pass) and of
// the row kernel (2T rows, tile twiddles, spectral and inverse four-step twiddles).
size_t smem_cols(const Shape& s, int T) {
    const size_t n = (size_t)s.N1 * s.G;
    const size_t fwd = 2 * n * T * s.csz + (size_t)s.N1 * s.csz + n * s.csz + n * s.rsz;
    const size_t inv = 2 * n * s.csz + (size_t)s.N1 * s.csz;
    return std::max(fwd, inv);
}
// (at least the scalar CTA's 4 MAXT + 1 doubles)
size_t smem_rows(const Shape& s, int T) {
    return std::max<size_t>(2 * (size_t)s.N2 * 2 * T * s.csz + 5 * (size_t)s.N2 * s.csz, (4 * MAXT + 1) * 8);
}

// Threads of a CTA whose passes cover `points` points: one per radix-8 butterfly,
// between 32 and cap.
int threads_for(int points, int cap = 256) {
    int t = points / 8;
    if (t > cap) t = cap;
    if (t < 32) t = 32;
    return (t + 31) & ~31;
}

// Per-system part of the workspace.
struct Layout {
    size_t tw, twc, twr, tws, W, Y, G2, ybuf, vec, half, stateB, mpart, fpart, sqpart, aux, rsc, shadow, log_t, log_h,
        log_e, log_a, total;
    size_t vstride;  // elements between work vectors
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
    L.tw = take((size_t)s.Mp * s.csz);
    L.twc = take((size_t)s.Mp * s.csz);
    L.twr = take((size_t)s.Mp * s.csz);
    L.tws = take((size_t)s.Mp * s.csz);
    L.W = take((size_t)Tm * s.Mp * s.rsz);
    L.Y = take((size_t)Tm * s.Mp * s.csz);
    L.G2 = take((size_t)s.Mp * s.csz);
    L.ybuf = take((size_t)s.Mp * s.rsz);
    L.vstride = align256((size_t)s.Mp * s.rsz) / s.rsz;
    L.vec = take((size_t)NVEC * L.vstride * s.rsz);
    L.half = take((size_t)s.Mp * 8);
    L.stateB = take((size_t)s.Mp * 8);
    L.mpart = take((size_t)Tm * s.N2 * 2 * 8);  // sized for G = 1 (G may shrink at init)
    L.fpart = take((size_t)std::max(s.nfin, s.N2) * FPW * 8);  // finish CTAs or column CTAs
    L.sqpart = take((size_t)s.N2 * 8);
    L.aux = take((size_t)(MAXT + 1) * 8);
    L.rsc = take((size_t)(MAXT + 2) * 8 + 2 * MAXT * 4);
    L.shadow = take(2 * align256((size_t)s.Mp * s.rsz));
    L.log_t = take((size_t)log_cap * 8);
    L.log_h = take((size_t)log_cap * 8);
    L.log_e = take((size_t)log_cap * 8);
    L.log_a = take((size_t)log_cap * 4);
    L.total = o;
    return L;
}

// Header of a batch workspace: control blocks, descriptors and block maps.
struct Header {
    size_t ctl, rctl, sys, sysr, mapC, mapB, mapF, bar, total;
    int nC, nB, nF;  // blocks of the column / row / finish launches
};

Header make_header(const std::vector<Shape>& sh) {
    Header H;
    const size_t n = sh.size();
    H.nC = H.nB = H.nF = 0;
    for (const Shape& s : sh) {
        H.nC += s.N2;  // room for G = 1; the launch count is set from the final maps
        H.nB += s.N1 / 2 + 1;  // row pairs and the scalar CTA
        H.nF += s.nfin;
    }
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += align256(bytes);
        return r;
    };
    H.ctl = take(n * sizeof(Ctl));
    H.rctl = take(n * sizeof(Ctl));
    H.sys = take(n * sizeof(SysDev));
    H.sysr = take(n * sizeof(SysDev));
    H.mapC = take((size_t)H.nC * sizeof(int2));
    H.mapB = take((size_t)H.nB * sizeof(int2));
    H.mapF = take((size_t)H.nF * sizeof(int2));
    H.bar = take(2 * BAR_GEN * sizeof(unsigned));  // grid barrier of the persistent attempt kernel
    H.total = o;
    return H;
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

static_assert(MAXR == SMOL_MAX_R, "rank limit of the C interface and the kernels");

// Largest M whose rule shape fits T distinct transforms in shared memory.
int64_t max_m_transforms(int32_t T, int32_t precision) {
    if (T < 1 || T > MAXT) return 0;
    int64_t best = 0;
    for (int lg = 2; lg <= 22; ++lg) {
        Shape s = make_shape((int64_t)1 << lg, precision);
        if (smem_cols(s, T) <= SMEM_LIMIT && smem_rows(s, T) <= SMEM_LIMIT) best = (int64_t)1 << lg;
    }
    return best;
}

// Largest M for rank R with no shared transforms (T = 2R).
int64_t max_m_for(int32_t R, int32_t precision) {
    if (R < 1 || R > MAXR) return 0;
    return max_m_transforms(2 * R, precision);
}

// A batch counts as wide when its systems together hold more than 2^20 sizes.
bool is_wide(int count, const int64_t* M) {
    int64_t tot = 0;
    for (int q = 0; q < count; ++q) tot += M[q];
    return count > 1 && tot > ((int64_t)1 << 20);
}

size_t batch_bytes(int count, const int64_t* M, int R, const smol_opts& o) {
    if (count < 1 || count > MAX_BATCH || R < 1 || R > MAXR) return 0;
    // the factors' actual T (<= 2R) is known only at init, which refuses shapes that do
    // not fit; here any M that fits with one transform
    const int64_t mm = max_m_transforms(1, o.precision);
    std::vector<Shape> sh;
    size_t tot = 0;
    const bool wide = is_wide(count, M);
    for (int q = 0; q < count; ++q) {
        if (M[q] < 1 || M[q] > mm) return 0;
        sh.push_back(engine_shape(count, M[q], o, wide));
        tot += make_layout(sh.back(), R, std::max(o.log_capacity, 0)).total;
    }
    return make_header(sh).total + tot;
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

}  // namespace

// The engine behind both opaque handles: a batch of `count` systems (count = 1 for
// smol_system).
struct Engine {
    int count = 0, R = 0;
    smol_opts o{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only for graph capture
    char* ws = nullptr;
    Header H{};
    std::vector<Shape> sh;
    std::vector<Layout> lay;
    std::vector<size_t> base;  // byte offset of each system's region
    std::vector<int> T;
    SysDev* d_sys = nullptr;   // descriptors used by integrations (control blocks ctl)
    SysDev* d_sysr = nullptr;  // descriptors of standalone evaluations (control blocks rctl)
    SysDev h_one{}, h_oner{};  // host copies for single-system launches (passed by value)
    std::vector<SysDev> hs, hsr;  // host copies of every system's descriptors
    Ctl* d_ctl = nullptr;
    Ctl* d_rctl = nullptr;
    int2 *mapC = nullptr, *mapB = nullptr, *mapF = nullptr;
    size_t smemC = 0, smemB = 0;
    int thrC = 32, thrB = 32;
    int thrCW = 32;  // column CTAs with SMOL_FLAG_WIDE_COLS (single system)
    Ctl* h_ctl = nullptr;  // pinned host copies of the control blocks
    cudaEvent_t ev_rb[2] = {nullptr, nullptr};  // completions of read-backs into h_ctl
    cudaEvent_t ev_hctl = nullptr;  // the last stream operation that reads or writes h_ctl
    cudaGraphExec_t gexec = nullptr;
    int64_t gkey = -1;
    std::vector<int64_t> last_attempts;
    bool running = false;
    int run_scheme = 0;
    int64_t run_attempts = 1;
    std::vector<double*> run_dn;
    std::vector<double> tau0;  // per system: first step of the next integration (<= 0: opts.tau0)
    // persistent attempt kernel (single system, RKF45, SMOL_FLAG_PERSISTENT)
    unsigned* d_bar = nullptr;
    bool persist_run = false;
    const void* pkern = nullptr;
    int pgrid = 0, pblock = 0;
    size_t psmem = 0;
    PersistPlan plan{};
};

struct smol_system : Engine {};
struct smol_batch : Engine {};

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
namespace {

// Every kernel of an attempt asks for the same (largest) shared-memory carveout: with
// programmatic dependent launch the next kernel's CTAs are placed on SMs while the
// previous kernel still runs there, and an SM whose L1 / shared split would have to
// change cannot take them, which crowds the early CTAs onto few SMs.
template <typename K>
bool carve(K k) {
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared) == cudaSuccess;
}

// The limits only rise (smol_attr.h): a smaller system created later must not lower the
// limit a larger live system (or the no-allocation entry point) launches with.
template <typename R>
int set_smem_attrs(const Engine* E) {
    using smol_host::raise_smem;
    const int sc = (int)E->smemC, sb = (int)E->smemB;
    if (raise_smem(k_fwd_cols<R>, sc) != cudaSuccess || raise_smem(k_inv_cols<R>, sc) != cudaSuccess ||
        raise_smem(k_inv_fwd<R>, sc) != cudaSuccess || raise_smem(k_inv_finish<R>, sc) != cudaSuccess ||
        raise_smem(k_rows<R>, sb) != cudaSuccess)
        return SMOL_ECUDA;
    if (!(carve(k_fwd_cols<R>) && carve(k_rows<R>) && carve(k_inv_cols<R>) && carve(k_inv_fwd<R>) &&
          carve(k_inv_finish<R>) && carve(k_finish<R>) && carve(k_lincomb<R>) && carve(k_persist<R>)))
        return SMOL_ECUDA;
    if (E->count == 1 && raise_smem(k_persist<R>, std::max(sc, sb)) != cudaSuccess) return SMOL_ECUDA;
    return SMOL_OK;
}

// Descriptor arguments of a launch: a single system passes its descriptor by value and
// no map; a batch passes the device array and the block maps.
struct LaunchArgs {
    const SysDev* sys;
    const int2 *mapC, *mapB, *mapF;
    SysDev one;
};

LaunchArgs args_for(const Engine* E, bool rhs) {
    LaunchArgs a;
    a.sys = rhs ? E->d_sysr : E->d_sys;
    if (E->count == 1) {
        a.mapC = a.mapB = a.mapF = nullptr;
        a.one = rhs ? E->h_oner : E->h_one;
    } else {
        a.mapC = E->mapC;
        a.mapB = E->mapB;
        a.mapF = E->mapF;
        memset(&a.one, 0, sizeof(a.one));
    }
    return a;
}

// Launches kernel k with programmatic stream serialisation (the kernel may start while
// its predecessor in the stream runs; it waits for it in griddep_wait) unless the
// options disable it.
template <typename... KArgs, typename... Args>
void launch(const Engine* E, int kind, void (*k)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
            Args&&... args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = (E->o.flags & (SMOL_FLAG_NO_PDL | (SMOL_FLAG_NO_PDL_FWD_COLS << kind))) ? 0 : 1;
    cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Threads of the column CTAs of this engine's launches.
int col_threads(const Engine* E) {
    return ((E->o.flags & SMOL_FLAG_WIDE_COLS) && E->count == 1) ? E->thrCW : E->thrC;
}

template <typename R>
void launch_eval(const Engine* E, const LaunchArgs& A, const StageIn& in, const EpiOut& eo, cudaStream_t st,
                 Prof* pr) {
    {
        ProfScope ps(pr, st, SMOL_PROF_FWD_COLS);
        launch(E, SMOL_PROF_FWD_COLS, k_fwd_cols<R>, E->H.nC, col_threads(E), E->smemC, st, A.sys, A.mapC, A.one, in);
    }
    {
        ProfScope ps(pr, st, SMOL_PROF_ROWS);
        launch(E, SMOL_PROF_ROWS, k_rows<R>, E->H.nB, E->thrB, E->smemB, st, A.sys, A.mapB, A.one, in);
    }
    {
        ProfScope ps(pr, st, SMOL_PROF_INV_COLS);
        launch(E, SMOL_PROF_INV_COLS, k_inv_cols<R>, E->H.nC, col_threads(E), E->smemC, st, A.sys, A.mapC, A.one, in, eo);
    }
}

// Emits the kernels of an attempt. Consecutive evaluations share a column kernel: the
// inverse pass of one and the forward pass of the next run in k_inv_fwd, and the last
// inverse pass runs with the final combination in k_inv_finish (unless the options
// disable fusion). A half-step combination (k_lincomb) between two evaluations ends a
// fused chain.
template <typename R>
struct Seq {
    const Engine* E;
    LaunchArgs A;
    cudaStream_t st;
    Prof* pr;
    bool fuse;
    bool pending = false;  // an evaluation whose inverse pass is not yet launched
    StageIn pin;
    EpiOut peo;

    void eval(const StageIn& in, const EpiOut& eo) {
        if (pending && fuse) {
            ProfScope ps(pr, st, SMOL_PROF_INV_FWD);
            launch(E, SMOL_PROF_INV_COLS, k_inv_fwd<R>, E->H.nC, col_threads(E), E->smemC, st, A.sys, A.mapC, A.one, pin, peo,
                   in);
        } else {
            flush();
            ProfScope ps(pr, st, SMOL_PROF_FWD_COLS);
            launch(E, SMOL_PROF_FWD_COLS, k_fwd_cols<R>, E->H.nC, col_threads(E), E->smemC, st, A.sys, A.mapC, A.one, in);
        }
        {
            ProfScope ps(pr, st, SMOL_PROF_ROWS);
            launch(E, SMOL_PROF_ROWS, k_rows<R>, E->H.nB, E->thrB, E->smemB, st, A.sys, A.mapB, A.one, in);
        }
        pending = true;
        pin = in;
        peo = eo;
    }
    void finish(const Comb2& c, const CtlParams& P) {
        if (pending && fuse) {
            ProfScope ps(pr, st, SMOL_PROF_INV_STEP);
            launch(E, SMOL_PROF_STEP, k_inv_finish<R>, E->H.nC, col_threads(E), E->smemC, st, A.sys, A.mapC, A.one, pin, peo,
                   c, P);
            pending = false;
            return;
        }
        flush();
        ProfScope ps(pr, st, SMOL_PROF_STEP);
        launch(E, SMOL_PROF_STEP, k_finish<R>, E->H.nF, FIN_THREADS, 0, st, A.sys, A.mapF, A.one, c, P);
    }
    void lincomb(const StageIn& in) {
        flush();
        ProfScope ps(pr, st, SMOL_PROF_STEP);
        launch(E, SMOL_PROF_STEP, k_lincomb<R>, E->H.nF, FIN_THREADS, 0, st, A.sys, A.mapF, A.one, in);
    }
    void flush() {
        if (!pending) return;
        ProfScope ps(pr, st, SMOL_PROF_INV_COLS);
        launch(E, SMOL_PROF_INV_COLS, k_inv_cols<R>, E->H.nC, col_threads(E), E->smemC, st, A.sys, A.mapC, A.one, pin, peo);
        pending = false;
    }
};

// Union of the candidate and error combinations of the final kernel.
Comb2 comb2(const StageIn& cand, const StageIn& del) {
    Comb2 c;
    memset(&c, 0, sizeof(c));
    auto add = [&](int slot, double cc, double dd) {
        for (int j = 0; j < c.in.nv; ++j)
            if (c.in.slot[j] == slot) {
                c.in.c[j] += cc;
                c.d[j] += dd;
                return;
            }
        const int j = c.in.nv++;
        c.in.slot[j] = slot;
        c.in.c[j] = cc;
        c.d[j] = dd;
    };
    for (int j = 0; j < cand.nv; ++j) add(cand.slot[j], cand.c[j], 0.0);
    for (int j = 0; j < del.nv; ++j) add(del.slot[j], 0.0, del.c[j]);
    for (int j = 0; j < c.in.nv; ++j) {
        c.ch[j] = (float)c.in.c[j];
        c.cl[j] = (float)(c.in.c[j] - (double)c.ch[j]);
        c.dh[j] = (float)c.d[j];
        c.dl[j] = (float)(c.d[j] - (double)c.dh[j]);
    }
    return c;
}

StageIn stage(std::initializer_list<std::pair<int, double>> terms) {
    // term index: SLOT_* (< 0) or a work vector k >= 0
    StageIn in;
    memset(&in, 0, sizeof(in));
    for (auto& tc : terms) {
        const int j = in.nv++;
        in.slot[j] = tc.first;
        in.c[j] = tc.second;
        in.cf[j] = (float)tc.second;
        in.cl[j] = (float)(tc.second - (double)in.cf[j]);
    }
    return in;
}

EpiOut epi_k(int slot, double hfac, int sq) {
    EpiOut e;
    memset(&e, 0, sizeof(e));
    e.out_slot = slot;
    e.hfac = hfac;
    e.sq = sq;
    return e;
}

// The RKF45 attempt of Sec. 2: stage inputs n + sum_j a_ij k_j (k_j = h S), the fourth-
// order candidate and the difference of the two weight rows of the tableau (the error).
void rkf45_stages(StageIn in[6], StageIn& cand, StageIn& del) {
    const int N = SLOT_CUR;
    in[0] = stage({{N, 1.0}});
    in[1] = stage({{N, 1.0}, {0, 0.25}});
    in[2] = stage({{N, 1.0}, {0, 3.0 / 32.0}, {1, 9.0 / 32.0}});
    in[3] = stage({{N, 1.0}, {0, 1932.0 / 2197.0}, {1, -7200.0 / 2197.0}, {2, 7296.0 / 2197.0}});
    in[4] = stage({{N, 1.0}, {0, 439.0 / 216.0}, {1, -8.0}, {2, 3680.0 / 513.0}, {3, -845.0 / 4104.0}});
    in[5] = stage({{N, 1.0}, {0, -8.0 / 27.0}, {1, 2.0}, {2, -3544.0 / 2565.0}, {3, 1859.0 / 4104.0}, {4, -11.0 / 40.0}});
    cand = stage({{N, 1.0}, {0, 25.0 / 216.0}, {2, 1408.0 / 2565.0}, {3, 2197.0 / 4104.0}, {4, -1.0 / 5.0}});
    del = stage({{0, 16.0 / 135.0 - 25.0 / 216.0},
                 {2, 6656.0 / 12825.0 - 1408.0 / 2565.0},
                 {3, 28561.0 / 56430.0 - 2197.0 / 4104.0},
                 {4, -9.0 / 50.0 + 1.0 / 5.0},
                 {5, 2.0 / 55.0}});
}

// A stage input as the kernels of form R take it: the first evaluation of an attempt is
// marked (a retry reuses it), and the FP32 / double-float forms read the state's shadow.
template <typename R>
StageIn stage_for(StageIn in, bool first) {
    in.first = first ? 1 : 0;
    if (Tr<R>::shadowed)
        for (int j = 0; j < in.nv; ++j)
            if (in.slot[j] == SLOT_CUR) in.slot[j] = SLOT_CURF;
    return in;
}

// The persistent kernel's plan of one RKF45 attempt (the graph path's sequence).
template <typename R>
PersistPlan make_plan(const CtlParams& P) {
    PersistPlan pl;
    memset(&pl, 0, sizeof(pl));
    StageIn in[6], cand, del;
    rkf45_stages(in, cand, del);
    for (int i = 0; i < 6; ++i) {
        pl.in[i] = stage_for<R>(in[i], i == 0);
        pl.eo[i] = epi_k(i, 1.0, (i == 0 && P.steady) ? 1 : 0);
    }
    pl.fin = comb2(cand, del);
    pl.P = P;
    return pl;
}

// Enqueues one step attempt of every system of the batch on stream st.
template <typename R>
void enqueue_attempt(Engine* E, int scheme, bool fixed, const CtlParams& P, cudaStream_t st, Prof* pr) {
    Seq<R> q;
    q.E = E;
    q.A = args_for(E, false);
    q.st = st;
    q.pr = pr;
    q.fuse = !(E->o.flags & SMOL_FLAG_NO_FUSE);
    auto Ev = [&](StageIn in, int k, double hfac, bool first) {
        // S(n^k) (first) is reused by the retry of a rejected attempt
        q.eval(stage_for<R>(in, first), epi_k(k, hfac, (first && P.steady) ? 1 : 0));
    };
    auto finish = [&](const StageIn& cand, const StageIn& del) { q.finish(comb2(cand, del), P); };
    auto half = [&](const StageIn& in) { q.lincomb(in); };
    const int N = SLOT_CUR, H = SLOT_HALF;
    if (scheme == SCHEME_RKF45) {
        StageIn in[6], cand, del;
        rkf45_stages(in, cand, del);
        for (int i = 0; i < 6; ++i) Ev(in[i], i, 1.0, i == 0);
        finish(cand, del);
        return;
    }
    if (scheme == SCHEME_RK2) {
        Ev(stage({{N, 1.0}}), 0, 1.0, true);            // k1 = h S(n)
        Ev(stage({{N, 1.0}, {0, 1.0}}), 1, 1.0, false);  // k2 = h S(n + k1)
        if (fixed) {
            finish(stage({{N, 1.0}, {0, 0.5}, {1, 0.5}}), stage({{0, 0.0}}));
            return;
        }
        // half step 1: l1 = k1/2, l2 = (h/2) S(n + k1/2); n_half = n + (l1 + l2)/2
        Ev(stage({{N, 1.0}, {0, 0.5}}), 2, 0.5, false);
        half(stage({{N, 1.0}, {0, 0.25}, {2, 0.5}}));
        // half step 2 from n_half: m1, m2; error n_hat - n^{k+1}
        Ev(stage({{H, 1.0}}), 4, 0.5, false);
        Ev(stage({{H, 1.0}, {4, 1.0}}), 5, 0.5, false);
        finish(stage({{H, 1.0}, {4, 0.5}, {5, 0.5}}),
               stage({{H, 1.0}, {4, 0.5}, {5, 0.5}, {N, -1.0}, {0, -0.5}, {1, -0.5}}));
        return;
    }
    // RK4
    Ev(stage({{N, 1.0}}), 0, 1.0, true);            // k1
    Ev(stage({{N, 1.0}, {0, 0.5}}), 1, 1.0, false);  // k2
    Ev(stage({{N, 1.0}, {1, 0.5}}), 2, 1.0, false);  // k3
    Ev(stage({{N, 1.0}, {2, 1.0}}), 3, 1.0, false);  // k4
    if (fixed) {
        finish(stage({{N, 1.0}, {0, 1.0 / 6.0}, {1, 1.0 / 3.0}, {2, 1.0 / 3.0}, {3, 1.0 / 6.0}}), stage({{0, 0.0}}));
        return;
    }
    // half step 1 with h/2: l1 = k1/2
    Ev(stage({{N, 1.0}, {0, 0.25}}), 4, 0.5, false);  // l2 = (h/2) S(n + l1/2)
    Ev(stage({{N, 1.0}, {4, 0.5}}), 5, 0.5, false);   // l3
    Ev(stage({{N, 1.0}, {5, 1.0}}), 6, 0.5, false);   // l4
    half(stage({{N, 1.0}, {0, 1.0 / 12.0}, {4, 1.0 / 3.0}, {5, 1.0 / 3.0}, {6, 1.0 / 6.0}}));
    Ev(stage({{H, 1.0}}), 8, 0.5, false);              // m1
    Ev(stage({{H, 1.0}, {8, 0.5}}), 9, 0.5, false);    // m2
    Ev(stage({{H, 1.0}, {9, 0.5}}), 10, 0.5, false);   // m3
    Ev(stage({{H, 1.0}, {10, 1.0}}), 11, 0.5, false);  // m4
    // n_hat and n_hat - n^{k+1} (the full step of length h)
    finish(stage({{H, 1.0}, {8, 1.0 / 6.0}, {9, 1.0 / 3.0}, {10, 1.0 / 3.0}, {11, 1.0 / 6.0}}),
           stage({{H, 1.0},
                  {8, 1.0 / 6.0},
                  {9, 1.0 / 3.0},
                  {10, 1.0 / 3.0},
                  {11, 1.0 / 6.0},
                  {N, -1.0},
                  {0, -1.0 / 6.0},
                  {1, -1.0 / 3.0},
                  {2, -1.0 / 3.0},
                  {3, -1.0 / 6.0}}));
}

CtlParams make_params(const Engine* E, int scheme) {
    CtlParams P;
    memset(&P, 0, sizeof(P));
    const bool fixed = E->o.fixed_tau > 0.0;
    P.scheme = scheme;
    P.ctrl = E->o.ctrl;
    P.rel_norm = E->o.norm == SMOL_NORM_REL;
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
    P.tau_min_rel = E->o.tau_min_rel;
    P.steady_rtol = E->o.steady_rtol;
    P.steady = E->o.steady_rtol > 0.0;
    P.fac_min = E->o.fac_min;
    P.fac_max = E->o.fac_max;
    P.max_attempts = E->o.max_attempts;
    P.log_cap = E->o.log_capacity;
    return P;
}

void enqueue_attempt_any(Engine* E, int scheme, bool fixed, const CtlParams& P, cudaStream_t st, Prof* pr) {
    if (E->o.precision == SMOL_FP32CONV) enqueue_attempt<float>(E, scheme, fixed, P, st, pr);
    else if (E->o.precision == SMOL_DF64) enqueue_attempt<dd>(E, scheme, fixed, P, st, pr);
    else enqueue_attempt<double>(E, scheme, fixed, P, st, pr);
}

#define CK(x)                                      \
    do {                                           \
        if ((x) != cudaSuccess) return SMOL_ECUDA; \
    } while (0)

template <typename R>
void to_type(const std::vector<double>& src, std::vector<unsigned char>& dst) {
    dst.resize(src.size() * sizeof(R));
    R* p = reinterpret_cast<R*>(dst.data());
    for (size_t q = 0; q < src.size(); ++q) p[q] = (R)src[q];
}

// Builds the engine: per system the distinct transforms of U and V, the weights and
// twiddles, the descriptor; then the block maps; uploads everything.
int engine_init(Engine* E, int count, const int64_t* Ms, int R, const double* const* hU, const double* const* hV,
                const double* lam, const smol_opts& o, void* d_ws, size_t ws_bytes) {
    E->count = count;
    E->R = R;
    E->o = o;
    if (E->o.chunk == 0) E->o.chunk = 32;
    E->stream = (cudaStream_t)o.stream;
    E->ws = (char*)d_ws;
    const int prec = o.precision;
    const int logc = std::max(o.log_capacity, 0);
    const bool wide = is_wide(count, Ms);
    for (int q = 0; q < count; ++q) {
        E->sh.push_back(engine_shape(count, Ms[q], o, wide));
        E->lay.push_back(make_layout(E->sh.back(), R, logc));
    }
    E->H = make_header(E->sh);
    size_t off = E->H.total;
    for (int q = 0; q < count; ++q) {
        E->base.push_back(off);
        off += E->lay[q].total;
    }
    if (off > ws_bytes) return SMOL_ENOSPACE;
    char* ws = E->ws;
    E->d_ctl = (Ctl*)(ws + E->H.ctl);
    E->d_rctl = (Ctl*)(ws + E->H.rctl);
    E->d_sys = (SysDev*)(ws + E->H.sys);
    E->d_sysr = (SysDev*)(ws + E->H.sysr);
    E->mapC = (int2*)(ws + E->H.mapC);
    E->mapB = (int2*)(ws + E->H.mapB);
    E->mapF = (int2*)(ws + E->H.mapF);
    E->d_bar = (unsigned*)(ws + E->H.bar);
    E->last_attempts.assign(count, 0);
    cudaStream_t st = E->stream;
    std::vector<SysDev> hs(count), hsr(count);
    std::vector<int2> mC, mB, mF;
    std::vector<std::pair<int, std::vector<double>>> twcache;  // twiddles per FFT size
    for (int q = 0; q < count; ++q) {
        const Shape& s = E->sh[q];
        const Layout& L = E->lay[q];
        const int Mi = s.M;
        const double* U = hU[q];
        const double* V = hV[q];
        if (!U || !V || !(lam[q] >= 0.0)) return SMOL_EINVAL;
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
                ucol[i] = U[(size_t)i * R + al];
                vrow[i] = V[(size_t)al * Mi + i];
                uz = uz && ucol[i] == 0.0;
                vz = vz && vrow[i] == 0.0;
                if (!isfinite(ucol[i]) || !isfinite(vrow[i])) return SMOL_EINVAL;
            }
            if (uz || vz) continue;  // the term vanishes
            double cu, cv;
            const int u = find_or_add(ucol, &cu);
            const int v = find_or_add(vrow, &cv);
            au.push_back(u);
            av.push_back(v);
            acoef.push_back(cu * cv);
        }
        if (W.empty()) {  // K == 0: one zero transform keeps every path well formed
            W.push_back(std::vector<double>(Mi, 0.0));
            au.push_back(0);
            av.push_back(0);
            acoef.push_back(0.0);
        }
        const int T = (int)W.size();
        E->T.push_back(T);
        Shape& sm = E->sh[q];
        while (smem_cols(sm, T) > SMEM_LIMIT && sm.G > 1) sm.G /= 2;  // wide shapes may not fit
        if (smem_rows(s, T) > SMEM_LIMIT || smem_cols(s, T) > SMEM_LIMIT) return SMOL_EUNSUPPORTED;
        E->smemC = std::max(E->smemC, smem_cols(s, T));
        E->smemB = std::max(E->smemB, smem_rows(s, T));
        // one thread per radix-8 butterfly of the column tiles, and at least one per
        // stage-input pair (so that all stage-input loads of a CTA are in flight at once)
        E->thrC = std::max(E->thrC, std::max(threads_for(s.N1 * s.G * T), std::min(256, (s.N1 * s.G / 2 + 31) & ~31)));
        // wide column CTAs: one thread per element pair (the per-pair phases of the
        // column kernels are chains of dependent FP64 operations, which more warps hide)
        const int wmax = o.precision == SMOL_FP32CONV ? 256 : COL_THREADS_MAX;  // the kernels' launch bounds
        E->thrCW = std::max(E->thrCW, std::max(threads_for(s.N1 * s.G * T, wmax), std::min(wmax, (s.N1 * s.G / 2 + 31) & ~31)));
        E->thrB = std::max(E->thrB, threads_for(s.N2 * 2 * T));
        char* b = ws + E->base[q];
        SysDev& d = hs[q];
        memset(&d, 0, sizeof(d));
        d.M = Mi;
        d.Mp = s.Mp;
        d.lgMp = s.lgMp;
        d.N1 = s.N1;
        d.N2 = s.N2;
        d.lgN1 = s.lgN1;
        d.lgN2 = s.lgN2;
        d.G = s.G;
        d.T = T;
        d.R = (int)au.size();
        d.nbx = s.N2 / s.G;
        d.lambda = lam[q];
        d.W = b + L.W;
        d.tw = b + L.tw;
        d.twc = b + L.twc;
        d.twr = b + L.twr;
        d.tws = b + L.tws;
        d.Y = b + L.Y;
        d.G2 = b + L.G2;
        d.ybuf = b + L.ybuf;
        d.vec = b + L.vec;
        d.half = (double*)(b + L.half);
        d.mpart = (double*)(b + L.mpart);
        d.fpart = (double*)(b + L.fpart);
        d.sqpart = (double*)(b + L.sqpart);
        d.aux = (double*)(b + L.aux);
        d.rsc = (double*)(b + L.rsc);
        if (prec != SMOL_FP64) {  // R-typed shadows of the state buffers
            d.shadow0 = b + L.shadow;
            d.shadow1 = b + L.shadow + align256((size_t)s.Mp * s.rsz);
        }
        d.log_t = (double*)(b + L.log_t);
        d.log_h = (double*)(b + L.log_h);
        d.log_e = (double*)(b + L.log_e);
        d.log_a = (int32_t*)(b + L.log_a);
        d.vstride = (int64_t)L.vstride;
        d.nfin = s.nfin;
        d.bnorm = 0.5 / (double)s.Mp;
        for (int al = 0; al < d.R; ++al) {
            d.au[al] = au[al];
            d.av[al] = av[al];
            d.acoef[al] = acoef[al];
        }
        // unordered pairs for the spectral product: (u,v) and (v,u) give the same product
        d.npairs = 0;
        for (int al = 0; al < d.R; ++al) {
            int a = au[al], c = av[al];
            if (a > c) std::swap(a, c);
            int p = 0;
            for (; p < d.npairs; ++p)
                if (d.pu[p] == a && d.pv[p] == c) break;
            if (p == d.npairs) {
                d.pu[p] = a;
                d.pv[p] = c;
                d.pcoef[p] = 0.0;
                d.npairs++;
            }
            d.pcoef[p] += acoef[al];
        }
        for (int t = 0; t < T; ++t) {
            double mx = 0.0;
            for (int i = 0; i < Mi; ++i) mx = fmax(mx, fabs(W[t][i]));
            d.wexp[t] = mx > 0.0 ? ilogb(mx) : 0;
        }
        d.ctl = E->d_ctl + q;
        hsr[q] = d;
        hsr[q].ctl = E->d_rctl + q;
        for (int c = 0; c < s.N2 / s.G; ++c) mC.push_back(make_int2(q, c));
        for (int c = 0; c <= s.N1 / 2; ++c) mB.push_back(make_int2(q, c));  // 0: scalar CTA
        for (int c = 0; c < s.nfin; ++c) mF.push_back(make_int2(q, c));

        // Host images of the tables: weights (zero beyond M) and twiddles
        // W_{2Mp}^e = exp(-i pi e / Mp), e < Mp, in extended precision.
        std::vector<double> hW((size_t)T * s.Mp, 0.0);
        for (int t = 0; t < T; ++t)
            for (int i = 0; i < Mi; ++i) hW[(size_t)t * s.Mp + i] = W[t][i];
        const std::vector<double>* twp = nullptr;
        for (auto& c : twcache)
            if (c.first == s.Mp) twp = &c.second;
        if (!twp) {
            std::vector<double> tw64(2 * (size_t)s.Mp);
            for (int e = 0; e < s.Mp; ++e) {
                const long double th = 3.141592653589793238462643383279502884L * (long double)e / (long double)s.Mp;
                tw64[2 * e] = (double)cosl(th);
                tw64[2 * e + 1] = (double)-sinl(th);
            }
            twcache.emplace_back(s.Mp, std::move(tw64));
            twp = &twcache.back().second;
        }
        const std::vector<double>& tw64 = *twp;
        // four-step and spectral twiddles in the layouts the kernels read contiguously:
        //   twc[n2][k1] = W_Mp^{n2 k1} = W_{2Mp}^{2 n2 k1 mod 2Mp}, twr[k1][n2] = its conjugate,
        //   tws[k1][k2] = W_{2Mp}^{k1 + N1 k2}
        std::vector<double> twc((size_t)2 * s.Mp), twr((size_t)2 * s.Mp), tws((size_t)2 * s.Mp);
        auto wv = [&](uint64_t e, double* re, double* im) {  // W_{2Mp}^e, any e
            e %= 2 * (uint64_t)s.Mp;
            const double sgn = e >= (uint64_t)s.Mp ? -1.0 : 1.0;
            if (e >= (uint64_t)s.Mp) e -= s.Mp;
            *re = sgn * tw64[2 * e];
            *im = sgn * tw64[2 * e + 1];
        };
        for (int n2 = 0; n2 < s.N2; ++n2)
            for (int k1 = 0; k1 < s.N1; ++k1) {
                double re, im;
                wv(2 * (uint64_t)n2 * k1, &re, &im);
                const size_t c = (size_t)n2 * s.N1 + k1, r = (size_t)k1 * s.N2 + n2;
                twc[2 * c] = re;
                twc[2 * c + 1] = im;
                twr[2 * r] = re;
                twr[2 * r + 1] = -im;
                wv((uint64_t)k1 + (uint64_t)s.N1 * n2, &re, &im);
                tws[2 * r] = re;
                tws[2 * r + 1] = im;
            }
        std::vector<unsigned char> Wb, twb, tcb, trb, tsb;
        if (prec == SMOL_FP32CONV) {
            to_type<float>(hW, Wb);
            to_type<float>(tw64, twb);
            to_type<float>(twc, tcb);
            to_type<float>(twr, trb);
            to_type<float>(tws, tsb);
        } else if (prec == SMOL_DF64) {
            to_type<dd>(hW, Wb);
            to_type<dd>(tw64, twb);
            to_type<dd>(twc, tcb);
            to_type<dd>(twr, trb);
            to_type<dd>(tws, tsb);
        } else {
            to_type<double>(hW, Wb);
            to_type<double>(tw64, twb);
            to_type<double>(twc, tcb);
            to_type<double>(twr, trb);
            to_type<double>(tws, tsb);
        }
        CK(cudaMemcpyAsync(b + L.W, Wb.data(), Wb.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b + L.tw, twb.data(), twb.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b + L.twc, tcb.data(), tcb.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b + L.twr, trb.data(), trb.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b + L.tws, tsb.data(), tsb.size(), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(b + L.vec, 0, (size_t)NVEC * L.vstride * s.rsz, st));
        CK(cudaMemsetAsync(b + L.ybuf, 0, (size_t)s.Mp * s.rsz, st));
        CK(cudaMemsetAsync(b + L.half, 0, (size_t)s.Mp * 8, st));
        CK(cudaMemsetAsync(b + L.stateB, 0, (size_t)s.Mp * 8, st));
        // the host images are freed at the end of this iteration
        CK(cudaStreamSynchronize(st));
    }
    E->H.nC = (int)mC.size();
    E->H.nB = (int)mB.size();
    E->H.nF = (int)mF.size();
    CK(cudaMemsetAsync(ws + E->H.ctl, 0, (size_t)count * sizeof(Ctl), st));
    CK(cudaMemsetAsync(ws + E->H.rctl, 0, (size_t)count * sizeof(Ctl), st));
    CK(cudaMemsetAsync(ws + E->H.bar, 0, 2 * BAR_GEN * sizeof(unsigned), st));
    CK(cudaMemcpyAsync(E->d_sys, hs.data(), count * sizeof(SysDev), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(E->d_sysr, hsr.data(), count * sizeof(SysDev), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(E->mapC, mC.data(), mC.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(E->mapB, mB.data(), mB.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(E->mapF, mF.data(), mF.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    E->h_one = hs[0];
    E->h_oner = hsr[0];
    E->hs = hs;
    E->hsr = hsr;
    CK(cudaHostAlloc((void**)&E->h_ctl, (size_t)count * sizeof(Ctl), cudaHostAllocDefault));
    for (cudaEvent_t* e : {&E->ev_rb[0], &E->ev_rb[1], &E->ev_hctl})
        CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    CK(cudaStreamCreateWithFlags(&E->cap, cudaStreamNonBlocking));
    if (prec == SMOL_FP32CONV) return set_smem_attrs<float>(E);
    if (prec == SMOL_DF64) return set_smem_attrs<dd>(E);
    return set_smem_attrs<double>(E);
}

void engine_free(Engine* E) {
    if (!E) return;
    if (E->gexec) cudaGraphExecDestroy(E->gexec);
    if (E->cap) cudaStreamDestroy(E->cap);
    if (E->h_ctl) cudaFreeHost(E->h_ctl);
    for (cudaEvent_t e : {E->ev_rb[0], E->ev_rb[1], E->ev_hctl})
        if (e) cudaEventDestroy(e);
}

int check_opts(const smol_opts& o) {
    if (o.precision != SMOL_FP64 && o.precision != SMOL_FP32CONV && o.precision != SMOL_DF64) return SMOL_EINVAL;
    if (o.log_capacity < 0 || o.chunk < 0) return SMOL_EINVAL;
    if (o.fft_lgn1 < 0 || o.fft_lgn1 > 30 || o.fft_g < 0 || o.fft_g > 64 || (o.fft_g & (o.fft_g - 1)))
        return SMOL_EINVAL;
    for (int k = 0; k < SMOL_SIZE_CLASSES; ++k) {
        const int lg = o.batch_lgn1[k], g = o.batch_g[k];
        if (lg < 0 || lg > 30 || g < 0 || g > 64 || (g & (g - 1))) return SMOL_EINVAL;
    }
    return SMOL_OK;
}

int integrate_start(Engine* E, double* const* d_n, double t0, double t1, double tol, int32_t scheme) {
    if (!E || !d_n) return SMOL_EINVAL;
    for (int q = 0; q < E->count; ++q)
        if (!d_n[q] || ((uintptr_t)d_n[q] & 15)) return SMOL_EINVAL;
    if (!(t1 >= t0) || !isfinite(t0) || !isfinite(t1)) return SMOL_EINVAL;
    if (scheme < SMOL_RK2 || scheme > SMOL_RKF45) return SMOL_EINVAL;
    const bool fixed = E->o.fixed_tau > 0.0;
    if (!fixed && !(tol > 0.0)) return SMOL_EINVAL;
    cudaStream_t st = E->stream;
    // the pinned blocks may still be read or written by an earlier copy: wait for that
    // copy only (not for the rest of the stream)
    CK(cudaEventSynchronize(E->ev_hctl));
    for (int q = 0; q < E->count; ++q) {
        Ctl& h = E->h_ctl[q];
        memset(&h, 0, sizeof(h));
        h.t = t0;
        h.t1 = t1;
        h.tol = tol;
        h.itol2 = tol > 0.0 ? 1.0 / (tol * tol) : 0.0;
        const double tq = (q < (int)E->tau0.size() && E->tau0[q] > 0.0) ? E->tau0[q] : E->o.tau0;
        h.tau = tq > 0.0 ? tq : (fixed ? E->o.fixed_tau : 0.0);
        h.state[0] = d_n[q];
        h.state[1] = (double*)(E->ws + E->base[q] + E->lay[q].stateB);
    }
    CK(cudaMemcpyAsync(E->d_ctl, E->h_ctl, (size_t)E->count * sizeof(Ctl), cudaMemcpyHostToDevice, st));
    CK(cudaEventRecord(E->ev_hctl, st));
    const LaunchArgs A = args_for(E, false);
    if (E->o.precision == SMOL_FP32CONV) {
        k_prep1<float><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one);
        k_prep2<float><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one, E->o.euler_a);
    } else if (E->o.precision == SMOL_DF64) {
        k_prep1<dd><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one);
        k_prep2<dd><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one, E->o.euler_a);
    } else {
        k_prep1<double><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one);
        k_prep2<double><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one, E->o.euler_a);
    }
    CK(cudaGetLastError());

    // One CUDA graph holds `chunk` attempts (fewer if max_attempts is smaller); kernels
    // of attempts after termination return at once (they read ctl->done first).
    int64_t na = E->o.chunk > 0 ? E->o.chunk : 32;
    if (E->o.max_attempts < na) na = E->o.max_attempts;
    if (na < 1) na = 1;
    // Persistent attempt kernel instead of the graph: a single RKF45 system, when all
    // its CTAs can be resident at once (else the graph path).
    E->persist_run = false;
    if ((E->o.flags & SMOL_FLAG_PERSISTENT) && E->count == 1 && scheme == SMOL_RKF45 && !fixed) {
        const CtlParams P = make_params(E, scheme);
        if (E->o.precision == SMOL_FP32CONV) {
            E->pkern = (const void*)k_persist<float>;
            E->plan = make_plan<float>(P);
        } else if (E->o.precision == SMOL_DF64) {
            E->pkern = (const void*)k_persist<dd>;
            E->plan = make_plan<dd>(P);
        } else {
            E->pkern = (const void*)k_persist<double>;
            E->plan = make_plan<double>(P);
        }
        int dev = 0, sms = 0, per = 0;
        E->pblock = std::max(E->thrC, E->thrB);
        E->psmem = std::max(E->smemC, E->smemB);
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, E->pkern, E->pblock, E->psmem) == cudaSuccess &&
            per > 0) {
            const int units = std::max(E->H.nC, E->H.nB);
            E->pgrid = std::min(units, per * sms);
            E->persist_run = true;
        }
        cudaGetLastError();  // an occupancy query that failed leaves the graph path
    }
    if (E->persist_run) {
        E->run_dn.assign(d_n, d_n + E->count);
        E->run_scheme = scheme;
        E->run_attempts = na;
        E->running = true;
        return SMOL_OK;
    }
    const int64_t key = ((na * 64 + scheme * 16 + (fixed ? 8 : 0) + (E->o.steady_rtol > 0.0 ? 4 : 0)) << 8) +
                        (E->o.flags & 0xff);
    if (E->gkey != key) {
        if (E->gexec) {
            cudaGraphExecDestroy(E->gexec);
            E->gexec = nullptr;
        }
        E->gkey = -1;
        CtlParams P = make_params(E, scheme);
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(E->cap, cudaStreamCaptureModeThreadLocal));
        for (int64_t q = 0; q < na; ++q) enqueue_attempt_any(E, scheme, fixed, P, E->cap, nullptr);
        cudaError_t e1 = cudaStreamEndCapture(E->cap, &g);
        if (e1 != cudaSuccess) return SMOL_ECUDA;
        e1 = cudaGraphInstantiate(&E->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e1 != cudaSuccess) {
            E->gexec = nullptr;
            return SMOL_ECUDA;
        }
        E->gkey = key;
    }
    E->run_dn.assign(d_n, d_n + E->count);
    E->run_scheme = scheme;
    E->run_attempts = na;
    E->running = true;
    return SMOL_OK;
}

// One chunk of attempts on stream st: the captured graph, or one launch of the
// persistent attempt kernel.
cudaError_t launch_chunk(Engine* E, cudaStream_t st) {
    if (E->persist_run) {
        int na = (int)E->run_attempts;
        void* args[] = {(void*)&E->h_one, (void*)&E->plan, (void*)&na, (void*)&E->d_bar};
        return cudaLaunchCooperativeKernel(E->pkern, dim3((unsigned)E->pgrid), dim3((unsigned)E->pblock), args,
                                           E->psmem, st);
    }
    return cudaGraphLaunch(E->gexec, st);
}

int integrate_advance(Engine* E) {
    if (!E || !E->running || (!E->gexec && !E->persist_run)) return SMOL_EINVAL;
    CK(launch_chunk(E, E->stream));
    return SMOL_OK;
}

void fill_stats(const Ctl& c, smol_stats* s) {
    s->t = c.t;
    s->tau_next = c.tau;
    s->err_last = c.err_last;
    s->mass = c.mass;
    s->rhs_evals = c.rhs_evals;
    s->rhs_evals_paper = c.rhs_paper;
    s->accepted = c.accepted;
    s->rejected = c.rejected;
    s->attempts = c.attempts;
    s->status = c.status;
    s->reserved = 0;
}

// Synchronises, copies states held in the engine's buffers back to the callers'
// vectors, fills stats (count entries) and returns the first error status, else
// SMOL_STEADY if any system stopped there, else SMOL_OK.
int integrate_finish(Engine* E, smol_stats* stats) {
    if (!E || !E->running) return SMOL_EINVAL;
    cudaStream_t st = E->stream;
    // the state back into the callers' buffers (on the device), then one read-back of
    // the control blocks and one synchronisation
    const LaunchArgs A = args_for(E, false);
    if (E->o.precision == SMOL_FP32CONV) k_restore<float><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one);
    else if (E->o.precision == SMOL_DF64) k_restore<dd><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one);
    else k_restore<double><<<E->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(E->h_ctl, E->d_ctl, (size_t)E->count * sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(E->ev_hctl, st));
    CK(cudaStreamSynchronize(st));
    int rc = SMOL_OK;
    for (int q = 0; q < E->count; ++q) {
        const Ctl& c = E->h_ctl[q];
        E->last_attempts[q] = c.attempts;
        if (stats) fill_stats(c, stats + q);
        if (c.status < 0 && rc >= 0) rc = c.status;
        else if (c.status == SMOL_STEADY && rc == SMOL_OK) rc = SMOL_STEADY;
    }
    return rc;
}

bool all_done(const Engine* E) {
    for (int q = 0; q < E->count; ++q)
        if (!E->h_ctl[q].done) return false;
    return true;
}

int integrate_all(Engine* E, double* const* d_n, double t0, double t1, double tol, int32_t scheme,
                  smol_stats* stats) {
    int rc = integrate_start(E, d_n, t0, t1, tol, scheme);
    if (rc != SMOL_OK) return rc;
    if (!(t1 > t0)) return integrate_finish(E, stats);  // nothing to integrate
    cudaStream_t st = E->stream;
    // Launch chunks, keeping one in flight while the status of the previous one is read
    // from pinned copies of the control blocks. A run that one chunk covers
    // (max_attempts <= chunk) reads nothing back before integrate_finish.
    cudaEvent_t* ev = E->ev_rb;
    const size_t cbytes = (size_t)E->count * sizeof(Ctl);
    const int64_t maxa = E->o.max_attempts;
    int64_t launched = E->run_attempts;  // attempts enqueued so far
    int cur = 0;
    if (launch_chunk(E, st) != cudaSuccess) rc = SMOL_ECUDA;
    if (rc == SMOL_OK && launched < maxa &&
        (cudaMemcpyAsync(E->h_ctl, E->d_ctl, cbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaEventRecord(ev[cur], st) != cudaSuccess || cudaEventRecord(E->ev_hctl, st) != cudaSuccess))
        rc = SMOL_ECUDA;
    while (rc == SMOL_OK && launched < maxa) {
        if (launch_chunk(E, st) != cudaSuccess) {
            rc = SMOL_ECUDA;
            break;
        }
        launched += E->run_attempts;
        if (cudaEventSynchronize(ev[cur]) != cudaSuccess) {
            rc = SMOL_ECUDA;
            break;
        }
        if (all_done(E) || launched >= maxa) break;
        if (cudaMemcpyAsync(E->h_ctl, E->d_ctl, cbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaEventRecord(ev[cur ^ 1], st) != cudaSuccess || cudaEventRecord(E->ev_hctl, st) != cudaSuccess) {
            rc = SMOL_ECUDA;
            break;
        }
        cur ^= 1;
    }
    if (rc != SMOL_OK) {
        cudaStreamSynchronize(st);
        return rc;
    }
    return integrate_finish(E, stats);  // synchronises once
}

int get_log(Engine* E, int q, double* h_t, double* h_tau, double* h_err, int32_t* h_acc, int32_t cap,
            int64_t* count) {
    if (!E || cap < 0 || q < 0 || q >= E->count) return SMOL_EINVAL;
    const int64_t n = E->last_attempts[q];
    if (count) *count = n;
    const int lc = E->o.log_capacity;
    if (lc <= 0 || cap == 0 || n == 0) return SMOL_OK;
    const int64_t keep = n < lc ? n : lc;
    const int64_t take = keep < cap ? keep : cap;
    std::vector<double> t(lc), hh(lc), e(lc);
    std::vector<int32_t> a(lc);
    const char* b = E->ws + E->base[q];
    const Layout& L = E->lay[q];
    CK(cudaMemcpy(t.data(), b + L.log_t, lc * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hh.data(), b + L.log_h, lc * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(e.data(), b + L.log_e, lc * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(a.data(), b + L.log_a, lc * 4, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < take; ++k) {
        const int64_t att = n - take + k;  // 0-based attempt index, oldest first
        const int64_t slot = att % lc;
        if (h_t) h_t[k] = t[slot];
        if (h_tau) h_tau[k] = hh[slot];
        if (h_err) h_err[k] = e[slot];
        if (h_acc) h_acc[k] = a[slot];
    }
    return SMOL_OK;
}

int rhs_common(smol_system* S, const double* d_n, double* d_out, double* d_birth, double* d_loss, double* d_src) {
    if (!S || !d_n) return SMOL_EINVAL;
    if (((uintptr_t)d_n & 15) || ((uintptr_t)d_out & 15) || ((uintptr_t)d_birth & 15) || ((uintptr_t)d_loss & 15))
        return SMOL_EINVAL;
    cudaStream_t st = S->stream;
    StageIn in;
    memset(&in, 0, sizeof(in));
    in.nv = 1;
    in.direct = 1;
    in.slot[0] = SLOT_EXT;
    in.c[0] = 1.0;
    in.cf[0] = 1.0f;
    in.ext = d_n;
    EpiOut eo;
    memset(&eo, 0, sizeof(eo));
    eo.out_slot = -1;
    eo.out = d_out;
    eo.birth = d_birth;
    eo.loss = d_loss;
    eo.source = d_src;
    eo.hfac = 1.0;
    const LaunchArgs A = args_for(S, true);
    if (S->o.precision == SMOL_FP32CONV) {
        k_absmax<<<S->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one, d_n, 1);
        k_tilt<<<S->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one, d_n);
        launch_eval<float>(S, A, in, eo, st, nullptr);
    } else if (S->o.precision == SMOL_DF64) {
        k_absmax<<<S->H.nF, FIN_THREADS, 0, st>>>(A.sys, A.mapF, A.one, d_n, 0);
        launch_eval<dd>(S, A, in, eo, st, nullptr);
    } else {
        launch_eval<double>(S, A, in, eo, st, nullptr);
    }
    return cudaGetLastError() == cudaSuccess ? SMOL_OK : SMOL_ECUDA;
}

// Schedule autotuner: mean time of one step attempt of engine E, run from copies of
// the states d_n0 (into d_work), over `attempts` attempts after one warm-up chunk, in
// microseconds; < 0 if a call failed or a system ended during the timing.
double time_attempts(Engine* E, double* const* d_work, const double* const* d_n0, double tol, int scheme,
                     int attempts) {
    cudaStream_t st = E->stream;
    for (int q = 0; q < E->count; ++q)
        if (cudaMemcpyAsync(d_work[q], d_n0[q], (size_t)E->sh[q].M * 8, cudaMemcpyDeviceToDevice, st) !=
            cudaSuccess)
            return -1.0;
    if (integrate_start(E, d_work, 0.0, 1e300, tol, scheme) != SMOL_OK) return -1.0;
    const int64_t chunks = std::max<int64_t>(1, (attempts + E->run_attempts - 1) / E->run_attempts);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double us = -1.0;
    if (integrate_advance(E) == SMOL_OK && cudaEventCreate(&e0) == cudaSuccess &&
        cudaEventCreate(&e1) == cudaSuccess && cudaEventRecord(e0, st) == cudaSuccess) {
        bool ok = true;
        for (int64_t c = 0; c < chunks && ok; ++c) ok = integrate_advance(E) == SMOL_OK;
        float ms = 0.f;
        if (ok && cudaEventRecord(e1, st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
            cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
            us = 1000.0 * ms / (double)(chunks * E->run_attempts);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // an error status or a steady stop ends the timing's validity
    if (integrate_finish(E, nullptr) != SMOL_OK) return -1.0;
    return us;
}

// Launch modes the tuner tries (programmatic launch, fusion of the column passes).
constexpr int TUNE_FLAGS[] = {0, SMOL_FLAG_NO_PDL, SMOL_FLAG_NO_PDL_FWD_COLS, SMOL_FLAG_NO_FUSE,
                              SMOL_FLAG_NO_FUSE | SMOL_FLAG_NO_PDL};
constexpr int PDL_BITS = SMOL_FLAG_NO_PDL | SMOL_FLAG_NO_PDL_FWD_COLS | SMOL_FLAG_NO_PDL_ROWS |
                         SMOL_FLAG_NO_PDL_INV_COLS | SMOL_FLAG_NO_PDL_STEP | SMOL_FLAG_NO_FUSE | SMOL_FLAG_PERSISTENT |
                         SMOL_FLAG_WIDE_COLS;

}  // namespace

// ---------------------------------------------------------------------------
// Point sources of Eq. (3)
// ---------------------------------------------------------------------------
namespace {
static_assert(SMOL_MAX_SOURCES == MAXSRC, "source capacity of the C interface and the kernels");
int set_sources(Engine* E, int q, int32_t count, const int64_t* sizes, const double* values) {
    if (!E || q < 0 || q >= E->count || count < 0 || count > MAXSRC) return SMOL_EINVAL;
    if (count > 0 && (!sizes || !values)) return SMOL_EINVAL;
    for (int k = 0; k < count; ++k)
        if (sizes[k] < 1 || sizes[k] > E->sh[q].M || !isfinite(values[k])) return SMOL_EINVAL;
    for (SysDev* d : {&E->hs[q], &E->hsr[q]}) {
        d->nsrc = count;
        for (int k = 0; k < MAXSRC; ++k) {
            d->src_i[k] = k < count ? (int)(sizes[k] - 1) : 0;
            d->src_v[k] = k < count ? values[k] : 0.0;
        }
    }
    cudaStream_t st = E->stream;
    CK(cudaMemcpyAsync(E->d_sys + q, &E->hs[q], sizeof(SysDev), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(E->d_sysr + q, &E->hsr[q], sizeof(SysDev), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    if (q == 0) {
        E->h_one = E->hs[0];
        E->h_oner = E->hsr[0];
    }
    // captured graphs hold the old descriptor (single systems pass it by value); a run
    // started before cannot be continued with smol_integrate_advance
    if (E->gexec) {
        cudaGraphExecDestroy(E->gexec);
        E->gexec = nullptr;
    }
    E->gkey = -1;
    E->running = false;
    return SMOL_OK;
}
}  // namespace

// ---------------------------------------------------------------------------
// C interface: single system
// ---------------------------------------------------------------------------
extern "C" {

void smol_default_opts(smol_opts* opts) {
    if (opts) default_opts(opts);
}

int64_t smol_max_m(int32_t R, int32_t precision) { return max_m_for(R, precision); }

int64_t smol_max_m_transforms(int32_t T, int32_t precision) { return max_m_transforms(T, precision); }

size_t smol_workspace_bytes(int64_t M, int32_t R, const smol_opts* opts) {
    smol_opts o;
    if (opts) o = *opts;
    else default_opts(&o);
    return batch_bytes(1, &M, R, o);
}

int smol_init_system(smol_system** out, int64_t M, int32_t R, const double* h_U, const double* h_V, double lambda,
                     const smol_opts* opts, void* d_workspace, size_t workspace_bytes) {
    if (!out || !h_U || !h_V || !d_workspace || M < 1 || R < 1 || R > MAXR || !(lambda >= 0.0)) return SMOL_EINVAL;
    *out = nullptr;
    smol_opts o;
    if (opts) o = *opts;
    else default_opts(&o);
    int rc = check_opts(o);
    if (rc != SMOL_OK) return rc;
    if (M > max_m_transforms(1, o.precision)) return SMOL_EUNSUPPORTED;
    if (((uintptr_t)d_workspace & 255) != 0) return SMOL_EINVAL;
    if (workspace_bytes < batch_bytes(1, &M, R, o)) return SMOL_ENOSPACE;
    smol_system* S = new smol_system();
    rc = engine_init(S, 1, &M, R, &h_U, &h_V, &lambda, o, d_workspace, workspace_bytes);
    if (rc != SMOL_OK) {
        engine_free(S);
        delete S;
        return rc;
    }
    *out = S;
    return SMOL_OK;
}

int smol_set_stream(smol_system* S, void* stream) {
    if (!S) return SMOL_EINVAL;
    S->stream = (cudaStream_t)stream;
    S->o.stream = stream;
    return SMOL_OK;
}

int smol_num_transforms(const smol_system* S) { return S ? S->T[0] : 0; }

int smol_set_tau0(smol_system* S, double tau0) {
    if (!S || !(tau0 >= 0.0) || !isfinite(tau0)) return SMOL_EINVAL;
    S->tau0.assign(1, tau0);
    return SMOL_OK;
}

int smol_batch_set_tau0(smol_batch* B, const double* tau0) {
    if (!B || !tau0) return SMOL_EINVAL;
    for (int q = 0; q < B->count; ++q)
        if (!(tau0[q] >= 0.0) || !isfinite(tau0[q])) return SMOL_EINVAL;
    B->tau0.assign(tau0, tau0 + B->count);
    return SMOL_OK;
}

int smol_rhs(smol_system* S, const double* d_n, double* d_out) {
    if (!d_out) return SMOL_EINVAL;
    return rhs_common(S, d_n, d_out, nullptr, nullptr, nullptr);
}

int smol_rhs_terms(smol_system* S, const double* d_n, double* d_birth, double* d_loss, double* d_source) {
    return rhs_common(S, d_n, nullptr, d_birth, d_loss, d_source);
}

int smol_integrate_start(smol_system* S, double* d_n, double t0, double t1, double tol, int32_t scheme) {
    if (!S) return SMOL_EINVAL;
    return integrate_start(S, &d_n, t0, t1, tol, scheme);
}

int smol_integrate_advance(smol_system* S) { return integrate_advance(S); }

int smol_integrate_finish(smol_system* S, smol_stats* stats) { return integrate_finish(S, stats); }

int smol_integrate(smol_system* S, double* d_n, double t0, double t1, double tol, int32_t scheme, smol_stats* stats) {
    if (!S) return SMOL_EINVAL;
    return integrate_all(S, &d_n, t0, t1, tol, scheme, stats);
}

int smol_profile_attempts(smol_system* S, int32_t reps, double* kernel_ms, int64_t* kernel_launches, int32_t nkinds) {
    if (!S || !S->running || reps < 1 || !kernel_ms || nkinds < SMOL_PROF_KINDS) return SMOL_EINVAL;
    cudaStream_t st = S->stream;
    Prof pr;
    memset(&pr, 0, sizeof(pr));
    for (int q = 0; q < PROF_MAX; ++q) {
        CK(cudaEventCreate(&pr.ev0[q]));
        CK(cudaEventCreate(&pr.ev1[q]));
    }
    const bool fixed = S->o.fixed_tau > 0.0;
    CtlParams P = make_params(S, S->run_scheme);
    double acc[SMOL_PROF_KINDS] = {0};
    int64_t cnt[SMOL_PROF_KINDS] = {0};
    int rc = SMOL_OK;
    for (int r = 0; r < reps && rc == SMOL_OK; ++r) {
        pr.n = 0;
        // ~0.5 ms of device work first, so that the whole attempt is enqueued before the
        // device reaches it and the events time the kernels, not the host launches
        k_delay<<<1, 32, 0, st>>>(1000000LL);
        enqueue_attempt_any(S, S->run_scheme, fixed, P, st, &pr);
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
    return get_log(S, 0, h_t, h_tau, h_err, h_acc, cap, count);
}

void smol_destroy(smol_system* S) {
    if (!S) return;
    engine_free(S);
    delete S;
}

int smol_tune(int64_t M, int32_t R, const double* h_U, const double* h_V, double lambda, const double* d_n0,
              double tol, int32_t scheme, int32_t attempts, smol_opts* opts, double* us_per_attempt) {
    if (!h_U || !h_V || !d_n0 || !opts || M < 1 || R < 1 || R > MAXR || !(lambda >= 0.0) || attempts < 1 ||
        scheme < SMOL_RK2 || scheme > SMOL_RKF45 || !(tol > 0.0) || ((uintptr_t)d_n0 & 15))
        return SMOL_EINVAL;
    smol_opts base = *opts;
    int rc = check_opts(base);
    if (rc != SMOL_OK) return rc;
    if (M > max_m_transforms(1, base.precision)) return SMOL_EUNSUPPORTED;
    base.max_attempts = (int64_t)1 << 62;
    base.fixed_tau = 0.0;
    double* d_work = nullptr;
    if (cudaMalloc((void**)&d_work, (size_t)M * 8) != cudaSuccess) return SMOL_ECUDA;
    const Shape def = make_shape(M, base.precision);
    double best = -1.0;
    smol_opts bo = base;
    for (int dl : {0, -1, -2, 1}) {
        const int lg = def.lgN1 + dl;
        if (lg < 1 || lg >= def.lgMp) continue;
        const int g0 = make_shape(M, base.precision, false, lg, 0).G;
        for (int gm : {1, 2, 4, 8}) {
            const int g = g0 * gm;
            if (g > 64 || g > (1 << (def.lgMp - lg))) continue;  // beyond the columns there are
            smol_opts c = base;
            c.fft_lgn1 = lg;
            c.fft_g = g;
            const size_t bytes = batch_bytes(1, &M, R, c);
            if (bytes == 0) continue;
            void* ws = nullptr;
            if (cudaMalloc(&ws, bytes + 256) != cudaSuccess) continue;
            void* wsa = (void*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
            smol_system* S = new smol_system();
            if (engine_init(S, 1, &M, R, &h_U, &h_V, &lambda, c, wsa, bytes) == SMOL_OK &&
                S->sh[0].G == g) {  // skip a G that the shared-memory limit reduced
                // the launch modes, and for RKF45 the persistent attempt kernel
                int modes[12], nm = 0;
                for (int fl : TUNE_FLAGS) modes[nm++] = fl;
                modes[nm++] = SMOL_FLAG_WIDE_COLS | SMOL_FLAG_NO_PDL;
                modes[nm++] = SMOL_FLAG_WIDE_COLS | SMOL_FLAG_NO_PDL_FWD_COLS;
                if (scheme == SMOL_RKF45) modes[nm++] = SMOL_FLAG_PERSISTENT;
                for (int k = 0; k < nm; ++k) {
                    const int fl = modes[k];
                    S->o.flags = (base.flags & ~PDL_BITS) | fl;
                    const double us = time_attempts(S, &d_work, &d_n0, tol, scheme, attempts);
                    if (us > 0.0 && (best < 0.0 || us < best)) {
                        best = us;
                        bo = c;
                        bo.flags = S->o.flags;
                    }
                }
            }
            engine_free(S);
            delete S;
            cudaFree(ws);
        }
    }
    cudaFree(d_work);
    if (best < 0.0) return SMOL_ECUDA;
    opts->fft_lgn1 = bo.fft_lgn1;
    opts->fft_g = bo.fft_g;
    opts->flags = bo.flags;
    if (us_per_attempt) *us_per_attempt = best;
    return SMOL_OK;
}

// ---------------------------------------------------------------------------
// C interface: batch of independent systems
// ---------------------------------------------------------------------------
size_t smol_batch_workspace_bytes(int32_t count, const int64_t* M, int32_t R, const smol_opts* opts) {
    if (!M) return 0;
    smol_opts o;
    if (opts) o = *opts;
    else default_opts(&o);
    return batch_bytes(count, M, R, o);
}

int smol_batch_init(smol_batch** out, int32_t count, const int64_t* M, int32_t R, const double* const* h_U,
                    const double* const* h_V, const double* lambda, const smol_opts* opts, void* d_workspace,
                    size_t workspace_bytes) {
    if (!out || !M || !h_U || !h_V || !lambda || !d_workspace || count < 1 || count > MAX_BATCH || R < 1 ||
        R > MAXR)
        return SMOL_EINVAL;
    *out = nullptr;
    smol_opts o;
    if (opts) o = *opts;
    else default_opts(&o);
    int rc = check_opts(o);
    if (rc != SMOL_OK) return rc;
    const int64_t mm = max_m_transforms(1, o.precision);  // the exact check (actual T) is in init
    for (int q = 0; q < count; ++q) {
        if (M[q] < 1) return SMOL_EINVAL;
        if (M[q] > mm) return SMOL_EUNSUPPORTED;
    }
    if (((uintptr_t)d_workspace & 255) != 0) return SMOL_EINVAL;
    if (workspace_bytes < batch_bytes(count, M, R, o)) return SMOL_ENOSPACE;
    smol_batch* B = new smol_batch();
    rc = engine_init(B, count, M, R, h_U, h_V, lambda, o, d_workspace, workspace_bytes);
    if (rc != SMOL_OK) {
        engine_free(B);
        delete B;
        return rc;
    }
    *out = B;
    return SMOL_OK;
}

int smol_batch_integrate(smol_batch* B, double* const* d_n, double t0, double t1, double tol, int32_t scheme,
                         smol_stats* stats) {
    if (!B) return SMOL_EINVAL;
    return integrate_all(B, d_n, t0, t1, tol, scheme, stats);
}

int smol_batch_integrate_start(smol_batch* B, double* const* d_n, double t0, double t1, double tol, int32_t scheme) {
    if (!B) return SMOL_EINVAL;
    return integrate_start(B, d_n, t0, t1, tol, scheme);
}

int smol_batch_integrate_advance(smol_batch* B) { return integrate_advance(B); }

int smol_batch_integrate_finish(smol_batch* B, smol_stats* stats) { return integrate_finish(B, stats); }

int smol_batch_get_log(smol_batch* B, int32_t system, double* h_t, double* h_tau, double* h_err, int32_t* h_acc,
                       int32_t cap, int64_t* count) {
    return get_log(B, system, h_t, h_tau, h_err, h_acc, cap, count);
}

int smol_batch_set_stream(smol_batch* B, void* stream) {
    if (!B) return SMOL_EINVAL;
    B->stream = (cudaStream_t)stream;
    B->o.stream = stream;
    return SMOL_OK;
}

int smol_batch_tune(smol_batch* B, double* const* d_n, double tol, int32_t scheme, int32_t attempts,
                    int32_t* flags, double* us_per_attempt) {
    if (!B || !d_n || attempts < 1 || scheme < SMOL_RK2 || scheme > SMOL_RKF45 || !(tol > 0.0)) return SMOL_EINVAL;
    for (int q = 0; q < B->count; ++q)
        if (!d_n[q] || ((uintptr_t)d_n[q] & 15)) return SMOL_EINVAL;
    std::vector<double*> work(B->count, nullptr);
    int rc = SMOL_OK;
    for (int q = 0; q < B->count && rc == SMOL_OK; ++q)
        if (cudaMalloc((void**)&work[q], (size_t)B->sh[q].M * 8) != cudaSuccess) rc = SMOL_ECUDA;
    const int base = B->o.flags;
    const int64_t maxa = B->o.max_attempts;
    const double ftau = B->o.fixed_tau;
    B->o.max_attempts = (int64_t)1 << 62;
    B->o.fixed_tau = 0.0;
    double best = -1.0;
    int bf = base;
    for (int fl : TUNE_FLAGS) {
        if (rc != SMOL_OK) break;
        B->o.flags = (base & ~PDL_BITS) | fl;
        const double us = time_attempts(B, work.data(), d_n, tol, scheme, attempts);
        if (us > 0.0 && (best < 0.0 || us < best)) {
            best = us;
            bf = B->o.flags;
        }
    }
    B->o.max_attempts = maxa;
    B->o.fixed_tau = ftau;
    B->o.flags = bf;
    B->gkey = -1;  // recapture with the chosen launch mask
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    B->running = false;  // the timings ran on scratch copies: nothing to continue
    for (double* w : work)
        if (w) cudaFree(w);
    if (rc == SMOL_OK && best < 0.0) rc = SMOL_ECUDA;
    if (rc != SMOL_OK) return rc;
    if (flags) *flags = bf;
    if (us_per_attempt) *us_per_attempt = best;
    return SMOL_OK;
}

int smol_batch_tune_schedules(int32_t count, const int64_t* M, int32_t R, const double* const* h_U,
                              const double* const* h_V, const double* lambda, double* const* d_n0, double tol,
                              int32_t scheme, int32_t attempts, smol_opts* opts, double* us_per_attempt) {
    if (!M || !h_U || !h_V || !lambda || !d_n0 || !opts || count < 1 || count > MAX_BATCH || R < 1 || R > MAXR ||
        attempts < 1 || scheme < SMOL_RK2 || scheme > SMOL_RKF45 || !(tol > 0.0))
        return SMOL_EINVAL;
    smol_opts base = *opts;
    int rc = check_opts(base);
    if (rc != SMOL_OK) return rc;
    const int64_t mm = max_m_transforms(1, base.precision);
    for (int q = 0; q < count; ++q) {
        if (M[q] < 1 || !d_n0[q] || ((uintptr_t)d_n0[q] & 15)) return SMOL_EINVAL;
        if (M[q] > mm) return SMOL_EUNSUPPORTED;
    }
    base.max_attempts = (int64_t)1 << 62;
    base.fixed_tau = 0.0;
    std::vector<double*> work(count, nullptr);
    for (int q = 0; q < count && rc == SMOL_OK; ++q)
        if (cudaMalloc((void**)&work[q], (size_t)M[q] * 8) != cudaSuccess) rc = SMOL_ECUDA;
    // one whole-batch timing of the options c (-1 where it does not fit or fails)
    auto timeit = [&](const smol_opts& c) -> double {
        const size_t bytes = batch_bytes(count, M, R, c);
        if (bytes == 0) return -1.0;
        void* ws = nullptr;
        if (cudaMalloc(&ws, bytes + 256) != cudaSuccess) {
            cudaGetLastError();
            return -1.0;
        }
        void* wsa = (void*)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
        smol_batch* B = new smol_batch();
        double us = -1.0;
        if (engine_init(B, count, M, R, h_U, h_V, lambda, c, wsa, bytes) == SMOL_OK)
            us = time_attempts(B, work.data(), d_n0, tol, scheme, attempts);
        engine_free(B);
        delete B;
        cudaFree(ws);
        return us;
    };
    // the size classes present, the one holding the most sizes first
    const bool wide = is_wide(count, M);
    std::vector<std::pair<int64_t, int>> cls;
    for (int q = 0; q < count; ++q) {
        const int k = ilog2(M[q] < 4 ? 4 : M[q]);
        bool found = false;
        for (auto& c : cls)
            if (c.second == k) {
                c.first += M[q];
                found = true;
            }
        if (!found) cls.push_back({M[q], k});
    }
    std::sort(cls.begin(), cls.end(), [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
        return a.first != b.first ? a.first > b.first : a.second > b.second;
    });
    smol_opts cur = base;
    double best = rc == SMOL_OK ? timeit(cur) : -1.0;
    if (rc == SMOL_OK && best < 0.0) rc = SMOL_ECUDA;
    for (size_t ci = 0; ci < cls.size() && rc == SMOL_OK; ++ci) {
        const int k = cls[ci].second;
        if (k >= SMOL_SIZE_CLASSES) continue;
        const int64_t Mk = (int64_t)1 << k;
        const Shape now = engine_shape(2, Mk, cur, wide);  // the class's schedule so far
        const Shape rule = make_shape(Mk, base.precision, wide);
        for (int dl : {-2, -1, 0, 1}) {
            const int lg = rule.lgN1 + dl;
            if (lg < 1 || lg >= k) continue;
            const int g0 = make_shape(Mk, base.precision, wide, lg, 0).G;
            for (int gm : {1, 2, 4, 8}) {
                const int g = g0 * gm;
                if (g > 64 || g > (1 << (k - lg))) continue;
                if (lg == now.lgN1 && g == now.G) continue;
                smol_opts c = cur;
                c.batch_lgn1[k] = (int8_t)lg;
                c.batch_g[k] = (int8_t)g;
                const double us = timeit(c);
                if (us > 0.0 && us < best) {
                    best = us;
                    cur = c;
                }
            }
        }
    }
    for (double* w : work)
        if (w) cudaFree(w);
    if (rc != SMOL_OK) return rc;
    memcpy(opts->batch_lgn1, cur.batch_lgn1, sizeof(cur.batch_lgn1));
    memcpy(opts->batch_g, cur.batch_g, sizeof(cur.batch_g));
    if (us_per_attempt) *us_per_attempt = best;
    return SMOL_OK;
}

void smol_batch_destroy(smol_batch* B) {
    if (!B) return;
    engine_free(B);
    delete B;
}

// ---------------------------------------------------------------------------
// C interface: point sources of Eq. (3)
// ---------------------------------------------------------------------------
int smol_set_sources(smol_system* S, int32_t count, const int64_t* sizes, const double* values) {
    return set_sources(S, 0, count, sizes, values);
}
int smol_batch_set_sources(smol_batch* B, int32_t system, int32_t count, const int64_t* sizes,
                           const double* values) {
    return set_sources(B, system, count, sizes, values);
}

// ---------------------------------------------------------------------------
// C interface: partition of a batch across GPUs (host only)
// ---------------------------------------------------------------------------
int smol_partition(int32_t count, const int64_t* M, const double* weight, int32_t nranks, int32_t* rank_of,
                   double* load) {
    if (count < 1 || !M || nranks < 1 || !rank_of) return SMOL_EINVAL;
    // cost of a system: its work per attempt, Mp log2 Mp (the FFT route's O(M log M)),
    // times the caller's weight (expected attempts; 1 if none)
    std::vector<double> cost(count);
    for (int q = 0; q < count; ++q) {
        if (M[q] < 1 || (weight && !(weight[q] >= 0.0))) return SMOL_EINVAL;
        const int lg = ilog2(M[q] < 4 ? 4 : M[q]);
        cost[q] = (double)((int64_t)1 << lg) * (double)(lg + 1) * (weight ? weight[q] : 1.0);
    }
    // longest processing time first: systems by decreasing cost (ties by index), each
    // to the least-loaded rank (ties by the lower rank); within 4/3 of the optimum
    std::vector<int> ord(count);
    for (int q = 0; q < count; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> ld(nranks, 0.0);
    for (int q : ord) {
        int r = 0;
        for (int k = 1; k < nranks; ++k)
            if (ld[k] < ld[r]) r = k;
        rank_of[q] = r;
        ld[r] += cost[q];
    }
    if (load)
        for (int k = 0; k < nranks; ++k) load[k] = ld[k];
    return SMOL_OK;
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
