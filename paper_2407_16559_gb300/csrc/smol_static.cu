// smol_static.cu - smol_rhs_static: one FP64 evaluation of S(n) that allocates
// nothing. It is for callers that cannot call cudaMalloc or hand over a workspace:
// code that runs while a CUDA graph is being captured, allocator-free embedded hosts,
// or plug-in environments where the memory of the process belongs to someone else.
// Its scratch memory is the file-scope device array below, which every GPU that loads
// the library holds until the process exits.
//
// Limits: M <= SMOL_STATIC_MAX_M (65536), R <= SMOL_STATIC_MAX_R (3). All calls on one
// device share the array and it keeps the last call's contents; calls that overlap on
// the GPU (for instance on two streams) race on it and must be serialised by the
// caller.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "../../include/smol.h"
#include "smol_attr.h"
#include "smol_rhs.cuh"

using namespace smol;

namespace {

constexpr int SMAX_M = SMOL_STATIC_MAX_M;
constexpr int SMAX_R = SMOL_STATIC_MAX_R;
constexpr int SMAX_T = 2 * SMAX_R;
constexpr size_t A256 = 256;
constexpr size_t al(size_t x) { return (x + A256 - 1) / A256 * A256; }

// Layout of the scratch array (byte offsets); sized for M = SMAX_M, T = 2 SMAX_R.
constexpr size_t OFF_CTL = 0;
constexpr size_t OFF_TW = OFF_CTL + al(sizeof(Ctl));
constexpr size_t OFF_TWC = OFF_TW + al((size_t)SMAX_M * 16);
constexpr size_t OFF_TWR = OFF_TWC + al((size_t)SMAX_M * 16);
constexpr size_t OFF_TWS = OFF_TWR + al((size_t)SMAX_M * 16);
constexpr size_t OFF_W = OFF_TWS + al((size_t)SMAX_M * 16);
constexpr size_t OFF_Y = OFF_W + al((size_t)SMAX_T * SMAX_M * 8);
constexpr size_t OFF_G2 = OFF_Y + al((size_t)SMAX_T * SMAX_M * 16);
constexpr size_t OFF_YBUF = OFF_G2 + al((size_t)SMAX_M * 16);
constexpr size_t OFF_MPART = OFF_YBUF + al((size_t)SMAX_M * 8);
constexpr size_t OFF_SYS = OFF_MPART + al((size_t)SMAX_T * 1024 * 2 * 8);
constexpr size_t OFF_MAPC = OFF_SYS + al(sizeof(SysDev));
constexpr size_t OFF_MAPB = OFF_MAPC + al((size_t)1024 * sizeof(int2));
constexpr size_t OFF_RSC = OFF_MAPB + al((size_t)1024 * sizeof(int2));
constexpr size_t SCRATCH_BYTES = OFF_RSC + al((size_t)(MAXT + 2) * 8 + 2 * MAXT * 4);

// The scratch memory of smol_rhs_static.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];
static_assert(SCRATCH_BYTES == 15321344, "the scratch size documented in smol.h");

constexpr int MAX_DEVICES = 64;
// Per device: the device address of g_scratch, published by the release store of
// g_ready (set-up runs once per device under g_setup_mutex, so two host threads making
// their first call at the same time do not race).
unsigned char* g_scratch_ptr[MAX_DEVICES];
std::atomic<bool> g_ready[MAX_DEVICES];
std::mutex g_setup_mutex;

// Weights: W_t = column t of U (t < R) and row t - R of V (t >= R), zero beyond M.
__global__ void k_static_weights(const double* __restrict__ U, const double* __restrict__ V, int M, int Mp, int R,
                                 double* W) {
    const int T = 2 * R;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < T * Mp; q += gridDim.x * blockDim.x) {
        const int t = q / Mp, i = q % Mp;
        double w = 0.0;
        if (i < M) w = (t < R) ? U[(size_t)i * R + t] : V[(size_t)(t - R) * M + i];
        W[q] = w;
    }
}

// Twiddles exp(-i pi e / Mp), e < Mp, and the four-step / spectral tables in the
// layouts the kernels read: twc[n2][k1] = W_Mp^{n2 k1}, twr[k1][n2] = its conjugate,
// tws[k1][k2] = W_{2Mp}^{k1 + N1 k2}.
__global__ void k_static_twiddles(int Mp, int N1, int N2, double2* tw, double2* twc, double2* twr, double2* tws) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Mp; e += gridDim.x * blockDim.x) {
        double s, c;
        sincospi((double)e / (double)Mp, &s, &c);
        tw[e] = make_double2(c, -s);
        const int n2 = e / N1, k1 = e % N1;
        const long long f = (2LL * n2 * k1) % (2LL * Mp);
        sincospi((double)f / (double)Mp, &s, &c);
        twc[e] = make_double2(c, -s);
        twr[(size_t)k1 * N2 + n2] = make_double2(c, s);
        const int r = e / N2, k2 = e % N2;
        sincospi((double)(r + (long long)N1 * k2) / (double)Mp, &s, &c);
        tws[e] = make_double2(c, -s);
    }
}

// Writes this call's descriptor and block maps into the scratch array (the host
// passes them as kernel arguments, so nothing is copied from host memory).
__global__ void k_static_setup(const SysDev d, SysDev* dst, int2* mapC, int nC, int2* mapB, int nB) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = d;
    for (int q = threadIdx.x; q < nC; q += blockDim.x) mapC[q] = make_int2(0, q);
    for (int q = threadIdx.x; q < nB; q += blockDim.x) mapB[q] = make_int2(0, q);
}

int ilog2i(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v) ++l;
    return l;
}

// Once per device, with that device current: the device address of the scratch array
// (host code cannot use the symbol itself) and the shared-memory limits of the kernels.
// The shared-memory limits are raised, never lowered (smol_attr.h), so a system created
// later with smaller needs cannot break this entry point, and it cannot break them.
int setup_device(int dev) {
    if (dev < 0 || dev >= MAX_DEVICES) return SMOL_EUNSUPPORTED;
    if (g_ready[dev].load(std::memory_order_acquire)) return SMOL_OK;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (g_ready[dev].load(std::memory_order_relaxed)) return SMOL_OK;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return SMOL_ECUDA;
    const int smax = 2 * 256 * 2 * SMAX_T * 16 + 5 * 256 * 16;  // row pass at Mp = SMAX_M
    if (smol_host::raise_smem(k_rows<double>, smax) != cudaSuccess ||
        smol_host::raise_smem(k_fwd_cols<double>, 96 * 1024) != cudaSuccess ||
        smol_host::raise_smem(k_inv_cols<double>, 96 * 1024) != cudaSuccess)
        return SMOL_ECUDA;
    g_scratch_ptr[dev] = (unsigned char*)p;
    g_ready[dev].store(true, std::memory_order_release);
    return SMOL_OK;
}

int threads_for_s(int points) {
    int t = points / 8;
    if (t > 256) t = 256;
    if (t < 32) t = 32;
    return (t + 31) & ~31;
}

}  // namespace

extern "C" int smol_rhs_static(int64_t M, int32_t R, const double* d_U, const double* d_V, double lambda,
                               const double* d_n, double* d_out, void* stream) {
    if (M < 1 || R < 1 || !d_U || !d_V || !d_n || !d_out || !(lambda >= 0.0)) return SMOL_EINVAL;
    if (M > SMAX_M || R > SMAX_R) return SMOL_EUNSUPPORTED;
    if (((uintptr_t)d_n & 15) || ((uintptr_t)d_out & 15)) return SMOL_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SMOL_ECUDA;
    int rc = setup_device(dev);
    if (rc != SMOL_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = g_scratch_ptr[dev];

    const int lgMp = ilog2i(M < 4 ? 4 : M);
    const int Mp = 1 << lgMp;
    const int lgN1 = (lgMp + 1) / 2, lgN2 = lgMp / 2;
    const int N1 = 1 << lgN1, N2 = 1 << lgN2;
    int G = 256 / N1;
    if (G < 1) G = 1;
    if (G > N2) G = N2;
    const int T = 2 * R;

    SysDev d;
    memset(&d, 0, sizeof(d));
    d.M = (int)M;
    d.Mp = Mp;
    d.lgMp = lgMp;
    d.N1 = N1;
    d.N2 = N2;
    d.lgN1 = lgN1;
    d.lgN2 = lgN2;
    d.G = G;
    d.T = T;
    d.R = R;
    d.lambda = lambda;
    d.bnorm = 0.5 / (double)Mp;
    d.nbx = N2 / G;
    d.npairs = R;
    for (int a = 0; a < R; ++a) {
        d.au[a] = a;
        d.av[a] = R + a;
        d.acoef[a] = 1.0;
        d.pu[a] = a;
        d.pv[a] = R + a;
        d.pcoef[a] = 1.0;
    }
    d.W = base + OFF_W;
    d.tw = base + OFF_TW;
    d.twc = base + OFF_TWC;
    d.twr = base + OFF_TWR;
    d.tws = base + OFF_TWS;
    d.Y = base + OFF_Y;
    d.G2 = base + OFF_G2;
    d.ybuf = base + OFF_YBUF;
    d.mpart = (double*)(base + OFF_MPART);
    d.rsc = (double*)(base + OFF_RSC);
    d.ctl = (Ctl*)(base + OFF_CTL);
    SysDev* dsys = (SysDev*)(base + OFF_SYS);
    int2* mapC = (int2*)(base + OFF_MAPC);
    int2* mapB = (int2*)(base + OFF_MAPB);

    // The control block must read "not done" and the weights must be zero beyond M:
    // both are rewritten on every call, since the array keeps the previous call's data.
    if (cudaMemsetAsync(d.ctl, 0, sizeof(Ctl), st) != cudaSuccess) return SMOL_ECUDA;
    k_static_setup<<<1, 256, 0, st>>>(d, dsys, mapC, N2 / G, mapB, N1 / 2 + 1);
    k_static_weights<<<256, 256, 0, st>>>(d_U, d_V, (int)M, Mp, R, (double*)(base + OFF_W));
    k_static_twiddles<<<64, 256, 0, st>>>(Mp, N1, N2, (double2*)(base + OFF_TW), (double2*)(base + OFF_TWC),
                                          (double2*)(base + OFF_TWR), (double2*)(base + OFF_TWS));

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
    eo.hfac = 1.0;
    const size_t n = (size_t)N1 * G;
    const size_t sc = 2 * n * T * 16 + (size_t)N1 * 16 + n * 16 + n * 8;  // >= the inverse pass's need
    const size_t sr = std::max<size_t>(2 * (size_t)N2 * 2 * T * 16 + 5 * (size_t)N2 * 16, (4 * MAXT + 1) * 8);
    SysDev none;
    memset(&none, 0, sizeof(none));
    k_fwd_cols<double><<<N2 / G, threads_for_s(N1 * G * T), sc, st>>>(dsys, mapC, none, in);
    k_rows<double><<<N1 / 2 + 1, threads_for_s(N2 * 2 * T), sr, st>>>(dsys, mapB, none, in);
    k_inv_cols<double><<<N2 / G, threads_for_s(N1 * G), sc, st>>>(dsys, mapC, none, in, eo);
    return cudaGetLastError() == cudaSuccess ? SMOL_OK : SMOL_ECUDA;
}
