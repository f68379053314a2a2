// smol_persist.cuh - the persistent attempt kernel: a chunk of RKF45 attempts of one
// system (Sec. 2) in a single cooperative launch.
//
// The graph path launches 13 kernels per attempt (forward columns, 6 x rows, 5 x fused
// inverse + forward columns, inverse + combination); at the sizes of the paper's
// workloads each of them is short and bound by its own latency. Here one grid of CTAs,
// all resident at once (cooperative launch), runs the same phases back to back,
// separated by grid-wide barriers: column phase (inverse pass of the previous stage and
// forward pass of the next), barrier, row phase (row transforms, product sum, inverse
// rows; unit 0 forms the evaluation's scalars), barrier, ... and the final column phase
// with the combination and the controller, barrier, next attempt. Each phase runs the
// same device functions as the separate kernels, on the same element-to-unit maps, so
// the results are those of the graph path. Every CTA takes the units u = blockIdx.x,
// + gridDim.x, ... of a phase; data written by another CTA earlier in the kernel is read
// through L2 (ld.cg, cp.async.cg), never from an SM's L1.
//
// Barrier waits are bounded: a CTA that waits longer than about BAR_WAIT_CYCLES clocks
// marks the system's status SMOL_ETIMEOUT (done) and returns; the others then time out
// or see the status, so the kernel always ends.
#pragma once
#include "smol_int.cuh"

namespace smol {

enum { ST_ETIMEOUT = -6 };
constexpr long long BAR_WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// The stages of one RKF45 attempt and its final combination.
struct PersistPlan {
    StageIn in[6];
    EpiOut eo[6];
    Comb2 fin;
    CtlParams P;
};

// GPU-scope acquire load and release store (PTX memory model; the acquire-release
// atomic add is in smol_rhs.cuh): the CTA's writes, ordered before its thread 0 by the
// block barrier, are released with the arrival and acquired by every CTA that sees the
// new generation (cumulativity), without a full fence on either side.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier of a cooperative launch on bar[0] (arrival count) and bar[BAR_GEN]
// (generation, on its own 128-byte line, so that the polling does not contend with the
// arrivals). Returns false when the wait gave up (and then marks the status).
constexpr int BAR_GEN = 32;
__device__ __forceinline__ bool grid_barrier(unsigned* bar, Ctl* ctl, int* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned gen = ld_acquire(bar + BAR_GEN);  // read before arriving: it cannot advance before then
        int ok = 1;
        if (atom_add_acq_rel(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0u;  // ordered before the release below; every CTA has arrived
            st_release(bar + BAR_GEN, gen + 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(bar + BAR_GEN) == gen) {
                if (clock64() - t0 > BAR_WAIT_CYCLES) {
                    ok = 0;
                    break;
                }
            }
        }
        if (!ok) {
            atomicExch(&ctl->status, (int)ST_ETIMEOUT);
            atomicExch(&ctl->done, 1);
        }
        *flag = ok;
    }
    __syncthreads();
    return *flag != 0;
}

template <typename R>
__global__ void __launch_bounds__(256, 1) k_persist(const __grid_constant__ SysDev one,
                                                 const __grid_constant__ PersistPlan pl, int nattempts,
                                                 unsigned* bar) {
    __shared__ __align__(16) SysDev S;
    __shared__ CtlView cv;
    __shared__ InvSm<R> sm;
    __shared__ double red[2 * MAXT][8];
    __shared__ FinSm f;
    __shared__ __align__(16) Ctl cs;
    __shared__ R pc[MAXR];
    __shared__ int bflag;
    extern __shared__ __align__(16) unsigned char smraw[];
    load_desc(nullptr, nullptr, one, S);
    const int nC = S.nbx, nB = (S.N1 >> 1) + 1;
    for (int att = 0; att < nattempts; ++att) {
        load_ctl_fields(S, cv);
        if (cv.done) return;
        for (int e = 0; e < 6; ++e) {
            // column phase: inverse pass of stage e - 1 and forward pass of stage e
            for (int bx = blockIdx.x; bx < nC; bx += gridDim.x) {
                const ColSm<R> m = col_sm<R>(S, smraw);
                stage_tw(m.twP, S.lgN1, reinterpret_cast<const cx<R>*>(S.tw), S.lgMp);
                typename vec2<R>::T wpre[WPRE];
                fwd_prologue<R>(S, bx, m, wpre);
                if (e == 0) {
                    if (reused(pl.in[0], cv)) {
                        cp_async_wait();
                    } else {
                        fwd_body<R>(S, cv, pl.in[0], bx, m, wpre, true, red);
                    }
                } else {
                    if (reused(pl.in[e - 1], cv)) {
                        cp_async_wait();
                        stage_tw_fix(m.twP, S.lgN1, S.lgMp);
                        rescale_k1<R>(S, cv, pl.eo[e - 1], bx);
                    } else {
                        inv_body<R, true>(S, cv, pl.in[e - 1], pl.eo[e - 1], bx, m, sm);
                    }
                    __syncthreads();  // the forward pass reuses the tile buffers
                    fwd_body<R>(S, cv, pl.in[e], bx, m, wpre, false, red);
                }
                __syncthreads();  // shared memory of the next unit
            }
            if (!grid_barrier(bar, S.ctl, &bflag)) return;
            // row phase: unit 0 the evaluation's scalars, unit b + 1 row pair b
            if (!reused(pl.in[e], cv)) {
                for (int u = blockIdx.x; u < nB; u += gridDim.x) {
                    if (u == 0) {
                        double* sh = reinterpret_cast<double*>(smraw);
                        scalar_prologue<R>(S, sh);
                        __syncthreads();
                        finalize_scalars<R>(S, cv, pl.in[e], sh);
                    } else {
                        const RowSm<R> m = row_sm<R>(S, smraw);
                        row_prologue<R>(S, u - 1, m);
                        row_body<R, true>(S, cv, u - 1, m, pc);
                    }
                    __syncthreads();
                }
            }
            if (!grid_barrier(bar, S.ctl, &bflag)) return;
        }
        // final column phase: inverse pass of stage 5, combination, error, controller
        for (int bx = blockIdx.x; bx < nC; bx += gridDim.x) {
            const ColSm<R> m = col_sm<R>(S, smraw);
            stage_tw(m.twP, S.lgN1, reinterpret_cast<const cx<R>*>(S.tw), S.lgMp);
            copy_ctl(S.ctl, cs);
            inv_body<R, true>(S, cv, pl.in[5], pl.eo[5], bx, m, sm);
            double* outp = const_cast<double*>(cv.cur ? cv.s0 : cv.s1);
            void* shad = cv.cur ? S.shadow0 : S.shadow1;
            const Terms<R> tp = resolve_terms<R>(pl.fin.in, S, cv, false);
            FinAcc acc = fin_acc();
            const Div DG = mkdiv(S.G);
            const int half = (S.N1 >> 1) * S.G;
            for (int idx = threadIdx.x; idx < half; idx += blockDim.x) {
                const int i = col_elem(S, DG, bx, idx);
                if (i < S.M) fin_pair<R>(S, pl.fin, tp, outp, shad, i, acc, cv.tlog);
            }
            fin_tail<R>(S, pl.P, S.ctl, cs, bx, nC, acc, f);
            __syncthreads();
        }
        if (!grid_barrier(bar, S.ctl, &bflag)) return;
    }
}

}  // namespace smol
