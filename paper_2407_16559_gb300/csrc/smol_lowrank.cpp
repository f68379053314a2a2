// smol_lowrank.cpp - smol_lowrank_kernel: low-rank factors K ~= U V of a collision
// kernel that has no exact low rank (the free-molecular kernel of Sec. 3.1), so that the
// O(M R log M) right-hand side of Sec. 1 applies to it. The paper takes such factors
// from the cross (skeleton) approximation of its reference [matveev2015fast]; this is a
// symmetric adaptive cross approximation of the kernel matrix, host code only.
//
// Method. The matrix is scaled to G = D^-1 K D^-1 with D = diag(sqrt |K_ii|), so that
// every diagonal entry is +-1 and the approximation error is measured relative to the
// local size of K. Each step takes the row p of largest residual diagonal |R_pp| and
// evaluates the residual row R_p. = G_p. - sum_l s_l u_l[p] u_l (the kernel is
// evaluated only on that row: O(k M) work per step). If |R_pp| >= alpha max |R_p.| the
// step is a 1 x 1 pivot, u = R_p. / sqrt |R_pp| with sign s = sign R_pp (the adaptive
// cross approximation of Bebendorf, Numer. Math. 86 (2000), with diagonal pivots, i.e.
// the pivoted Cholesky decomposition of Harbrecht, Peters and Schneider, Appl. Numer.
// Math. 62 (2012), extended to indefinite matrices by signs); otherwise it is a 2 x 2
// pivot on rows p and q = argmax |R_p.| (the partial pivoting of Bunch and Kaufman,
// Math. Comp. 31 (1977), alpha = (1 + sqrt 17) / 8), whose 2 x 2 block is diagonalised
// into two signed terms. The residual diagonal is updated after every term; the
// iteration stops when it and the last residual row are below tol (relative to the
// largest entry of G), or at max_rank terms.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/smol.h"

namespace {

double kernel_entry(int kind, const double* par, double i, double j) {
    switch (kind) {
        case SMOL_KERNEL_CONST:
            return 1.0;
        case SMOL_KERNEL_BROWNIAN: {
            const double a = par ? par[0] : 0.0, c = par ? par[1] : 0.0;
            return pow(i / j, a) + pow(j / i, a) + c;
        }
        case SMOL_KERNEL_FREE_MOLECULAR: {
            const double s = cbrt(i) + cbrt(j);
            return s * s * sqrt(1.0 / i + 1.0 / j);
        }
        default:
            return NAN;
    }
}

struct Cross {
    int kind;
    const double* par;
    int64_t M;
    std::vector<double> dsc;           // D: sqrt |K_ii|
    std::vector<std::vector<double>> u;  // terms u_l (scaled), length M each
    std::vector<double> s;             // their signs

    // residual row p of G: G_p. - sum_l s_l u_l[p] u_l
    void residual_row(int64_t p, std::vector<double>& r) const {
        const double ip = (double)(p + 1), dp = dsc[p];
        for (int64_t j = 0; j < M; ++j) r[j] = kernel_entry(kind, par, ip, (double)(j + 1)) / (dp * dsc[j]);
        for (size_t l = 0; l < u.size(); ++l) {
            const double c = s[l] * u[l][p];
            if (c == 0.0) continue;
            const double* ul = u[l].data();
            for (int64_t j = 0; j < M; ++j) r[j] -= c * ul[j];
        }
    }
};

}  // namespace

extern "C" int smol_lowrank_kernel(int32_t kind, const double* params, int64_t M, double tol, int32_t max_rank,
                                   double* h_U, double* h_V, int32_t* rank, double* err_est) {
    if (M < 1 || !(tol > 0.0) || max_rank < 1 || !h_U || !h_V || !rank) return SMOL_EINVAL;
    if (kind != SMOL_KERNEL_CONST && kind != SMOL_KERNEL_BROWNIAN && kind != SMOL_KERNEL_FREE_MOLECULAR)
        return SMOL_EINVAL;
    if (kind == SMOL_KERNEL_BROWNIAN && (!params || !isfinite(params[0]) || !isfinite(params[1]))) return SMOL_EINVAL;
    Cross X;
    X.kind = kind;
    X.par = params;
    X.M = M;
    X.dsc.resize(M);
    std::vector<double> d(M);  // residual diagonal of G
    for (int64_t i = 0; i < M; ++i) {
        const double kii = kernel_entry(kind, params, (double)(i + 1), (double)(i + 1));
        if (!isfinite(kii) || kii == 0.0) return SMOL_EINVAL;  // the scaling needs a nonzero diagonal
        X.dsc[i] = sqrt(fabs(kii));
        d[i] = kii > 0.0 ? 1.0 : -1.0;
    }
    const double alpha = (1.0 + sqrt(17.0)) / 8.0;
    std::vector<double> rp(M), rq(M);
    double gmax = 1.0;  // largest |G| seen (the diagonal's is 1)
    while ((int)X.u.size() < max_rank) {
        int64_t p = 0;
        for (int64_t i = 1; i < M; ++i)
            if (fabs(d[i]) > fabs(d[p])) p = i;
        X.residual_row(p, rp);
        int64_t q = 0;
        double rmax = 0.0;
        for (int64_t j = 0; j < M; ++j)
            if (fabs(rp[j]) > rmax) {
                rmax = fabs(rp[j]);
                q = j;
            }
        gmax = std::max(gmax, rmax);
        if (rmax <= tol * gmax && fabs(d[p]) <= tol * gmax) break;
        const double rpp = rp[p];
        if (fabs(rpp) >= alpha * rmax || (int)X.u.size() + 1 == max_rank || q == p) {
            // 1 x 1 pivot
            const double sc = 1.0 / sqrt(fabs(rpp));
            std::vector<double> u(M);
            for (int64_t j = 0; j < M; ++j) u[j] = rp[j] * sc;
            const double sg = rpp > 0.0 ? 1.0 : -1.0;
            for (int64_t j = 0; j < M; ++j) d[j] -= sg * u[j] * u[j];
            X.u.push_back(std::move(u));
            X.s.push_back(sg);
        } else {
            // 2 x 2 pivot on rows p, q: R ~= [r_p r_q]^T P^-1 [r_p r_q], P = [[a, b], [b, c]]
            X.residual_row(q, rq);
            const double a = rp[p], b = rp[q], c = rq[q];
            // P = Q diag(l1, l2) Q^T (symmetric 2 x 2 eigen-decomposition)
            const double tr = 0.5 * (a + c), df = 0.5 * (a - c);
            const double rad = sqrt(df * df + b * b);
            const double l1 = tr + rad, l2 = tr - rad;
            double cs, sn;  // eigenvector of l1: (cs, sn)
            if (rad == 0.0) {
                cs = 1.0;
                sn = 0.0;
            } else {
                const double th = 0.5 * atan2(b, df);
                cs = cos(th);
                sn = sin(th);
            }
            // P^-1 = Q diag(1/l1, 1/l2) Q^T; terms u_k = (Q^T [r_p; r_q])_k / sqrt |l_k|
            const double lam[2] = {l1, l2};
            const double q0[2] = {cs, -sn}, q1[2] = {sn, cs};  // rows of Q^T: (cs, sn), (-sn, cs)
            for (int k = 0; k < 2; ++k) {
                if (lam[k] == 0.0) continue;
                const double ca = k == 0 ? q0[0] : q0[1], cb = k == 0 ? q1[0] : q1[1];
                const double sc = 1.0 / sqrt(fabs(lam[k]));
                std::vector<double> u(M);
                for (int64_t j = 0; j < M; ++j) u[j] = (ca * rp[j] + cb * rq[j]) * sc;
                const double sg = lam[k] > 0.0 ? 1.0 : -1.0;
                for (int64_t j = 0; j < M; ++j) d[j] -= sg * u[j] * u[j];
                X.u.push_back(std::move(u));
                X.s.push_back(sg);
            }
        }
    }
    const int r = (int)X.u.size();
    if (r == 0) return SMOL_EINVAL;
    // U (M x r, row-major) = D u, V (r x M, row-major) = s D u^T
    for (int64_t i = 0; i < M; ++i)
        for (int k = 0; k < r; ++k) h_U[(size_t)i * r + k] = X.dsc[i] * X.u[k][i];
    for (int k = 0; k < r; ++k)
        for (int64_t j = 0; j < M; ++j) h_V[(size_t)k * M + j] = X.s[k] * X.dsc[j] * X.u[k][j];
    *rank = r;
    if (err_est) {
        // largest relative entry error max |K^ - K| / |K| on sampled rows: the first and
        // last 8, and every ceil(M / 64)-th
        double e = 0.0;
        const int64_t stride = std::max<int64_t>(1, (M + 63) / 64);
        std::vector<int64_t> rows;
        for (int64_t i = 0; i < std::min<int64_t>(8, M); ++i) rows.push_back(i);
        for (int64_t i = 8; i < M - 8; i += stride) rows.push_back(i);
        for (int64_t i = std::max<int64_t>(8, M - 8); i < M; ++i) rows.push_back(i);
        for (int64_t i : rows)
            for (int64_t j = 0; j < M; ++j) {
                double kh = 0.0;
                for (int k = 0; k < r; ++k) kh += h_U[(size_t)i * r + k] * h_V[(size_t)k * M + j];
                const double kx = kernel_entry(kind, params, (double)(i + 1), (double)(j + 1));
                e = std::max(e, fabs(kh - kx) / fabs(kx));
            }
        *err_est = e;
    }
    return SMOL_OK;
}
