// FP64 host arithmetic of the set-up (shared by the single-problem and the
// batched plans): local blocks, their inverses, alpha, omega*, and the
// transfer matrices.
#pragma once

#include <math.h>

#include "tmg_plan.h"

namespace tmg_host {

// ------------------------------------------------ FP64 set-up arithmetic --
//
// Shifted Legendre basis psi_k(s) = P_k(2s-1) on the reference interval.
// Legendre identities give the local matrices of Section 2 in closed form:
//   K[k,l] = 1 - 2 [l < k and k + l odd]   (from P_k(1) = 1 and the expansion of P_k')
//   Mhat   = diag(1 / (2k + 1))             (orthogonality)
//   a_k    = P_k(-1) = (-1)^k,  b_l = P_l(1) = 1.

inline void local_blocks(int d, double z, double* A) {
    for (int k = 0; k < d; ++k)
        for (int l = 0; l < d; ++l) {
            double v = (l < k && ((k + l) & 1)) ? -1.0 : 1.0;
            if (k == l) v += z / (2.0 * k + 1.0);
            A[k * d + l] = v;
        }
}

// Gauss-Jordan inversion with partial pivoting; returns false if singular.
inline bool invert(int d, const double* A, double* Ainv) {
    double M[tmg::kMaxDWide][2 * tmg::kMaxDWide];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < 2 * d; ++j) M[i][j] = j < d ? A[i * d + j] : (j - d == i ? 1.0 : 0.0);
    for (int c = 0; c < d; ++c) {
        int piv = c;
        for (int r = c + 1; r < d; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (M[piv][c] == 0.0) return false;
        if (piv != c)
            for (int j = 0; j < 2 * d; ++j) {
                double t = M[c][j];
                M[c][j] = M[piv][j];
                M[piv][j] = t;
            }
        const double inv = 1.0 / M[c][c];
        for (int j = 0; j < 2 * d; ++j) M[c][j] *= inv;
        for (int r = 0; r < d; ++r) {
            if (r == c || M[r][c] == 0.0) continue;
            const double m = M[r][c];
            for (int j = 0; j < 2 * d; ++j) M[r][j] -= m * M[c][j];
        }
    }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Ainv[i * d + j] = M[i][j + d];
    return true;
}

// Constants of L^T written in reversed time: diagonal block A^T with coupling
// a' = 1, b' = a, so g' = A^{-T} 1 = (b^T A^{-1})^T = c, c' = a^T A^{-T} = g,
// and alpha' = a^T A^{-T} 1 = alpha (the same omega*).
inline void level_setup_adjoint(int d, const tmg_level_host& F, tmg_level_host* L) {
    L->N = F.N;
    L->z = F.z;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            L->A[i * d + j] = F.A[j * d + i];
            L->Ainv[i * d + j] = F.Ainv[j * d + i];
        }
    for (int k = 0; k < d; ++k) {
        L->g[k] = F.c[k];
        L->c[k] = F.g[k];
    }
    L->alpha = F.alpha;
    L->omega = F.omega;
}

inline void level_setup(int d, double z, double omega_user, tmg_level_host* L) {
    L->z = z;
    local_blocks(d, z, L->A);
    invert(d, L->A, L->Ainv);
    double al = 0.0;
    for (int k = 0; k < d; ++k) {
        double gk = 0.0, ck = 0.0;
        for (int l = 0; l < d; ++l) {
            gk += L->Ainv[k * d + l] * ((l & 1) ? -1.0 : 1.0);   // A^{-1} a
            ck += L->Ainv[l * d + k];                              // (b^T A^{-1})_k
        }
        L->g[k] = gk;
        L->c[k] = ck;
        al += gk;                                                  // b^T A^{-1} a
    }
    L->alpha = al;
    // Lemma chap4_lemma7: omega* = 1/(1+alpha^2) for alpha >= 0, else 1
    L->omega = omega_user > 0.0 ? omega_user : (al >= 0.0 ? 1.0 / (1.0 + al * al) : 1.0);
}

// Prolongation matrices of Section 4.2: column k of P1 (P2) holds the Legendre
// coefficients, on the fine interval, of coarse basis function k restricted to
// the first (second) half.  With x the fine variable on [-1,1] the coarse
// argument is (x - 1)/2 on the first half and (x + 1)/2 on the second, so the
// columns follow from composing P_k with that affine map and converting the
// monomial coefficients back to the Legendre basis (exact polynomial algebra).
// For blocks wider than 11 coefficients the monomial route loses digits (the
// monomial coefficients of P_20 reach 1e5 and cancel), so the columns come
// from the three-term recurrence written in the Legendre basis itself:
// P_{k+1}(y) = ((2k+1) y P_k(y) - k P_{k-1}(y)) / (k+1) with y = (x -+ 1)/2,
// where multiplying a Legendre series by x maps coefficient c_i to
// (i+1)/(2i+1) on P_{i+1} and i/(2i+1) on P_{i-1}.
inline void transfer_setup_recurrence(int d, double* P1, double* P2) {
    constexpr int M = tmg::kMaxDWide;
    for (int half = 0; half < 2; ++half) {
        const double shift = half == 0 ? -1.0 : 1.0;
        double* P = half == 0 ? P1 : P2;
        double prev[M + 1] = {0}, cur[M + 1] = {0};
        cur[0] = 1.0;                          // P_0
        for (int k = 0; k < d; ++k) {
            for (int j = 0; j < d; ++j) P[j * d + k] = j <= k ? cur[j] : 0.0;
            if (k + 1 == d) break;
            double y[M + 1] = {0};            // y * (series cur), y = (x + shift) / 2
            for (int j = 0; j <= k + 1 && j < M; ++j) {
                double xv = 0.0;
                if (j >= 1) xv += cur[j - 1] * j / (2.0 * j - 1.0);
                if (j + 1 <= k) xv += cur[j + 1] * (j + 1.0) / (2.0 * j + 3.0);
                y[j] = 0.5 * (xv + shift * cur[j]);
            }
            double next[M + 1] = {0};
            for (int j = 0; j <= k + 1 && j < M; ++j) next[j] = ((2.0 * k + 1.0) * y[j] - k * prev[j]) / (k + 1.0);
            for (int j = 0; j < M; ++j) {
                prev[j] = cur[j];
                cur[j] = next[j];
            }
        }
    }
}

inline void transfer_setup(int d, double* P1, double* P2) {
    if (d > 11) {
        transfer_setup_recurrence(d, P1, P2);
        return;
    }
    constexpr int M = tmg::kMaxDWide;
    double leg[M][M] = {{0}};   // monomial coefficients of P_0..P_{d-1}
    leg[0][0] = 1.0;
    if (d > 1) leg[1][1] = 1.0;
    for (int k = 1; k + 1 < d; ++k)   // (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}
        for (int j = 0; j < M; ++j) {
            double v = -k * leg[k - 1][j];
            if (j > 0) v += (2.0 * k + 1.0) * leg[k][j - 1];
            leg[k + 1][j] = v / (k + 1.0);
        }
    for (int half = 0; half < 2; ++half) {
        const double shift = half == 0 ? -1.0 : 1.0;
        double* P = half == 0 ? P1 : P2;
        for (int k = 0; k < d; ++k) {
            // q(x) = P_k((x + shift) / 2) in monomials
            double q[M] = {0};
            for (int j = 0; j < d; ++j) {
                if (leg[k][j] == 0.0) continue;
                // ((x + shift)/2)^j = 2^-j sum_i C(j,i) x^i shift^(j-i)
                double binom = 1.0;
                for (int i = 0; i <= j; ++i) {
                    if (i > 0) binom = binom * (j - i + 1) / i;
                    q[i] += leg[k][j] * ldexp(binom * pow(shift, j - i), -j);
                }
            }
            // convert to Legendre coefficients, highest degree first
            for (int j = d - 1; j >= 0; --j) {
                const double cj = q[j] / leg[j][j];
                P[j * d + k] = cj;
                for (int i = 0; i <= j; ++i) q[i] -= cj * leg[j][i];
            }
        }
    }
}

}  // namespace tmg_host
