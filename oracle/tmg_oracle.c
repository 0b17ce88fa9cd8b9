/*
 * Oracle for the time-multigrid solve of Gander & Neumueller, "Analysis of a
 * Time Multigrid Algorithm for DG-Discretizations in Time" (arXiv:1409.5254).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct FP64 C.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no code, header or constant with the CUDA path.
 *
 * Everything here follows the paper's definitions literally:
 *   - local DG matrices K, M, N and the per-interval system, Section 2
 *     ("Linear system", eq. chap4_generalLinearSystemODE), built by Gauss
 *     quadrature from the definitions of K[k,l], M[k,l], N[k,l];
 *   - the block forward substitution that solves that block lower-bidiagonal
 *     system exactly (Section 2, the system itself);
 *   - the damped block Jacobi smoother, eq. chap4_ODESmoother (Section 3);
 *   - restriction/prolongation R = [R1 R2], P = R^T with R_i^T = M^{-1} Mtilde^i,
 *     eqs. chap4_restrictionTime / chap4_prolongationTime (Section 4.2);
 *   - the two-grid / multigrid cycle of eq. chap4_errorTwoGridCycle, recursed
 *     on the nested meshes of Section 3 (V-cycle gamma=1, W-cycle gamma=2);
 *   - the optimised damping omega* of Lemma chap4_lemma7 (Section 4.1);
 *   - the transposed system L^T mu = g solved backward in time (adjoint).
 *
 * Basis: shifted Legendre polynomials psi_k(s) = P_k(2s-1) on the reference
 * interval s in [0,1] (the paper allows any basis of P^{p_t}).  For the
 * generalised model u' + lambda u = f every local matrix depends on the step
 * only through z = lambda * tau: A(z) = K + z * Mhat with Mhat the reference
 * mass matrix, because K and N do not depend on tau and M_tau = tau * Mhat.
 *
 * Vectors are interval-major: u[n*d + k] is coefficient k of interval n
 * (0-based), d = p+1.  The initial value u0 enters the first interval's right
 * hand side as a*u0 (the term u^{n-1}(t_{n-1}) v(t_{n-1}) of eq.
 * chap4_discreteVarFormODE for n = 1).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Degrees p = 0..20 (d <= 21).  The 22-point Gauss rule integrates every
 * product of two basis functions (degree <= 2p = 40) exactly. */
#define ORC_MAXD 21
#define ORC_PI 3.14159265358979323846
#define ORC_NQ 22

/* ---------------------------------------------------------------- basis -- */

/* The quadratures below run in long double so that the FP64 blocks are the
 * correctly rounded values of their definitions (the same rule summed in
 * double leaves errors of a few 1e-15 already in the p = 3 entries). */
typedef long double ldbl;

/* Largest degree p the oracle accepts. */
int orc_max_degree(void) { return ORC_MAXD - 1; }

/* Legendre P_k(x) and P_k'(x) for k = 0..n-1 by the three-term recurrence. */
static void legendre(int n, ldbl x, ldbl *P, ldbl *dP) {
    P[0] = 1.0L; dP[0] = 0.0L;
    if (n > 1) { P[1] = x; dP[1] = 1.0L; }
    for (int k = 1; k + 1 < n; ++k) {
        P[k + 1] = ((2.0L * k + 1.0L) * x * P[k] - k * P[k - 1]) / (k + 1.0L);
        dP[k + 1] = dP[k - 1] + (2.0L * k + 1.0L) * P[k];
    }
}

/* Gauss-Legendre nodes/weights on [0,1] by Newton's method on P_q. */
static void gauss01(int q, ldbl *x01, ldbl *w01) {
    ldbl P[ORC_NQ + 2], dP[ORC_NQ + 2];
    for (int i = 0; i < q; ++i) {
        ldbl x = cosl(ORC_PI * (i + 0.75L) / (q + 0.5L));
        for (int it = 0; it < 100; ++it) {
            legendre(q + 1, x, P, dP);
            ldbl dx = P[q] / dP[q];
            x -= dx;
            if (fabsl(dx) < 1e-30L) break;
        }
        legendre(q + 1, x, P, dP);
        x01[i] = 0.5L * (x + 1.0L);
        w01[i] = 0.5L * 2.0L / ((1.0L - x * x) * dP[q] * dP[q]);
    }
}

/* Shifted basis psi_k(s) = P_k(2s-1) and its s-derivative. */
static void shifted(int d, ldbl s, ldbl *psi, ldbl *dpsi) {
    ldbl P[ORC_MAXD], dP[ORC_MAXD];
    legendre(d, 2.0L * s - 1.0L, P, dP);
    for (int k = 0; k < d; ++k) { psi[k] = P[k]; dpsi[k] = 2.0L * dP[k]; }
}

/*
 * Local matrices on the reference interval (Section 2, definitions of
 * K_tau, M_tau, N_tau):
 *   K[k,l]   = -int_0^1 psi_l psi_k' ds + psi_l(1) psi_k(1)   (tau cancels)
 *   Mhat[k,l]=  int_0^1 psi_l psi_k ds                        (M_tau = tau*Mhat)
 *   N[k,l]   =  psi_l(1) psi_k(0) = a_k b_l  with a_k = psi_k(0), b_l = psi_l(1)
 * (psi_l^{n-1}(t_{n-1}) is the previous interval's basis at its right end.)
 * Row-major d x d.
 */
void orc_blocks(int p, double *K, double *Mhat, double *a, double *b) {
    int d = p + 1;
    ldbl xq[ORC_NQ], wq[ORC_NQ], psi[ORC_MAXD], dpsi[ORC_MAXD];
    ldbl Kl[ORC_MAXD * ORC_MAXD] = {0}, Ml[ORC_MAXD * ORC_MAXD] = {0};
    gauss01(ORC_NQ, xq, wq);
    for (int q = 0; q < ORC_NQ; ++q) {
        shifted(d, xq[q], psi, dpsi);
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) {
                Kl[k * d + l] -= wq[q] * psi[l] * dpsi[k];
                Ml[k * d + l] += wq[q] * psi[l] * psi[k];
            }
    }
    ldbl psi0[ORC_MAXD], psi1[ORC_MAXD];
    shifted(d, 0.0L, psi0, dpsi);
    shifted(d, 1.0L, psi1, dpsi);
    for (int k = 0; k < d; ++k) {
        a[k] = (double)psi0[k];
        b[k] = (double)psi1[k];
        for (int l = 0; l < d; ++l) {
            K[k * d + l] = (double)(Kl[k * d + l] + psi1[l] * psi1[k]);
            Mhat[k * d + l] = (double)Ml[k * d + l];
        }
    }
}

/* Diagonal block A(z) = K + z*Mhat of the system for step z = lambda*tau. */
static void block_A(int p, double z, double *A, double *a, double *b) {
    int d = p + 1;
    double K[ORC_MAXD * ORC_MAXD], Mh[ORC_MAXD * ORC_MAXD];
    orc_blocks(p, K, Mh, a, b);
    for (int i = 0; i < d * d; ++i) A[i] = K[i] + z * Mh[i];
}

/* ------------------------------------------------------- dense algebra -- */

/*
 * Solve A x = rhs (n x n, row-major) by Gaussian elimination with partial
 * pivoting.  A and rhs are copied; x may alias rhs.  Returns 0, or -1 if a
 * pivot is exactly zero.
 */
int orc_gesv(int n, const double *A_in, const double *rhs, double *x) {
    double *A = (double *)malloc(sizeof(double) * n * n);
    double *y = (double *)malloc(sizeof(double) * n);
    memcpy(A, A_in, sizeof(double) * n * n);
    memcpy(y, rhs, sizeof(double) * n);
    int status = 0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r * n + c]) > fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) { status = -1; break; }
        if (piv != c) {
            for (int j = 0; j < n; ++j) {
                double t = A[c * n + j]; A[c * n + j] = A[piv * n + j]; A[piv * n + j] = t;
            }
            double t = y[c]; y[c] = y[piv]; y[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double m = A[r * n + c] / A[c * n + c];
            if (m == 0.0) continue;
            for (int j = c; j < n; ++j) A[r * n + j] -= m * A[c * n + j];
            y[r] -= m * y[c];
        }
    }
    if (status == 0)
        for (int r = n - 1; r >= 0; --r) {
            double s = y[r];
            for (int j = r + 1; j < n; ++j) s -= A[r * n + j] * x[j];
            x[r] = s / A[r * n + r];
        }
    free(A);
    free(y);
    return status;
}

/* Small fixed-size solve with a local copy (d <= ORC_MAXD). */
static void solve_small(int d, const double *A, const double *rhs, double *x) {
    double tmp[ORC_MAXD];
    memcpy(tmp, rhs, sizeof(double) * d);
    orc_gesv(d, A, tmp, x);
}

static void transpose(int d, const double *A, double *At) {
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) At[j * d + i] = A[i * d + j];
}

/* alpha(z) = b^T A(z)^{-1} a: the nonzero eigenvalue of A^{-1}N (Lemma
 * chap4_theorem2), i.e. the stability function of the scheme at -z. */
double orc_alpha(int p, double z) {
    int d = p + 1;
    double A[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD], g[ORC_MAXD];
    block_A(p, z, A, a, b);
    solve_small(d, A, a, g);
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += b[k] * g[k];
    return s;
}

/* Asymptotically optimal damping of Lemma chap4_lemma7. */
double orc_omega_star(int p, double z) {
    double al = orc_alpha(p, z);
    return al >= 0.0 ? 1.0 / (1.0 + al * al) : 1.0;
}

/*
 * Local prolongation matrices (Section 4.2): P1 = R1^T = M^{-1} Mtilde^1 and
 * P2 = R2^T = M^{-1} Mtilde^2, where Mtilde^i[k,l] integrates the coarse basis
 * function l against fine basis function k over the i-th half of the coarse
 * interval.  In reference coordinates the fine variable is s in [0,1] and the
 * coarse variable is (s + i - 1)/2, and tau cancels against M^{-1}.
 * The second-half integral is read with the fine basis shifted to that half.
 */
void orc_transfer(int p, double *P1, double *P2) {
    int d = p + 1;
    ldbl xq[ORC_NQ], wq[ORC_NQ], psi[ORC_MAXD], dpsi[ORC_MAXD];
    ldbl cps[ORC_MAXD], cdps[ORC_MAXD];
    ldbl Mt1[ORC_MAXD * ORC_MAXD] = {0}, Mt2[ORC_MAXD * ORC_MAXD] = {0};
    ldbl Mh[ORC_MAXD * ORC_MAXD] = {0};
    gauss01(ORC_NQ, xq, wq);
    for (int q = 0; q < ORC_NQ; ++q) {
        shifted(d, xq[q], psi, dpsi);
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) Mh[k * d + l] += wq[q] * psi[k] * psi[l];
        shifted(d, 0.5L * xq[q], cps, cdps);          /* first half  */
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) Mt1[k * d + l] += wq[q] * cps[l] * psi[k];
        shifted(d, 0.5L * (xq[q] + 1.0L), cps, cdps);  /* second half */
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) Mt2[k * d + l] += wq[q] * cps[l] * psi[k];
    }
    /* The projected mass matrix is diagonal for an orthogonal basis but is
     * solved as a general system: P = Mh^{-1} Mt, column by column, by
     * Gaussian elimination in long double. */
    for (int half = 0; half < 2; ++half) {
        const ldbl *Mt = half == 0 ? Mt1 : Mt2;
        double *P = half == 0 ? P1 : P2;
        for (int l = 0; l < d; ++l) {
            ldbl Ag[ORC_MAXD][ORC_MAXD + 1];
            for (int k = 0; k < d; ++k) {
                for (int j = 0; j < d; ++j) Ag[k][j] = Mh[k * d + j];
                Ag[k][d] = Mt[k * d + l];
            }
            for (int c = 0; c < d; ++c) {
                int piv = c;
                for (int r = c + 1; r < d; ++r)
                    if (fabsl(Ag[r][c]) > fabsl(Ag[piv][c])) piv = r;
                for (int j = 0; j <= d; ++j) { ldbl t = Ag[c][j]; Ag[c][j] = Ag[piv][j]; Ag[piv][j] = t; }
                for (int r = c + 1; r < d; ++r) {
                    ldbl m = Ag[r][c] / Ag[c][c];
                    for (int j = c; j <= d; ++j) Ag[r][j] -= m * Ag[c][j];
                }
            }
            for (int r = d - 1; r >= 0; --r) {
                ldbl sacc = Ag[r][d];
                for (int j = r + 1; j < d; ++j) sacc -= Ag[r][j] * (ldbl)P[j * d + l];
                P[r * d + l] = (double)(sacc / Ag[r][r]);
            }
        }
    }
}

/* ------------------------------------------------- exact block solves -- */

/*
 * Block forward substitution for the system of eq.
 * chap4_generalLinearSystemODE with z = lambda*tau:
 *   (K + z Mhat) u_n = f_n + N u_{n-1},  N u_{n-1} = a (b^T u_{n-1}),
 * with b^T u_0 replaced by the initial value u0.  Each block solve is
 * Gaussian elimination.
 */
void orc_fsub(int p, double z, long N, const double *f, double u0, double *u) {
    int d = p + 1;
    double A[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD], rhs[ORC_MAXD];
    block_A(p, z, A, a, b);
    double e_prev = u0;
    for (long n = 0; n < N; ++n) {
        for (int k = 0; k < d; ++k) rhs[k] = f[n * d + k] + a[k] * e_prev;
        solve_small(d, A, rhs, &u[n * d]);
        double e = 0.0;
        for (int k = 0; k < d; ++k) e += b[k] * u[n * d + k];
        e_prev = e;
    }
}

/*
 * Brute force: assemble the whole (N d) x (N d) matrix of eq.
 * chap4_generalLinearSystemODE (diagonal blocks K + z Mhat, sub-diagonal
 * blocks -N) and solve it by Gaussian elimination.  For small N only.
 * Returns 0 on success.
 */
int orc_dense_solve(int p, double z, long N, const double *f, double u0, double *u) {
    int d = p + 1;
    long n = N * d;
    double A[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD];
    block_A(p, z, A, a, b);
    double *L = (double *)calloc((size_t)(n * n), sizeof(double));
    double *rhs = (double *)malloc(sizeof(double) * n);
    for (long blk = 0; blk < N; ++blk)
        for (int k = 0; k < d; ++k) {
            for (int l = 0; l < d; ++l) {
                L[(blk * d + k) * n + blk * d + l] = A[k * d + l];
                if (blk > 0) L[(blk * d + k) * n + (blk - 1) * d + l] = -a[k] * b[l];
            }
            rhs[blk * d + k] = f[blk * d + k] + (blk == 0 ? a[k] * u0 : 0.0);
        }
    int st = orc_gesv((int)n, L, rhs, u);
    free(L);
    free(rhs);
    return st;
}

/*
 * Apply L (eq. chap4_equationLinearSystemODE, zero initial value):
 * (L u)_n = A u_n - a (b^T u_{n-1}).
 */
static void apply_L(int d, const double *A, const double *a, const double *b,
                    long N, const double *u, double *out) {
    double e_prev = 0.0;
    for (long n = 0; n < N; ++n) {
        for (int k = 0; k < d; ++k) {
            double s = 0.0;
            for (int l = 0; l < d; ++l) s += A[k * d + l] * u[n * d + l];
            out[n * d + k] = s - a[k] * e_prev;
        }
        double e = 0.0;
        for (int k = 0; k < d; ++k) e += b[k] * u[n * d + k];
        e_prev = e;
    }
}

/* ------------------------------------------------------- multigrid -- */

typedef struct {
    int p, d, nlev, nu1, nu2, gamma;
    long *Nl;     /* intervals per level */
    double *z;    /* z_l = lambda * tau_l, tau_l = 2^l tau */
    double *om;   /* damping per level */
    double P1[ORC_MAXD * ORC_MAXD], P2[ORC_MAXD * ORC_MAXD];
    double a[ORC_MAXD], b[ORC_MAXD];
} orc_hier;

/* Levels: coarsen by two while the level has an even number of intervals,
 * more than n_min of them, and fewer than max_levels levels exist.  */
int orc_num_levels(long N, long n_min, int max_levels) {
    int L = 1;
    long n = N;
    while ((max_levels <= 0 || L < max_levels) && n % 2 == 0 && n > n_min && n / 2 >= 1) {
        n /= 2;
        ++L;
    }
    return L;
}

static void smooth(const orc_hier *h, int lev, long N, double *u, const double *f, int sweeps) {
    int d = h->d;
    double A[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD], rl[ORC_MAXD], c[ORC_MAXD];
    block_A(h->p, h->z[lev], A, a, b);
    double *Lu = (double *)malloc(sizeof(double) * N * d);
    for (int s = 0; s < sweeps; ++s) {
        /* eq. chap4_ODESmoother: u <- u + omega D^{-1} (f - L u) */
        apply_L(d, A, a, b, N, u, Lu);
        for (long n = 0; n < N; ++n) {
            for (int k = 0; k < d; ++k) rl[k] = f[n * d + k] - Lu[n * d + k];
            solve_small(d, A, rl, c);
            for (int k = 0; k < d; ++k) u[n * d + k] += h->om[lev] * c[k];
        }
    }
    free(Lu);
}

/* A cycle cut at level `stop`: mode 0 stops the way down there and hands out
 * that level's right-hand side; mode 1 takes that level's correction from the
 * caller instead of recursing (the coarse part of the cycle solved elsewhere,
 * e.g. on the gathered coarse problem of several time slabs). */
typedef struct {
    int stop, mode;
    double *fc_out;
    const double *uc_in;
} orc_split;

static void mg_cycle_s(const orc_hier *h, int lev, double *u, const double *f, const orc_split *sp);

static void mg_cycle(const orc_hier *h, int lev, double *u, const double *f) { mg_cycle_s(h, lev, u, f, NULL); }

static void mg_cycle_s(const orc_hier *h, int lev, double *u, const double *f, const orc_split *sp) {
    int d = h->d;
    long N = h->Nl[lev];
    if (sp && lev == sp->stop) {
        if (sp->mode == 0) memcpy(sp->fc_out, f, sizeof(double) * N * d);
        else memcpy(u, sp->uc_in, sizeof(double) * N * d);
        return;
    }
    if (lev == h->nlev - 1) {          /* coarsest level: exact solve */
        orc_fsub(h->p, h->z[lev], N, f, 0.0, u);
        return;
    }
    double A[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD];
    block_A(h->p, h->z[lev], A, a, b);
    smooth(h, lev, N, u, f, h->nu1);
    /* residual r = f - L u */
    double *r = (double *)malloc(sizeof(double) * N * d);
    apply_L(d, A, a, b, N, u, r);
    for (long i = 0; i < N * d; ++i) r[i] = f[i] - r[i];
    /* restriction f_c,m = R1 r_{2m} + R2 r_{2m+1}, R_i = P_i^T */
    long Nc = N / 2;
    double *fc = (double *)calloc((size_t)(Nc * d), sizeof(double));
    double *uc = (double *)calloc((size_t)(Nc * d), sizeof(double));
    for (long m = 0; m < Nc; ++m)
        for (int k = 0; k < d; ++k) {
            double s = 0.0;
            for (int l = 0; l < d; ++l)
                s += h->P1[l * d + k] * r[(2 * m) * d + l] + h->P2[l * d + k] * r[(2 * m + 1) * d + l];
            fc[m * d + k] = s;
        }
    for (int g = 0; g < h->gamma; ++g) mg_cycle_s(h, lev + 1, uc, fc, sp);
    if (sp && sp->mode == 0) {         /* the way down ended at sp->stop */
        free(r);
        free(fc);
        free(uc);
        return;
    }
    /* prolongation u_{2m} += P1 uc_m, u_{2m+1} += P2 uc_m */
    for (long m = 0; m < Nc; ++m)
        for (int k = 0; k < d; ++k) {
            double s1 = 0.0, s2 = 0.0;
            for (int l = 0; l < d; ++l) {
                s1 += h->P1[k * d + l] * uc[m * d + l];
                s2 += h->P2[k * d + l] * uc[m * d + l];
            }
            u[(2 * m) * d + k] += s1;
            u[(2 * m + 1) * d + k] += s2;
        }
    smooth(h, lev, N, u, f, h->nu2);
    free(r);
    free(fc);
    free(uc);
}

/*
 * Multigrid solve of L u = F (F = f with a*u0 added to the first interval).
 * Starts from u (initial guess, overwritten by the result).  Records the
 * relative residual ||F - L u_k||_2 / ||F||_2 before every cycle k in
 * hist[0..max_cycles] and returns the number of cycles done.  omega <= 0 means
 * omega*(alpha(z_l)) per level.  n_min/max_levels fix the hierarchy.
 */
int orc_mg_solve(int p, double z, long N, const double *f, double u0, double *u,
                 long n_min, int max_levels, int nu1, int nu2, int gamma, double omega,
                 double tol, int max_cycles, double *hist) {
    orc_hier h;
    int d = p + 1;
    h.p = p; h.d = d; h.nu1 = nu1; h.nu2 = nu2; h.gamma = gamma;
    h.nlev = orc_num_levels(N, n_min, max_levels);
    h.Nl = (long *)malloc(sizeof(long) * h.nlev);
    h.z = (double *)malloc(sizeof(double) * h.nlev);
    h.om = (double *)malloc(sizeof(double) * h.nlev);
    for (int l = 0; l < h.nlev; ++l) {
        h.Nl[l] = N >> l;
        h.z[l] = ldexp(z, l);
        h.om[l] = omega > 0.0 ? omega : orc_omega_star(p, h.z[l]);
    }
    orc_transfer(p, h.P1, h.P2);
    double K[ORC_MAXD * ORC_MAXD], Mh[ORC_MAXD * ORC_MAXD];
    orc_blocks(p, K, Mh, h.a, h.b);

    double *F = (double *)malloc(sizeof(double) * N * d);
    memcpy(F, f, sizeof(double) * N * d);
    for (int k = 0; k < d; ++k) F[k] += h.a[k] * u0;
    double A[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD];
    block_A(p, z, A, a, b);
    double *r = (double *)malloc(sizeof(double) * N * d);
    double nF = 0.0;
    for (long i = 0; i < N * d; ++i) nF += F[i] * F[i];
    nF = sqrt(nF);
    int k = 0;
    for (;; ++k) {
        apply_L(d, A, a, b, N, u, r);
        double nr = 0.0;
        for (long i = 0; i < N * d; ++i) { double t = F[i] - r[i]; nr += t * t; }
        double rel = nF > 0.0 ? sqrt(nr) / nF : sqrt(nr);
        if (hist) hist[k] = rel;
        if (rel <= tol || k >= max_cycles) break;
        mg_cycle(&h, 0, u, F);
    }
    free(r); free(F); free(h.Nl); free(h.z); free(h.om);
    return k;
}

/* One multigrid cycle applied to u for right hand side F (u0 already folded
 * into F).  For one-cycle parity checks. */
void orc_mg_one_cycle(int p, double z, long N, const double *F, double *u,
                      long n_min, int max_levels, int nu1, int nu2, int gamma, double omega) {
    orc_hier h;
    int d = p + 1;
    h.p = p; h.d = d; h.nu1 = nu1; h.nu2 = nu2; h.gamma = gamma;
    h.nlev = orc_num_levels(N, n_min, max_levels);
    h.Nl = (long *)malloc(sizeof(long) * h.nlev);
    h.z = (double *)malloc(sizeof(double) * h.nlev);
    h.om = (double *)malloc(sizeof(double) * h.nlev);
    for (int l = 0; l < h.nlev; ++l) {
        h.Nl[l] = N >> l;
        h.z[l] = ldexp(z, l);
        h.om[l] = omega > 0.0 ? omega : orc_omega_star(p, h.z[l]);
    }
    orc_transfer(p, h.P1, h.P2);
    double K[ORC_MAXD * ORC_MAXD], Mh[ORC_MAXD * ORC_MAXD];
    orc_blocks(p, K, Mh, h.a, h.b);
    mg_cycle(&h, 0, u, F);
    free(h.Nl); free(h.z); free(h.om);
}

/* One V-cycle on L u = F (u0 folded into F) cut at level `stop` of its
 * hierarchy (0 < stop < number of levels).  mode 0: the way down only, on a
 * copy of u (u is left unchanged); the right-hand side of level `stop`,
 * N/2^stop intervals, is written to fc_out.  mode 1: the same way down again
 * (the same arithmetic), then uc_in as the correction of level `stop`, and
 * the way up, updating u.  With uc_in = one cycle of the level-stop problem
 * from zero the two calls apply exactly orc_mg_one_cycle. */
void orc_mg_cycle_split(int p, double z, long N, const double *F, double *u, long n_min, int max_levels, int nu1,
                        int nu2, double omega, int stop, int mode, double *fc_out, const double *uc_in) {
    orc_hier h;
    int d = p + 1;
    h.p = p; h.d = d; h.nu1 = nu1; h.nu2 = nu2; h.gamma = 1;
    h.nlev = orc_num_levels(N, n_min, max_levels);
    h.Nl = (long *)malloc(sizeof(long) * h.nlev);
    h.z = (double *)malloc(sizeof(double) * h.nlev);
    h.om = (double *)malloc(sizeof(double) * h.nlev);
    for (int l = 0; l < h.nlev; ++l) {
        h.Nl[l] = N >> l;
        h.z[l] = ldexp(z, l);
        h.om[l] = omega > 0.0 ? omega : orc_omega_star(p, h.z[l]);
    }
    orc_transfer(p, h.P1, h.P2);
    double K[ORC_MAXD * ORC_MAXD], Mh[ORC_MAXD * ORC_MAXD];
    orc_blocks(p, K, Mh, h.a, h.b);
    orc_split sp = {stop, mode, fc_out, uc_in};
    if (mode == 0) {
        double *w = (double *)malloc(sizeof(double) * N * d);
        memcpy(w, u, sizeof(double) * N * d);
        mg_cycle_s(&h, 0, w, F, &sp);
        free(w);
    } else {
        mg_cycle_s(&h, 0, u, F, &sp);
    }
    free(h.Nl); free(h.z); free(h.om);
}

/* Residual F - L u with u0 folded into the first interval. */
void orc_residual(int p, double z, long N, const double *f, double u0, const double *u, double *r) {
    int d = p + 1;
    double A[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD];
    block_A(p, z, A, a, b);
    apply_L(d, A, a, b, N, u, r);
    for (long i = 0; i < N * d; ++i) r[i] = f[i] - r[i];
    for (int k = 0; k < d; ++k) r[k] += a[k] * u0;
}

/* ---------------------------------------------------------- adjoint -- */

/*
 * Transposed system L^T mu = g solved backward in time.  L^T has diagonal
 * blocks A^T and super-diagonal blocks -N^T = -b a^T, so
 *   mu_{N-1} = A^{-T} g_{N-1},  mu_n = A^{-T} (g_n + b (a^T mu_{n+1})).
 */
void orc_adj_sweep(int p, double z, long N, const double *g, double *mu) {
    int d = p + 1;
    double A[ORC_MAXD * ORC_MAXD], At[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD], rhs[ORC_MAXD];
    block_A(p, z, A, a, b);
    transpose(d, A, At);
    double h_next = 0.0;    /* a^T mu_{n+1} */
    for (long n = N - 1; n >= 0; --n) {
        for (int k = 0; k < d; ++k) rhs[k] = g[n * d + k] + b[k] * h_next;
        solve_small(d, At, rhs, &mu[n * d]);
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += a[k] * mu[n * d + k];
        h_next = s;
    }
}

/*
 * Gradients of a loss J(u) with dJ/du = g at the solution u of L u = F:
 * mu = L^{-T} g; dJ/df = mu; dJ/du0 = a^T mu_0 (u0 enters F_0 as a*u0);
 * dJ/dlambda = -tau * sum_n mu_n^T Mhat u_n (dL/dlambda = I (x) tau*Mhat).
 */
void orc_adjoint_grads(int p, double lambda, double tau, long N, const double *g, const double *u,
                       double *dJdf, double *dJdu0, double *dJdlambda) {
    int d = p + 1;
    double K[ORC_MAXD * ORC_MAXD], Mh[ORC_MAXD * ORC_MAXD], a[ORC_MAXD], b[ORC_MAXD];
    orc_blocks(p, K, Mh, a, b);
    orc_adj_sweep(p, lambda * tau, N, g, dJdf);
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += a[k] * dJdf[k];
    *dJdu0 = s;
    double acc = 0.0;
    for (long n = 0; n < N; ++n)
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) acc += dJdf[n * d + k] * Mh[k * d + l] * u[n * d + l];
    *dJdlambda = -tau * acc;
}
