// Space-time multigrid for the heat equation (the paper's outlook, Section 7):
// u_t - Delta u = f on the unit square with zero Dirichlet boundary values,
// the 5-point Laplacian A_h on an n x n interior grid (h = 1/(n+1),
// n = 2^k - 1) and the DG-in-time discretisation of Section 2.  Every time
// interval carries p_t + 1 spatial fields; the system is block
// lower-bidiagonal with diagonal blocks G_tau = K (x) I + tau Mhat (x) A_h and
// sub-diagonal blocks -(a b^T) (x) I (eq. chap4_generalLinearSystemODE with
// lambda replaced by A_h).
//
// The cycle is the time multigrid of Section 3 with the damped block Jacobi
// smoother of eq. chap4_ODESmoother, omega_t = 1/2 (the uniform damping that
// bounds the smoothing factor of every spatial mode), in which the block
// inverse G_tau^{-1} is replaced by ONE multigrid V(1,1)-cycle in space --
// damped point-block Jacobi (omega_s = 4/5, the (p+1) x (p+1) block
// K + tau (4/h^2) Mhat of a grid point), full-weighting restriction, bilinear
// prolongation, re-discretised coarse grids down to one point, solved
// exactly.  Time coarsens by two down to one interval, whose block is solved
// by nu_c spatial V-cycles; restriction and prolongation in time act on the
// Legendre coefficients of every grid point (eqs. chap4_restrictionTime,
// chap4_prolongationTime).  FP64 throughout.
//
// Layout: [interval][coefficient][row][column], row-major, FP64.  Every
// spatial V-cycle runs on all intervals of a time level at once; the kernels
// are grid-stride loops over (interval, row, column) points or values.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/tmg.h"
#include "tmg_nvtx.h"
#include "tmg_setup_math.h"

namespace {

constexpr int kHT = 256;
constexpr double kOmegaT = 0.5;
constexpr double kOmegaS = 0.8;

// Constants of one (time level, spatial level): the block G_tau on grid
// spacing h, its point block's inverse, the damping.
template <int D>
struct HeatK {
    double K[D * D];      // upwind DG stiffness block (Section 2)
    double Mh[D];         // reference mass matrix diagonal 1/(2k+1)
    double Dinv[D * D];   // (K + tau (4/h^2) Mhat)^{-1}
    double tau;
    double h2inv;         // 1/h^2
};

template <int D>
HeatK<D> heat_consts(double tau, int n) {
    HeatK<D> C;
    double A[tmg::kMaxDWide * tmg::kMaxDWide], Ai[tmg::kMaxDWide * tmg::kMaxDWide];
    tmg_host::local_blocks(D, 0.0, A);   // K
    for (int i = 0; i < D * D; ++i) C.K[i] = A[i];
    for (int k = 0; k < D; ++k) C.Mh[k] = 1.0 / (2.0 * k + 1.0);
    const double h = 1.0 / (n + 1);
    C.h2inv = 1.0 / (h * h);
    C.tau = tau;
    tmg_host::local_blocks(D, tau * 4.0 * C.h2inv, A);   // K + tau (4/h^2) Mhat
    tmg_host::invert(D, A, Ai);
    for (int i = 0; i < D * D; ++i) C.Dinv[i] = Ai[i];
    return C;
}

// (G x)_k at one grid point: K x + tau Mhat (A_h x); x at (m, i, j) for every
// coefficient and the four neighbours' values (zero outside the grid).
template <int D>
__device__ __forceinline__ void block_at(const HeatK<D>& C, const double* __restrict__ x, int64_t base, int n, int i,
                                         int j, double (&xc)[D], double (&gx)[D]) {
    const int64_t nn = (int64_t)n * n;
    double lap[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const double* xk = x + base + k * nn;
        const int64_t o = (int64_t)i * n + j;
        const double c = xk[o];
        double s = 4.0 * c;
        if (i > 0) s -= xk[o - n];
        if (i + 1 < n) s -= xk[o + n];
        if (j > 0) s -= xk[o - 1];
        if (j + 1 < n) s -= xk[o + 1];
        xc[k] = c;
        lap[k] = s * C.h2inv;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        double s = C.tau * C.Mh[k] * lap[k];
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(C.K[k * D + l], xc[l], s);
        gx[k] = s;
    }
}

// Point (m, i, j) of a grid-stride loop over npts = N n^2 points.
struct Pt {
    int64_t m;
    int i, j;
    int64_t base;   // offset of (m, 0, 0, 0)
    int64_t o;      // i n + j
};

template <int D>
__device__ __forceinline__ Pt point(int64_t t, int n) {
    const int64_t nn = (int64_t)n * n;
    Pt p;
    p.m = t / nn;
    p.o = t - p.m * nn;
    p.i = (int)(p.o / n);
    p.j = (int)(p.o - (int64_t)p.i * n);
    p.base = p.m * D * nn;
    return p;
}

// Time residual g = F + a e_{m-1} - G_tau u (a_k = (-1)^k, e = sum_k u_k of
// the previous interval; u0 before the first one, or 0 when u0 is nullptr);
// with norm2 != nullptr also sum g^2 (atomic per block).
template <int D>
__global__ void __launch_bounds__(kHT) kh_time_resid(const double* __restrict__ F, const double* __restrict__ u,
                                                     const double* __restrict__ u0, double* __restrict__ g, int64_t N,
                                                     int n, HeatK<D> C, double* __restrict__ norm2) {
    const int64_t nn = (int64_t)n * n, npts = N * nn;
    double ss = 0.0;
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < npts; t += (int64_t)gridDim.x * kHT) {
        const Pt p = point<D>(t, n);
        double xc[D], gx[D];
        block_at<D>(C, u, p.base, n, p.i, p.j, xc, gx);
        double e = 0.0;
        if (p.m > 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) e += u[p.base - D * nn + k * nn + p.o];
        } else if (u0 != nullptr) {
            e = u0[p.o];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int64_t idx = p.base + k * nn + p.o;
            const double v = F[idx] + ((k & 1) ? -e : e) - gx[k];
            g[idx] = v;
            ss = fma(v, v, ss);
        }
    }
    if (norm2 != nullptr) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(norm2, ss);
    }
}

// x = omega_s Dinv r (the first Jacobi sweep from zero); with n = 1 and
// omega = 1 the exact solve of a one-point grid.
template <int D>
__global__ void __launch_bounds__(kHT) kh_smooth0(const double* __restrict__ r, double* __restrict__ x, int64_t npts,
                                                  int64_t nn, HeatK<D> C, double omega) {
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < npts; t += (int64_t)gridDim.x * kHT) {
        const int64_t m = t / nn, o = t - m * nn, base = m * D * nn + o;
        double rv[D];
#pragma unroll
        for (int k = 0; k < D; ++k) rv[k] = r[base + k * nn];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < D; ++l) s = fma(C.Dinv[k * D + l], rv[l], s);
            x[base + k * nn] = omega * s;
        }
    }
}

// y = r - G x (mode 0), or y = x + omega_s Dinv (r - G x) (mode 1: a Jacobi
// sweep, out of place).
template <int D>
__global__ void __launch_bounds__(kHT) kh_sweep(const double* __restrict__ r, const double* __restrict__ x,
                                                double* __restrict__ y, int64_t N, int n, HeatK<D> C, int mode,
                                                double omega) {
    const int64_t nn = (int64_t)n * n, npts = N * nn;
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < npts; t += (int64_t)gridDim.x * kHT) {
        const Pt p = point<D>(t, n);
        double xc[D], gx[D], res[D];
        block_at<D>(C, x, p.base, n, p.i, p.j, xc, gx);
#pragma unroll
        for (int k = 0; k < D; ++k) res[k] = r[p.base + k * nn + p.o] - gx[k];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double v = res[k];
            if (mode == 1) {
                double s = 0.0;
#pragma unroll
                for (int l = 0; l < D; ++l) s = fma(C.Dinv[k * D + l], res[l], s);
                v = fma(omega, s, xc[k]);
            }
            y[p.base + k * nn + p.o] = v;
        }
    }
}

// Full weighting onto the coarse grid (nc = (n-1)/2): coarse (I, J) sits on
// fine (2I+1, 2J+1); weights 4 centre, 2 edge neighbours, 1 corners, / 16.
// One thread per coarse value (interval, coefficient, I, J).
__global__ void __launch_bounds__(kHT) kh_restrict_space(const double* __restrict__ y, double* __restrict__ rc,
                                                         int64_t nvals_c, int n, int nc) {
    const int64_t ncc = (int64_t)nc * nc, nnf = (int64_t)n * n;
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < nvals_c; t += (int64_t)gridDim.x * kHT) {
        const int64_t f = t / ncc, o = t - f * ncc;   // f = interval * D + coefficient
        const int I = (int)(o / nc), J = (int)(o - (int64_t)I * nc);
        const double* yf = y + f * nnf;
        const int i = 2 * I + 1, j = 2 * J + 1;
        auto at = [&](int a, int b) { return yf[(int64_t)a * n + b]; };
        double s = 4.0 * at(i, j);
        s += 2.0 * (at(i - 1, j) + at(i + 1, j) + at(i, j - 1) + at(i, j + 1));
        s += at(i - 1, j - 1) + at(i + 1, j - 1) + at(i - 1, j + 1) + at(i + 1, j + 1);
        rc[t] = s * 0.0625;
    }
}

// x += bilinear interpolation of the coarse correction; one thread per fine
// value.  Fine (i, j) lies between coarse rows (i-1)/2 .. (i+1)/2 (zero
// beyond the boundary).
__global__ void __launch_bounds__(kHT) kh_prolong_add(const double* __restrict__ xc, double* __restrict__ x,
                                                      int64_t nvals, int n, int nc) {
    const int64_t nnf = (int64_t)n * n, ncc = (int64_t)nc * nc;
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < nvals; t += (int64_t)gridDim.x * kHT) {
        const int64_t f = t / nnf, o = t - f * nnf;
        const int i = (int)(o / n), j = (int)(o - (int64_t)i * n);
        const double* c = xc + f * ncc;
        auto cv = [&](int a, int b) { return (a < 0 || b < 0 || a >= nc || b >= nc) ? 0.0 : c[(int64_t)a * nc + b]; };
        // coarse index of fine point i: odd i = 2I+1 -> on a coarse row; even i -> between rows i/2-1 and i/2
        double v;
        const bool ri = i & 1, rj = j & 1;
        const int I = ri ? (i - 1) / 2 : i / 2 - 1, J = rj ? (j - 1) / 2 : j / 2 - 1;
        if (ri && rj) v = cv(I, J);
        else if (ri) v = 0.5 * (cv(I, J) + cv(I, J + 1));
        else if (rj) v = 0.5 * (cv(I, J) + cv(I + 1, J));
        else v = 0.5 * (0.5 * (cv(I, J) + cv(I + 1, J)) + 0.5 * (cv(I, J + 1) + cv(I + 1, J + 1)));
        x[t] += v;
    }
}

// Time restriction of the residual: fc[m] = P1^T g[2m] + P2^T g[2m+1] on the
// Legendre axis of every grid point (eq. chap4_restrictionTime).
template <int D>
__global__ void __launch_bounds__(kHT) kh_restrict_time(const double* __restrict__ g, double* __restrict__ fc,
                                                        int64_t Nc, int64_t nn, tmg::Xfer<double, D> X) {
    const int64_t npts = Nc * nn;
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < npts; t += (int64_t)gridDim.x * kHT) {
        const int64_t m = t / nn, o = t - m * nn;
        double a[D], b[D];
#pragma unroll
        for (int l = 0; l < D; ++l) {
            a[l] = g[(2 * m) * D * nn + l * nn + o];
            b[l] = g[(2 * m + 1) * D * nn + l * nn + o];
        }
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double s = 0.0;
#pragma unroll
            for (int l = 0; l < D; ++l) s = fma(X.P1[l * D + k], a[l], fma(X.P2[l * D + k], b[l], s));
            fc[m * D * nn + k * nn + o] = s;
        }
    }
}

// Time prolongation: u[2m] += P1 uc[m], u[2m+1] += P2 uc[m] (eq.
// chap4_prolongationTime).
template <int D>
__global__ void __launch_bounds__(kHT) kh_prolong_time(const double* __restrict__ uc, double* __restrict__ u,
                                                       int64_t Nc, int64_t nn, tmg::Xfer<double, D> X) {
    const int64_t npts = Nc * nn;
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < npts; t += (int64_t)gridDim.x * kHT) {
        const int64_t m = t / nn, o = t - m * nn;
        double c[D];
#pragma unroll
        for (int l = 0; l < D; ++l) c[l] = uc[m * D * nn + l * nn + o];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double s1 = 0.0, s2 = 0.0;
#pragma unroll
            for (int l = 0; l < D; ++l) {
                s1 = fma(X.P1[k * D + l], c[l], s1);
                s2 = fma(X.P2[k * D + l], c[l], s2);
            }
            u[(2 * m) * D * nn + k * nn + o] += s1;
            u[(2 * m + 1) * D * nn + k * nn + o] += s2;
        }
    }
}

// u += omega x
__global__ void __launch_bounds__(kHT) kh_axpy(double* __restrict__ u, const double* __restrict__ x, int64_t nv,
                                               double omega) {
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < nv; t += (int64_t)gridDim.x * kHT)
        u[t] = fma(omega, x[t], u[t]);
}

}  // namespace

struct tmg_heat {
    int p, d, n;
    double tau;
    int64_t N;
    int nt;                       // time levels: N, N/2, ..., 1
    int ns;                       // spatial levels: n, (n-1)/2, ..., 1
    std::vector<int> nsz;         // grid size of every spatial level
    int nu1, nu2, nu_c;
    double tol;
    int max_cycles;
    cudaStream_t s;
    bool own_stream;
    int max_blocks;
    void* ws;                     // one allocation for every buffer below
    std::vector<double*> ft, ut;  // time levels l >= 1: right-hand side and correction
    std::vector<double*> rs, xs, ys;   // spatial levels: right-hand side, iterate, Jacobi output
    double* g;                    // time residual of the current time level
    double* g2;                   // coarsest time level: residual of the block solve
    double* cx;                   // coarsest time level: accumulated block solution
    double* norm2;                // device ||g||^2 of the level-0 residual
    double* host2;                // pinned copy
    double P1[tmg::kMaxD * tmg::kMaxD], P2[tmg::kMaxD * tmg::kMaxD];
    int last_cycles;
    double last_rel;
    std::vector<double> hist;
};

namespace {

thread_local int g_heat_cuda = 0;

#define TH_CUDA(call)                                    \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) {                         \
            g_heat_cuda = (int)_e;                       \
            return TMG_ECUDA;                            \
        }                                                \
    } while (0)

int grid_of(const tmg_heat* H, int64_t n) {
    int64_t b = (n + kHT - 1) / kHT;
    if (b > H->max_blocks) b = H->max_blocks;
    return (int)(b < 1 ? 1 : b);
}

template <int D>
struct HeatImpl {
    static tmg::Xfer<double, D> xfer(const tmg_heat* H) {
        tmg::Xfer<double, D> X;
        for (int i = 0; i < D * D; ++i) {
            X.P1[i] = H->P1[i];
            X.P2[i] = H->P2[i];
        }
        return X;
    }

    // One spatial V(1,1)-cycle from zero on G_tau x = rhs for N intervals at
    // spatial level sl; returns the buffer holding x.
    static const double* vcycle(tmg_heat* H, int sl, const double* rhs, int64_t N, double tau) {
        const tmg::NvtxRange r_lev("tmg heat spatial level %d", sl);
        const int n = H->nsz[sl];
        const int64_t nn = (int64_t)n * n, npts = N * nn;
        const HeatK<D> C = heat_consts<D>(tau, n);
        if (n == 1) {   // one grid point: G_tau is its point block, solved exactly
            kh_smooth0<D><<<grid_of(H, npts), kHT, 0, H->s>>>(rhs, H->xs[sl], npts, nn, C, 1.0);
            return H->xs[sl];
        }
        const int nc = H->nsz[sl + 1];
        kh_smooth0<D><<<grid_of(H, npts), kHT, 0, H->s>>>(rhs, H->xs[sl], npts, nn, C, kOmegaS);
        kh_sweep<D><<<grid_of(H, npts), kHT, 0, H->s>>>(rhs, H->xs[sl], H->ys[sl], N, n, C, 0, 0.0);
        const int64_t nvc = N * D * (int64_t)nc * nc;
        kh_restrict_space<<<grid_of(H, nvc), kHT, 0, H->s>>>(H->ys[sl], H->rs[sl + 1], nvc, n, nc);
        const double* xc = vcycle(H, sl + 1, H->rs[sl + 1], N, tau);
        const int64_t nv = N * D * nn;
        kh_prolong_add<<<grid_of(H, nv), kHT, 0, H->s>>>(xc, H->xs[sl], nv, n, nc);
        kh_sweep<D><<<grid_of(H, npts), kHT, 0, H->s>>>(rhs, H->xs[sl], H->ys[sl], N, n, C, 1, kOmegaS);
        return H->ys[sl];
    }

    // Time residual of level l into H->g (and ||g||^2 into H->norm2 when asked).
    static void time_resid(tmg_heat* H, const double* F, const double* u, const double* u0, int64_t N, double tau,
                           bool norm) {
        const int64_t npts = N * (int64_t)H->n * H->n;
        kh_time_resid<D><<<grid_of(H, npts), kHT, 0, H->s>>>(F, u, u0, H->g, N, H->n, heat_consts<D>(tau, H->n),
                                                            norm ? H->norm2 : nullptr);
    }

    // One smoothing step of every interval: u += omega_t (one spatial V-cycle on g).
    static void smooth(tmg_heat* H, double* u, int64_t N, double tau) {
        const double* x = vcycle(H, 0, H->g, N, tau);
        const int64_t nv = N * D * (int64_t)H->n * H->n;
        kh_axpy<<<grid_of(H, nv), kHT, 0, H->s>>>(u, x, nv, kOmegaT);
    }

    // One V-cycle in time at level l on L_l u = F (u0 only at level 0);
    // g_ready: H->g already holds this level's residual of u.
    static void tcycle(tmg_heat* H, int l, const double* F, double* u, const double* u0, bool g_ready) {
        const tmg::NvtxRange r_lev("tmg heat time level %d", l);
        const int64_t N = H->N >> l;
        const double tau = ldexp(H->tau, l);
        const int64_t nn = (int64_t)H->n * H->n, nv = N * D * nn;
        if (N == 1) {
            // nu_c spatial V-cycles on the block: x = 0; x += V(r - G x)
            if (!g_ready) time_resid(H, F, u, u0, 1, tau, false);
            const HeatK<D> C = heat_consts<D>(tau, H->n);
            for (int c = 0; c < H->nu_c; ++c) {
                if (c == 0) {
                    const double* x = vcycle(H, 0, H->g, 1, tau);
                    cudaMemcpyAsync(H->cx, x, sizeof(double) * nv, cudaMemcpyDeviceToDevice, H->s);
                } else {
                    kh_sweep<D><<<grid_of(H, nn), kHT, 0, H->s>>>(H->g, H->cx, H->g2, 1, H->n, C, 0, 0.0);
                    const double* x = vcycle(H, 0, H->g2, 1, tau);
                    kh_axpy<<<grid_of(H, nv), kHT, 0, H->s>>>(H->cx, x, nv, 1.0);
                }
            }
            kh_axpy<<<grid_of(H, nv), kHT, 0, H->s>>>(u, H->cx, nv, 1.0);
            return;
        }
        for (int k = 0; k < H->nu1; ++k) {
            if (!(g_ready && k == 0)) time_resid(H, F, u, u0, N, tau, false);
            smooth(H, u, N, tau);
        }
        if (!(g_ready && H->nu1 == 0)) time_resid(H, F, u, u0, N, tau, false);
        const tmg::Xfer<double, D> X = xfer(H);
        kh_restrict_time<D><<<grid_of(H, (N / 2) * nn), kHT, 0, H->s>>>(H->g, H->ft[l + 1], N / 2, nn, X);
        cudaMemsetAsync(H->ut[l + 1], 0, sizeof(double) * (nv / 2), H->s);
        tcycle(H, l + 1, H->ft[l + 1], H->ut[l + 1], nullptr, false);
        kh_prolong_time<D><<<grid_of(H, (N / 2) * nn), kHT, 0, H->s>>>(H->ut[l + 1], u, N / 2, nn, X);
        for (int k = 0; k < H->nu2; ++k) {
            time_resid(H, F, u, u0, N, tau, false);
            smooth(H, u, N, tau);
        }
    }
};

template <int D>
tmg_status run_heat(tmg_heat* H, const double* F, const double* u0, double* u, bool solve) {
    const int64_t nv = H->N * D * (int64_t)H->n * H->n;
    if (solve) TH_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * nv, H->s));
    H->hist.clear();
    double nF = 0.0;
    for (int k = 0;; ++k) {
        // residual of the current iterate and its norm; it also serves the
        // cycle's first smoothing step
        TH_CUDA(cudaMemsetAsync(H->norm2, 0, sizeof(double), H->s));
        HeatImpl<D>::time_resid(H, F, u, u0, H->N, H->tau, true);
        if (solve) {
            TH_CUDA(cudaMemcpyAsync(H->host2, H->norm2, sizeof(double), cudaMemcpyDeviceToHost, H->s));
            TH_CUDA(cudaStreamSynchronize(H->s));
            const double nr = sqrt(*H->host2);
            if (k == 0) nF = nr;
            const double rel = nF > 0.0 ? nr / nF : nr;
            H->hist.push_back(rel);
            H->last_cycles = k;
            H->last_rel = rel;
            if (!(rel == rel) || rel > 1e300) return TMG_ENUMERIC;
            if (rel <= H->tol) return TMG_OK;
            if (k >= H->max_cycles) return TMG_ENOTCONV;
        }
        HeatImpl<D>::tcycle(H, 0, F, u, u0, true);
        TH_CUDA(cudaGetLastError());
        if (!solve) {
            TH_CUDA(cudaStreamSynchronize(H->s));
            return TMG_OK;
        }
    }
}

tmg_status run_heat_d(tmg_heat* H, const double* F, const double* u0, double* u, bool solve) {
    switch (H->d) {
        case 1: return run_heat<1>(H, F, u0, u, solve);
        case 2: return run_heat<2>(H, F, u0, u, solve);
        case 3: return run_heat<3>(H, F, u0, u, solve);
        case 4: return run_heat<4>(H, F, u0, u, solve);
        case 5: return run_heat<5>(H, F, u0, u, solve);
        default: return run_heat<6>(H, F, u0, u, solve);
    }
}

bool aligned16(const void* p) { return p != nullptr && (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

tmg_status tmg_heat_setup(tmg_heat** out, int p_t, double tau, int n, int64_t N, const tmg_opts* opts, int nu_c,
                          void* stream) {
    if (!out) return TMG_EINVAL;
    *out = nullptr;
    tmg_opts o;
    tmg_opts_default(&o);
    if (opts) o = *opts;
    bool pow2n = n >= 1, pow2N = N >= 1;
    for (int64_t m = n + 1; pow2n && m > 1; m >>= 1) pow2n = (m & 1) == 0;
    for (int64_t m = N; pow2N && m > 1; m >>= 1) pow2N = (m & 1) == 0;
    if (p_t < 0 || p_t > tmg::kMaxD - 1 || !(tau > 0.0) || !isfinite(tau) || !pow2n || !pow2N || nu_c < 1 ||
        nu_c > 16 || o.nu1 < 0 || o.nu1 > 8 || o.nu2 < 0 || o.nu2 > 8 || o.nu1 + o.nu2 < 1 || o.gamma != 1 ||
        o.max_cycles < 0 || !(o.tol >= 0.0))
        return TMG_EINVAL;
    tmg_heat* H = new (std::nothrow) tmg_heat();
    if (!H) return TMG_ENOMEM;
    H->p = p_t;
    H->d = p_t + 1;
    H->n = n;
    H->tau = tau;
    H->N = N;
    H->nu1 = o.nu1;
    H->nu2 = o.nu2;
    H->nu_c = nu_c;
    H->tol = o.tol;
    H->max_cycles = o.max_cycles;
    H->last_rel = NAN;
    H->nt = 1;
    for (int64_t m = N; m > 1; m >>= 1) ++H->nt;
    for (int m = n; m >= 1; m = (m - 1) / 2) {
        H->nsz.push_back(m);
        if (m == 1) break;
    }
    H->ns = (int)H->nsz.size();
    H->s = static_cast<cudaStream_t>(stream);
    if (!H->s) {
        if (cudaStreamCreate(&H->s) != cudaSuccess) {
            delete H;
            return TMG_ECUDA;
        }
        H->own_stream = true;
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        tmg_heat_destroy(H);
        return TMG_ECUDA;
    }
    H->max_blocks = nsm * 8;
    double P1[tmg::kMaxDWide * tmg::kMaxDWide], P2[tmg::kMaxDWide * tmg::kMaxDWide];
    tmg_host::transfer_setup(H->d, P1, P2);
    for (int i = 0; i < H->d * H->d; ++i) {
        H->P1[i] = P1[i];
        H->P2[i] = P2[i];
    }
    // workspace: time levels 1.., the residual, the spatial hierarchy for the
    // level-0 batch, the coarse-level block solve
    const int64_t nv0 = N * H->d * (int64_t)n * n, blk = (int64_t)H->d * n * n;
    std::vector<int64_t> sizes;
    for (int l = 1; l < H->nt; ++l) {
        sizes.push_back(nv0 >> l);   // ft
        sizes.push_back(nv0 >> l);   // ut
    }
    sizes.push_back(nv0);            // g
    for (int sl = 0; sl < H->ns; ++sl) {
        const int64_t v = N * H->d * (int64_t)H->nsz[sl] * H->nsz[sl];
        if (sl > 0) sizes.push_back(v);   // rs (level 0 reads the time residual)
        sizes.push_back(v);          // xs
        sizes.push_back(v);          // ys
    }
    sizes.push_back(blk);            // g2
    sizes.push_back(blk);            // cx
    sizes.push_back(1);              // norm2
    size_t bytes = 0;
    for (int64_t v : sizes) bytes += ((size_t)v * sizeof(double) + 255) / 256 * 256;
    if (cudaMalloc(&H->ws, bytes) != cudaSuccess) {
        H->ws = nullptr;
        tmg_heat_destroy(H);
        return TMG_ENOMEM;
    }
    char* b = static_cast<char*>(H->ws);
    size_t off = 0, k = 0;
    auto take = [&](void) {
        double* p = reinterpret_cast<double*>(b + off);
        off += ((size_t)sizes[k++] * sizeof(double) + 255) / 256 * 256;
        return p;
    };
    H->ft.assign(H->nt, nullptr);
    H->ut.assign(H->nt, nullptr);
    for (int l = 1; l < H->nt; ++l) {
        H->ft[l] = take();
        H->ut[l] = take();
    }
    H->g = take();
    for (int sl = 0; sl < H->ns; ++sl) {
        H->rs.push_back(sl > 0 ? take() : nullptr);
        H->xs.push_back(take());
        H->ys.push_back(take());
    }
    H->g2 = take();
    H->cx = take();
    H->norm2 = take();
    if (cudaMallocHost(&H->host2, sizeof(double)) != cudaSuccess) {
        H->host2 = nullptr;
        tmg_heat_destroy(H);
        return TMG_ENOMEM;
    }
    *out = H;
    return TMG_OK;
}

tmg_status tmg_heat_solve(tmg_heat* H, const double* f, const double* u0, double* u) {
    if (!H || !aligned16(f) || !aligned16(u) || !u0 || (reinterpret_cast<uintptr_t>(u0) & 7u)) return TMG_EINVAL;
    const tmg::NvtxRange r("tmg_heat_solve");
    return run_heat_d(H, f, u0, u, true);
}

tmg_status tmg_heat_cycle(tmg_heat* H, const double* f, const double* u0, double* u) {
    if (!H || !aligned16(f) || !aligned16(u) || !u0 || (reinterpret_cast<uintptr_t>(u0) & 7u)) return TMG_EINVAL;
    return run_heat_d(H, f, u0, u, false);
}

tmg_status tmg_heat_residual(tmg_heat* H, const double* f, const double* u0, const double* u, double* r) {
    if (!H || !aligned16(f) || !aligned16(u) || !aligned16(r) || !u0 || (reinterpret_cast<uintptr_t>(u0) & 7u))
        return TMG_EINVAL;
    const int64_t npts = H->N * (int64_t)H->n * H->n;
    switch (H->d) {
#define TMG_HEAT_RES(DD)                                                                                    \
    case DD:                                                                                                \
        kh_time_resid<DD><<<grid_of(H, npts), kHT, 0, H->s>>>(f, u, u0, r, H->N, H->n,                      \
                                                              heat_consts<DD>(H->tau, H->n), nullptr);     \
        break;
        TMG_HEAT_RES(1)
        TMG_HEAT_RES(2)
        TMG_HEAT_RES(3)
        TMG_HEAT_RES(4)
        TMG_HEAT_RES(5)
        TMG_HEAT_RES(6)
#undef TMG_HEAT_RES
        default: return TMG_EINVAL;
    }
    TH_CUDA(cudaGetLastError());
    TH_CUDA(cudaStreamSynchronize(H->s));
    return TMG_OK;
}

tmg_status tmg_heat_stats(const tmg_heat* H, int* cycles, double* rel_res, double* hist, int hist_len) {
    if (!H) return TMG_EINVAL;
    if (cycles) *cycles = H->last_cycles;
    if (rel_res) *rel_res = H->last_rel;
    if (hist)
        for (int i = 0; i < hist_len; ++i) hist[i] = i < (int)H->hist.size() ? H->hist[i] : NAN;
    return TMG_OK;
}

void tmg_heat_destroy(tmg_heat* H) {
    if (!H) return;
    if (H->s) cudaStreamSynchronize(H->s);
    if (H->ws) cudaFree(H->ws);
    if (H->host2) cudaFreeHost(H->host2);
    if (H->own_stream) cudaStreamDestroy(H->s);
    delete H;
}

}  // extern "C"
