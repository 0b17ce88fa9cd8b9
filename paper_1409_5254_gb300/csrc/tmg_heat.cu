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
// chap4_prolongationTime).
//
// Two precisions.  TMG_FP64: every step in FP64 (the textbook iterates).
// TMG_MIXED: the residual of the FP64 iterate is formed in FP64 and rounded
// to FP32, one cycle in FP32 computes the correction c from zero, u += c in
// FP64 -- iterative refinement, which reaches the FP64 solution because the
// FP32 cycle contracts the error of every correction.
//
// Kernels.  The spatial V-cycle keeps no smoothed iterate in memory: the
// first Jacobi sweep from zero is pointwise (x = omega Dinv r), so the
// "pre" kernel recomputes x from r, forms the residual r - G x and restricts
// it by full weighting in one pass; the "post" kernel recomputes x, adds the
// bilinear prolongation of the coarse correction, applies the second sweep
// and writes (or accumulates into the time iterate) the result.  Per spatial
// level: read r twice, the coarse values once, write the result once.  Both
// stream a warp down the rows of one interval with the stencil's rows in
// registers: whole rows (4, 2 or 1 columns per lane) for grids up to 127
// points a side, overlapping 64-column strips above.
// In the mixed form the residual of the FP64 iterate is kept as a float pair
// and updated by r -= L c after every cycle (float-pair arithmetic on the
// exact FP32 correction), with one FP64 residual to confirm convergence.
//
// Layout: [interval][coefficient][row][column], row-major.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <type_traits>
#include <vector>

#include "../../include/tmg.h"
#include "tmg_bounds.h"
#include "tmg_nvtx.h"
#include "tmg_setup_math.h"

namespace {

constexpr int kHT = 256;
constexpr double kOmegaT = 0.5;
constexpr double kOmegaS = 0.8;

// Constants of one (time level, spatial level): the block G_tau on grid
// spacing h and its point block's inverse.
template <int D, typename T>
struct HeatK {
    T K[D * D];      // upwind DG stiffness block (Section 2)
    T Mh[D];         // reference mass matrix diagonal 1/(2k+1), times tau / h^2
    T Dinv[D * D];   // (K + tau (4/h^2) Mhat)^{-1}
};

template <int D, typename T>
HeatK<D, T> heat_consts(double tau, int n) {
    HeatK<D, T> C;
    double A[tmg::kMaxDWide * tmg::kMaxDWide], Ai[tmg::kMaxDWide * tmg::kMaxDWide];
    tmg_host::local_blocks(D, 0.0, A);   // K
    for (int i = 0; i < D * D; ++i) C.K[i] = (T)A[i];
    const double h = 1.0 / (n + 1), h2inv = 1.0 / (h * h);
    for (int k = 0; k < D; ++k) C.Mh[k] = (T)(tau * h2inv / (2.0 * k + 1.0));
    tmg_host::local_blocks(D, tau * 4.0 * h2inv, A);   // K + tau (4/h^2) Mhat
    tmg_host::invert(D, A, Ai);
    for (int i = 0; i < D * D; ++i) C.Dinv[i] = (T)Ai[i];
    return C;
}

// (G x)_k at one grid point from x there (c) and the sum of its four
// neighbours (nb, zero outside the grid): K c + (tau/h^2) Mhat (4 c - nb).
template <int D, typename T>
__device__ __forceinline__ void apply_G(const HeatK<D, T>& C, const T (&c)[D], const T (&nb)[D], T (&gx)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T s = C.Mh[k] * (T(4) * c[k] - nb[k]);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(C.K[k * D + l], c[l], s);
        gx[k] = s;
    }
}

// y = Dinv v
template <int D, typename T>
__device__ __forceinline__ void apply_Dinv(const HeatK<D, T>& C, const T (&v)[D], T (&y)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(C.Dinv[k * D + l], v[l], s);
        y[k] = s;
    }
}

// ---------------------------------------------------------------- row tasks
// Kernels on the full spatial grid of a time level (residuals, updates,
// transfers in time) run one CTA-wide task per (interval, block of kRB grid
// rows), kRT threads across the row, each thread down the kRB rows of its
// column; offsets within an interval are 32-bit (D n^2 < 2^31).
constexpr int kRT = 128;
constexpr int kRB = 4;   // rows per task: four independent points per thread keep loads in flight

struct RowTask {
    int64_t m;
    int i0;
};

__device__ __forceinline__ int row_blocks(int n) { return (n + kRB - 1) / kRB; }

__device__ __forceinline__ RowTask row_task(int64_t t, int nrb) {
    RowTask r;
    r.m = t / nrb;
    r.i0 = (int)(t - r.m * nrb) * kRB;
    return r;
}

// x at (i, j) of one interval (pointer at its coefficient 0) and the sum of
// its four neighbours, zero outside the grid.
template <int D, typename T>
__device__ __forceinline__ void stencil_at(const T* __restrict__ x, int nn, int n, int i, int j, T (&c)[D],
                                           T (&nb)[D]) {
    const int o = i * n + j;
    const bool ok = TMG_IN(o, nn, 43);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const T* xk = x + (int64_t)k * nn;
        c[k] = ok ? xk[o] : T(0);
        T s = T(0);
        if (i > 0) s += xk[o - n];
        if (i + 1 < n) s += xk[o + n];
        if (j > 0) s += xk[o - 1];
        if (j + 1 < n) s += xk[o + 1];
        nb[k] = s;
    }
}

template <bool NORM>
__device__ __forceinline__ void norm_flush(double ss, double* __restrict__ norm2) {
    if (NORM) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(norm2, ss);
    }
}

// Residual g = F + a e_{m-1} - G_tau u (TIME: a_k = (-1)^k, e = sum_k u_k of
// the previous interval, u0 before the first one or 0 when u0 is nullptr;
// without TIME the residual r - G x of independent block solves), computed
// in T and stored as TO.  PAIR: stored as the float pair (g, gl) with
// g + gl = the FP64 value to 2^-48.  NORM: sum of squares into *norm2.
template <int D, typename T, typename TO, bool TIME, bool NORM, bool PAIR>
__global__ void __launch_bounds__(kRT) kh_resid(const T* __restrict__ F, const T* __restrict__ u,
                                                const double* __restrict__ u0, TO* __restrict__ g,
                                                float* __restrict__ gl, int64_t N, int n, HeatK<D, T> C,
                                                double* __restrict__ norm2) {
    const int nn = n * n;
    const int nrb = row_blocks(n);
    const int64_t tasks = N * nrb;
    double ss = 0.0;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const RowTask rt = row_task(t, nrb);
        const int64_t base = rt.m * D * (int64_t)nn;
        const T* um = u + base;
        for (int j = threadIdx.x; j < n; j += kRT)
#pragma unroll
        for (int rr = 0; rr < kRB; ++rr) {
            const int i = rt.i0 + rr;
            if (i >= n) break;
            const int o = i * n + j;
            if (!TMG_IN(o, nn, 37)) continue;
            T c[D], nb[D], gx[D];
            stencil_at<D, T>(um, nn, n, i, j, c, nb);
            apply_G<D, T>(C, c, nb, gx);
            T e = T(0);
            if (TIME) {
                if (rt.m > 0) {
#pragma unroll
                    for (int k = 0; k < D; ++k) e += um[(int64_t)(k - D) * nn + o];
                } else if (u0 != nullptr) {
                    e = (T)u0[o];
                }
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int64_t idx = base + (int64_t)k * nn + o;
                const T v = F[idx] + ((k & 1) ? -e : e) - gx[k];
                if (PAIR) {
                    const float h = (float)v;
                    g[idx] = (TO)h;
                    gl[idx] = (float)(v - (T)h);
                } else {
                    g[idx] = (TO)v;
                }
                if (NORM) ss = fma((double)v, (double)v, ss);
            }
        }
    }
    norm_flush<NORM>(ss, norm2);
}

// Residual of u = 0 as a float pair: r = F, plus a (x) u0 in the first
// interval; sum of squares into *norm2.
template <int D>
__global__ void __launch_bounds__(kRT) kh_init_pair(const double* __restrict__ F, const double* __restrict__ u0,
                                                    float* __restrict__ rh, float* __restrict__ rl, int64_t N, int n,
                                                    double* __restrict__ norm2) {
    const int nn = n * n;
    const int nrb = row_blocks(n);
    const int64_t tasks = N * nrb;
    double ss = 0.0;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const RowTask rt = row_task(t, nrb);
        const int64_t base = rt.m * D * (int64_t)nn;
        for (int j = threadIdx.x; j < n; j += kRT)
#pragma unroll
        for (int rr = 0; rr < kRB; ++rr) {
            const int i = rt.i0 + rr;
            if (i >= n) break;
            const int o = i * n + j;
            if (!TMG_IN(o, nn, 37)) continue;
            const double e = rt.m == 0 ? u0[o] : 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const int64_t idx = base + (int64_t)k * nn + o;
                const double v = F[idx] + ((k & 1) ? -e : e);
                const float h = (float)v;
                rh[idx] = h;
                rl[idx] = (float)(v - (double)h);
                ss = fma(v, v, ss);
            }
        }
    }
    norm_flush<true>(ss, norm2);
}

// Float-pair arithmetic (a value h + l, |l| <= ulp(h)/2): the error-free sum
// of Knuth and the FMA-based error-free product; the products use __fmul_rn
// so that no multiply is contracted into an FMA that would change them.
struct FF {
    float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ FF quick_two_sum(float a, float b) {   // |a| >= |b| or a = 0
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    FF s = two_sum(a.h, b.h);
    const FF t = two_sum(a.l, b.l);
    s = quick_two_sum(s.h, s.l + t.h);
    return quick_two_sum(s.h, s.l + t.l);
}

__device__ __forceinline__ FF ff_add_f(FF a, float b) {
    const FF s = two_sum(a.h, b);
    return quick_two_sum(s.h, s.l + a.l);
}

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.h, -a.l}; }

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = fmaf(a.h, b.h, -p);
    return quick_two_sum(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}

// tau Mhat_kk / h^2 of one time level as float pairs (the K entries are +-1,
// exact in any precision).
template <int D>
struct PairK {
    float mh[D], ml[D];
    float K[D * D];
};

template <int D>
PairK<D> pair_consts(double tau, int n) {
    PairK<D> P;
    double A[tmg::kMaxDWide * tmg::kMaxDWide];
    tmg_host::local_blocks(D, 0.0, A);
    for (int i = 0; i < D * D; ++i) P.K[i] = (float)A[i];
    const double h = 1.0 / (n + 1), h2inv = 1.0 / (h * h);
    for (int k = 0; k < D; ++k) {
        const double mu = tau * h2inv / (2.0 * k + 1.0);
        P.mh[k] = (float)mu;
        P.ml[k] = (float)(mu - (double)P.mh[k]);
    }
    return P;
}

// The mixed form's update after one FP32 correction cycle: u += c (FP64),
// r -= L c in float-pair arithmetic (c is exact in FP32, so L c is formed to
// about 2^-44 of its size and the updated residual follows the true residual
// of u across the cycles), sum of r_h^2 into *norm2.  (L c)_m =
// G_tau c_m - a (b^T c_{m-1}); the first interval has no predecessor term
// (u0 is part of the initial residual).
// (12 blocks per SM: 40 registers with a few spilled, 1.42 ms against
// 1.52 ms at 64 registers on the 127^2 x 4096 level)
template <int D>
__global__ void __launch_bounds__(kRT, 12) kh_update_pair(double* __restrict__ u, const float* __restrict__ c,
                                                      float* __restrict__ rh, float* __restrict__ rl, int64_t N,
                                                      int n, PairK<D> P, double* __restrict__ norm2) {
    const int nn = n * n;
    const int nrb = row_blocks(n);
    const int64_t tasks = N * nrb;
    float ss = 0.0f;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const RowTask rt = row_task(t, nrb);
        const int64_t base = rt.m * D * (int64_t)nn;
        const float* cm = c + base;
        for (int j = threadIdx.x; j < n; j += kRT)
#pragma unroll
        for (int rr = 0; rr < kRB; ++rr) {
            const int i = rt.i0 + rr;
            if (i >= n) break;
            const int o = i * n + j;
            if (!TMG_IN(o, nn, 37)) continue;
            float cv[D];
#pragma unroll
            for (int k = 0; k < D; ++k) cv[k] = cm[(int64_t)k * nn + o];
            FF e = {0.0f, 0.0f};   // b^T c_{m-1}
            if (rt.m > 0) {
#pragma unroll
                for (int k = 0; k < D; ++k) e = ff_add_f(e, cm[(int64_t)(k - D) * nn + o]);
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float* ck = cm + (int64_t)k * nn;
                const float up = i > 0 ? ck[o - n] : 0.0f, dn = i + 1 < n ? ck[o + n] : 0.0f;
                const float lt = j > 0 ? ck[o - 1] : 0.0f, rt_ = j + 1 < n ? ck[o + 1] : 0.0f;
                // 4 c - (up + dn + lt + rt), then times tau Mhat_kk / h^2
                FF d = ff_add(two_sum(up, dn), two_sum(lt, rt_));
                d = ff_add_f(ff_neg(d), 4.0f * cv[k]);
                FF tk = ff_mul(FF{P.mh[k], P.ml[k]}, d);
#pragma unroll
                for (int l = 0; l < D; ++l) tk = ff_add_f(tk, P.K[k * D + l] * cv[l]);
                tk = ff_add(tk, (k & 1) ? e : ff_neg(e));   // - a_k e, a_k = (-1)^k
                const int64_t idx = base + (int64_t)k * nn + o;
                const FF r = ff_add(FF{rh[idx], rl[idx]}, ff_neg(tk));
                rh[idx] = r.h;
                rl[idx] = r.l;
                ss = fmaf(r.h, r.h, ss);
                u[idx] += (double)cv[k];
            }
        }
    }
    norm_flush<true>((double)ss, norm2);
}

// ------------------------------------------------------------- warp strips
// The spatial V-cycle kernels run one warp per (interval, strip of columns,
// chunk of rows).  Lane L holds the adjacent local columns q = 2L and
// 2L + 1 of a 64-column window and streams down the rows with a three-row
// window of the smoothed iterate in registers; the columns next to a lane's
// pair come from the neighbouring lanes by shuffles.  Windows overlap: the
// outermost local columns only feed their neighbours, so strips advance by
// 62 (post) or 60 (pre: 30 coarse columns) fine columns and no lane runs
// extra halo code.  The loads of row i + 2 are issued before row i is
// computed.
constexpr int kPreRows = 16;    // coarse rows per pre task (at most; fewer when that leaves SMs idle)
constexpr int kPostRows = 32;   // fine rows per post task (at most)
constexpr int kPreStride = 30;  // coarse columns per pre strip
constexpr int kPostStride = 62; // fine columns per post strip

template <typename T>
__device__ __forceinline__ T shup(T v) {
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ T shdn(T v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}

// r at fine (i, j) of one interval, zero outside the grid.
template <int D, typename T>
__device__ __forceinline__ void r_at(const T* __restrict__ r, int nn, int n, int i, int j, T (&rv)[D]) {
    const bool in = (unsigned)i < (unsigned)n && (unsigned)j < (unsigned)n;
    const int o = in ? i * n + j : 0;
    const bool ok = in && TMG_IN(o, nn, 30);
#pragma unroll
    for (int k = 0; k < D; ++k) rv[k] = ok ? r[k * nn + o] : T(0);
}

// d = omega Dinv r (the first Jacobi sweep from zero).
template <int D, typename T>
__device__ __forceinline__ void smooth0(const HeatK<D, T>& C, T omega, const T (&rv)[D], T (&dv)[D]) {
    T t[D];
    apply_Dinv<D, T>(C, rv, t);
#pragma unroll
    for (int k = 0; k < D; ++k) dv[k] = omega * t[k];
}

// Pre-smoothing, residual and full weighting in one pass: x = omega Dinv r,
// y = r - G x, rc = FW(y) on the coarse grid nc = (n-1)/2 (coarse (I, J) on
// fine (2I+1, 2J+1), weights [1 2 1]^T [1 2 1] / 16: across the columns at
// the odd ones, then down the rows).  Window origin c0 = 60s - 2: lane L's
// odd column c0 + 2L + 1 is coarse column 30s - 1 + L, written by lanes
// 1..30.
template <int D, typename T>
__global__ void __launch_bounds__(kHT) kh_pre_w(const T* __restrict__ r, T* __restrict__ rc, int64_t N, int n,
                                                int nc, int rows, HeatK<D, T> C, T omega) {
    const int lane = threadIdx.x & 31;
    const int nn = n * n, ncc = nc * nc;
    const int strips = (nc + kPreStride - 1) / kPreStride, chunks = (nc + rows - 1) / rows;
    const int per = strips * chunks;
    const int64_t tasks = N * per;
    const int64_t nw = ((int64_t)gridDim.x * kHT) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * kHT + threadIdx.x) >> 5; w < tasks; w += nw) {
        const int64_t m = w / per;
        const int rem = (int)(w - m * per);
        const int s = rem / chunks, ch = rem - s * chunks;
        const int I0 = ch * rows, I1 = min(I0 + rows, nc);
        const T* rm = r + m * D * (int64_t)nn;
        T* rcm = rc + m * D * (int64_t)ncc;
        const int c0 = 2 * kPreStride * s - 2;
        const int ce = c0 + 2 * lane, co = ce + 1;   // this lane's even and odd fine column
        const int J = kPreStride * s - 1 + lane;     // coarse column of co
        const bool writer = lane >= 1 && lane <= 30 && J < nc;
        const int f0 = 2 * I0, f1 = 2 * I1;           // fine rows f0 .. f1
        T xe[3][D], xo[3][D], re[D], ro[D], ren[D], ron[D], pe[D], po[D], acc[D];
        {
            T t0[D], t1[D];
            r_at<D, T>(rm, nn, n, f0 - 1, ce, t0);
            r_at<D, T>(rm, nn, n, f0 - 1, co, t1);
            smooth0<D, T>(C, omega, t0, xe[0]);
            smooth0<D, T>(C, omega, t1, xo[0]);
        }
        r_at<D, T>(rm, nn, n, f0, ce, re);
        r_at<D, T>(rm, nn, n, f0, co, ro);
        smooth0<D, T>(C, omega, re, xe[1]);
        smooth0<D, T>(C, omega, ro, xo[1]);
        r_at<D, T>(rm, nn, n, f0 + 1, ce, ren);
        r_at<D, T>(rm, nn, n, f0 + 1, co, ron);
        smooth0<D, T>(C, omega, ren, xe[2]);
        smooth0<D, T>(C, omega, ron, xo[2]);
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = T(0);
        for (int i = f0;; ++i) {
            // loads of row i + 2, consumed after row i is done
            r_at<D, T>(rm, nn, n, i + 2, ce, pe);
            r_at<D, T>(rm, nn, n, i + 2, co, po);
            // y = r - G x at row i; H = y(even) + 2 y(odd) + y(next lane's even)
            T nbe[D], nbo[D], ge[D], go[D], H[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T left = shup(xo[1][k]), right = shdn(xe[1][k]);
                nbe[k] = (xe[0][k] + xe[2][k]) + (left + xo[1][k]);
                nbo[k] = (xo[0][k] + xo[2][k]) + (xe[1][k] + right);
            }
            apply_G<D, T>(C, xe[1], nbe, ge);
            apply_G<D, T>(C, xo[1], nbo, go);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T ye = re[k] - ge[k], yo = ro[k] - go[k];
                H[k] = (ye + shdn(ye)) + T(2) * yo;
            }
            // down the rows: coarse row I takes fine rows 2I, 2I+1, 2I+2 with weights 1, 2, 1
            if ((i & 1) == 0) {
                if (i > f0) {
                    const int I = i / 2 - 1;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        acc[k] += H[k];
                        if (writer && TMG_IN(I * nc + J, ncc, 33)) rcm[k * ncc + I * nc + J] = acc[k] * T(0.0625);
                    }
                }
                if (i == f1) break;
#pragma unroll
                for (int k = 0; k < D; ++k) acc[k] = H[k];
            } else {
#pragma unroll
                for (int k = 0; k < D; ++k) acc[k] += T(2) * H[k];
            }
            // advance the window to row i + 1
#pragma unroll
            for (int k = 0; k < D; ++k) {
                xe[0][k] = xe[1][k];
                xe[1][k] = xe[2][k];
                xo[0][k] = xo[1][k];
                xo[1][k] = xo[2][k];
                re[k] = ren[k];
                ro[k] = ron[k];
                ren[k] = pe[k];
                ron[k] = po[k];
            }
            smooth0<D, T>(C, omega, pe, xe[2]);
            smooth0<D, T>(C, omega, po, xo[2]);
        }
    }
}

// Coarse-grid correction and post-smoothing in one pass: x = omega Dinv r +
// P xc (the pre-smoothed iterate recomputed, plus the bilinear prolongation
// of the coarse correction, rows interpolated first), z = x + omega Dinv
// (r - G x); out = alpha z (acc = 0) or out += alpha z (acc = 1).  Window
// origin c0 = 62s - 1: lane L's first column c0 + 2L is odd and lies on
// coarse column Jl = 31s - 1 + L, its second column lies between Jl and
// Jl + 1 (the next lane's); z is written at local columns 1..62.
template <int D, typename T>
__global__ void __launch_bounds__(kHT) kh_post_w(const T* __restrict__ r, const T* __restrict__ xc,
                                                 T* __restrict__ out, int64_t N, int n, int nc, int rows,
                                                 HeatK<D, T> C, T omega, T alpha, int acc) {
    const int lane = threadIdx.x & 31;
    const int nn = n * n, ncc = nc * nc;
    const int strips = (n + kPostStride - 1) / kPostStride, chunks = (n + rows - 1) / rows;
    const int per = strips * chunks;
    const int64_t tasks = N * per;
    const int64_t nw = ((int64_t)gridDim.x * kHT) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * kHT + threadIdx.x) >> 5; w < tasks; w += nw) {
        const int64_t m = w / per;
        const int rem = (int)(w - m * per);
        const int s = rem / chunks, ch = rem - s * chunks;
        const int i0 = ch * rows, i1 = min(i0 + rows, n);
        const T* rm = r + m * D * (int64_t)nn;
        const T* cm = xc + m * D * (int64_t)ncc;
        T* om = out + m * D * (int64_t)nn;
        const int c0 = kPostStride * s - 1;
        const int ca = c0 + 2 * lane, cb = ca + 1;    // odd and even fine column of this lane
        const int Jl = (ca - 1) >> 1;                 // coarse column of ca (31s - 1 + L)
        const bool wa = lane >= 1 && ca < n, wb = lane <= 30 && cb < n;
        const bool jin = (unsigned)Jl < (unsigned)nc, jin1 = (unsigned)(Jl + 1) < (unsigned)nc;
        // coarse values of fine row a at Jl (q) and Jl + 1 (q1, lane 31 only: the
        // others take it from the next lane): rows (a-1)/2 for odd a, else the
        // two rows a/2 - 1 and a/2 (zero outside the coarse grid)
        auto cload = [&](int a, T (&q)[D], T (&q2)[D], T (&q1)[D], T (&q12)[D]) {
            const int Ia = (a & 1) ? (a - 1) >> 1 : (a >> 1) - 1, Ib = (a & 1) ? -1 : a >> 1;
            const bool ia = (unsigned)Ia < (unsigned)nc, ib = (unsigned)Ib < (unsigned)nc;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T* ck = cm + k * ncc;
                q[k] = (ia && jin && TMG_IN(Ia * nc + Jl, ncc, 32)) ? ck[Ia * nc + Jl] : T(0);
                q2[k] = (ib && jin && TMG_IN(Ib * nc + Jl, ncc, 32)) ? ck[Ib * nc + Jl] : T(0);
                q1[k] = (lane == 31 && ia && jin1) ? ck[Ia * nc + Jl + 1] : T(0);
                q12[k] = (lane == 31 && ib && jin1) ? ck[Ib * nc + Jl + 1] : T(0);
            }
        };
        // x at fine row a from its loads: d = omega Dinv r plus the prolongation
        auto xrow = [&](int a, const T (&ra)[D], const T (&rb)[D], const T (&q)[D], const T (&q2)[D],
                        const T (&q1)[D], const T (&q12)[D], T (&xa)[D], T (&xb)[D]) {
            T da[D], db[D];
            smooth0<D, T>(C, omega, ra, da);
            smooth0<D, T>(C, omega, rb, db);
            const bool odd = a & 1, rowin = (unsigned)a < (unsigned)n;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T cr = odd ? q[k] : T(0.5) * (q[k] + q2[k]);       // row-interpolated at Jl
                const T cr1l = odd ? q1[k] : T(0.5) * (q1[k] + q12[k]);  // lane 31's own Jl + 1
                const T nxt = shdn(cr);
                const T cr1 = lane == 31 ? cr1l : nxt;
                xa[k] = (rowin && (unsigned)ca < (unsigned)n) ? da[k] + cr : T(0);
                xb[k] = (rowin && (unsigned)cb < (unsigned)n) ? db[k] + T(0.5) * (cr + cr1) : T(0);
            }
        };
        T xa[3][D], xb[3][D], ra[D], rb[D], ran[D], rbn[D], pa[D], pb[D];
        T q[D], q2[D], q1[D], q12[D];
        {
            T t0[D], t1[D];
            r_at<D, T>(rm, nn, n, i0 - 1, ca, t0);
            r_at<D, T>(rm, nn, n, i0 - 1, cb, t1);
            cload(i0 - 1, q, q2, q1, q12);
            xrow(i0 - 1, t0, t1, q, q2, q1, q12, xa[0], xb[0]);
        }
        r_at<D, T>(rm, nn, n, i0, ca, ra);
        r_at<D, T>(rm, nn, n, i0, cb, rb);
        cload(i0, q, q2, q1, q12);
        xrow(i0, ra, rb, q, q2, q1, q12, xa[1], xb[1]);
        r_at<D, T>(rm, nn, n, i0 + 1, ca, ran);
        r_at<D, T>(rm, nn, n, i0 + 1, cb, rbn);
        cload(i0 + 1, q, q2, q1, q12);
        xrow(i0 + 1, ran, rbn, q, q2, q1, q12, xa[2], xb[2]);
        for (int i = i0; i < i1; ++i) {
            // loads of row i + 2, consumed after row i is written
            r_at<D, T>(rm, nn, n, i + 2, ca, pa);
            r_at<D, T>(rm, nn, n, i + 2, cb, pb);
            cload(i + 2, q, q2, q1, q12);
            T nba[D], nbb[D], ga[D], gb[D], ea[D], eb[D], ya[D], yb[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T left = shup(xb[1][k]), right = shdn(xa[1][k]);
                nba[k] = (xa[0][k] + xa[2][k]) + (left + xb[1][k]);
                nbb[k] = (xb[0][k] + xb[2][k]) + (xa[1][k] + right);
            }
            apply_G<D, T>(C, xa[1], nba, ga);
            apply_G<D, T>(C, xb[1], nbb, gb);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                ea[k] = ra[k] - ga[k];
                eb[k] = rb[k] - gb[k];
            }
            apply_Dinv<D, T>(C, ea, ya);
            apply_Dinv<D, T>(C, eb, yb);
            T* oi = om + i * n;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T za = fma(omega, ya[k], xa[1][k]), zb = fma(omega, yb[k], xb[1][k]);
                if (wa && TMG_IN(i * n + ca, nn, 36)) {
                    T* p = oi + k * nn + ca;
                    *p = acc ? fma(alpha, za, *p) : alpha * za;
                }
                if (wb && TMG_IN(i * n + cb, nn, 36)) {
                    T* p = oi + k * nn + cb;
                    *p = acc ? fma(alpha, zb, *p) : alpha * zb;
                }
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                xa[0][k] = xa[1][k];
                xa[1][k] = xa[2][k];
                xb[0][k] = xb[1][k];
                xb[1][k] = xb[2][k];
                ra[k] = ran[k];
                rb[k] = rbn[k];
                ran[k] = pa[k];
                rbn[k] = pb[k];
            }
            xrow(i + 2, pa, pb, q, q2, q1, q12, xa[2], xb[2]);
        }
    }
}

// ----------------------------------------------------------- full-row warps
// For n + 1 <= 128 a warp spans whole grid rows, both boundary columns
// included: lane L' of a segment of SW = (n+1)/CPL lanes holds the local
// columns CPL L' + q (q < CPL), which are fine columns CPL L' + q - 1.  Local
// column 0 is the left boundary (x = 0); the right neighbour of the last
// local column is the right boundary.  No lane carries halo work and every
// lane holds grid columns; with n + 1 < 32 one warp holds 32/SW intervals.
template <int CPL>
struct RowGeom {
    int SW, IPW, ls, seg;
    __device__ RowGeom(int n, int lane) {
        SW = (n + 1) / CPL;
        IPW = 32 / SW;
        ls = lane % SW;
        seg = lane / SW;
    }
};

// Neighbour values of local column q at the current row from the row vector
// v[CPL][D] of every lane: left (q-1) and right (q+1), zero beyond the right
// boundary.  All lanes call it (shuffles).
template <int D, typename T, int CPL>
__device__ __forceinline__ void row_neighbours(const T (&v)[CPL][D], bool last, T (&lt)[CPL][D], T (&rt)[CPL][D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const T fromL = shup(v[CPL - 1][k]);
        const T fromR = shdn(v[0][k]);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            lt[q][k] = q > 0 ? v[q - 1][k] : fromL;
            rt[q][k] = q + 1 < CPL ? v[q + 1][k] : (last ? T(0) : fromR);
        }
    }
}

template <int D, typename T, int CPL>
__device__ __forceinline__ void row_load(const T* __restrict__ rm, int nn, int n, int i, int lc0, bool live,
                                         T (&v)[CPL][D]) {
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int j = lc0 + q - 1;
        const bool in = live && (unsigned)i < (unsigned)n && (unsigned)j < (unsigned)n;
        const int o = in ? i * n + j : 0;
        const bool ok = in && TMG_IN(o, nn, 31);
#pragma unroll
        for (int k = 0; k < D; ++k) v[q][k] = ok ? rm[k * nn + o] : T(0);
    }
}

// Pre-smoothing, residual and full weighting (as kh_pre_w) on full rows:
// coarse column J sits on the even local column 2J + 2; its weights take y
// at local columns 2J + 1, 2J + 2, 2J + 3.
// (at CPL = 4 in FP32, three blocks per SM: 80 registers, 12 bytes of spill;
// 0.155 ms against 0.182 ms on the 127^2 x 4096 level; the same bound on
// kh_post_f spills 112 bytes and makes it slower, 0.62 against 0.50 ms)
template <int D, typename T, int CPL>
__global__ void __launch_bounds__(kHT, (CPL == 4 && sizeof(T) == 4) ? 3 : 1) kh_pre_f(const T* __restrict__ r, T* __restrict__ rc, int64_t N, int n,
                                                int nc, int rows, HeatK<D, T> C, T omega) {
    constexpr int NO = CPL >= 2 ? CPL / 2 : 1;   // coarse outputs per lane
    const int lane = threadIdx.x & 31;
    const RowGeom<CPL> G(n, lane);
    const bool last = G.ls == G.SW - 1;
    const int nn = n * n, ncc = nc * nc;
    const int chunks = (nc + rows - 1) / rows;
    const int64_t groups = (N + G.IPW - 1) / G.IPW;
    const int64_t tasks = groups * chunks;
    const int64_t nw = ((int64_t)gridDim.x * kHT) >> 5;
    const int lc0 = CPL * G.ls;
    for (int64_t w = ((int64_t)blockIdx.x * kHT + threadIdx.x) >> 5; w < tasks; w += nw) {
        const int64_t g = w / chunks;
        const int ch = (int)(w - g * chunks);
        const int64_t m = g * G.IPW + G.seg;
        const bool live = m < N;
        const int I0 = ch * rows, I1 = min(I0 + rows, nc);
        const T* rm = r + (live ? m : 0) * D * (int64_t)nn;
        T* rcm = rc + (live ? m : 0) * D * (int64_t)ncc;
        const int f0 = 2 * I0, f1 = 2 * I1;
        T x[3][CPL][D], rv[CPL][D], rn[CPL][D], pf[CPL][D], acc[NO][D];
        {
            T t0[CPL][D];
            row_load<D, T, CPL>(rm, nn, n, f0 - 1, lc0, live, t0);
#pragma unroll
            for (int q = 0; q < CPL; ++q) smooth0<D, T>(C, omega, t0[q], x[0][q]);
        }
        row_load<D, T, CPL>(rm, nn, n, f0, lc0, live, rv);
        row_load<D, T, CPL>(rm, nn, n, f0 + 1, lc0, live, rn);
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            smooth0<D, T>(C, omega, rv[q], x[1][q]);
            smooth0<D, T>(C, omega, rn[q], x[2][q]);
        }
#pragma unroll
        for (int o = 0; o < NO; ++o)
#pragma unroll
            for (int k = 0; k < D; ++k) acc[o][k] = T(0);
        for (int i = f0;; ++i) {
            row_load<D, T, CPL>(rm, nn, n, i + 2, lc0, live, pf);
            // y = r - G x at row i
            T lt[CPL][D], rt[CPL][D], y[CPL][D];
            row_neighbours<D, T, CPL>(x[1], last, lt, rt);
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                T nb[D], gx[D];
#pragma unroll
                for (int k = 0; k < D; ++k) nb[k] = (x[0][q][k] + x[2][q][k]) + (lt[q][k] + rt[q][k]);
                apply_G<D, T>(C, x[1][q], nb, gx);
#pragma unroll
                for (int k = 0; k < D; ++k) y[q][k] = rv[q][k] - gx[k];
            }
            // across the columns at the even local columns: H = y(q-1) + 2 y(q) + y(q+1)
            T yl[CPL][D], yr[CPL][D], H[NO][D];
            row_neighbours<D, T, CPL>(y, last, yl, yr);
#pragma unroll
            for (int o = 0; o < NO; ++o) {
                const int q = CPL >= 2 ? 2 * o : 0;
#pragma unroll
                for (int k = 0; k < D; ++k) H[o][k] = (yl[q][k] + yr[q][k]) + T(2) * y[q][k];
            }
            if ((i & 1) == 0) {
                if (i > f0) {
                    const int I = i / 2 - 1;
#pragma unroll
                    for (int o = 0; o < NO; ++o) {
                        const int lc = lc0 + (CPL >= 2 ? 2 * o : 0);
                        const int J = (lc - 2) >> 1;
                        const bool wr = live && (lc & 1) == 0 && lc >= 2 && J < nc;
#pragma unroll
                        for (int k = 0; k < D; ++k) {
                            acc[o][k] += H[o][k];
                            if (wr && TMG_IN(I * nc + J, ncc, 34)) rcm[k * ncc + I * nc + J] = acc[o][k] * T(0.0625);
                        }
                    }
                }
                if (i == f1) break;
#pragma unroll
                for (int o = 0; o < NO; ++o)
#pragma unroll
                    for (int k = 0; k < D; ++k) acc[o][k] = H[o][k];
            } else {
#pragma unroll
                for (int o = 0; o < NO; ++o)
#pragma unroll
                    for (int k = 0; k < D; ++k) acc[o][k] += T(2) * H[o][k];
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    x[0][q][k] = x[1][q][k];
                    x[1][q][k] = x[2][q][k];
                    rv[q][k] = rn[q][k];
                    rn[q][k] = pf[q][k];
                }
#pragma unroll
            for (int q = 0; q < CPL; ++q) smooth0<D, T>(C, omega, pf[q], x[2][q]);
        }
    }
}

// Coarse-grid correction and post-smoothing (as kh_post_w) on full rows.
// A lane's fine columns lc0 - 1 .. lc0 + CPL - 2 read the row-interpolated
// coarse correction at coarse columns jlo .. jlo + NJ - 1; an odd fine column
// 2J+1 takes J, an even one 2J the mean of J-1 and J.
template <int D, typename T, int CPL>
__global__ void __launch_bounds__(kHT) kh_post_f(const T* __restrict__ r, const T* __restrict__ xc,
                                                 T* __restrict__ out, int64_t N, int n, int nc, int rows,
                                                 HeatK<D, T> C, T omega, T alpha, int acc) {
    constexpr int NJ = CPL >= 2 ? CPL / 2 + 1 : 2;
    const int lane = threadIdx.x & 31;
    const RowGeom<CPL> G(n, lane);
    const bool last = G.ls == G.SW - 1;
    const int nn = n * n, ncc = nc * nc;
    const int chunks = (n + rows - 1) / rows;
    const int64_t groups = (N + G.IPW - 1) / G.IPW;
    const int64_t tasks = groups * chunks;
    const int64_t nw = ((int64_t)gridDim.x * kHT) >> 5;
    const int lc0 = CPL * G.ls;
    const int j0 = lc0 - 1;                                   // fine column of q = 0
    const int jlo = (j0 & 1) ? (j0 - 1) >> 1 : (j0 >> 1) - 1;  // first coarse column read
    const bool j0odd = j0 & 1;
    for (int64_t w = ((int64_t)blockIdx.x * kHT + threadIdx.x) >> 5; w < tasks; w += nw) {
        const int64_t g = w / chunks;
        const int ch = (int)(w - g * chunks);
        const int64_t m = g * G.IPW + G.seg;
        const bool live = m < N;
        const int i0 = ch * rows, i1 = min(i0 + rows, n);
        const T* rm = r + (live ? m : 0) * D * (int64_t)nn;
        const T* cm = xc + (live ? m : 0) * D * (int64_t)ncc;
        T* om = out + (live ? m : 0) * D * (int64_t)nn;
        // x at fine row a from its r values
        auto xrow = [&](int a, const T (&ra)[CPL][D], T (&xa)[CPL][D]) {
            T cr[NJ][D];
            const int Ia = (a & 1) ? (a - 1) >> 1 : (a >> 1) - 1, Ib = (a & 1) ? -1 : a >> 1;
            const bool ia = live && (unsigned)Ia < (unsigned)nc, ib = live && (unsigned)Ib < (unsigned)nc;
#pragma unroll
            for (int t = 0; t < NJ; ++t) {
                const int J = jlo + t;
                const bool jin = (unsigned)J < (unsigned)nc;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T* ck = cm + k * ncc;
                    const T va = (ia && jin && TMG_IN(Ia * nc + J, ncc, 35)) ? ck[Ia * nc + J] : T(0);
                    if (a & 1) {
                        cr[t][k] = va;
                    } else {
                        const T vb = (ib && jin && TMG_IN(Ib * nc + J, ncc, 35)) ? ck[Ib * nc + J] : T(0);
                        cr[t][k] = T(0.5) * (va + vb);
                    }
                }
            }
            const bool rowin = (unsigned)a < (unsigned)n;
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                T d[D];
                smooth0<D, T>(C, omega, ra[q], d);
                const int j = j0 + q;
                const bool in = rowin && (unsigned)j < (unsigned)n;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    T p;
                    if (CPL >= 2) {   // j0 odd: even q on a coarse column, odd q between two
                        p = (q & 1) ? T(0.5) * (cr[(q - 1) / 2][k] + cr[(q + 1) / 2][k]) : cr[q / 2][k];
                    } else {
                        p = j0odd ? cr[0][k] : T(0.5) * (cr[0][k] + cr[1][k]);
                    }
                    xa[q][k] = in ? d[k] + p : T(0);
                }
            }
        };
        T x[3][CPL][D], rv[CPL][D], rn[CPL][D], pf[CPL][D];
        {
            T t0[CPL][D];
            row_load<D, T, CPL>(rm, nn, n, i0 - 1, lc0, live, t0);
            xrow(i0 - 1, t0, x[0]);
        }
        row_load<D, T, CPL>(rm, nn, n, i0, lc0, live, rv);
        xrow(i0, rv, x[1]);
        row_load<D, T, CPL>(rm, nn, n, i0 + 1, lc0, live, rn);
        xrow(i0 + 1, rn, x[2]);
        for (int i = i0; i < i1; ++i) {
            row_load<D, T, CPL>(rm, nn, n, i + 2, lc0, live, pf);
            T ov[CPL][D];   // the accumulated output of row i, loaded early
            if (acc) row_load<D, T, CPL>(om, nn, n, i, lc0, live, ov);
            T lt[CPL][D], rt[CPL][D];
            row_neighbours<D, T, CPL>(x[1], last, lt, rt);
            T* oi = om + i * n;
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                T nb[D], gx[D], e[D], y[D];
#pragma unroll
                for (int k = 0; k < D; ++k) nb[k] = (x[0][q][k] + x[2][q][k]) + (lt[q][k] + rt[q][k]);
                apply_G<D, T>(C, x[1][q], nb, gx);
#pragma unroll
                for (int k = 0; k < D; ++k) e[k] = rv[q][k] - gx[k];
                apply_Dinv<D, T>(C, e, y);
                const int j = j0 + q;
                if (live && (unsigned)j < (unsigned)n && TMG_IN(i * n + j, nn, 36)) {
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const T z = fma(omega, y[k], x[1][q][k]);
                        oi[k * nn + j] = acc ? fma(alpha, z, ov[q][k]) : alpha * z;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    x[0][q][k] = x[1][q][k];
                    x[1][q][k] = x[2][q][k];
                    rv[q][k] = rn[q][k];
                    rn[q][k] = pf[q][k];
                }
            xrow(i + 2, pf, x[2]);
        }
    }
}

// Time residual on full rows (as kh_resid with TIME, no norm, stored in T):
// g = F + a e_{m-1} - G u, with the three-row window of u in registers and
// the loads of row i + 2 issued before row i is computed.
template <int D, typename T, int CPL>
__global__ void __launch_bounds__(kHT) kh_resid_f(const T* __restrict__ F, const T* __restrict__ u,
                                                  const double* __restrict__ u0, T* __restrict__ g, int64_t N, int n,
                                                  int rows, HeatK<D, T> C) {
    const int lane = threadIdx.x & 31;
    const RowGeom<CPL> G(n, lane);
    const bool last = G.ls == G.SW - 1;
    const int nn = n * n;
    const int chunks = (n + rows - 1) / rows;
    const int64_t groups = (N + G.IPW - 1) / G.IPW;
    const int64_t tasks = groups * chunks;
    const int64_t nw = ((int64_t)gridDim.x * kHT) >> 5;
    const int lc0 = CPL * G.ls;
    for (int64_t w = ((int64_t)blockIdx.x * kHT + threadIdx.x) >> 5; w < tasks; w += nw) {
        const int64_t gi = w / chunks;
        const int ch = (int)(w - gi * chunks);
        const int64_t m = gi * G.IPW + G.seg;
        const bool live = m < N;
        const int i0 = ch * rows, i1 = min(i0 + rows, n);
        const int64_t base = (live ? m : 0) * D * (int64_t)nn;
        const T* um = u + base;
        const T* Fm = F + base;
        const T* up = (live && m > 0) ? um - D * (int64_t)nn : nullptr;   // previous interval
        T* gm = g + base;
        T x[3][CPL][D], pf[CPL][D];
        row_load<D, T, CPL>(um, nn, n, i0 - 1, lc0, live, x[0]);
        row_load<D, T, CPL>(um, nn, n, i0, lc0, live, x[1]);
        row_load<D, T, CPL>(um, nn, n, i0 + 1, lc0, live, x[2]);
        for (int i = i0; i < i1; ++i) {
            row_load<D, T, CPL>(um, nn, n, i + 2, lc0, live, pf);
            T fv[CPL][D], pv[CPL][D];
            row_load<D, T, CPL>(Fm, nn, n, i, lc0, live, fv);
            if (up != nullptr) row_load<D, T, CPL>(up, nn, n, i, lc0, live, pv);
            T lt[CPL][D], rt[CPL][D];
            row_neighbours<D, T, CPL>(x[1], last, lt, rt);
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const int j = lc0 + q - 1;
                T nb[D], gx[D];
#pragma unroll
                for (int k = 0; k < D; ++k) nb[k] = (x[0][q][k] + x[2][q][k]) + (lt[q][k] + rt[q][k]);
                apply_G<D, T>(C, x[1][q], nb, gx);
                T e = T(0);
                if (up != nullptr) {
#pragma unroll
                    for (int k = 0; k < D; ++k) e += pv[q][k];
                } else if (m == 0 && u0 != nullptr && (unsigned)j < (unsigned)n && TMG_IN(i * n + j, nn, 38)) {
                    e = (T)u0[i * n + j];
                }
                if (live && (unsigned)j < (unsigned)n && TMG_IN(i * n + j, nn, 38)) {
#pragma unroll
                    for (int k = 0; k < D; ++k) gm[k * nn + i * n + j] = fv[q][k] + ((k & 1) ? -e : e) - gx[k];
                }
            }
#pragma unroll
            for (int q = 0; q < CPL; ++q)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    x[0][q][k] = x[1][q][k];
                    x[1][q][k] = x[2][q][k];
                    x[2][q][k] = pf[q][k];
                }
        }
    }
}

// ----------------------------------------------------- small-grid V-cycle
// The whole spatial V(1,1)-cycle of a grid of at most kSmallN points a side
// (and every coarser level down to one point) in shared memory, one CTA per
// interval: the same steps as kh_pre_f / kh_post_f / kh_point_solve level by
// level, with every level's right-hand side, iterate and a scratch array
// on chip.  out = alpha x (acc = 0) or out += alpha x (acc = 1).
constexpr int kSmallN = 31;
constexpr int kSmallLevels = 5;   // 31, 15, 7, 3, 1
constexpr int kSmallNT = 256;

template <int D, typename T>
struct SmallK {
    HeatK<D, T> k[kSmallLevels];
    int n[kSmallLevels];
    int nl;   // levels, the last of one point
};

template <int D>
__host__ __device__ constexpr int small_values() {   // values per array over the levels 31, 15, 7, 3, 1
    return D * (31 * 31 + 15 * 15 + 7 * 7 + 3 * 3 + 1);
}

template <typename T>
size_t small_smem(int D) {
    return (size_t)3 * D * (31 * 31 + 15 * 15 + 7 * 7 + 3 * 3 + 1) * sizeof(T);
}

template <int D, typename T>
__global__ void __launch_bounds__(kSmallNT) kh_vsmall(const T* __restrict__ rhs, T* __restrict__ out, int64_t N,
                                                      SmallK<D, T> S, T omega, T alpha, int acc) {
    extern __shared__ __align__(16) unsigned char small_smem_raw[];
    T* R = reinterpret_cast<T*>(small_smem_raw);   // right-hand sides of every level
    T* X = R + small_values<D>();                   // iterates
    T* Y = X + small_values<D>();                   // scratch
    int off[kSmallLevels];
    {
        int o = 0;
        for (int l = 0; l < S.nl; ++l) {
            off[l] = o;
            o += D * S.n[l] * S.n[l];
        }
    }
    const int n0 = S.n[0], nn0 = n0 * n0;
    for (int64_t m = blockIdx.x; m < N; m += gridDim.x) {
        const T* rm = rhs + m * D * (int64_t)nn0;
        for (int p = threadIdx.x; p < D * nn0; p += kSmallNT)
            if (TMG_IN(p, D * nn0, 44)) R[p] = rm[p];
        __syncthreads();
        // down: x = omega Dinv r, y = r - G x, r_{l+1} = FW(y)
        for (int l = 0; l + 1 < S.nl; ++l) {
            const int n = S.n[l], nn = n * n, nc = S.n[l + 1], ncc = nc * nc;
            const HeatK<D, T>& C = S.k[l];
            T* r = R + off[l];
            T* x = X + off[l];
            T* y = Y + off[l];
            for (int p = threadIdx.x; p < nn; p += kSmallNT) {
                T v[D], d[D];
#pragma unroll
                for (int k = 0; k < D; ++k) v[k] = r[k * nn + p];
                apply_Dinv<D, T>(C, v, d);
#pragma unroll
                for (int k = 0; k < D; ++k) x[k * nn + p] = omega * d[k];
            }
            __syncthreads();
            for (int p = threadIdx.x; p < nn; p += kSmallNT) {
                const int i = p / n, j = p - i * n;
                T c[D], nb[D], gx[D];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T* xk = x + k * nn;
                    c[k] = xk[p];
                    T s = T(0);
                    if (i > 0) s += xk[p - n];
                    if (i + 1 < n) s += xk[p + n];
                    if (j > 0) s += xk[p - 1];
                    if (j + 1 < n) s += xk[p + 1];
                    nb[k] = s;
                }
                apply_G<D, T>(C, c, nb, gx);
#pragma unroll
                for (int k = 0; k < D; ++k) y[k * nn + p] = r[k * nn + p] - gx[k];
            }
            __syncthreads();
            T* rc = R + off[l + 1];
            for (int p = threadIdx.x; p < ncc; p += kSmallNT) {
                const int I = p / nc, J = p - I * nc;
                const int q = (2 * I + 1) * n + (2 * J + 1);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T* Yk = y + k * nn;
                    T s = T(4) * Yk[q];
                    s += T(2) * ((Yk[q - n] + Yk[q + n]) + (Yk[q - 1] + Yk[q + 1]));
                    s += (Yk[q - n - 1] + Yk[q - n + 1]) + (Yk[q + n - 1] + Yk[q + n + 1]);
                    rc[k * ncc + p] = s * T(0.0625);
                }
            }
            __syncthreads();
        }
        // one grid point: G is its point block, solved exactly
        {
            const int l = S.nl - 1;
            if (threadIdx.x == 0) {
                T v[D], d[D];
#pragma unroll
                for (int k = 0; k < D; ++k) v[k] = R[off[l] + k];
                apply_Dinv<D, T>(S.k[l], v, d);
#pragma unroll
                for (int k = 0; k < D; ++k) X[off[l] + k] = d[k];
            }
            __syncthreads();
        }
        // up: x += P x_c, z = x + omega Dinv (r - G x)
        for (int l = S.nl - 2; l >= 0; --l) {
            const int n = S.n[l], nn = n * n, nc = S.n[l + 1], ncc = nc * nc;
            const HeatK<D, T>& C = S.k[l];
            const T* r = R + off[l];
            T* x = X + off[l];
            T* z = Y + off[l];
            const T* xc = X + off[l + 1];
            for (int p = threadIdx.x; p < nn; p += kSmallNT) {
                const int i = p / n, j = p - i * n;
                const bool ri = i & 1, rj = j & 1;
                const int I = ri ? (i - 1) / 2 : i / 2 - 1, J = rj ? (j - 1) / 2 : j / 2 - 1;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T* ck = xc + k * ncc;
                    auto cv = [&](int a, int b) -> T {
                        return (a < 0 || b < 0 || a >= nc || b >= nc) ? T(0) : ck[a * nc + b];
                    };
                    T v;
                    if (ri && rj) v = cv(I, J);
                    else if (ri) v = T(0.5) * (cv(I, J) + cv(I, J + 1));
                    else if (rj) v = T(0.5) * (cv(I, J) + cv(I + 1, J));
                    else v = T(0.5) * (T(0.5) * (cv(I, J) + cv(I + 1, J)) + T(0.5) * (cv(I, J + 1) + cv(I + 1, J + 1)));
                    x[k * nn + p] += v;
                }
            }
            __syncthreads();
            for (int p = threadIdx.x; p < nn; p += kSmallNT) {
                const int i = p / n, j = p - i * n;
                T c[D], nb[D], gx[D], e[D], d[D];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T* xk = x + k * nn;
                    c[k] = xk[p];
                    T s = T(0);
                    if (i > 0) s += xk[p - n];
                    if (i + 1 < n) s += xk[p + n];
                    if (j > 0) s += xk[p - 1];
                    if (j + 1 < n) s += xk[p + 1];
                    nb[k] = s;
                }
                apply_G<D, T>(C, c, nb, gx);
#pragma unroll
                for (int k = 0; k < D; ++k) e[k] = r[k * nn + p] - gx[k];
                apply_Dinv<D, T>(C, e, d);
#pragma unroll
                for (int k = 0; k < D; ++k) z[k * nn + p] = fma(omega, d[k], c[k]);
            }
            __syncthreads();
            if (l > 0) {   // the coarse level's result becomes its iterate for the next prolongation
                for (int p = threadIdx.x; p < D * nn; p += kSmallNT) x[p] = z[p];
                __syncthreads();
            }
        }
        T* om = out + m * D * (int64_t)nn0;
        for (int p = threadIdx.x; p < D * nn0; p += kSmallNT)
            if (TMG_IN(p, D * nn0, 45)) om[p] = acc ? fma(alpha, Y[p], om[p]) : alpha * Y[p];
        __syncthreads();
    }
}

// One grid point: G_tau is its point block, solved exactly.
// out = alpha Dinv r (acc = 0) or out += alpha Dinv r (acc = 1).
template <int D, typename T>
__global__ void __launch_bounds__(kHT) kh_point_solve(const T* __restrict__ r, T* __restrict__ out, int64_t N,
                                                      HeatK<D, T> C, T alpha, int acc) {
    for (int64_t m = (int64_t)blockIdx.x * kHT + threadIdx.x; m < N; m += (int64_t)gridDim.x * kHT) {
        T v[D], y[D];
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = r[m * D + k];
        apply_Dinv<D, T>(C, v, y);
#pragma unroll
        for (int k = 0; k < D; ++k) out[m * D + k] = acc ? fma(alpha, y[k], out[m * D + k]) : alpha * y[k];
    }
}

// Time restriction of the residual: fc[m] = P1^T g[2m] + P2^T g[2m+1] on the
// Legendre axis of every grid point (eq. chap4_restrictionTime).  Row tasks
// over the coarse intervals.
template <int D, typename T>
__global__ void __launch_bounds__(kRT) kh_restrict_time(const T* __restrict__ g, T* __restrict__ fc, int64_t Nc,
                                                        int n, tmg::Xfer<T, D> X) {
    const int nn = n * n;
    const int nrb = row_blocks(n);
    const int64_t tasks = Nc * nrb;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const RowTask rt = row_task(t, nrb);
        const T* g0 = g + 2 * rt.m * D * (int64_t)nn;
        const T* g1 = g0 + D * (int64_t)nn;
        T* f = fc + rt.m * D * (int64_t)nn;
        for (int j = threadIdx.x; j < n; j += kRT)
#pragma unroll
        for (int rr = 0; rr < kRB; ++rr) {
            const int i = rt.i0 + rr;
            if (i >= n) break;
            const int o = i * n + j;
            if (!TMG_IN(o, nn, 37)) continue;
            T a[D], b[D];
#pragma unroll
            for (int l = 0; l < D; ++l) {
                a[l] = g0[(int64_t)l * nn + o];
                b[l] = g1[(int64_t)l * nn + o];
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                T s = T(0);
#pragma unroll
                for (int l = 0; l < D; ++l) s = fma(X.P1[l * D + k], a[l], fma(X.P2[l * D + k], b[l], s));
                f[(int64_t)k * nn + o] = s;
            }
        }
    }
}

// Time prolongation: u[2m] += P1 uc[m], u[2m+1] += P2 uc[m] (eq.
// chap4_prolongationTime).
template <int D, typename T>
__global__ void __launch_bounds__(kRT) kh_prolong_time(const T* __restrict__ uc, T* __restrict__ u, int64_t Nc, int n,
                                                       tmg::Xfer<T, D> X) {
    const int nn = n * n;
    const int nrb = row_blocks(n);
    const int64_t tasks = Nc * nrb;
    for (int64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
        const RowTask rt = row_task(t, nrb);
        const T* c = uc + rt.m * D * (int64_t)nn;
        T* u0p = u + 2 * rt.m * D * (int64_t)nn;
        T* u1p = u0p + D * (int64_t)nn;
        for (int j = threadIdx.x; j < n; j += kRT)
#pragma unroll
        for (int rr = 0; rr < kRB; ++rr) {
            const int i = rt.i0 + rr;
            if (i >= n) break;
            const int o = i * n + j;
            if (!TMG_IN(o, nn, 37)) continue;
            T cv[D];
#pragma unroll
            for (int l = 0; l < D; ++l) cv[l] = c[(int64_t)l * nn + o];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                T s1 = T(0), s2 = T(0);
#pragma unroll
                for (int l = 0; l < D; ++l) {
                    s1 = fma(X.P1[k * D + l], cv[l], s1);
                    s2 = fma(X.P2[k * D + l], cv[l], s2);
                }
                u0p[(int64_t)k * nn + o] += s1;
                u1p[(int64_t)k * nn + o] += s2;
            }
        }
    }
}

// u += x
template <typename T>
__global__ void __launch_bounds__(kHT) kh_add(T* __restrict__ u, const T* __restrict__ x, int64_t nv) {
    for (int64_t t = (int64_t)blockIdx.x * kHT + threadIdx.x; t < nv; t += (int64_t)gridDim.x * kHT) u[t] += x[t];
}

}  // namespace

// Buffers of one cycle precision: time levels (right-hand side and
// correction; level 0 only for the correction cycle of the mixed form), the
// time residual, the spatial hierarchy (levels >= 1: restricted right-hand
// side and V-cycle result), the coarsest time level's block solve.
template <typename T>
struct HeatBufs {
    std::vector<T*> ft, ut, rs, ys;
    T* g = nullptr;
    T* g2 = nullptr;
    T* cx = nullptr;
};

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
    int precision;                // TMG_FP64 or TMG_MIXED
    int use_graph;
    cudaStream_t s;
    bool own_stream;
    int max_blocks;
    void* ws;                     // one allocation for every buffer
    HeatBufs<double> b64;
    HeatBufs<float> b32;
    float* rl;                    // mixed: low part of the residual pair (high part: b32.ft[0])
    bool fresh;                   // mixed: the pair was formed from u directly, not updated
    double* norm2;                // device ||F - L u||^2 of the FP64 iterate
    double* host2;                // pinned copy
    double P1[tmg::kMaxD * tmg::kMaxD], P2[tmg::kMaxD * tmg::kMaxD];
    cudaGraphExec_t graph;        // one cycle, captured for (gF, gu, gu0)
    const void *gF, *gu, *gu0;
    int last_cycles;
    double last_rel;
    std::vector<double> hist;
    int launches_per_cycle;       // kernels and memsets one cycle issues
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

// CTAs for a grid-stride loop over warp tasks (8 per CTA) or row tasks
// (one per CTA of kRT threads): at most what is resident at once.
int grid_warps(const tmg_heat* H, int64_t tasks) {
    const int64_t b = (tasks + kHT / 32 - 1) / (kHT / 32);
    return (int)(b < 1 ? 1 : (b > H->max_blocks ? H->max_blocks : b));
}

int host_row_blocks(int n) { return (n + kRB - 1) / kRB; }

int grid_rows(const tmg_heat* H, int64_t tasks) {
    const int64_t cap = 2 * (int64_t)H->max_blocks;
    return (int)(tasks < 1 ? 1 : (tasks > cap ? cap : tasks));
}

HeatBufs<double>& bufs_of(tmg_heat* H, double*) { return H->b64; }
HeatBufs<float>& bufs_of(tmg_heat* H, float*) { return H->b32; }

thread_local int g_launches = 0;   // kernels and memsets issued (counted while a cycle is issued)

template <int D, typename T>
struct HeatImpl {
    static HeatBufs<T>& B(tmg_heat* H) { return bufs_of(H, static_cast<T*>(nullptr)); }

    static tmg::Xfer<T, D> xfer(const tmg_heat* H) {
        tmg::Xfer<T, D> X;
        for (int i = 0; i < D * D; ++i) {
            X.P1[i] = (T)H->P1[i];
            X.P2[i] = (T)H->P2[i];
        }
        return X;
    }

    // One spatial V(1,1)-cycle from zero on G_tau x = rhs for N intervals at
    // spatial level sl: out = alpha x (acc = 0) or out += alpha x (acc = 1).
    static void vcycle(tmg_heat* H, int sl, const T* rhs, int64_t N, double tau, T* out, T alpha, int acc) {
        const tmg::NvtxRange r_lev("tmg heat spatial level %d", sl);
        HeatBufs<T>& b = B(H);
        const int n = H->nsz[sl];
        const HeatK<D, T> C = heat_consts<D, T>(tau, n);
        ++g_launches;
        if (n == 1) {
            kh_point_solve<D, T><<<grid_of(H, N), kHT, 0, H->s>>>(rhs, out, N, C, alpha, acc);
            return;
        }
        if (n <= kSmallN) {   // this level and all coarser ones in one kernel, in shared memory
            SmallK<D, T> S;
            S.nl = H->ns - sl;
            for (int l = 0; l < S.nl; ++l) {
                S.n[l] = H->nsz[sl + l];
                S.k[l] = heat_consts<D, T>(tau, S.n[l]);
            }
            const int64_t g = N < H->max_blocks ? N : H->max_blocks;
            kh_vsmall<D, T><<<(int)g, kSmallNT, small_smem<T>(D), H->s>>>(rhs, out, N, S, (T)kOmegaS, alpha, acc);
            return;
        }
        const int nc = H->nsz[sl + 1];
        pre(H, rhs, b.rs[sl + 1], N, n, nc, C);
        vcycle(H, sl + 1, b.rs[sl + 1], N, tau, b.ys[sl + 1], T(1), 0);
        ++g_launches;
        post(H, rhs, b.ys[sl + 1], out, N, n, nc, C, alpha, acc);
    }

    // Fused pre kernel of one spatial level: full-row warps up to n = 127,
    // 64-column strips above.
    // Full rows for n + 1 = 32 CPL with CPL = 1, or with a row window of at
    // most 32 bytes per lane and coefficient set (registers); strips otherwise.
    static bool full_rows(int n) {
        return n + 1 <= 32 || ((n + 1 == 64 || n + 1 == 128) && D * ((n + 1) / 32) * (int)sizeof(T) <= 32);
    }

    // Rows per warp task: the longest of max_rows, halving down to 4, that
    // still gives every SM 16 warps; short grids and coarse time levels
    // would otherwise leave few warps, each walking a long chain of rows.
    static int chunk_rows(const tmg_heat* H, int64_t row_sets, int total_rows, int max_rows) {
        const int64_t want = (int64_t)(H->max_blocks / 8) * 16;
        int rows = max_rows;
        while (rows > 4 && row_sets * ((total_rows + rows - 1) / rows) < want) rows /= 2;
        return rows;
    }

    // Warp tasks per row chunk: intervals x strips (strip kernels), intervals
    // (whole-row kernels, CPL >= 2), interval groups of 32 / (n + 1) (CPL = 1).
    static int64_t row_sets(int64_t N, int n, int cols, int stride) {
        if (!full_rows(n)) return N * ((cols + stride - 1) / stride);
        if (n + 1 <= 32) return (N + 32 / (n + 1) - 1) / (32 / (n + 1));
        return N;
    }

    static void pre(tmg_heat* H, const T* rhs, T* rc, int64_t N, int n, int nc, const HeatK<D, T>& C) {
        const T w = (T)kOmegaS;
        const int64_t sets = row_sets(N, n, nc, kPreStride);
        const int rows = chunk_rows(H, sets, nc, kPreRows);
        const int64_t tasks = sets * ((nc + rows - 1) / rows);
        const int g = grid_warps(H, tasks);
        if (!full_rows(n))
            kh_pre_w<D, T><<<g, kHT, 0, H->s>>>(rhs, rc, N, n, nc, rows, C, w);
        else if (n + 1 <= 32)
            kh_pre_f<D, T, 1><<<g, kHT, 0, H->s>>>(rhs, rc, N, n, nc, rows, C, w);
        else if (n + 1 == 64)
            kh_pre_f<D, T, 2><<<g, kHT, 0, H->s>>>(rhs, rc, N, n, nc, rows, C, w);
        else
            kh_pre_f<D, T, 4><<<g, kHT, 0, H->s>>>(rhs, rc, N, n, nc, rows, C, w);
    }

    static void post(tmg_heat* H, const T* rhs, const T* xc, T* out, int64_t N, int n, int nc,
                     const HeatK<D, T>& C, T alpha, int acc) {
        const T w = (T)kOmegaS;
        const int64_t sets = row_sets(N, n, n, kPostStride);
        const int rows = chunk_rows(H, sets, n, kPostRows);
        const int64_t tasks = sets * ((n + rows - 1) / rows);
        const int g = grid_warps(H, tasks);
        if (!full_rows(n))
            kh_post_w<D, T><<<g, kHT, 0, H->s>>>(rhs, xc, out, N, n, nc, rows, C, w, alpha, acc);
        else if (n + 1 <= 32)
            kh_post_f<D, T, 1><<<g, kHT, 0, H->s>>>(rhs, xc, out, N, n, nc, rows, C, w, alpha, acc);
        else if (n + 1 == 64)
            kh_post_f<D, T, 2><<<g, kHT, 0, H->s>>>(rhs, xc, out, N, n, nc, rows, C, w, alpha, acc);
        else
            kh_post_f<D, T, 4><<<g, kHT, 0, H->s>>>(rhs, xc, out, N, n, nc, rows, C, w, alpha, acc);
    }

    // Time residual of level l (u0 only at level 0) into b.g.
    static cudaError_t set_smem() {
        return cudaFuncSetAttribute(kh_vsmall<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)small_smem<T>(D));
    }

    static const T* resid(tmg_heat* H, const T* F, const T* u, const double* u0, int64_t N, double tau) {
        HeatBufs<T>& b = B(H);
        ++g_launches;
        const int n = H->n;
        const HeatK<D, T> C = heat_consts<D, T>(tau, n);
        if (full_rows(n) && n > 1) {
            const int64_t sets = row_sets(N, n, n, kPostStride);
            const int rows = chunk_rows(H, sets, n, kPostRows);
            const int gsz = grid_warps(H, sets * ((n + rows - 1) / rows));
            if (n + 1 <= 32)
                kh_resid_f<D, T, 1><<<gsz, kHT, 0, H->s>>>(F, u, u0, b.g, N, n, rows, C);
            else if (n + 1 == 64)
                kh_resid_f<D, T, 2><<<gsz, kHT, 0, H->s>>>(F, u, u0, b.g, N, n, rows, C);
            else
                kh_resid_f<D, T, 4><<<gsz, kHT, 0, H->s>>>(F, u, u0, b.g, N, n, rows, C);
        } else {
            kh_resid<D, T, T, true, false, false><<<grid_rows(H, N * host_row_blocks(n)), kRT, 0, H->s>>>(
                F, u, u0, b.g, nullptr, N, n, C, nullptr);
        }
        return b.g;
    }

    // One V-cycle in time at level l on L_l u = F (u0 only at level 0).
    // g0: the residual of u, when the caller already has it; zero: u is zero
    // on entry (its residual is F, and the first smoothing step writes u).
    static void tcycle(tmg_heat* H, int l, const T* F, T* u, const double* u0, const T* g0, bool zero) {
        const tmg::NvtxRange r_lev("tmg heat time level %d", l);
        HeatBufs<T>& b = B(H);
        const int64_t N = H->N >> l;
        const double tau = ldexp(H->tau, l);
        const int64_t nn = (int64_t)H->n * H->n, nv = N * D * nn;
        const T wt = (T)kOmegaT;
        if (N == 1) {
            // nu_c spatial V-cycles on the block: x = V(g); x += V(g - G x)
            const T* g = g0 ? g0 : resid(H, F, u, u0, 1, tau);
            T* x = zero ? u : b.cx;
            for (int c = 0; c < H->nu_c; ++c) {
                if (c == 0) {
                    vcycle(H, 0, g, 1, tau, x, T(1), 0);
                } else {
                    ++g_launches;
                    kh_resid<D, T, T, false, false, false><<<grid_rows(H, host_row_blocks(H->n)), kRT, 0, H->s>>>(
                        g, x, nullptr, b.g2, nullptr, 1, H->n, heat_consts<D, T>(tau, H->n), nullptr);
                    vcycle(H, 0, b.g2, 1, tau, x, T(1), 1);
                }
            }
            if (!zero) {
                ++g_launches;
                kh_add<T><<<grid_of(H, nv), kHT, 0, H->s>>>(u, b.cx, nv);
            }
            return;
        }
        if (zero && H->nu1 == 0) {
            ++g_launches;
            cudaMemsetAsync(u, 0, sizeof(T) * nv, H->s);
        }
        for (int k = 0; k < H->nu1; ++k) {
            const T* rhs = (k == 0 && g0) ? g0 : resid(H, F, u, u0, N, tau);
            vcycle(H, 0, rhs, N, tau, u, wt, (zero && k == 0) ? 0 : 1);
        }
        const T* rhs = (H->nu1 == 0 && g0) ? g0 : resid(H, F, u, u0, N, tau);
        const tmg::Xfer<T, D> X = xfer(H);
        ++g_launches;
        kh_restrict_time<D, T><<<grid_rows(H, (N / 2) * host_row_blocks(H->n)), kRT, 0, H->s>>>(rhs, b.ft[l + 1], N / 2, H->n, X);
        tcycle(H, l + 1, b.ft[l + 1], b.ut[l + 1], nullptr, b.ft[l + 1], true);
        ++g_launches;
        kh_prolong_time<D, T><<<grid_rows(H, (N / 2) * host_row_blocks(H->n)), kRT, 0, H->s>>>(b.ut[l + 1], u, N / 2, H->n, X);
        for (int k = 0; k < H->nu2; ++k) vcycle(H, 0, resid(H, F, u, u0, N, tau), N, tau, u, wt, 1);
    }
};

// The work of one cycle after the residual of u has been formed: FP64 --
// the cycle on L u = F with the residual in b64.g; mixed -- the FP32 cycle on
// L c = r_h from c = 0, then u += c and r -= L c (float pair) with ||r||^2.
template <int D>
void cycle_body(tmg_heat* H, const double* F, double* u, const double* u0) {
    if (H->precision == TMG_FP64) {
        HeatImpl<D, double>::tcycle(H, 0, F, u, u0, H->b64.g, false);
    } else {
        HeatBufs<float>& b = H->b32;
        HeatImpl<D, float>::tcycle(H, 0, b.ft[0], b.ut[0], nullptr, b.ft[0], true);
        g_launches += 2;
        cudaMemsetAsync(H->norm2, 0, sizeof(double), H->s);
        kh_update_pair<D><<<grid_rows(H, H->N * host_row_blocks(H->n)), kRT, 0, H->s>>>(u, b.ut[0], b.ft[0], H->rl, H->N, H->n,
                                                                      pair_consts<D>(H->tau, H->n), H->norm2);
    }
}

// One cycle: replayed from a graph captured for these arrays (the FP64 form
// reads F, u and u0 inside the cycle; the mixed form only u), else issued.
template <int D>
tmg_status run_cycle(tmg_heat* H, const double* F, double* u, const double* u0) {
    const bool fp64 = H->precision == TMG_FP64;
    const void* kF = fp64 ? F : nullptr;
    const void* ku0 = fp64 ? u0 : nullptr;
    if (!H->use_graph) {
        g_launches = 0;
        cycle_body<D>(H, F, u, u0);
        H->launches_per_cycle = g_launches;
        TH_CUDA(cudaGetLastError());
        return TMG_OK;
    }
    if (!H->graph || H->gF != kF || H->gu != u || H->gu0 != ku0) {
        if (H->graph) {
            cudaGraphExecDestroy(H->graph);
            H->graph = nullptr;
        }
        TH_CUDA(cudaStreamBeginCapture(H->s, cudaStreamCaptureModeThreadLocal));
        g_launches = 0;
        cycle_body<D>(H, F, u, u0);
        cudaGraph_t g = nullptr;
        const cudaError_t e1 = cudaStreamEndCapture(H->s, &g);
        if (e1 != cudaSuccess || g == nullptr) {
            cudaGetLastError();
            g_heat_cuda = (int)e1;
            return TMG_ECUDA;
        }
        const cudaError_t e2 = cudaGraphInstantiate(&H->graph, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) {
            H->graph = nullptr;
            g_heat_cuda = (int)e2;
            return TMG_ECUDA;
        }
        H->launches_per_cycle = g_launches;
        H->gF = kF;
        H->gu = u;
        H->gu0 = ku0;
    }
    TH_CUDA(cudaGraphLaunch(H->graph, H->s));
    return TMG_OK;
}

// ||F - L u||^2 of the FP64 iterate into *norm2, the residual itself into
// b64.g (FP64 form) or the float pair (b32.ft[0], rl) (mixed form).
template <int D>
tmg_status residual_fp64(tmg_heat* H, const double* F, const double* u, const double* u0) {
    const HeatK<D, double> C = heat_consts<D, double>(H->tau, H->n);
    TH_CUDA(cudaMemsetAsync(H->norm2, 0, sizeof(double), H->s));
    const int grid = grid_rows(H, H->N * host_row_blocks(H->n));
    if (H->precision == TMG_FP64)
        kh_resid<D, double, double, true, true, false><<<grid, kRT, 0, H->s>>>(F, u, u0, H->b64.g, nullptr, H->N,
                                                                              H->n, C, H->norm2);
    else
        kh_resid<D, double, float, true, true, true><<<grid, kRT, 0, H->s>>>(F, u, u0, H->b32.ft[0], H->rl, H->N,
                                                                            H->n, C, H->norm2);
    TH_CUDA(cudaGetLastError());
    return TMG_OK;
}

tmg_status read_norm(tmg_heat* H, double* nr) {
    TH_CUDA(cudaMemcpyAsync(H->host2, H->norm2, sizeof(double), cudaMemcpyDeviceToHost, H->s));
    TH_CUDA(cudaStreamSynchronize(H->s));
    *nr = sqrt(*H->host2);
    return TMG_OK;
}

// solve: cycles from u = 0 until the relative residual is below tol; the
// mixed form confirms a converged float-pair residual by the FP64 residual
// of u before it stops.  !solve: one cycle applied to u.
template <int D>
tmg_status run_heat(tmg_heat* H, const double* F, const double* u0, double* u, bool solve) {
    const int64_t nv = H->N * D * (int64_t)H->n * H->n;
    const bool fp64 = H->precision == TMG_FP64;
    tmg_status st;
    if (!solve) {
        if ((st = residual_fp64<D>(H, F, u, u0)) != TMG_OK) return st;
        if ((st = run_cycle<D>(H, F, u, u0)) != TMG_OK) return st;
        TH_CUDA(cudaGetLastError());
        TH_CUDA(cudaStreamSynchronize(H->s));
        return TMG_OK;
    }
    TH_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * nv, H->s));
    H->hist.clear();
    if (fp64) {
        if ((st = residual_fp64<D>(H, F, u, u0)) != TMG_OK) return st;
    } else {
        TH_CUDA(cudaMemsetAsync(H->norm2, 0, sizeof(double), H->s));
        kh_init_pair<D><<<grid_rows(H, H->N * host_row_blocks(H->n)), kRT, 0, H->s>>>(F, u0, H->b32.ft[0], H->rl, H->N, H->n,
                                                                    H->norm2);
        TH_CUDA(cudaGetLastError());
    }
    H->fresh = true;
    double nF = 0.0;
    for (int k = 0;; ++k) {
        double nr = 0.0;
        if ((st = read_norm(H, &nr)) != TMG_OK) return st;
        if (k == 0) nF = nr;
        double rel = nF > 0.0 ? nr / nF : nr;
        if (!fp64 && rel <= H->tol && !H->fresh) {
            // confirm from u itself (this also restarts the pair from the true residual)
            if ((st = residual_fp64<D>(H, F, u, u0)) != TMG_OK) return st;
            if ((st = read_norm(H, &nr)) != TMG_OK) return st;
            rel = nF > 0.0 ? nr / nF : nr;
            H->fresh = true;
        }
        H->hist.push_back(rel);
        H->last_cycles = k;
        H->last_rel = rel;
        if (!(rel == rel) || rel > 1e300) return TMG_ENUMERIC;
        if (rel <= H->tol) return TMG_OK;
        if (k >= H->max_cycles) return TMG_ENOTCONV;
        if ((st = run_cycle<D>(H, F, u, u0)) != TMG_OK) return st;
        TH_CUDA(cudaGetLastError());
        H->fresh = false;
        if (fp64 && (st = residual_fp64<D>(H, F, u, u0)) != TMG_OK) return st;
    }
}

// Event timings (ms per launch, mean of reps) of the level-0 kernels on the
// plan's stream after one cycle has filled the buffers: [0] time residual in
// the cycle precision, [1] pre (spatial level 0), [2] post with
// accumulation (spatial level 0), [3] the mixed form's pair update or the
// FP64 form's FP64 residual, [4] one whole cycle.
template <int D>
tmg_status profile_heat(tmg_heat* H, const double* F, const double* u0, double* u, int reps, double* ms) {
    tmg_status st;
    if ((st = residual_fp64<D>(H, F, u, u0)) != TMG_OK) return st;
    if ((st = run_cycle<D>(H, F, u, u0)) != TMG_OK) return st;
    const int64_t N = H->N;
    const int n = H->n, nc = H->ns > 1 ? H->nsz[1] : 0;
    cudaEvent_t e0, e1;
    TH_CUDA(cudaEventCreate(&e0));
    TH_CUDA(cudaEventCreate(&e1));
    auto timed = [&](auto&& launch) -> double {
        cudaEventRecord(e0, H->s);
        for (int r = 0; r < reps; ++r) launch();
        cudaEventRecord(e1, H->s);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        return (double)t / reps;
    };
    auto level0 = [&](auto* tag, auto& b, const auto* rhs, const auto* uu, auto* out) {
        using T = typename std::remove_pointer<decltype(tag)>::type;
        const HeatK<D, T> C = heat_consts<D, T>(H->tau, n);
        ms[0] = timed([&] { HeatImpl<D, T>::resid(H, rhs, uu, nullptr, N, H->tau); });
        if (nc > 0) {
            ms[1] = timed([&] { HeatImpl<D, T>::pre(H, rhs, b.rs[1], N, n, nc, C); });
            ms[2] = timed([&] { HeatImpl<D, T>::post(H, rhs, b.ys[1], out, N, n, nc, C, (T)kOmegaT, 1); });
        }
    };
    ms[1] = ms[2] = 0.0;
    if (H->precision == TMG_FP64) {
        level0(static_cast<double*>(nullptr), H->b64, F, u, H->b64.g);
        ms[3] = timed([&] { residual_fp64<D>(H, F, u, u0); });
    } else {
        HeatBufs<float>& b = H->b32;
        level0(static_cast<float*>(nullptr), b, b.ft[0], b.ut[0], b.g);
        const PairK<D> P = pair_consts<D>(H->tau, n);
        ms[3] = timed([&] {
            kh_update_pair<D><<<grid_rows(H, N * host_row_blocks(n)), kRT, 0, H->s>>>(u, b.ut[0], b.ft[0], H->rl, N,
                                                                                     n, P, H->norm2);
        });
    }
    ms[4] = timed([&] { run_cycle<D>(H, F, u, u0); });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TH_CUDA(cudaGetLastError());
    TH_CUDA(cudaStreamSynchronize(H->s));
    return TMG_OK;
}

tmg_status profile_heat_d(tmg_heat* H, const double* F, const double* u0, double* u, int reps, double* ms) {
    switch (H->d) {
        case 1: return profile_heat<1>(H, F, u0, u, reps, ms);
        case 2: return profile_heat<2>(H, F, u0, u, reps, ms);
        case 3: return profile_heat<3>(H, F, u0, u, reps, ms);
        case 4: return profile_heat<4>(H, F, u0, u, reps, ms);
        case 5: return profile_heat<5>(H, F, u0, u, reps, ms);
        default: return profile_heat<6>(H, F, u0, u, reps, ms);
    }
}

cudaError_t set_smem_d(int d, bool fp64) {
    switch (d) {
#define TMG_HEAT_SMEM(DD) \
    case DD: return fp64 ? HeatImpl<DD, double>::set_smem() : HeatImpl<DD, float>::set_smem();
        TMG_HEAT_SMEM(1)
        TMG_HEAT_SMEM(2)
        TMG_HEAT_SMEM(3)
        TMG_HEAT_SMEM(4)
        TMG_HEAT_SMEM(5)
        TMG_HEAT_SMEM(6)
#undef TMG_HEAT_SMEM
        default: return cudaErrorInvalidValue;
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
    bool pow2n = n >= 1 && n < (1 << 14), pow2N = N >= 1 && N <= (int64_t(1) << 40);
    for (int64_t m = (int64_t)n + 1; pow2n && m > 1; m >>= 1) pow2n = (m & 1) == 0;
    for (int64_t m = N; pow2N && m > 1; m >>= 1) pow2N = (m & 1) == 0;
    if (p_t < 0 || p_t > tmg::kMaxD - 1 || !(tau > 0.0) || !isfinite(tau) || !pow2n || !pow2N || nu_c < 1 ||
        nu_c > 16 || o.nu1 < 0 || o.nu1 > 8 || o.nu2 < 0 || o.nu2 > 8 || o.nu1 + o.nu2 < 1 || o.gamma != 1 ||
        o.max_cycles < 0 || !(o.tol >= 0.0) || (o.precision != TMG_FP64 && o.precision != TMG_MIXED))
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
    H->precision = o.precision;
    H->use_graph = o.use_graph ? 1 : 0;
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
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        set_smem_d(H->d, H->precision == TMG_FP64) != cudaSuccess) {
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
    // workspace, in the cycle precision: time levels (level 0 only for the
    // mixed form's correction), the time residual, the spatial hierarchy
    // below level 0, the coarsest time level's block solve
    const bool fp64 = H->precision == TMG_FP64;
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    const int64_t nv0 = N * H->d * (int64_t)n * n, blk = (int64_t)H->d * n * n;
    std::vector<int64_t> sizes;
    for (int l = fp64 ? 1 : 0; l < H->nt; ++l) {
        sizes.push_back(nv0 >> l);   // ft
        sizes.push_back(nv0 >> l);   // ut
    }
    sizes.push_back(nv0);            // g
    for (int sl = 1; sl < H->ns; ++sl) {
        const int64_t v = N * H->d * (int64_t)H->nsz[sl] * H->nsz[sl];
        sizes.push_back(v);          // rs
        sizes.push_back(v);          // ys
    }
    sizes.push_back(blk);            // g2
    sizes.push_back(blk);            // cx
    if (!fp64) sizes.push_back(nv0); // rl (float)
    auto padded = [](size_t b) { return (b + 255) / 256 * 256; };
    size_t bytes = padded(sizeof(double));   // norm2
    for (int64_t v : sizes) bytes += padded((size_t)v * es);
    if (cudaMalloc(&H->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        H->ws = nullptr;
        tmg_heat_destroy(H);
        return TMG_ENOMEM;
    }
    char* base = static_cast<char*>(H->ws);
    size_t off = 0, k = 0;
    H->norm2 = reinterpret_cast<double*>(base);
    off = padded(sizeof(double));
    auto take = [&]() -> void* {
        void* q = base + off;
        off += padded((size_t)sizes[k++] * es);
        return q;
    };
    auto carve = [&](auto& b) {
        using P = typename std::remove_reference<decltype(b.ft[0])>::type;
        b.ft.assign(H->nt, nullptr);
        b.ut.assign(H->nt, nullptr);
        for (int l = fp64 ? 1 : 0; l < H->nt; ++l) {
            b.ft[l] = static_cast<P>(take());
            b.ut[l] = static_cast<P>(take());
        }
        b.g = static_cast<P>(take());
        b.rs.assign(H->ns, nullptr);
        b.ys.assign(H->ns, nullptr);
        for (int sl = 1; sl < H->ns; ++sl) {
            b.rs[sl] = static_cast<P>(take());
            b.ys[sl] = static_cast<P>(take());
        }
        b.g2 = static_cast<P>(take());
        b.cx = static_cast<P>(take());
    };
    if (fp64) {
        carve(H->b64);
    } else {
        carve(H->b32);
        H->rl = static_cast<float*>(take());
    }
    if (cudaMallocHost(&H->host2, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
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
    switch (H->d) {
#define TMG_HEAT_RES(DD)                                                                                  \
    case DD:                                                                                              \
        kh_resid<DD, double, double, true, false, false><<<grid_rows(H, H->N * host_row_blocks(H->n)), kRT, 0, H->s>>>(   \
            f, u, u0, r, nullptr, H->N, H->n, heat_consts<DD, double>(H->tau, H->n), nullptr);            \
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

tmg_status tmg_heat_profile(tmg_heat* H, const double* f, const double* u0, double* u, int reps, double* ms,
                            int n_ms) {
    if (!H || !aligned16(f) || !aligned16(u) || !u0 || (reinterpret_cast<uintptr_t>(u0) & 7u) || reps < 1 ||
        !ms || n_ms < 5)
        return TMG_EINVAL;
    return profile_heat_d(H, f, u0, u, reps, ms);
}

tmg_status tmg_heat_stats(const tmg_heat* H, int* cycles, double* rel_res, double* hist, int hist_len) {
    if (!H) return TMG_EINVAL;
    if (cycles) *cycles = H->last_cycles;
    if (rel_res) *rel_res = H->last_rel;
    if (hist)
        for (int i = 0; i < hist_len; ++i) hist[i] = i < (int)H->hist.size() ? H->hist[i] : NAN;
    return TMG_OK;
}

tmg_status tmg_heat_info(const tmg_heat* H, int* time_levels, int* space_levels, int* launches_per_cycle,
                         size_t* workspace_bytes) {
    if (!H) return TMG_EINVAL;
    if (time_levels) *time_levels = H->nt;
    if (space_levels) *space_levels = H->ns;
    if (launches_per_cycle) *launches_per_cycle = H->launches_per_cycle;
    if (workspace_bytes) {
        size_t b = 0;
        const size_t es = H->precision == TMG_FP64 ? sizeof(double) : sizeof(float);
        const int64_t nv0 = H->N * H->d * (int64_t)H->n * H->n;
        for (int l = H->precision == TMG_FP64 ? 1 : 0; l < H->nt; ++l) b += 2 * (size_t)(nv0 >> l) * es;
        b += (size_t)nv0 * es;
        for (int sl = 1; sl < H->ns; ++sl) b += 2 * (size_t)(H->N * H->d * (int64_t)H->nsz[sl] * H->nsz[sl]) * es;
        if (H->precision != TMG_FP64) b += (size_t)nv0 * sizeof(float);
        *workspace_bytes = b;
    }
    return TMG_OK;
}

void tmg_heat_destroy(tmg_heat* H) {
    if (!H) return;
    if (H->s) cudaStreamSynchronize(H->s);
    if (H->graph) cudaGraphExecDestroy(H->graph);
    if (H->ws) cudaFree(H->ws);
    if (H->host2) cudaFreeHost(H->host2);
    if (H->own_stream) cudaStreamDestroy(H->s);
    delete H;
}

}  // extern "C"
