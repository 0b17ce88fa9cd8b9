// Device code of the time-multigrid solver (Gander & Neumueller, arXiv:1409.5254).
//
// Data layout: every level stores its vectors interval-major, [N_l][D] with
// D = p_t + 1 shifted-Legendre coefficients per interval.  The basis fixes
// a_k = psi_k(0) = (-1)^k and b_l = psi_l(1) = 1, so the coupling term
// N u_{n-1} = a (b^T u_{n-1}) only needs the previous interval's endpoint
// value e_{n-1} = sum_l u_{n-1}[l] (the one-value halo).
//
// Each cycle is written in correction form: level 0 forms r = F - L u in
// FP64, every level below starts from a zero guess, and the pre-smoothed
// iterate of a zero-started level is recomputed on the way up instead of
// being stored.  With a zero start the damped block Jacobi sweep of
// eq. chap4_ODESmoother gives u = omega A^{-1} f and A u = omega f, so the
// residual after pre-smoothing is formed without an explicit A u product
// (no cancellation in the cycle precision): we carry w = A u along.
//
// Streaming kernels map one lane to one coarse pair (two fine intervals,
// the unit of the restriction R = [R1 R2]).  Halo values move between lanes
// by warp shuffles; the first H lanes of every warp tile recompute the
// previous tile's last pairs so that warps never wait on each other.  Each
// sweep that needs e_{n-1} shifts the garbage entering lane 0 by one
// interval, so H = ceil(S/2) lanes cover S such sweeps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tmg_bounds.h"

#include <type_traits>

namespace tmg {

constexpr int kMaxD = 6;          // p_t <= 5: every kernel (two-level kernels, on-chip solver, fused level 0)
constexpr int kMaxDWide = 21;     // p_t = 10 and 20 (D = 11, 21): the per-level kernels and the grid-wide scan

// Block widths the library builds: p_t = 0..5, 10 and 20 (the degrees of the
// paper's scaling tables).
constexpr bool built_width(int d) { return (d >= 1 && d <= kMaxD) || d == 11 || d == kMaxDWide; }
constexpr int kMaxLevels = 48;
constexpr int kHist = 512;
constexpr unsigned kFull = 0xffffffffu;

// Constants of one level in the cycle precision T (row-major D x D blocks).
template <typename T, int D>
struct LevelK {
    T A[D * D];      // K + z_l Mhat
    T Ainv[D * D];   // its inverse
    T g[D];          // A^{-1} a
    T c[D];          // b^T A^{-1}
    T omega;         // damping of this level
    T alpha;         // b^T A^{-1} a
};

// Prolongation onto the two halves of a coarse interval: P1 = R1^T, P2 = R2^T.
template <typename T, int D>
struct Xfer {
    T P1[D * D];
    T P2[D * D];
};

// Level-0 residual constants: zm[k] = z_0 / (2k+1) in FP64 and as an
// unevaluated float pair zm_hi + zm_lo.
struct Res0 {
    double zm[kMaxDWide];
    float zm_hi[kMaxDWide];
    float zm_lo[kMaxDWide];
};

// Device-resident solve state.  Written by the last block of the residual
// kernel; every other kernel of a cycle returns at once when done != 0.
struct DevState {
    const double* F;      // load vector of the current solve
    double* u;            // solution of the current solve
    double u0;            // initial value of the current solve
    double nF;            // ||F||_2 (F with a*u0 folded in)
    double tol;
    int max_cycles;
    int cycle;            // residual evaluations done so far in this solve
    int done;             // 0 running, 1 converged, 2 cycle limit, 3 non-finite
    int nF_from_first;    // 1: the first residual (u = 0) defines ||F||
    int use_cond;         // 1: the solve runs as a graph while-loop
    int full;             // what the next level-0 down kernel evaluates from u in FP64: 0 nothing,
                          // 1 only the norm of F - L u (confirming an updated residual that met
                          // tol), 2 the residual itself, stored, with the restriction onto level 1
                          // (the start of a solve, and after a confirmation failed)
    int rsel;             // which of the two float-pair residual buffers holds the current residual
    int u_zero;           // 1: the solve starts from u = 0 (the first residual is F itself)
    unsigned ticket;      // last-block ticket
    unsigned ticket2;     // last-block ticket of the coarsest solve in the last down kernel
    float nscale;         // power of two that brings the residual near 1 (FP32 norm)
    long long nvals;      // values per residual vector, N * D
    unsigned long long cond;   // cudaGraphConditionalHandle of that loop
    double hist[kHist];   // relative residual before each cycle
};

// ------------------------------------------------------------ helpers --

// Programmatic dependent launch: a kernel of the cycle may be launched
// before its predecessor in the stream has finished; it waits here, before
// touching any memory, until the predecessor has completed and its writes are
// visible, and then lets its own successor launch.  Without a programmatic
// predecessor the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

// Coupling policy.  DIR = 0: the system of eq. chap4_generalLinearSystemODE,
// N = a b^T with a_k = (-1)^k, b_l = 1.  DIR = 1: its transpose written in
// reversed time, n -> N-1-n, which is again block lower-bidiagonal with
// diagonal block A^T and N' = a' b'^T, a'_k = 1, b'_l = (-1)^l (the adjoint
// solve runs the same cycle on reversed arrays).

// Sum of the coefficients, e = 1^T u.
template <typename T, int D>
__device__ __forceinline__ T endval(const T (&u)[D]) {
    T e = u[0];
#pragma unroll
    for (int k = 1; k < D; ++k) e += u[k];
    return e;
}

// The halo functional b^T u.
template <int DIR, typename T, int D>
__device__ __forceinline__ T bval(const T (&u)[D]) {
    T e = u[0];
#pragma unroll
    for (int k = 1; k < D; ++k) e += (DIR == 1 && (k & 1)) ? -u[k] : u[k];
    return e;
}

// a_k x.
template <int DIR, typename T>
__device__ __forceinline__ T acoef(int k, T x) {
    return (DIR == 0 && (k & 1)) ? -x : x;
}

template <typename T, int D>
__device__ __forceinline__ void matvec(const T* M, const T (&x)[D], T (&y)[D]) {
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = M[i * D] * x[0];
#pragma unroll
        for (int j = 1; j < D; ++j) s = fma(M[i * D + j], x[j], s);
        y[i] = s;
    }
}

template <typename T, int D>
__device__ __forceinline__ T dotc(const T* c, const T (&x)[D]) {
    T s = c[0] * x[0];
#pragma unroll
    for (int j = 1; j < D; ++j) s = fma(c[j], x[j], s);
    return s;
}

template <typename T>
__device__ __forceinline__ T shfl_prev(T v) {
    return __shfl_up_sync(kFull, v, 1);
}

// Vector load/store of NV contiguous T values.  The caller guarantees that
// p is aligned to the largest power of two (<= 16 bytes) dividing NV*sizeof(T).
template <typename T, int NV>
struct VecIO {
    static constexpr int B = NV * (int)sizeof(T);
    static constexpr int W = (B % 16 == 0) ? 16 : (B % 8 == 0) ? 8 : 4;
    using V = typename std::conditional<W == 16, uint4, typename std::conditional<W == 8, uint2, unsigned>::type>::type;
    union U {
        V w[B / W];
        T v[NV];
    };
    static __device__ __forceinline__ void load(const T* __restrict__ p, T (&out)[NV]) {
        U u;
        const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
        for (int i = 0; i < B / W; ++i) u.w[i] = q[i];
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i] = u.v[i];
    }
    static __device__ __forceinline__ void store(T* __restrict__ p, const T (&in)[NV]) {
        U u;
#pragma unroll
        for (int i = 0; i < NV; ++i) u.v[i] = in[i];
        V* q = reinterpret_cast<V*>(p);
#pragma unroll
        for (int i = 0; i < B / W; ++i) q[i] = u.w[i];
    }
};

// The level-vector helpers take the number of valid elements nq of their
// array (pairs, intervals, groups of M); the debug build checks q against it
// (q >= 0 only when nq < 0) and skips an access outside.
template <typename T, int D>
__device__ __forceinline__ void load_pair(const T* __restrict__ base, int64_t q, bool ok, T (&x)[2][D],
                                          int64_t nq = -1) {
    T v[2 * D];
    if (ok && TMG_IN(q, nq < 0 ? INT64_MAX : nq, 1)) {
        VecIO<T, 2 * D>::load(base + q * 2 * D, v);
    } else {
#pragma unroll
        for (int i = 0; i < 2 * D; ++i) v[i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        x[0][i] = v[i];
        x[1][i] = v[D + i];
    }
}

template <typename T, int D>
__device__ __forceinline__ void store_pair(T* __restrict__ base, int64_t q, const T (&x)[2][D], int64_t nq = -1) {
    if (!TMG_IN(q, nq < 0 ? INT64_MAX : nq, 2)) return;
    T v[2 * D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        v[i] = x[0][i];
        v[D + i] = x[1][i];
    }
    VecIO<T, 2 * D>::store(base + q * 2 * D, v);
}

template <typename T, int D>
__device__ __forceinline__ void load_one(const T* __restrict__ base, int64_t q, bool ok, T (&x)[D],
                                         int64_t nq = -1) {
    if (ok && TMG_IN(q, nq < 0 ? INT64_MAX : nq, 3)) {
        VecIO<T, D>::load(base + q * D, x);
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) x[i] = T(0);
    }
}

// ------------------------------------------- asynchronous tile staging --
//
// Level-0 kernels stage the next warp tile of their FP64 inputs in shared
// memory with cp.async while they compute the current one (two stages per
// warp).  Each lane copies and later reads only its own bytes, stored
// 16-byte-chunk-major so that a warp's reads of one chunk are contiguous.
// Lanes outside the array copy zeros (source size 0).

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// NB bytes (a multiple of 16) per lane; buffer layout [NB/16][32] of 16-byte chunks.
template <int NB>
struct LaneStage {
    static_assert(NB % 16 == 0, "staged lane data must be a multiple of 16 bytes");
    static constexpr int C = NB / 16;
    // Copy NB bytes at base + offset (in T elements); invalid lanes read nothing
    // (source size 0, the address stays at the array base) and store zeros.
    template <typename T>
    static __device__ __forceinline__ void issue(uint4* buf, const T* base, int64_t offset, bool valid, int lane) {
        const uint4* g = reinterpret_cast<const uint4*>(valid ? base + offset : base);
#pragma unroll
        for (int c = 0; c < C; ++c) cp_async16(&buf[c * 32 + lane], valid ? g + c : g, valid);
    }
    template <typename T, int NV>
    static __device__ __forceinline__ void read(const uint4* buf, int lane, T (&out)[NV]) {
        static_assert(NV * sizeof(T) == NB, "size mismatch");
        union {
            uint4 w[C];
            T v[NV];
        } u;
#pragma unroll
        for (int c = 0; c < C; ++c) u.w[c] = buf[c * 32 + lane];
#pragma unroll
        for (int i = 0; i < NV; ++i) out[i] = u.v[i];
    }
};

// ------------------------------------------------ smoother building blocks --

// Pre-smoothing from a zero guess for a coarse pair with right-hand side f:
// sweep 1 gives u = omega A^{-1} f, w = A u = omega f; sweeps 2..nu1 use the
// previous interval's endpoint value (warp shuffle).  h = A^{-1} f is kept.
template <int DIR, typename T, int D>
__device__ __forceinline__ void presmooth_zero(const LevelK<T, D>& K, const T (&f)[2][D], T (&h)[2][D],
                                               T (&u)[2][D], T (&w)[2][D], int nu1, bool first = false) {
    const T om = K.omega, om1 = T(1) - K.omega;
    const T om_first = nu1 > 0 ? om : T(0);     // no pre-smoothing leaves u = 0
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        matvec<T, D>(K.Ainv, f[i], h[i]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            u[i][k] = om_first * h[i][k];
            w[i][k] = om_first * f[i][k];
        }
    }
    for (int s = 1; s < nu1; ++s) {
        const T e0 = bval<DIR, T, D>(u[0]);
        const T ep_s = shfl_prev(bval<DIR, T, D>(u[1]));
        const T ep = first ? T(0) : ep_s;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            u[0][k] = om1 * u[0][k] + om * fma(K.g[k], ep, h[0][k]);
            w[0][k] = om1 * w[0][k] + om * (f[0][k] + acoef<DIR>(k, ep));
            u[1][k] = om1 * u[1][k] + om * fma(K.g[k], e0, h[1][k]);
            w[1][k] = om1 * w[1][k] + om * (f[1][k] + acoef<DIR>(k, e0));
        }
    }
}

// Pre-smoothing from a given iterate u (the second visit of a level in a
// W-cycle): w = A u, then nu1 damped block-Jacobi sweeps of u and w; h =
// A^{-1} f.  The same sweep as presmooth_zero's after its first.
template <int DIR, typename T, int D>
__device__ __forceinline__ void presmooth_from(const LevelK<T, D>& K, const T (&f)[2][D], T (&h)[2][D],
                                               T (&u)[2][D], T (&w)[2][D], int nu1, bool first = false) {
    const T om = K.omega, om1 = T(1) - K.omega;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        matvec<T, D>(K.Ainv, f[i], h[i]);
        matvec<T, D>(K.A, u[i], w[i]);
    }
    for (int s = 0; s < nu1; ++s) {
        const T e0 = bval<DIR, T, D>(u[0]);
        const T ep_s = shfl_prev(bval<DIR, T, D>(u[1]));
        const T ep = first ? T(0) : ep_s;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            u[0][k] = om1 * u[0][k] + om * fma(K.g[k], ep, h[0][k]);
            w[0][k] = om1 * w[0][k] + om * (f[0][k] + acoef<DIR>(k, ep));
            u[1][k] = om1 * u[1][k] + om * fma(K.g[k], e0, h[1][k]);
            w[1][k] = om1 * w[1][k] + om * (f[1][k] + acoef<DIR>(k, e0));
        }
    }
}

// Residual f + a e_{n-1} - A u of a pair, with A u = w carried along.
template <int DIR, typename T, int D>
__device__ __forceinline__ void residual_tracked(const T (&f)[2][D], const T (&u)[2][D], const T (&w)[2][D],
                                                 T (&r)[2][D], bool first = false) {
    const T e0 = bval<DIR, T, D>(u[0]);
    const T ep_s = shfl_prev(bval<DIR, T, D>(u[1]));
    const T ep = first ? T(0) : ep_s;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        r[0][k] = f[0][k] + acoef<DIR>(k, ep) - w[0][k];
        r[1][k] = f[1][k] + acoef<DIR>(k, e0) - w[1][k];
    }
}

// Restriction f_c = R1 r_{2m} + R2 r_{2m+1} with R_i = P_i^T (eq. chap4_restrictionTime).
template <typename T, int D>
__device__ __forceinline__ void restrict_pair(const Xfer<T, D>& X, const T (&r)[2][D], T (&fc)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(X.P1[l * D + k], r[0][l], fma(X.P2[l * D + k], r[1][l], s));
        fc[k] = s;
    }
}

// Prolongation u_{2m} += P1 uc, u_{2m+1} += P2 uc (eq. chap4_prolongationTime).
template <typename T, int D>
__device__ __forceinline__ void prolong_add(const Xfer<T, D>& X, const T (&uc)[D], T (&u)[2][D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T s1 = u[0][k], s2 = u[1][k];
#pragma unroll
        for (int l = 0; l < D; ++l) {
            s1 = fma(X.P1[k * D + l], uc[l], s1);
            s2 = fma(X.P2[k * D + l], uc[l], s2);
        }
        u[0][k] = s1;
        u[1][k] = s2;
    }
}

// nu post-smoothing sweeps: u <- (1-omega) u + omega (A^{-1} f + g e_{n-1}).
template <int DIR, typename T, int D>
__device__ __forceinline__ void postsmooth(const LevelK<T, D>& K, const T (&h)[2][D], T (&u)[2][D], int nu,
                                           bool first = false) {
    const T om = K.omega, om1 = T(1) - K.omega;
    for (int s = 0; s < nu; ++s) {
        const T e0 = bval<DIR, T, D>(u[0]);
        const T ep_s = shfl_prev(bval<DIR, T, D>(u[1]));
        const T ep = first ? T(0) : ep_s;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            u[0][k] = om1 * u[0][k] + om * fma(K.g[k], ep, h[0][k]);
            u[1][k] = om1 * u[1][k] + om * fma(K.g[k], e0, h[1][k]);
        }
    }
}

// ------------------------- M consecutive intervals per lane (two-level kernels) --
//
// The same building blocks for a lane that holds M consecutive intervals of
// one level; the halo of interval 0 is the previous lane's interval M-1.

template <int DIR, typename T, int D, int M>
__device__ __forceinline__ void presmooth_zero_m(const LevelK<T, D>& K, const T (&f)[M][D], T (&h)[M][D],
                                                 T (&u)[M][D], T (&w)[M][D], int nu1, bool first = false) {
    const T om = K.omega, om1 = T(1) - K.omega;
    const T om_first = nu1 > 0 ? om : T(0);
#pragma unroll
    for (int i = 0; i < M; ++i) {
        matvec<T, D>(K.Ainv, f[i], h[i]);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            u[i][k] = om_first * h[i][k];
            w[i][k] = om_first * f[i][k];
        }
    }
    for (int s = 1; s < nu1; ++s) {
        T e[M];
#pragma unroll
        for (int i = 0; i < M; ++i) e[i] = bval<DIR, T, D>(u[i]);
        const T ep_s = shfl_prev(e[M - 1]);
        const T ep0 = first ? T(0) : ep_s;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const T ep = i == 0 ? ep0 : e[i - 1];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                u[i][k] = om1 * u[i][k] + om * fma(K.g[k], ep, h[i][k]);
                w[i][k] = om1 * w[i][k] + om * (f[i][k] + acoef<DIR>(k, ep));
            }
        }
    }
}

template <int DIR, typename T, int D, int M>
__device__ __forceinline__ void residual_tracked_m(const T (&f)[M][D], const T (&u)[M][D], const T (&w)[M][D],
                                                   T (&r)[M][D], bool first = false) {
    T e[M];
#pragma unroll
    for (int i = 0; i < M; ++i) e[i] = bval<DIR, T, D>(u[i]);
    const T ep_s = shfl_prev(e[M - 1]);
    const T ep0 = first ? T(0) : ep_s;
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const T ep = i == 0 ? ep0 : e[i - 1];
#pragma unroll
        for (int k = 0; k < D; ++k) r[i][k] = f[i][k] + acoef<DIR>(k, ep) - w[i][k];
    }
}

template <int DIR, typename T, int D, int M>
__device__ __forceinline__ void postsmooth_m(const LevelK<T, D>& K, const T (&h)[M][D], T (&u)[M][D], int nu,
                                             bool first = false) {
    const T om = K.omega, om1 = T(1) - K.omega;
    for (int s = 0; s < nu; ++s) {
        T e[M];
#pragma unroll
        for (int i = 0; i < M; ++i) e[i] = bval<DIR, T, D>(u[i]);
        const T ep_s = shfl_prev(e[M - 1]);
        const T ep0 = first ? T(0) : ep_s;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const T ep = i == 0 ? ep0 : e[i - 1];
#pragma unroll
            for (int k = 0; k < D; ++k) u[i][k] = om1 * u[i][k] + om * fma(K.g[k], ep, h[i][k]);
        }
    }
}

// f_c = R1 a + R2 b for the two halves a, b of one coarse interval.
template <typename T, int D>
__device__ __forceinline__ void restrict2(const Xfer<T, D>& X, const T (&a)[D], const T (&b)[D], T (&fc)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s = fma(X.P1[l * D + k], a[l], fma(X.P2[l * D + k], b[l], s));
        fc[k] = s;
    }
}

// a += P1 uc, b += P2 uc.
template <typename T, int D>
__device__ __forceinline__ void prolong_add2(const Xfer<T, D>& X, const T (&uc)[D], T (&a)[D], T (&b)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        T s1 = a[k], s2 = b[k];
#pragma unroll
        for (int l = 0; l < D; ++l) {
            s1 = fma(X.P1[k * D + l], uc[l], s1);
            s2 = fma(X.P2[k * D + l], uc[l], s2);
        }
        a[k] = s1;
        b[k] = s2;
    }
}

template <typename T, int D, int M>
__device__ __forceinline__ void load_m(const T* __restrict__ base, int64_t q, bool ok, T (&x)[M][D],
                                       int64_t nq = -1) {
    T v[M * D];
    if (ok && TMG_IN(q, nq < 0 ? INT64_MAX : nq, 4)) {
        VecIO<T, M * D>::load(base + q * M * D, v);
    } else {
#pragma unroll
        for (int i = 0; i < M * D; ++i) v[i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) x[i][k] = v[i * D + k];
}

template <typename T, int D, int M>
__device__ __forceinline__ void store_m(T* __restrict__ base, int64_t q, const T (&x)[M][D], int64_t nq = -1) {
    if (!TMG_IN(q, nq < 0 ? INT64_MAX : nq, 5)) return;
    T v[M * D];
#pragma unroll
    for (int i = 0; i < M; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) v[i * D + k] = x[i][k];
    VecIO<T, M * D>::store(base + q * M * D, v);
}

// FP64 residual of one interval, r = F + a (b^T u_{n-1}) - A u_n, using the
// Legendre structure of the stiffness block.  ep = b^T u_{n-1}, E = 1^T u_n.
// DIR = 0: (K u)[k] = E - 2 S_k, S_k = sum of u[l], l < k, l of the other
//   parity than k, so r[k] = F[k] + a_k ep - E + 2 S_k - z/(2k+1) u[k].
// DIR = 1: (K^T u)[k] = E - 2 T_k, T_k = sum of u[l], l > k, l of the other
//   parity, and a'_k = 1: r[k] = F[k] + ep - E + 2 T_k - z/(2k+1) u[k].
// The nearly-cancelling endpoint difference is formed first.
template <int DIR, int D>
__device__ __forceinline__ void residual0(const double (&F)[D], const double (&u)[D], double ep, double E,
                                          const Res0& R, double (&r)[D]) {
    const double dp = ep - E;
    if constexpr (DIR == 0 && D <= 4) {
        r[0] = fma(-R.zm[0], u[0], F[0] + dp);
        if constexpr (D > 1) {
            const double sm = ep + E;
            r[1] = fma(-R.zm[1], u[1], fma(2.0, u[0], F[1] - sm));
            if constexpr (D > 2) r[2] = fma(-R.zm[2], u[2], fma(2.0, u[1], F[2] + dp));
            if constexpr (D > 3) r[3] = fma(-R.zm[3], u[3], fma(2.0, u[0] + u[2], F[3] - sm));
        }
    } else if constexpr (DIR == 0) {
        // S_k = sum of u[l], l < k, l of the other parity, as running sums
        // S_k = S_{k-2} + u[k-1] (one add per coefficient); a_k = (-1)^k
        const double sm = ep + E;
        double s_even = 0.0, s_odd = 0.0;    // S_k for even k / odd k
#pragma unroll
        for (int k = 0; k < D; ++k) {
            double sk;
            if (k & 1) {
                s_odd = k >= 1 ? s_odd + u[k - 1] : s_odd;
                sk = s_odd;
            } else {
                s_even = k >= 2 ? s_even + u[k - 1] : s_even;
                sk = s_even;
            }
            r[k] = fma(-R.zm[k], u[k], fma(2.0, sk, F[k] + ((k & 1) ? -sm : dp)));
        }
    } else {
        // T_k = sum of u[l], l > k, l of the other parity: T_k = T_{k+2} + u[k+1]
        double t[D];
        double t_next[2] = {0.0, 0.0};       // T_{k+2} for the two parities of k
#pragma unroll
        for (int k = D - 1; k >= 0; --k) {
            const double tk = k + 1 < D ? t_next[k & 1] + u[k + 1] : 0.0;
            t[k] = tk;
            t_next[k & 1] = tk;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) r[k] = fma(-R.zm[k], u[k], fma(2.0, t[k], F[k] + dp));
    }
}

// ------------------------------------- level-0 residual without FP64 math --
//
// GB300 issues about two FP64 operations per clock per SM, so the level-0
// residual of the mixed form is evaluated with one FP64 operation per
// interval.  Write e_n = u_n[0] + s_n with s_n = sum_{l>=1} u_n[l].  Then
// e_{n-1} - e_n = d + s_{n-1} - s_n with d = u_{n-1}[0] - u_n[0], and the
// Legendre form of r (see residual0) becomes
//   r[k] = F[k] + a_k (d + s_{n-1}) - s_n + 2 [k>=2] u_n[k-1] - z/(2k+1) u_n[k].
// Only d cancels two O(|u|) numbers; it is one FP64 subtraction (exact when
// the two values are within a factor two).  Every other term is of the size
// of the residual's own parts (tau-scale for smooth solutions), so each double
// is split into a float pair hi + lo with integer operations and the terms are
// summed with compensated FP32 arithmetic (error ~2^-48 of the terms).

struct ff {
    float hi, lo;
};

// x = hi + lo: hi is x truncated to 24 significant bits, lo the remaining 29
// bits truncated to 24.  Integer operations only.  |x| < 2^-126 gives 0;
// |x| >= 2^128 (or Inf/NaN) gives +-Inf so that the norm flags it.
__device__ __forceinline__ ff split_d_general(double x) {
    const unsigned hw = (unsigned)__double2hiint(x);
    const unsigned lw = (unsigned)__double2loint(x);
    const unsigned sign = hw & 0x80000000u;
    const int e = (int)((hw >> 20) & 0x7FFu);
    const unsigned m23 = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
    const unsigned r29 = lw & 0x1FFFFFFFu;
    ff out;
    if (e < 897) {
        out.hi = 0.f;
        out.lo = 0.f;
    } else if (e > 1150) {
        out.hi = __uint_as_float(sign | 0x7F800000u);
        out.lo = 0.f;
    } else {
        out.hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m23);
        const int lz = __clz(r29);                  // 32 when r29 == 0
        const int fe = e - 1075 + 31 - lz + 127;    // biased exponent of lo
        const unsigned mant = ((r29 << (lz & 31)) >> 8) & 0x7FFFFFu;
        out.lo = (r29 != 0u && fe > 0) ? __uint_as_float(sign | ((unsigned)fe << 23) | mant) : 0.f;
    }
    return out;
}

// The same split with lo rounded (instead of truncated) to 24 bits: for
// 2^-74 <= |x| < 2^128 the remaining 29 mantissa bits are converted as an
// integer and scaled by the exact power of two 2^(e - 1075), which the
// conversion unit does in one instruction where the general form needs a
// leading-zero count and a renormalisation.  Other x take split_d_general.
// Either way hi + lo = x to within 2^-47 |x|.
__device__ __forceinline__ ff split_d(double x) {
    const unsigned hw = (unsigned)__double2hiint(x);
    const unsigned lw = (unsigned)__double2loint(x);
    const int e = (int)((hw >> 20) & 0x7FFu);
    if ((unsigned)(e - 949) > 201u) return split_d_general(x);
    const unsigned sign = hw & 0x80000000u;
    const unsigned m23 = __funnelshift_l(lw, hw, 3) & 0x7FFFFFu;      // mantissa bits 51..29
    ff out;
    out.hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | m23);
    const float s = __uint_as_float((unsigned)(e - 948) << 23);         // 2^(e - 1075), a normal float
    out.lo = __uint_as_float(sign | __float_as_uint(__uint2float_rn(lw & 0x1FFFFFFFu) * s));
    return out;
}

// Compensated accumulation: (s, c) += th + tl, with the rounding error of the
// leading sum kept in c (Knuth's two-sum).
__device__ __forceinline__ void acc_add(float& s, float& c, float th, float tl) {
    const float t = s + th;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (th - bp);
    s = t;
    c += err + tl;
}

// a + b = hi + lo exactly (Knuth's two-sum).
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bp = s - a;
    return ff{s, (a - (s - bp)) + (b - bp)};
}

// Storage of the low part of a float pair (hi, lo) with |lo| <= ulp(hi)/2
// (hi the rounded sum, as two_sum leaves it): a 16-bit fixed-point multiple
// of 2^-15 ulp(hi), so the code lies in [-2^14, 2^14] and resolves 2^-16
// ulp(hi) -- hi + lo keeps about 39 significant bits in 6 bytes instead of
// 8.  Values with |hi| < 2^-88 keep no low part.
__device__ __forceinline__ short lo_encode(float hi, float lo) {
    const int E = (int)((__float_as_uint(hi) >> 23) & 0xFFu);
    if (E < 39) return 0;
    const float s = __uint_as_float((unsigned)(292 - E) << 23);   // 2^(165 - E)
    return (short)__float2int_rn(lo * s);
}

__device__ __forceinline__ float lo_decode(float hi, short q) {
    const int E = (int)((__float_as_uint(hi) >> 23) & 0xFFu);
    if (E < 39) return 0.f;
    const float s = __uint_as_float((unsigned)(E - 38) << 23);    // 2^(E - 165)
    return (float)q * s;
}

// (s, c) += t for a single float term.
__device__ __forceinline__ void acc_add1(float& s, float& c, float t) {
    const ff n = two_sum(s, t);
    s = n.hi;
    c += n.lo;
}

// float -> double by re-biasing the exponent with integer operations (the
// conversion instruction would occupy GB300's FP64 pipe).  Exact for zero
// and normal floats; a subnormal c (|c| < 2^-126) comes out within 2^-126 of
// its value, and Inf/NaN come out NaN (still caught by every norm test).
__device__ __forceinline__ double f2d_int(float c) {
    const unsigned b = __float_as_uint(c);
    const unsigned a = b & 0x7FFFFFFFu;
    unsigned hi = a >= 0x7F800000u ? 0x7FF80000u : (a >> 3) + 0x38000000u;
    hi = a == 0u ? 0u : (hi | (b & 0x80000000u));
    return __hiloint2double((int)hi, (int)(b << 29));
}

// Sum over the warp of the squares of every lane's n floats, as a double,
// with no FP64 operation per value (GB300's FP64 pipe is narrow).  All values
// are scaled by one power of two common to the warp, taken from the largest
// exponent among the lanes so that no square can overflow; the squares are
// summed in FP32 (relative error about 2^-17 for 32 n terms, far finer than a
// stopping test needs) and the total is widened and rescaled once.  Squares
// more than 2^-126 below the largest are flushed (a relative change of at
// most 32 n 2^-126).  An Inf or NaN value makes the total Inf or NaN.  All
// 32 lanes must call it; each receives the warp total.
template <int n>
__device__ __forceinline__ double warp_sumsq(const float (&v)[n]) {
    unsigned em = 0u;
#pragma unroll
    for (int i = 0; i < n; ++i) em = max(em, (__float_as_uint(v[i]) >> 23) & 0xFFu);
    em = __reduce_max_sync(kFull, em);
    int k = (int)em - 127;                           // every |v| < 2^(k+1)
    k = k < -126 ? -126 : (k > 126 ? 126 : k);
    const float s = __uint_as_float((unsigned)(127 - k) << 23);   // 2^-k, exact scaling
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const float x = v[i] * s;
        ss = fmaf(x, x, ss);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(kFull, ss, off);
    return f2d_int(ss) * __hiloint2double((2 * k + 1023) << 20, 0);   // times 2^(2k)
}

// Product of two float pairs (lo*lo dropped), as an unnormalised pair.
__device__ __forceinline__ ff mul_ff(float ah, float al, ff b) {
    ff p;
    p.hi = ah * b.hi;
    float e = fmaf(ah, b.hi, -p.hi);
    e = fmaf(ah, b.lo, e);
    p.lo = fmaf(al, b.hi, e);
    return p;
}

// Float-pair splits of one interval and the small parts of its two
// functionals: sE = sum_{l>=1} u[l] (of 1^T u) and sB = sum_{l>=1} b_l u[l]
// (of the halo functional b^T u; equal to sE for DIR = 0).
template <int DIR, int D>
__device__ __forceinline__ void small_sums(const double (&u)[D], ff (&us)[D], ff& sE, ff& sB) {
    sE = ff{0.f, 0.f};
    sB = ff{0.f, 0.f};
#pragma unroll
    for (int l = 0; l < D; ++l) us[l] = split_d(u[l]);
#pragma unroll
    for (int l = 1; l < D; ++l) {
        acc_add(sE.hi, sE.lo, us[l].hi, us[l].lo);
        if constexpr (DIR == 1) {
            const float sg = (l & 1) ? -1.f : 1.f;
            acc_add(sB.hi, sB.lo, sg * us[l].hi, sg * us[l].lo);
        }
    }
    if constexpr (DIR == 0) sB = sE;
}

// r[k] of one interval, rounded to float.  up0 = u_{n-1}[0], spB = the small
// part of b^T u_{n-1}, snE = the small part of 1^T u_n.  With d = up0 - u_n[0]:
// DIR = 0: r[k] = F[k] + a_k (d + spB) - snE + 2 S'_k - z/(2k+1) u[k], S'_k = u[k-1] + u[k-3] + ... (l >= 1)
// DIR = 1: r[k] = F[k] + (d + spB) - snE + 2 T_k - z/(2k+1) u[k]  (T_k as in residual0)
template <int DIR, int D>
__device__ __forceinline__ void residual0_ff(const double (&F)[D], const double (&u)[D], const ff (&us)[D],
                                             double up0, ff spB, ff snE, const Res0& R, float (&r)[D],
                                             float (&rlo)[D]) {
    const ff d = split_d(up0 - u[0]);
    // 2 S_k (DIR = 0: u[l], l < k of the other parity, without the u[0] term
    // of odd k, which a_k d already holds) or 2 T_k (DIR = 1: l > k of the
    // other parity).  Up to D = 6 each term enters the residual's compensated
    // sum directly; wider blocks keep compensated running sums per parity,
    // S_k = S_{k-2} + 2 u[k-1] (T_k = T_{k+2} + 2 u[k+1]): one pair add per
    // coefficient instead of O(D^2 / 4).
    ff run[D];
    if constexpr (D > 6) {
        ff par[2] = {ff{0.f, 0.f}, ff{0.f, 0.f}};
        if constexpr (DIR == 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if (k >= 2) acc_add(par[k & 1].hi, par[k & 1].lo, 2.f * us[k - 1].hi, 2.f * us[k - 1].lo);
                run[k] = par[k & 1];
            }
        } else {
#pragma unroll
            for (int k = D - 1; k >= 0; --k) {
                if (k + 1 < D) acc_add(par[k & 1].hi, par[k & 1].lo, 2.f * us[k + 1].hi, 2.f * us[k + 1].lo);
                run[k] = par[k & 1];
            }
        }
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const ff Fk = split_d(F[k]);
        float s = Fk.hi, c = Fk.lo;
        const float sg = (DIR == 0 && (k & 1)) ? -1.f : 1.f;
        acc_add(s, c, sg * d.hi, sg * d.lo);
        acc_add(s, c, sg * spB.hi, sg * spB.lo);
        acc_add(s, c, -snE.hi, -snE.lo);
        if constexpr (D > 6) {
            acc_add(s, c, run[k].hi, run[k].lo);
        } else if constexpr (DIR == 0) {
#pragma unroll
            for (int l = k - 1; l >= 1; l -= 2) acc_add(s, c, 2.f * us[l].hi, 2.f * us[l].lo);
        } else {
#pragma unroll
            for (int l = k + 1; l < D; l += 2) acc_add(s, c, 2.f * us[l].hi, 2.f * us[l].lo);
        }
        const ff zu = mul_ff(R.zm_hi[k], R.zm_lo[k], us[k]);
        acc_add(s, c, -zu.hi, -zu.lo);
        const ff n = two_sum(s, c);
        r[k] = n.hi;
        rlo[k] = n.lo;
    }
}

// Same, rounded to one float per value.
template <int DIR, int D>
__device__ __forceinline__ void residual0_ff(const double (&F)[D], const double (&u)[D], const ff (&us)[D],
                                             double up0, ff spB, ff snE, const Res0& R, float (&r)[D]) {
    float lo[D];
    residual0_ff<DIR, D>(F, u, us, up0, spB, snE, R, r, lo);
}

// Residual of the correction equation L c = r at a float correction c, as a
// float pair: (rh, rl) <- r + a ep - A c, where ep = b^T c_{n-1} (a float
// pair) and A c uses the Legendre structure of the stiffness block (see
// residual0).  Each float term (sums of c, 2 c[l], the pair product
// z/(2k+1) c[k]) enters a compensated sum, so the result carries ~2^-48 of
// the terms' size -- the residual of an FP64 iterate is updated without an
// FP64 operation.
template <int DIR, int D>
__device__ __forceinline__ void residual_update_ff(float (&rh)[D], float (&rl)[D], const float (&c)[D], ff ep,
                                                   const Res0& R) {
    ff E{c[0], 0.f};                       // 1^T c
#pragma unroll
    for (int l = 1; l < D; ++l) {
        const ff t = two_sum(E.hi, c[l]);
        E.hi = t.hi;
        E.lo += t.lo;
    }
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float s = rh[k], e = rl[k];
        const float sg = (DIR == 0 && (k & 1)) ? -1.f : 1.f;
        acc_add(s, e, sg * ep.hi, sg * ep.lo);
        acc_add(s, e, -E.hi, -E.lo);
        if constexpr (DIR == 0) {
#pragma unroll
            for (int l = k - 1; l >= 0; l -= 2) acc_add1(s, e, 2.f * c[l]);
        } else {
#pragma unroll
            for (int l = k + 1; l < D; l += 2) acc_add1(s, e, 2.f * c[l]);
        }
        const ff zu = mul_ff(R.zm_hi[k], R.zm_lo[k], ff{c[k], 0.f});
        acc_add(s, e, -zu.hi, -zu.lo);
        const ff n = two_sum(s, e);
        rh[k] = n.hi;
        rl[k] = n.lo;
    }
}

// b^T c of a float vector as a float pair.
template <int DIR, int D>
__device__ __forceinline__ ff bsum_ff(const float (&c)[D]) {
    ff b{c[0], 0.f};
#pragma unroll
    for (int l = 1; l < D; ++l) {
        const ff t = two_sum(b.hi, (DIR == 1 && (l & 1)) ? -c[l] : c[l]);
        b.hi = t.hi;
        b.lo += t.lo;
    }
    return b;
}

// ------------------------------------------------- norm and stopping test --

// First kernel of a cycle: a finished solve must also end the graph loop.
__device__ __forceinline__ bool cycle_finished(const DevState* st) {
    if (!st->done) return false;
    if (st->use_cond && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, 0u);
    return true;
}

// How a residual norm enters the solve state.
//   kFinPlain: the residual of the current iterate, from u (one per cycle).
//   kFinFull: the same where level 0 keeps an updated residual: at the start
//     of a solve a new entry; later a confirmation of the updated residual of
//     the same iterate (it replaces that entry; the solve stops only here).
//   kFinUpdated: the updated residual of the new iterate; meeting tol asks
//     for a confirmation from u instead of stopping.
enum : int { kFinPlain = 0, kFinFull = 1, kFinUpdated = 2 };

__device__ __forceinline__ void finalize_state(DevState* st, double ss, int mode) {
    const bool confirm = mode == kFinFull && st->cycle > 0;
    const int k = confirm ? st->cycle - 1 : st->cycle;
    const double nrm = sqrt(ss);
    if (k == 0 && !confirm && st->nF_from_first) st->nF = nrm;
    const double rel = st->nF > 0.0 ? nrm / st->nF : nrm;
    st->hist[k < kHist ? k : kHist - 1] = rel;
    // scale for the next FP32 norm: 2^-round(log2(rms)), kept well inside FP32 range
    const double rms = st->nvals > 0 ? nrm / sqrt((double)st->nvals) : 0.0;
    int ex = 0;
    if (rms > 0.0 && rms < 1.0e300) ex = -ilogb(rms);
    ex = ex < -100 ? -100 : (ex > 100 ? 100 : ex);
    st->nscale = ldexpf(1.0f, ex);
    int done = 0;
    if (!(rel == rel) || rel > 1.0e300) done = 3;
    else if (rel <= st->tol) done = mode == kFinUpdated ? 0 : 1;
    else if (k >= st->max_cycles) done = 2;
    if (mode == kFinFull) {
        // a failed norm-only confirmation asks for the residual itself next time
        st->full = (confirm && done == 0 && st->full == 1) ? 2 : 0;
    }
    if (mode == kFinUpdated) {
        st->rsel ^= 1;      // the kernel wrote the other buffer
        if (done == 0 && rel <= st->tol && st->full == 0) st->full = 1;
    }
    if (!confirm) st->cycle = k + 1;
    st->done = done;
    if (done && st->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, 0u);
}

// Deterministic grid sum of ss: block partials in a fixed order, reduced by
// the last block to finish (ticket), which then applies the stopping test.
template <int NT>
__device__ __forceinline__ void grid_norm_finalize(double ss, double* __restrict__ partials, DevState* st,
                                                   int mode = kFinPlain) {
    __shared__ double red[NT / 32];
    __shared__ int last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(kFull, ss, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < NT / 32; ++i) s += red[i];
        partials[blockIdx.x] = s;
        __threadfence();
        const unsigned t = atomicAdd(&st->ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += NT) s += __ldcg(&partials[i]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(kFull, s, off);
    __syncthreads();
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int i = 0; i < NT / 32; ++i) tot += red[i];
        st->ticket = 0u;
        finalize_state(st, tot, mode);
    }
}

// ------------------------------------------------------ streaming kernels --

constexpr int kNT = 256;   // threads per block of the streaming kernels

// Exact solve of a coarsest level of at most 64 intervals by one warp: two
// intervals per lane, the affine maps e_n = alpha e_{n-1} + c^T f_n (e_{-1} =
// 0) combined by a warp scan, then u_n = A^{-1} f_n + g e_{n-1}.  f is read
// through L2 (it was written by other blocks of the same launch).
template <typename T, int D>
__device__ __forceinline__ void warp_coarse_solve(const LevelK<T, D>& K, const T* f, T* u, int Nc) {
    const int lane = threadIdx.x & 31;
    const int n0 = 2 * lane, n1 = 2 * lane + 1;
    T f0[D], f1[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        f0[k] = n0 < Nc ? __ldcg(f + n0 * D + k) : T(0);
        f1[k] = n1 < Nc ? __ldcg(f + n1 * D + k) : T(0);
    }
    const T b0 = dotc<T, D>(K.c, f0), b1 = dotc<T, D>(K.c, f1);
    T A = n1 < Nc ? K.alpha * K.alpha : (n0 < Nc ? K.alpha : T(1));
    T B = n1 < Nc ? fma(K.alpha, b0, b1) : (n0 < Nc ? b0 : T(0));
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T Ap = __shfl_up_sync(kFull, A, off);
        const T Bp = __shfl_up_sync(kFull, B, off);
        if (lane >= off) {
            B = fma(A, Bp, B);
            A = A * Ap;
        }
    }
    T ein = __shfl_up_sync(kFull, B, 1);   // e_{2 lane - 1}: inclusive prefix of the lane before
    if (lane == 0) ein = T(0);
    T x0[D], x1[D];
    matvec<T, D>(K.Ainv, f0, x0);
    matvec<T, D>(K.Ainv, f1, x1);
    const T emid = fma(K.alpha, ein, b0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        if (n0 < Nc) u[n0 * D + k] = fma(K.g[k], ein, x0[k]);
        if (n1 < Nc) u[n1 * D + k] = fma(K.g[k], emid, x1[k]);
    }
}

// The coarsest level solved by the last block of the last down kernel of a
// cycle (u == nullptr: not this kernel's job).  Each block, after its tiles,
// fences its writes and takes a ticket; the block that takes the last ticket
// reads the whole coarsest right-hand side and solves it with one warp.  No
// block waits for another.
template <typename T, int D>
struct CoarseTail {
    const LevelK<T, D>* K;    // constants of the coarsest level (device)
    const T* f;               // its right-hand side, written by this kernel
    T* u;                     // its solution
    int Nc;                   // intervals, at most 64
    unsigned* ticket;         // zero between launches
};

template <typename T, int D>
__device__ __forceinline__ void coarse_tail_last_block(const CoarseTail<T, D>& ct) {
    if (ct.u == nullptr) return;
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ct.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        const LevelK<T, D> K = *ct.K;
        warp_coarse_solve<T, D>(K, ct.f, ct.u, ct.Nc);
    }
    if (threadIdx.x == 0) *ct.ticket = 0u;
}

// Level l >= 1, zero guess: pre-smooth, residual, restrict.  f: [2*nchunks][D],
// fc: [nchunks][D].
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT) k_down(const T* __restrict__ f, T* __restrict__ fc, int64_t nchunks,
                                              LevelK<T, D> K, Xfer<T, D> X, int nu1, int H,
                                              const DevState* __restrict__ st, CoarseTail<T, D> ct) {
    pdl_enter();
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        T fv[2][D], h[2][D], u[2][D], w[2][D], r[2][D], out[D];
        load_pair<T, D>(f, q, inb, fv);
        presmooth_zero<DIR, T, D>(K, fv, h, u, w, nu1);
        residual_tracked<DIR, T, D>(fv, u, w, r);
        restrict_pair<T, D>(X, r, out);
        if (inb && lane >= H) VecIO<T, D>::store(fc + q * D, out);
    }
    coarse_tail_last_block<T, D>(ct);
}

// Level l >= 1, zero guess: recompute the pre-smoothed iterate, add the
// prolongated coarse correction uc: [nchunks][D], post-smooth, write u.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT) k_up(const T* __restrict__ f, const T* __restrict__ uc, T* __restrict__ u,
                                            int64_t nchunks, LevelK<T, D> K, Xfer<T, D> X, int nu1, int nu2,
                                            int H, const DevState* __restrict__ st) {
    pdl_enter();
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        T fv[2][D], h[2][D], v[2][D], w[2][D], c[D];
        load_pair<T, D>(f, q, inb, fv);
        load_one<T, D>(uc, q, inb, c);
        presmooth_zero<DIR, T, D>(K, fv, h, v, w, nu1);
        prolong_add<T, D>(X, c, v);
        postsmooth<DIR, T, D>(K, h, v, nu2);
        if (inb && lane >= H) store_pair<T, D>(u, q, v);
    }
}

// The second visit of level l >= 1 in a W-cycle (nonzero start u_in, the
// result of the first visit): pre-smooth from u_in, residual, restrict.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT) k_down_nz(const T* __restrict__ f, const T* __restrict__ u_in,
                                                 T* __restrict__ fc, int64_t nchunks, LevelK<T, D> K, Xfer<T, D> X,
                                                 int nu1, int H, const DevState* __restrict__ st) {
    pdl_enter();
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        T fv[2][D], h[2][D], u[2][D], w[2][D], r[2][D], out[D];
        load_pair<T, D>(f, q, inb, fv);
        load_pair<T, D>(u_in, q, inb, u);
        presmooth_from<DIR, T, D>(K, fv, h, u, w, nu1);
        residual_tracked<DIR, T, D>(fv, u, w, r);
        restrict_pair<T, D>(X, r, out);
        if (inb && lane >= H) VecIO<T, D>::store(fc + q * D, out);
    }
}

// The way up of that second visit: recompute the pre-smoothing from u_in, add
// the prolongated coarse correction uc, post-smooth, write u_out (another
// buffer than u_in: neighbouring tiles still read u_in).
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT) k_up_nz(const T* __restrict__ f, const T* __restrict__ u_in,
                                               const T* __restrict__ uc, T* __restrict__ u_out, int64_t nchunks,
                                               LevelK<T, D> K, Xfer<T, D> X, int nu1, int nu2, int H,
                                               const DevState* __restrict__ st) {
    pdl_enter();
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        T fv[2][D], h[2][D], v[2][D], w[2][D], c[D];
        load_pair<T, D>(f, q, inb, fv);
        load_pair<T, D>(u_in, q, inb, v);
        load_one<T, D>(uc, q, inb, c);
        presmooth_from<DIR, T, D>(K, fv, h, v, w, nu1);
        prolong_add<T, D>(X, c, v);
        postsmooth<DIR, T, D>(K, h, v, nu2);
        if (inb && lane >= H) store_pair<T, D>(u_out, q, v);
    }
}

// Levels l and l+1 at once, zero guess on both (the way down): each lane
// takes four consecutive intervals of level l (two coarse pairs), which
// restrict to one pair of level l+1 and then to one interval of level l+2.
// f_l: [4*nquads][D], f_{l+2}: [nquads][D]; f_{l+1} is never stored (the
// way up recomputes it from f_l).  K0, K1: constants of levels l and l+1.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT) k_down2(const T* __restrict__ f, T* __restrict__ fcc, int64_t nquads,
                                               LevelK<T, D> K0, LevelK<T, D> K1, Xfer<T, D> X, int nu1, int H,
                                               const DevState* __restrict__ st, CoarseTail<T, D> ct) {
    pdl_enter();
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nquads + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nquads;
        T fv[4][D], h[4][D], u[4][D], w[4][D], r[4][D];
        load_m<T, D, 4>(f, q, inb, fv);
        presmooth_zero_m<DIR, T, D, 4>(K0, fv, h, u, w, nu1);
        residual_tracked_m<DIR, T, D, 4>(fv, u, w, r);
        T f1[2][D], h1[2][D], u1[2][D], w1[2][D], r1[2][D], out[D];
        restrict2<T, D>(X, r[0], r[1], f1[0]);
        restrict2<T, D>(X, r[2], r[3], f1[1]);
        presmooth_zero<DIR, T, D>(K1, f1, h1, u1, w1, nu1);
        residual_tracked<DIR, T, D>(f1, u1, w1, r1);
        restrict_pair<T, D>(X, r1, out);
        if (inb && lane >= H) VecIO<T, D>::store(fcc + q * D, out);
    }
    coarse_tail_last_block<T, D>(ct);
}

// Levels l+1 and l at once on the way up: recompute level l's pre-smoothed
// iterate and residual and level l+1's right-hand side and pre-smoothed
// iterate from f_l, add the prolongated level-(l+2) correction ucc, post-smooth
// on level l+1, prolongate onto level l, post-smooth there and write u_l.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT) k_up2(const T* __restrict__ f, const T* __restrict__ ucc, T* __restrict__ u,
                                             int64_t nquads, LevelK<T, D> K0, LevelK<T, D> K1, Xfer<T, D> X, int nu1,
                                             int nu2, int H, const DevState* __restrict__ st) {
    pdl_enter();
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nquads + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nquads;
        T fv[4][D], h[4][D], v[4][D], w[4][D], r[4][D], cc[D];
        load_m<T, D, 4>(f, q, inb, fv);
        load_one<T, D>(ucc, q, inb, cc);
        presmooth_zero_m<DIR, T, D, 4>(K0, fv, h, v, w, nu1);
        residual_tracked_m<DIR, T, D, 4>(fv, v, w, r);
        T f1[2][D], h1[2][D], v1[2][D], w1[2][D];
        restrict2<T, D>(X, r[0], r[1], f1[0]);
        restrict2<T, D>(X, r[2], r[3], f1[1]);
        presmooth_zero<DIR, T, D>(K1, f1, h1, v1, w1, nu1);
        prolong_add<T, D>(X, cc, v1);
        postsmooth<DIR, T, D>(K1, h1, v1, nu2);
        prolong_add2<T, D>(X, v1[0], v[0], v[1]);
        prolong_add2<T, D>(X, v1[1], v[2], v[3]);
        postsmooth_m<DIR, T, D, 4>(K0, h, v, nu2);
        if (inb && lane >= H) store_m<T, D, 4>(u, q, v);
    }
}

// Level 0: r = F - L u in FP64 (u0 is the halo before the first interval),
// ||r||^2 for the stopping test, r stored in the cycle precision T; then,
// when fc != nullptr, the zero-guess pre-smoothing, residual and restriction
// of the correction equation L c = r onto level 1.
// k_down0 stages its u and F pairs through shared memory (cp.async, two
// stages) up to D = 6.  Wider blocks load them straight from global memory:
// at D = 11 the stages take 180 KB per block, one block of 8 warps per SM,
// too few to hide the latency; at D = 21 they would take 344 KB.
template <int D>
__host__ __device__ constexpr bool k_down0_staged() {
    return D <= kMaxD;
}

// Dynamic shared memory of k_down0: 2 stages x (u, F) x 32 lanes x 2*D doubles per warp.
template <int D>
__host__ __device__ constexpr size_t k_down0_smem_bytes() {
    return k_down0_staged<D>() ? (size_t)(kNT / 32) * 2 * 2 * 32 * (2 * D * 8) : 0;
}

// The main loop of k_down0; FP64NORM selects the norm arithmetic at compile
// time (FP64 squares in the first cycle, scaled FP32 squares afterwards) so
// that no branch between the two sits inside the loop.
template <bool FP64NORM, int DIR, typename T, int D, bool NORM_ONLY = false>
__device__ __forceinline__ double down0_loop(T* __restrict__ rT, short* __restrict__ rlo, T* __restrict__ fc,
                                             int64_t nchunks,
                                             const Res0& R, const LevelK<T, D>& K, const Xfer<T, D>& X, int nu1,
                                             int H, const DevState* st) {
    const double* __restrict__ F = st->F;
    const double* __restrict__ uu = st->u;
    const double u0 = st->u0;
    constexpr bool kMixed = std::is_same<T, float>::value;
    constexpr int kPairBytes = 2 * D * 8;
    using Stage = LaneStage<kPairBytes>;
    // two stages x (u, F) per warp, in dynamic shared memory (k_down0_smem_bytes)
    extern __shared__ __align__(16) unsigned char k_down0_stage[];
    auto stage = reinterpret_cast<uint4 (*)[2][2][Stage::C * 32]>(k_down0_stage);
    const float nsc = st->nscale;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    double ss = 0.0;
    float ssf = 0.f;
    int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5;
    int sb = 0;
    if constexpr (k_down0_staged<D>()) {
        if (tw < ntiles) {
            const int64_t q = tw * per + lane - H;
            const bool inb = q >= 0 && q < nchunks;
            Stage::issue(stage[wib][0][0], uu, q * 2 * D, inb, lane);
            Stage::issue(stage[wib][0][1], F, q * 2 * D, inb, lane);
        }
        cp_async_commit();
    }
    for (; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        const bool own = inb && lane >= H;
        double uv[2][D], Fv[2][D];
        if constexpr (k_down0_staged<D>()) {
            {   // prefetch the warp's next tile
                const int64_t qn = (tw + nwarps) * per + lane - H;
                const bool nb = tw + nwarps < ntiles && qn >= 0 && qn < nchunks;
                Stage::issue(stage[wib][sb ^ 1][0], uu, qn * 2 * D, nb, lane);
                Stage::issue(stage[wib][sb ^ 1][1], F, qn * 2 * D, nb, lane);
                cp_async_commit();
            }
            cp_async_wait_prev();
            double uvf[2 * D], Fvf[2 * D];
            Stage::template read<double, 2 * D>(stage[wib][sb][0], lane, uvf);
            Stage::template read<double, 2 * D>(stage[wib][sb][1], lane, Fvf);
            sb ^= 1;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                uv[0][k] = uvf[k];
                uv[1][k] = uvf[D + k];
                Fv[0][k] = Fvf[k];
                Fv[1][k] = Fvf[D + k];
            }
        } else {
            load_pair<double, D>(uu, q, inb, uv);
            load_pair<double, D>(F, q, inb, Fv);
        }
        T rt[2][D];
        short rtl[2][D];     // low parts of the float-pair residual (mixed form), encoded
        if constexpr (kMixed) {
            ff us0[D], us1[D], sE0, sB0, sE1, sB1;
            small_sums<DIR, D>(uv[0], us0, sE0, sB0);
            small_sums<DIR, D>(uv[1], us1, sE1, sB1);
            double h0 = uv[1][0];
            ff hB = sB1;
            if (q < 0) {                        // the value before the first interval: b^T u = u0
                h0 = u0;
                hB = ff{0.f, 0.f};
            }
            const double up0 = shfl_prev(h0);
            const ff sp{shfl_prev(hB.hi), shfl_prev(hB.lo)};
            float r0[D], r1[D], l0[D], l1[D];
            residual0_ff<DIR, D>(Fv[0], uv[0], us0, up0, sp, sE0, R, r0, l0);
            residual0_ff<DIR, D>(Fv[1], uv[1], us1, uv[0][0], sB0, sE1, R, r1, l1);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                rt[0][k] = inb ? r0[k] : 0.f;
                rt[1][k] = inb ? r1[k] : 0.f;
                rtl[0][k] = lo_encode(r0[k], l0[k]);
                rtl[1][k] = lo_encode(r1[k], l1[k]);
            }
        } else {
            double r[2][D];
            const double b0 = bval<DIR, double, D>(uv[0]);
            double b1 = bval<DIR, double, D>(uv[1]);
            if (q < 0) b1 = u0;                   // the value before the first interval
            const double ep = shfl_prev(b1);
            const double E0 = DIR == 0 ? b0 : endval<double, D>(uv[0]);
            const double E1 = DIR == 0 ? b1 : endval<double, D>(uv[1]);
            residual0<DIR, D>(Fv[0], uv[0], ep, E0, R, r[0]);
            residual0<DIR, D>(Fv[1], uv[1], b0, E1, R, r[1]);
            // Lanes outside the array carry u0 only as the halo of the FP64
            // residual; for the correction equation L c = r their r is zero.
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) rt[i][k] = inb ? (T)r[i][k] : T(0);
        }
        if constexpr (FP64NORM && kMixed) {
            float sq[2 * D];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) sq[i * D + k] = own ? (float)rt[i][k] : 0.f;
            const double t = warp_sumsq<2 * D>(sq);
            if (lane == 0) ss += t;
        }
        if (own) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    if constexpr (FP64NORM) {
                        if constexpr (!kMixed) ss = fma((double)rt[i][k], (double)rt[i][k], ss);
                    } else {
                        const float v = (float)rt[i][k] * nsc;
                        ssf = fmaf(v, v, ssf);
                    }
                }
            if constexpr (!NORM_ONLY) {
                store_pair<T, D>(rT, q, rt);
                if constexpr (kMixed) {
                    if (rlo != nullptr) store_pair<short, D>(rlo, q, rtl);
                }
            }
        }
        if (!NORM_ONLY && fc != nullptr) {
            T h[2][D], c[2][D], w[2][D], rc[2][D], out[D];
            presmooth_zero<DIR, T, D>(K, rt, h, c, w, nu1);
            residual_tracked<DIR, T, D>(rt, c, w, rc);
            restrict_pair<T, D>(X, rc, out);
            if (own) VecIO<T, D>::store(fc + q * D, out);
        }
    }
    if constexpr (k_down0_staged<D>()) cp_async_wait_all();
    if constexpr (!FP64NORM) ss = (double)ssf / ((double)nsc * (double)nsc);
    return ss;
}

//
// With rlo != nullptr (mixed form with an updated residual) the residual is
// stored as a float pair (rT, rlo; low parts encoded by lo_encode) into buffer
// st->rsel of two (each nchunks * 2 * D values) and the kernel runs only when
// st->full is set: to evaluate the residual (the start of a solve, or after a
// failed confirmation), or only its norm (to confirm an updated residual that
// met the tolerance); in every other cycle k_updown0 has done its work.
// Mixed form, first residual of a solve that starts from u = 0: r = F (with
// a u0 in the first interval) needs no product with u, so F is split into
// float pairs directly; then the pre-smoothing and restriction of L c = r.
template <int DIR, int D>
__device__ __forceinline__ double start0_loop(float* __restrict__ rT, short* __restrict__ rlo,
                                              float* __restrict__ fc, int64_t nchunks, const LevelK<float, D>& K,
                                              const Xfer<float, D>& X, int nu1, int H, const DevState* st) {
    const double* __restrict__ F = st->F;
    const double u0 = st->u0;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    double ss = 0.0;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        const bool own = inb && lane >= H;
        double Fv[2][D];
        load_pair<double, D>(F, q, inb, Fv);
        if (q == 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) Fv[0][k] += acoef<DIR>(k, u0);
        }
        float rt[2][D];
        short rq[2][D];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const ff sp = split_d(Fv[i][k]);
                const ff n = two_sum(sp.hi, sp.lo);      // rounded high part, |lo| <= ulp/2
                rt[i][k] = n.hi;
                rq[i][k] = lo_encode(n.hi, n.lo);
            }
        {
            float sq[2 * D];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) sq[i * D + k] = own ? rt[i][k] : 0.f;
            const double t = warp_sumsq<2 * D>(sq);
            if (lane == 0) ss += t;
        }
        if (own) {
            store_pair<float, D>(rT, q, rt);
            store_pair<short, D>(rlo, q, rq);
        }
        float h[2][D], c[2][D], w[2][D], rc[2][D], out[D];
        presmooth_zero<DIR, float, D>(K, rt, h, c, w, nu1);
        residual_tracked<DIR, float, D>(rt, c, w, rc);
        restrict_pair<float, D>(X, rc, out);
        if (own) VecIO<float, D>::store(fc + q * D, out);
    }
    return ss;
}

// At D = 11 two blocks per SM (128 registers, a few hundred bytes of spill
// per thread) beat one block at 160 registers: p_t = 10 mixed solve 46.9 ms
// against 52.6 ms; three blocks (80 registers) spill 2.7 KB and take 54.8 ms,
// and two blocks at D = 21 take 62.9 ms against 56.0 ms.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT, (D > 6 && D <= 11) ? 2 : 1) k_down0(T* __restrict__ rT, short* __restrict__ rlo, T* __restrict__ fc,
                                               int64_t nchunks, Res0 R, LevelK<T, D> K, Xfer<T, D> X, int nu1,
                                               int H, double* __restrict__ partials, DevState* st) {
    pdl_enter();
    if (cycle_finished(st)) return;
    if (rlo != nullptr) {
        if (!st->full) return;
        const int64_t nv = nchunks * 2 * D;
        rT += st->rsel * nv;
        rlo += st->rsel * nv;
    }
    constexpr bool kMixed = std::is_same<T, float>::value;
    // FP32 norm with a power-of-two scale, except in the first cycle whose
    // residual magnitude is not known yet (FP64 then)
    double ss;
    if constexpr (kMixed) {
        if (rlo != nullptr && st->cycle == 0 && st->u_zero) {
            ss = start0_loop<DIR, D>(rT, rlo, fc, nchunks, K, X, nu1, H, st);
            grid_norm_finalize<kNT>(ss, partials, st, kFinFull);
            return;
        }
    }
    if (!kMixed || st->cycle == 0) ss = down0_loop<true, DIR, T, D>(rT, rlo, fc, nchunks, R, K, X, nu1, H, st);
    else if (rlo != nullptr && st->full == 1)   // confirmation: the norm only
        ss = down0_loop<false, DIR, T, D, true>(rT, rlo, fc, nchunks, R, K, X, nu1, H, st);
    else ss = down0_loop<false, DIR, T, D>(rT, rlo, fc, nchunks, R, K, X, nu1, H, st);
    grid_norm_finalize<kNT>(ss, partials, st, rlo != nullptr ? kFinFull : kFinPlain);
}

// Level 0 on the way up: recompute the pre-smoothed correction from r, add
// the prolongated level-1 correction, post-smooth, and update u += c in FP64.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT, (D > 6 && D <= 11) ? 2 : 1) k_up0(const T* __restrict__ rT, const T* __restrict__ uc, int64_t nchunks,
                                             LevelK<T, D> K, Xfer<T, D> X, int nu1, int nu2, int H,
                                             const DevState* __restrict__ st) {
    pdl_enter();
    if (st->done) return;
    double* __restrict__ uu = st->u;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        const bool own = inb && lane >= H;
        T rt[2][D], h[2][D], c[2][D], w[2][D], cc[D];
        double uv[2][D];
        load_pair<T, D>(rT, q, inb, rt);
        load_one<T, D>(uc, q, inb, cc);
        load_pair<double, D>(uu, q, own, uv);      // issued early: its latency overlaps the sweeps
        presmooth_zero<DIR, T, D>(K, rt, h, c, w, nu1);
        prolong_add<T, D>(X, cc, c);
        postsmooth<DIR, T, D>(K, h, c, nu2);
        if (own) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    if constexpr (std::is_same<T, float>::value) uv[i][k] += f2d_int(c[i][k]);
                    else uv[i][k] += (double)c[i][k];
                }
            store_pair<double, D>(uu, q, uv);
        }
    }
}

// Level 0 of the mixed form between two cycles: the way up of one cycle
// fused with the way down of the next, with the level-0 residual updated
// instead of recomputed from u.  The residual is kept as a float pair
// (rh, rl), about 39 significant bits in storage (lo_encode).  Per coarse pair: recompute the
// pre-smoothed correction from rh, add the prolongated level-1 correction,
// post-smooth (this cycle's correction c); u += c in FP64; (rh, rl) <- r - L c
// (residual_update_ff), whose norm feeds the stopping test; then the
// zero-start pre-smoothing, residual and restriction of the next cycle's
// correction equation L c' = rh write the level-1 right-hand side.
//
// Sweeps that read the previous interval: those of k_up0, one for L c, and
// those of k_down's part, so H = ceil(S/2) with S = sweeps_up + 1 + sweeps_down.
// The updated residual differs from F - L u by the FP64 rounding of u += c
// and ~2^-48 of each update's terms; before the solve stops on it, k_down0
// recomputes it from u in FP64 (st->full).
//
// The residual is read from buffer st->rsel and written to the other one:
// the halo lanes of a tile read pairs that another warp owns and updates, so
// an in-place update would race.  rh (floats) and rl (16-bit encoded low
// parts, lo_encode) each hold two buffers of nchunks * 2 * D values.
template <int DIR, int D>
__global__ void __launch_bounds__(kNT, D <= 2 ? 4 : 2) k_updown0(float* __restrict__ rh, short* __restrict__ rl,
                                                 const float* __restrict__ uc, float* __restrict__ fc,
                                                 int64_t nchunks, Res0 R, LevelK<float, D> K, Xfer<float, D> X,
                                                 int nu1, int nu2, int H, double* __restrict__ partials,
                                                 DevState* st) {
    pdl_enter();
    if (st->done) return;
    double* __restrict__ uu = st->u;
    const float nsc = st->nscale;
    const int64_t nv = nchunks * 2 * D;
    const int sel = st->rsel;
    const float* __restrict__ rh_in = rh + sel * nv;
    const short* __restrict__ rl_in = rl + sel * nv;
    float* __restrict__ rh_out = rh + (1 - sel) * nv;
    short* __restrict__ rl_out = rl + (1 - sel) * nv;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = (nchunks + per - 1) / per;
    const int64_t nwarps = ((int64_t)gridDim.x * kNT) >> 5;
    float ssf = 0.f;
    for (int64_t tw = ((int64_t)blockIdx.x * kNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const int64_t q = tw * per + lane - H;
        const bool inb = q >= 0 && q < nchunks;
        const bool own = inb && lane >= H;
        float r[2][D], rlo[2][D], cc[D];
        short rq[2][D];
        double uv[2][D];
        load_pair<float, D>(rh_in, q, inb, r);
        load_pair<short, D>(rl_in, q, inb, rq);
        load_one<float, D>(uc, q, inb, cc);
        load_pair<double, D>(uu, q, own, uv);      // issued early: its latency overlaps the sweeps
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) rlo[i][k] = lo_decode(r[i][k], rq[i][k]);
        float h[2][D], c[2][D], w[2][D];
        presmooth_zero<DIR, float, D>(K, r, h, c, w, nu1);
        prolong_add<float, D>(X, cc, c);
        postsmooth<DIR, float, D>(K, h, c, nu2);
        if (!inb) {                                 // the correction is zero outside the array
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) c[i][k] = 0.f;
        }
        // r <- r - L c
        const ff b0 = bsum_ff<DIR, D>(c[0]);
        const ff b1 = bsum_ff<DIR, D>(c[1]);
        const ff bp{shfl_prev(b1.hi), shfl_prev(b1.lo)};
        residual_update_ff<DIR, D>(r[0], rlo[0], c[0], bp, R);
        residual_update_ff<DIR, D>(r[1], rlo[1], c[1], b0, R);
        if (own) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    uv[i][k] += f2d_int(c[i][k]);
                    const float v = r[i][k] * nsc;
                    ssf = fmaf(v, v, ssf);
                }
            store_pair<double, D>(uu, q, uv);
            store_pair<float, D>(rh_out, q, r);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) rq[i][k] = lo_encode(r[i][k], rlo[i][k]);
            store_pair<short, D>(rl_out, q, rq);
        }
        // the next cycle's way down on L c' = rh
        float rc[2][D], out[D];
        presmooth_zero<DIR, float, D>(K, r, h, c, w, nu1);
        residual_tracked<DIR, float, D>(r, c, w, rc);
        restrict_pair<float, D>(X, rc, out);
        if (own) VecIO<float, D>::store(fc + q * D, out);
    }
    const double ss = (double)ssf / ((double)nsc * (double)nsc);
    grid_norm_finalize<kNT>(ss, partials, st, kFinUpdated);
}

// Level 0 residual only, one interval per thread (any N): used when the
// on-chip solver handles the whole correction cycle.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kNT) k_res0(T* __restrict__ rT, int64_t N, Res0 R, double* __restrict__ partials,
                                              DevState* st) {
    pdl_enter();
    if (cycle_finished(st)) return;
    const double* __restrict__ F = st->F;
    const double* __restrict__ uu = st->u;
    const double u0 = st->u0;
    double ss = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kNT;
    for (int64_t n = (int64_t)blockIdx.x * kNT + threadIdx.x; n < N; n += stride) {
        double uv[D], Fv[D], up[D], r[D];
        load_one<double, D>(uu, n, true, uv);
        load_one<double, D>(F, n, true, Fv);
        double ep = u0;
        if (n > 0) {
            load_one<double, D>(uu, n - 1, true, up);
            ep = bval<DIR, double, D>(up);
        }
        residual0<DIR, D>(Fv, uv, ep, endval<double, D>(uv), R, r);
        T rt[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            rt[k] = (T)r[k];
            ss = fma(r[k], r[k], ss);
        }
        VecIO<T, D>::store(rT + n * D, rt);
    }
    grid_norm_finalize<kNT>(ss, partials, st);
}

// u += c (FP64 accumulation of a level-0 correction held in precision T).
template <typename T>
__global__ void __launch_bounds__(kNT) k_update0(const T* __restrict__ c, int64_t n_values,
                                                 const DevState* __restrict__ st) {
    pdl_enter();
    if (st->done) return;
    double* __restrict__ uu = st->u;
    const int64_t stride = (int64_t)gridDim.x * kNT;
    for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < n_values; i += stride) uu[i] += (double)c[i];
}

// r = F - L u into an FP64 array (public residual entry point).
template <int DIR, int D>
__global__ void __launch_bounds__(kNT) k_residual_out(const double* __restrict__ F, const double* __restrict__ u,
                                                      double u0, double* __restrict__ r, int64_t N, Res0 R) {
    const int64_t stride = (int64_t)gridDim.x * kNT;
    for (int64_t n = (int64_t)blockIdx.x * kNT + threadIdx.x; n < N; n += stride) {
        double uv[D], Fv[D], up[D], rr[D];
        load_one<double, D>(u, n, true, uv);
        load_one<double, D>(F, n, true, Fv);
        double ep = u0;
        if (n > 0) {
            load_one<double, D>(u, n - 1, true, up);
            ep = bval<DIR, double, D>(up);
        }
        residual0<DIR, D>(Fv, uv, ep, endval<double, D>(uv), R, rr);
        VecIO<double, D>::store(r + n * D, rr);
    }
}

// ||F||_2 with a*u0 folded into the first interval (for a caller-given start).
template <int DIR, int D>
__global__ void __launch_bounds__(kNT) k_normF(int64_t N, double* __restrict__ partials, DevState* st) {
    const double* __restrict__ F = st->F;
    const double u0 = st->u0;
    double ss = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kNT;
    for (int64_t n = (int64_t)blockIdx.x * kNT + threadIdx.x; n < N; n += stride) {
        double Fv[D];
        load_one<double, D>(F, n, true, Fv);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double v = (n == 0) ? Fv[k] + acoef<DIR>(k, u0) : Fv[k];
            ss = fma(v, v, ss);
        }
    }
    // reuse the ticketed reduction, but only to store ||F||
    __shared__ double red[kNT / 32];
    __shared__ int last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(kFull, ss, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < kNT / 32; ++i) s += red[i];
        partials[blockIdx.x] = s;
        __threadfence();
        last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (unsigned i = 0; i < gridDim.x; ++i) tot += __ldcg(&partials[i]);
        st->nF = sqrt(tot);
        st->ticket = 0u;
    }
}

// --------------------------------------------------- on-chip coarse solver --

constexpr int kTailNT = 512;
// Levels one CTA may hold: 8192 intervals (the largest on-chip level) halve
// to 1 in 14 steps.
constexpr int kTailLevels = 16;

// Shared-memory image of the coarse hierarchy handled by one CTA.
template <typename T, int D>
struct TailView {
    T* f[kTailLevels];
    T* u[kTailLevels];
    T* w;        // A u during pre-smoothing
    T* e;        // endpoint values of one pass
    T* scanA;    // [kTailNT/32] warp-total slopes of the coarsest scan
    T* scanB;    // [2*kTailNT/32] warp-total offsets, then inclusive warp prefixes
    int64_t N[kTailLevels];
};

template <typename T, int D>
__device__ __forceinline__ void sm_load(const T* p, T (&x)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = p[k];
}
template <typename T, int D>
__device__ __forceinline__ void sm_store(T* p, const T (&x)[D]) {
#pragma unroll
    for (int k = 0; k < D; ++k) p[k] = x[k];
}

// Endpoint values e[n] = b^T u_n of a whole level.
template <int DIR, typename T, int D>
__device__ __forceinline__ void tail_endvals(const T* u, T* e, int64_t N) {
    for (int64_t n = threadIdx.x; n < N; n += kTailNT) {
        T x[D];
        sm_load<T, D>(u + n * D, x);
        e[n] = bval<DIR, T, D>(x);
    }
}

// One damped block-Jacobi sweep of a level held in shared memory; w = A u is
// updated alongside when track_w.
template <int DIR, typename T, int D>
__device__ void tail_sweep(const LevelK<T, D>& K, const T* f, T* u, T* w, T* e, int64_t N, bool track_w) {
    tail_endvals<DIR, T, D>(u, e, N);
    __syncthreads();
    const T om = K.omega, om1 = T(1) - K.omega;
    for (int64_t n = threadIdx.x; n < N; n += kTailNT) {
        T fv[D], h[D], x[D];
        sm_load<T, D>(f + n * D, fv);
        sm_load<T, D>(u + n * D, x);
        matvec<T, D>(K.Ainv, fv, h);
        const T ep = n > 0 ? e[n - 1] : T(0);
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = om1 * x[k] + om * fma(K.g[k], ep, h[k]);
        sm_store<T, D>(u + n * D, x);
        if (track_w) {
            T y[D];
            sm_load<T, D>(w + n * D, y);
#pragma unroll
            for (int k = 0; k < D; ++k) y[k] = om1 * y[k] + om * (fv[k] + acoef<DIR>(k, ep));
            sm_store<T, D>(w + n * D, y);
        }
    }
    __syncthreads();
}

// Exact solve of the level by a block-wide prefix scan over the affine maps
// e_n = alpha e_{n-1} + c^T f_n (e_{-1} = 0), then u_n = A^{-1} f_n + g e_{n-1}.
template <typename T, int D>
__device__ void tail_exact(const LevelK<T, D>& K, const T* f, T* u, T* scanA, T* scanB, int64_t N) {
    const int t = threadIdx.x;
    const int64_t per = (N + kTailNT - 1) / kTailNT;
    const int64_t n0 = t * per, n1 = (n0 + per < N) ? n0 + per : N;
    T Aacc = T(1), Bacc = T(0);
    for (int64_t n = n0; n < n1; ++n) {
        T fv[D];
        sm_load<T, D>(f + n * D, fv);
        Bacc = fma(K.alpha, Bacc, dotc<T, D>(K.c, fv));
        Aacc *= K.alpha;
    }
    // inclusive scan of (A, B) over threads: compose left-to-right
    const int lane = t & 31, warp = t >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const T Ap = __shfl_up_sync(kFull, Aacc, off);
        const T Bp = __shfl_up_sync(kFull, Bacc, off);
        if (lane >= off) {
            Bacc = fma(Aacc, Bp, Bacc);
            Aacc = Aacc * Ap;
        }
    }
    if (lane == 31) {
        scanA[warp] = Aacc;
        scanB[warp] = Bacc;
    }
    __syncthreads();
    if (warp == 0) {
        T Aw = lane < kTailNT / 32 ? scanA[lane] : T(1);
        T Bw = lane < kTailNT / 32 ? scanB[lane] : T(0);
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T Ap = __shfl_up_sync(kFull, Aw, off);
            const T Bp = __shfl_up_sync(kFull, Bw, off);
            if (lane >= off) {
                Bw = fma(Aw, Bp, Bw);
                Aw = Aw * Ap;
            }
        }
        if (lane < kTailNT / 32) scanB[kTailNT / 32 + lane] = Bw;   // inclusive warp prefixes
    }
    __syncthreads();
    // exclusive prefix for this thread: warps before, then lanes before
    const T ew = warp > 0 ? scanB[kTailNT / 32 + warp - 1] : T(0);
    T Ain = __shfl_up_sync(kFull, Aacc, 1), Bin = __shfl_up_sync(kFull, Bacc, 1);
    if (lane == 0) {
        Ain = T(1);
        Bin = T(0);
    }
    T e = fma(Ain, ew, Bin);
    for (int64_t n = n0; n < n1; ++n) {
        T fv[D], h[D];
        sm_load<T, D>(f + n * D, fv);
        matvec<T, D>(K.Ainv, fv, h);
#pragma unroll
        for (int k = 0; k < D; ++k) h[k] = fma(K.g[k], e, h[k]);
        sm_store<T, D>(u + n * D, h);
        e = fma(K.alpha, e, dotc<T, D>(K.c, fv));
    }
    __syncthreads();
}

// Carve the shared-memory image of nl levels starting with Nt intervals out
// of p (layout of tail_smem_bytes).
template <typename T, int D>
__device__ __forceinline__ TailView<T, D> tail_view(T* p, int64_t Nt, int nl) {
    TailView<T, D> V;
    for (int j = 0; j < nl; ++j) {
        V.N[j] = Nt >> j;
        V.f[j] = p;
        p += V.N[j] * D;
    }
    for (int j = 0; j < nl; ++j) {
        V.u[j] = p;
        p += V.N[j] * D;
    }
    V.w = p;
    p += Nt * D;
    V.e = p;
    p += Nt;
    V.scanA = p;
    p += kTailNT / 32;
    V.scanB = p;
    return V;
}

// Debug build: the view ends inside the dynamic shared memory that starts
// at dyn (the launch's size); false (and recorded) otherwise, and the
// kernel skips the work.
template <typename T, int D>
__device__ __forceinline__ bool tail_view_fits(const TailView<T, D>& V, const void* dyn) {
#ifdef TMG_BOUNDS
    unsigned dyn_bytes;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
    const long long end = (long long)(reinterpret_cast<const char*>(V.scanB + 2 * (kTailNT / 32)) -
                                      reinterpret_cast<const char*>(dyn));
    return TMG_IN(end - 1, (long long)dyn_bytes, 10);
#else
    (void)V;
    (void)dyn;
    return true;
#endif
}

// One cycle on the levels held in V (tail index j = 0..nl-1), from a zero
// start (or, with init0, from the iterate V.u[0] holds): V (gamma = 1) or W
// (gamma = 2) recursion written as a loop, the coarsest level solved exactly.
// V.f[0] holds the right-hand side, V.u[0] receives the correction.  lk[j] are the constants of tail level j.  All
// threads of the CTA take part; ends with the block synchronised.
template <int DIR, typename T, int D>
__device__ void tail_cycle(const TailView<T, D>& V, const LevelK<T, D>* __restrict__ lk, const Xfer<T, D>& X, int nl,
                           int nu1, int nu2, int gamma, bool init0 = false) {
    int visits[kTailLevels];
    bool has_init[kTailLevels];
    for (int j = 0; j < nl; ++j) {
        visits[j] = 0;
        has_init[j] = false;
    }
    has_init[0] = init0;   // V.u[0] holds the start iterate
    int j = 0;
    bool down = true;
    while (true) {
        const LevelK<T, D>& K = lk[j];
        const int64_t N = V.N[j];
        if (down) {
            if (j == nl - 1) {
                tail_exact<T, D>(K, V.f[j], V.u[j], V.scanA, V.scanB, N);
                if (j == 0) break;
                --j;
                down = false;
                continue;
            }
            // pre-smoothing; a zero start gives u = omega A^{-1} f, A u = omega f
            int sweeps = nu1;
            if (!has_init[j]) {
                const T om_first = nu1 > 0 ? K.omega : T(0);
                for (int64_t n = threadIdx.x; n < N; n += kTailNT) {
                    T fv[D], h[D], x[D], y[D];
                    sm_load<T, D>(V.f[j] + n * D, fv);
                    matvec<T, D>(K.Ainv, fv, h);
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        x[k] = om_first * h[k];
                        y[k] = om_first * fv[k];
                    }
                    sm_store<T, D>(V.u[j] + n * D, x);
                    sm_store<T, D>(V.w + n * D, y);
                }
                __syncthreads();
                sweeps = nu1 > 0 ? nu1 - 1 : 0;
            } else {
                for (int64_t n = threadIdx.x; n < N; n += kTailNT) {
                    T x[D], y[D];
                    sm_load<T, D>(V.u[j] + n * D, x);
                    matvec<T, D>(K.A, x, y);
                    sm_store<T, D>(V.w + n * D, y);
                }
                __syncthreads();
            }
            for (int s = 0; s < sweeps; ++s) tail_sweep<DIR, T, D>(K, V.f[j], V.u[j], V.w, V.e, N, true);
            // residual f + a e_{n-1} - A u, restricted onto level j+1
            tail_endvals<DIR, T, D>(V.u[j], V.e, N);
            __syncthreads();
            for (int64_t m = threadIdx.x; m < N / 2; m += kTailNT) {
                T r[2][D], out[D];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int64_t n = 2 * m + i;
                    const T ep = n > 0 ? V.e[n - 1] : T(0);
#pragma unroll
                    for (int k = 0; k < D; ++k) r[i][k] = V.f[j][n * D + k] + acoef<DIR>(k, ep) - V.w[n * D + k];
                }
                restrict_pair<T, D>(X, r, out);
                sm_store<T, D>(V.f[j + 1] + m * D, out);
            }
            __syncthreads();
            visits[j] = 0;
            has_init[j + 1] = false;
            ++j;
            continue;
        }
        // back from level j+1
        if (++visits[j] < gamma) {
            has_init[j + 1] = true;
            ++j;
            down = true;
            continue;
        }
        for (int64_t m = threadIdx.x; m < N / 2; m += kTailNT) {
            T x[2][D], c[D];
            sm_load<T, D>(V.u[j] + (2 * m) * D, x[0]);
            sm_load<T, D>(V.u[j] + (2 * m + 1) * D, x[1]);
            sm_load<T, D>(V.u[j + 1] + m * D, c);
            prolong_add<T, D>(X, c, x);
            sm_store<T, D>(V.u[j] + (2 * m) * D, x[0]);
            sm_store<T, D>(V.u[j] + (2 * m + 1) * D, x[1]);
        }
        __syncthreads();
        for (int s = 0; s < nu2; ++s) tail_sweep<DIR, T, D>(K, V.f[j], V.u[j], V.w, V.e, N, false);
        if (j == 0) break;
        --j;
    }
}

// The coarse part of the cycle, levels lt..lt+nl-1 (tail index j = l - lt),
// entirely in shared memory (tail_cycle).  f_in is the right-hand side of
// level lt, u_out receives its correction; u_init (or nullptr for zero) is
// the start iterate of level lt (the second visit in a W-cycle).
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kTailNT) k_tail(const T* __restrict__ f_in, T* __restrict__ u_out,
                                                  const LevelK<T, D>* __restrict__ lk, Xfer<T, D> X, int nl,
                                                  int64_t Nt, int nu1, int nu2, int gamma,
                                                  const DevState* __restrict__ st, const T* __restrict__ u_init) {
    pdl_enter();
    if (st != nullptr && st->done) return;
    extern __shared__ __align__(16) unsigned char tail_smem[];
    const TailView<T, D> V = tail_view<T, D>(reinterpret_cast<T*>(tail_smem), Nt, nl);
    if (!tail_view_fits<T, D>(V, tail_smem)) return;
    for (int64_t i = threadIdx.x; i < Nt * D; i += kTailNT) {
        V.f[0][i] = f_in[i];
        if (u_init != nullptr) V.u[0][i] = u_init[i];
    }
    __syncthreads();
    tail_cycle<DIR, T, D>(V, lk, X, nl, nu1, nu2, gamma, u_init != nullptr);
    for (int64_t i = threadIdx.x; i < Nt * D; i += kTailNT) u_out[i] = V.u[0][i];
}

// Shared-memory bytes of the tail for nl levels starting with Nt intervals.
template <typename T, int D>
inline size_t tail_smem_bytes(int64_t Nt, int nl) {
    int64_t tot = 0;
    for (int j = 0; j < nl; ++j) tot += 2 * (Nt >> j) * D;
    tot += Nt * D + Nt + 3 * (kTailNT / 32);   // w, e, scanA, scanB (twice as long)
    return (size_t)tot * sizeof(T);
}

}  // namespace tmg
