// Exact solve of a whole level by a parallel prefix scan over affine maps.
//
// Because N = a b^T has rank one, the block forward substitution of eq.
// chap4_generalLinearSystemODE reduces to a scalar first-order recurrence for
// the halo values e_n = b^T u_n:
//     e_n = alpha e_{n-1} + c^T f_n,   u_n = A^{-1} f_n + g e_{n-1},
// with c^T = b^T A^{-1}, g = A^{-1} a, alpha = b^T A^{-1} a and e_{-1} the
// initial value (u0 on the original system, 0 for a correction equation).
// Each interval is the affine map e -> alpha e + beta_n; maps compose
// associatively, so the recurrence is a scan.  Three passes, no block waits
// for another: (1) every block reduces its tile of intervals to one map and
// stores, per thread, the map from the tile's incoming value to the value
// entering that thread's chunk; (2) one block scans the tile maps into the
// incoming value of every tile; (3) every thread replays its chunk from its
// stored map and the tile's incoming value and writes u.  On GB300 the scan is
// bound by FP64 arithmetic, so pass 3 does not recompute pass 1's maps.
// Tiles are staged in shared memory with coalesced loads; each thread owns a
// contiguous chunk of kScanPT intervals.
#pragma once

#include "tmg_kernels.cuh"

namespace tmg {

constexpr int kScanNT = 256;
constexpr int kScanPT = 8;                    // tile maps per thread in the prefix pass
constexpr int kScanTileMin = kScanNT * 4;     // the smallest tile: the host sizes the scan workspace with it

// Intervals per thread chunk: 8, or 4 for blocks wider than 11 coefficients
// (a tile of 256 x 8 intervals of 21 FP64 coefficients would need 346 KB of
// shared memory).
template <int D>
__host__ __device__ constexpr int scan_pt() {
    return D > 11 ? 4 : 8;
}

template <int D>
__host__ __device__ constexpr int scan_tile() {
    return kScanNT * scan_pt<D>();
}

template <typename S, int D>
struct ScanK {
    S Ainv[D * D];
    S g[D];
    S c[D];
    S alpha;
};

template <int D, typename TIn>
constexpr size_t scan_smem_bytes() {
    return (size_t)kScanNT * (scan_pt<D>() * D + 1) * sizeof(TIn);
}

// Stage the tile [t0, t0 + scan_tile<D>()) of f (values beyond N read as 0) into
// shared memory, padded by one element per thread chunk (bank spread).
template <int D, typename TIn>
__device__ __forceinline__ void scan_stage(const TIn* __restrict__ f, int64_t N, int64_t t0, TIn* sm) {
    constexpr int PT = scan_pt<D>();
    const int64_t base = t0 * D;
    const int64_t total = N * D;
    for (int i = threadIdx.x; i < scan_tile<D>() * D; i += kScanNT) {
        const int64_t gi = base + i;
        const int t = i / (PT * D), j = i - t * (PT * D);
        sm[t * (PT * D + 1) + j] = gi < total ? f[gi] : TIn(0);
    }
    __syncthreads();
}

// Map of this thread's chunk: e_out = A e_in + B.
template <typename S, int D, typename TIn>
__device__ __forceinline__ void chunk_map(const ScanK<S, D>& K, const TIn* sm, S& A, S& B) {
    const TIn* p = sm + threadIdx.x * (scan_pt<D>() * D + 1);
    A = S(1);
    B = S(0);
#pragma unroll
    for (int i = 0; i < scan_pt<D>(); ++i) {
        S beta = S(0);
#pragma unroll
        for (int k = 0; k < D; ++k) beta = fma(K.c[k], (S)p[i * D + k], beta);
        B = fma(K.alpha, B, beta);
        A *= K.alpha;
    }
}

// Block-wide inclusive scan of maps (A, B) in thread order; returns the
// exclusive prefix of this thread and the block total.
template <typename S>
__device__ __forceinline__ void block_scan_maps(S A, S B, S& exA, S& exB, S& totA, S& totB) {
    __shared__ S wA[kScanNT / 32], wB[kScanNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const S Ap = __shfl_up_sync(kFull, A, off);
        const S Bp = __shfl_up_sync(kFull, B, off);
        if (lane >= off) {
            B = fma(A, Bp, B);
            A = A * Ap;
        }
    }
    if (lane == 31) {
        wA[warp] = A;
        wB[warp] = B;
    }
    __syncthreads();
    // prefix over the warps before this one
    S pA = S(1), pB = S(0);
    for (int w = 0; w < warp; ++w) {
        pB = fma(wA[w], pB, wB[w]);
        pA = pA * wA[w];
    }
    S iA = __shfl_up_sync(kFull, A, 1), iB = __shfl_up_sync(kFull, B, 1);
    if (lane == 0) {
        iA = S(1);
        iB = S(0);
    }
    // exclusive map of this thread = (lanes before in this warp) o (warps before)
    exB = fma(iA, pB, iB);
    exA = iA * pA;
    totA = S(1);
    totB = S(0);
    for (int w = 0; w < kScanNT / 32; ++w) {
        totB = fma(wA[w], totB, wB[w]);
        totA = totA * wA[w];
    }
    __syncthreads();
}

// Pass 1: one map per tile, and the exclusive map of every thread's chunk
// within its tile (thrA/thrB [ntiles][kScanNT]).
template <typename S, int D, typename TIn>
__global__ void __launch_bounds__(kScanNT) k_scan_tiles(const TIn* __restrict__ f, int64_t N, ScanK<S, D> K,
                                                        S* __restrict__ aggA, S* __restrict__ aggB,
                                                        S* __restrict__ thrA, S* __restrict__ thrB,
                                                        const DevState* __restrict__ st) {
    pdl_enter();
    if (st != nullptr && st->done) return;
    extern __shared__ __align__(16) unsigned char scan_sm[];
    TIn* sm = reinterpret_cast<TIn*>(scan_sm);
    const int64_t ntiles = (N + scan_tile<D>() - 1) / scan_tile<D>();
    for (int64_t b = blockIdx.x; b < ntiles; b += gridDim.x) {
        scan_stage<D, TIn>(f, N, b * scan_tile<D>(), sm);
        S A, B, eA, eB, tA, tB;
        chunk_map<S, D, TIn>(K, sm, A, B);
        block_scan_maps<S>(A, B, eA, eB, tA, tB);
        thrA[b * kScanNT + threadIdx.x] = eA;
        thrB[b * kScanNT + threadIdx.x] = eB;
        if (threadIdx.x == 0) {
            aggA[b] = tA;
            aggB[b] = tB;
        }
    }
}

// Pass 2 (one block): incoming value of every tile, ein[b], from e_{-1} = e0
// (e0 given, or read from *e0p when e0p != nullptr).
template <typename S>
__global__ void __launch_bounds__(kScanNT) k_scan_prefix(const S* __restrict__ aggA, const S* __restrict__ aggB,
                                                         int64_t ntiles, S e0, const double* e0p,
                                                         S* __restrict__ ein, const DevState* __restrict__ st) {
    pdl_enter();
    if (st != nullptr && st->done) return;
    S carry = e0p != nullptr ? (S)(*e0p) : e0;
    for (int64_t base = 0; base < ntiles; base += kScanNT * kScanPT) {
        // each thread composes up to kScanPT consecutive tile maps
        const int64_t t0 = base + (int64_t)threadIdx.x * kScanPT;
        S A = S(1), B = S(0);
        for (int i = 0; i < kScanPT; ++i) {
            const int64_t t = t0 + i;
            if (t < ntiles) {
                B = fma(aggA[t], B, aggB[t]);
                A = A * aggA[t];
            }
        }
        S eA, eB, tA, tB;
        block_scan_maps<S>(A, B, eA, eB, tA, tB);
        S e = fma(eA, carry, eB);            // value entering this thread's first tile
        for (int i = 0; i < kScanPT; ++i) {
            const int64_t t = t0 + i;
            if (t < ntiles) {
                ein[t] = e;
                e = fma(aggA[t], e, aggB[t]);
            }
        }
        carry = fma(tA, carry, tB);
    }
}

// Pass 3: replay every tile from its incoming value; u_n = A^{-1} f_n + g e_{n-1}.
template <typename S, int D, typename TIn, typename TOut>
__global__ void __launch_bounds__(kScanNT) k_scan_apply(const TIn* __restrict__ f, TOut* __restrict__ u, int64_t N,
                                                        ScanK<S, D> K, const S* __restrict__ ein,
                                                        const S* __restrict__ thrA, const S* __restrict__ thrB,
                                                        const DevState* __restrict__ st) {
    pdl_enter();
    if (st != nullptr && st->done) return;
    extern __shared__ __align__(16) unsigned char scan_sm[];
    TIn* sm = reinterpret_cast<TIn*>(scan_sm);
    constexpr int PT = scan_pt<D>();
    const int64_t ntiles = (N + scan_tile<D>() - 1) / scan_tile<D>();
    for (int64_t b = blockIdx.x; b < ntiles; b += gridDim.x) {
        const int64_t t0 = b * scan_tile<D>();
        scan_stage<D, TIn>(f, N, t0, sm);
        S e = fma(thrA[b * kScanNT + threadIdx.x], ein[b], thrB[b * kScanNT + threadIdx.x]);
        TIn* p = sm + threadIdx.x * (PT * D + 1);   // this thread's chunk; results overwrite it
#pragma unroll
        for (int i = 0; i < PT; ++i) {
            S x[D], beta = S(0);
#pragma unroll
            for (int k = 0; k < D; ++k) beta = fma(K.c[k], (S)p[i * D + k], beta);
#pragma unroll
            for (int r = 0; r < D; ++r) {
                S s = K.g[r] * e;
#pragma unroll
                for (int k = 0; k < D; ++k) s = fma(K.Ainv[r * D + k], (S)p[i * D + k], s);
                x[r] = s;
            }
            e = fma(K.alpha, e, beta);
#pragma unroll
            for (int r = 0; r < D; ++r) p[i * D + r] = (TIn)x[r];
        }
        __syncthreads();
        // coalesced write-back of the tile
        const int64_t total = N * D;
        for (int i = threadIdx.x; i < scan_tile<D>() * D; i += kScanNT) {
            const int64_t gi = t0 * D + i;
            const int t = i / (PT * D), j = i - t * (PT * D);
            if (gi < total) u[gi] = (TOut)sm[t * (PT * D + 1) + j];
        }
        __syncthreads();
    }
}

}  // namespace tmg
