// Residual and residual norm of the DG-in-time system without any device
// allocation.
//
// Who needs this: code that may not call cudaMalloc at the point where it
// wants to check a solution -- real-time loops that cannot afford the
// implicit device synchronisation an allocation may cause, and applications
// that hand all device memory to their own pool at start-up.  tmg_setup
// allocates a workspace, so those callers cannot build a plan at that point;
// this entry point needs no plan and no allocation.
//
// The per-block partial sums of ||r||^2 and the completion ticket live in one
// file-scope __device__ array of fixed size (kScratchBlocks partials, about
// 8 KB), which every GPU that loads the library keeps until the process
// exits.  All calls share it: two calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/tmg.h"
#include "tmg_kernels.cuh"

namespace {

constexpr int kScratchBlocks = 1024;                     // partial sums held by the scratch array
constexpr int kPerThread = 8;                            // intervals per thread
constexpr int64_t kPerBlock = (int64_t)tmg::kNT * kPerThread;
constexpr int64_t kMaxIntervals = kScratchBlocks * kPerBlock;   // 2^21 intervals
constexpr int kMaxDevices = 64;

struct NormScratch {
    double partial[kScratchBlocks];
    unsigned ticket;
};

static __device__ __align__(256) NormScratch g_norm_scratch;

// One block per kPerBlock intervals; the last block to finish adds the
// partials in a fixed order (deterministic) and writes the norm.
template <int D>
__global__ void __launch_bounds__(tmg::kNT) k_residual_norm_static(const double* __restrict__ F,
                                                                    const double* __restrict__ u, double u0,
                                                                    double* __restrict__ r, int64_t N, tmg::Res0 R,
                                                                    NormScratch* __restrict__ scratch,
                                                                    double* __restrict__ norm_out) {
    using namespace tmg;
    double ss = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kPerBlock + threadIdx.x;
#pragma unroll 1
    for (int i = 0; i < kPerThread; ++i) {
        const int64_t n = base + (int64_t)i * kNT;
        if (n >= N) break;
        double uv[D], Fv[D], up[D], rr[D];
        load_one<double, D>(u, n, true, uv);
        load_one<double, D>(F, n, true, Fv);
        double ep = u0;
        if (n > 0) {
            load_one<double, D>(u, n - 1, true, up);
            ep = endval<double, D>(up);
        }
        residual0<0, D>(Fv, uv, ep, endval<double, D>(uv), R, rr);
        VecIO<double, D>::store(r + n * D, rr);
#pragma unroll
        for (int k = 0; k < D; ++k) ss = fma(rr[k], rr[k], ss);
    }
    __shared__ double red[kNT / 32];
    __shared__ int last;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(kFull, ss, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kNT / 32; ++w) s += red[w];
        scratch->partial[blockIdx.x] = s;
        __threadfence();
        last = (atomicAdd(&scratch->ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) tot += __ldcg(&scratch->partial[b]);
        *norm_out = sqrt(tot);
        scratch->ticket = 0u;
    }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.
std::mutex g_scratch_mutex;
NormScratch* g_scratch_addr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(NormScratch** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_norm_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<NormScratch*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" tmg_status tmg_residual_norm_noalloc(int p_t, double tau, double lambda, int64_t N, const double* f,
                                                double u0, const double* u, double* r, double* norm,
                                                void* stream) {
    if (p_t < 0 || p_t > tmg::kMaxD - 1 || !(tau > 0.0) || !isfinite(tau) || !(lambda >= 0.0) || !isfinite(lambda) || N < 1 ||
        !isfinite(u0) || !f || !u || !r || !norm)
        return TMG_EINVAL;
    if ((reinterpret_cast<uintptr_t>(f) | reinterpret_cast<uintptr_t>(u) | reinterpret_cast<uintptr_t>(r)) & 15u)
        return TMG_EINVAL;
    if ((reinterpret_cast<uintptr_t>(norm) & 7u) != 0) return TMG_EINVAL;
    if (N > kMaxIntervals) return TMG_EUNSUPPORTED;   // more blocks than the scratch holds partials for

    NormScratch* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return TMG_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the ticket must start at zero even if an earlier call was interrupted
    e = cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return TMG_ECUDA;

    tmg::Res0 R;
    for (int k = 0; k < tmg::kMaxD; ++k) {
        R.zm[k] = lambda * tau / (2.0 * k + 1.0);
        R.zm_hi[k] = (float)R.zm[k];
        R.zm_lo[k] = (float)(R.zm[k] - (double)R.zm_hi[k]);
    }
    const int blocks = (int)((N + kPerBlock - 1) / kPerBlock);
    switch (p_t) {
        case 0: k_residual_norm_static<1><<<blocks, tmg::kNT, 0, s>>>(f, u, u0, r, N, R, scratch, norm); break;
        case 1: k_residual_norm_static<2><<<blocks, tmg::kNT, 0, s>>>(f, u, u0, r, N, R, scratch, norm); break;
        case 2: k_residual_norm_static<3><<<blocks, tmg::kNT, 0, s>>>(f, u, u0, r, N, R, scratch, norm); break;
        case 3: k_residual_norm_static<4><<<blocks, tmg::kNT, 0, s>>>(f, u, u0, r, N, R, scratch, norm); break;
        case 4: k_residual_norm_static<5><<<blocks, tmg::kNT, 0, s>>>(f, u, u0, r, N, R, scratch, norm); break;
        default: k_residual_norm_static<6><<<blocks, tmg::kNT, 0, s>>>(f, u, u0, r, N, R, scratch, norm); break;
    }
    return cudaGetLastError() == cudaSuccess ? TMG_OK : TMG_ECUDA;
}
