// Helpers of the adjoint solve (interval reversal, the gradient reductions)
// and of the error check against the exact FP64 solve.
//
// For a loss J(u) of the solution of L u = F (F = f with a*u0 in the first
// interval), mu = L^{-T} dJ/du gives dJ/df = mu, dJ/du0 = a^T mu_0 and
// dJ/dlambda = -tau sum_n mu_n^T Mhat u_n (L depends on lambda only through
// the mass term lambda*tau*Mhat of every diagonal block, Section 2).
#include <stdint.h>

#include "tmg_plan.h"

namespace {

constexpr int kThreads = 256;

// One thread per interval (no integer division in the index arithmetic).
__global__ void __launch_bounds__(kThreads) k_reverse(const double* __restrict__ src, double* __restrict__ dst,
                                                      int64_t N, int d) {
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t n = (int64_t)blockIdx.x * kThreads + threadIdx.x; n < N; n += stride) {
        const double* s = src + n * d;
        double* o = dst + (N - 1 - n) * d;
        for (int k = 0; k < d; ++k) o[k] = s[k];
    }
}

// Deterministic grid reduction of sum_n sum_k mu[n][k] u[n][k] / (2k+1); the
// last block adds the partials in order and writes both gradients.  Each
// thread takes whole intervals and keeps one sum per coefficient k; the
// weights 1/(2k+1) are applied once per block.
__global__ void __launch_bounds__(kThreads) k_adjoint_grads(const double* __restrict__ mu, const double* __restrict__ u,
                                                            int64_t N, int d, double tau,
                                                            double* __restrict__ partials, unsigned* ticket,
                                                            double* __restrict__ dJdu0,
                                                            double* __restrict__ dJdlambda) {
    double sk[tmg::kMaxDWide];
#pragma unroll
    for (int k = 0; k < tmg::kMaxDWide; ++k) sk[k] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t n = (int64_t)blockIdx.x * kThreads + threadIdx.x; n < N; n += stride) {
        const double* a = mu + n * d;
        const double* b = u + n * d;
#pragma unroll
        for (int k = 0; k < tmg::kMaxDWide; ++k)
            if (k < d) sk[k] = fma(a[k], b[k], sk[k]);
    }
    __shared__ double red[tmg::kMaxDWide][kThreads / 32];
    __shared__ int last;
#pragma unroll
    for (int k = 0; k < tmg::kMaxDWide; ++k) {
        double s = sk[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < d; ++k) {
            double tk = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) tk += red[k][w];
            t += tk / (2.0 * k + 1.0);
        }
        partials[blockIdx.x] = t;
        __threadfence();
        last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double tot = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) tot += __ldcg(&partials[b]);
    *dJdlambda = -tau * tot;
    double g0 = 0.0;
    for (int k = 0; k < d; ++k) g0 += (k & 1) ? -mu[k] : mu[k];   // a^T mu_0, a_k = (-1)^k
    *dJdu0 = g0;
    *ticket = 0u;
}

// max |u - v| and max |v| over n values into out[0], out[1] as the bit
// patterns of non-negative doubles (their order as unsigned integers is the
// order of the values, so atomicMax on the bits is a max of the values).  A
// non-finite difference counts as infinite.
__global__ void __launch_bounds__(kThreads) k_maxabs2(const double* __restrict__ u, const double* __restrict__ v,
                                                      int64_t n, unsigned long long* __restrict__ out) {
    double md = 0.0, mv = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        const double a = u[i], b = v[i];
        const double dv = fabs(a - b);
        md = (dv == dv && dv <= 1.0e308) ? fmax(md, dv) : INFINITY;
        mv = fmax(mv, fabs(b));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        md = fmax(md, __shfl_xor_sync(0xffffffffu, md, off));
        mv = fmax(mv, __shfl_xor_sync(0xffffffffu, mv, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(md));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(mv));
    }
}

}  // namespace

cudaError_t tmg_launch_maxabs2(const double* u, const double* v, int64_t n, unsigned long long* out2, int max_blocks,
                               cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (n + kThreads - 1) / kThreads;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    k_maxabs2<<<(int)blocks, kThreads, 0, s>>>(u, v, n, out2);
    return cudaGetLastError();
}

cudaError_t tmg_launch_reverse(const double* src, double* dst, int64_t N, int d, cudaStream_t s) {
    int64_t blocks = (N + kThreads - 1) / kThreads;
    if (blocks > 4096) blocks = 4096;
    k_reverse<<<(int)blocks, kThreads, 0, s>>>(src, dst, N, d);
    return cudaGetLastError();
}

cudaError_t tmg_launch_adjoint_grads(const double* mu, const double* u, int64_t N, int d, double tau,
                                     double* partials, int max_blocks, unsigned* ticket, double* dJdu0,
                                     double* dJdlambda, cudaStream_t s) {
    int64_t blocks = (N + kThreads - 1) / kThreads;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    k_adjoint_grads<<<(int)blocks, kThreads, 0, s>>>(mu, u, N, d, tau, partials, ticket, dJdu0, dJdlambda);
    return cudaGetLastError();
}
