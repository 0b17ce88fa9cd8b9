// Batched solver kernels for degrees p_t = 3..5 (D = 4..6), compiled apart
// from tmg_batched.cu so that the two translation units build in parallel.
#include <type_traits>

#include "tmg_batched_host.h"

namespace tmgb {

template <typename T, int DIR>
cudaError_t enqueue_hi_t(tmg_batch* B, tmg_batch_group* G) {
    switch (G->d) {
        case 4: return enqueue_cycle<T, 4, DIR>(B, G);
        case 5: return enqueue_cycle<T, 5, DIR>(B, G);
        case 6: return enqueue_cycle<T, 6, DIR>(B, G);
        default: return enqueue_wide(B, G, std::is_same<T, float>::value, DIR);
    }
}

template <typename T, int DIR>
cudaError_t launch_cta_hi_t(tmg_batch* B, tmg_batch_group* G, const double* F, double* u, const double* u0) {
    switch (G->d) {
        case 4: return launch_cta<T, 4, DIR>(B, G, F, u, u0);
        case 5: return launch_cta<T, 5, DIR>(B, G, F, u, u0);
        case 6: return launch_cta<T, 6, DIR>(B, G, F, u, u0);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t enqueue_hi(tmg_batch* B, tmg_batch_group* G, bool mixed, int dir) {
    if (mixed) return dir == 0 ? enqueue_hi_t<float, 0>(B, G) : enqueue_hi_t<float, 1>(B, G);
    return dir == 0 ? enqueue_hi_t<double, 0>(B, G) : enqueue_hi_t<double, 1>(B, G);
}

cudaError_t launch_cta_hi(tmg_batch* B, tmg_batch_group* G, const double* F, double* u, const double* u0,
                          bool mixed, int dir) {
    if (mixed) return dir == 0 ? launch_cta_hi_t<float, 0>(B, G, F, u, u0) : launch_cta_hi_t<float, 1>(B, G, F, u, u0);
    return dir == 0 ? launch_cta_hi_t<double, 0>(B, G, F, u, u0) : launch_cta_hi_t<double, 1>(B, G, F, u, u0);
}

}  // namespace tmgb
