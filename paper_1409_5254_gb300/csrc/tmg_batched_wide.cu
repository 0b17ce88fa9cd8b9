// Batched solver kernels for the wide degrees p_t = 10 and 20 (D = 11, 21),
// compiled apart so that the units build in parallel.  As for one problem at
// these degrees: per-level streaming kernels (no two-level kernels), the
// level-0 residual recomputed from u in every cycle (no updated float pair),
// the coarsest level (at most 64 intervals) by one warp per instance, V-cycles
// and the grid schedule only.
#include <type_traits>

#include "tmg_batched_host.h"

namespace tmgb {

template <typename T, int DIR>
cudaError_t enqueue_wide_t(tmg_batch* B, tmg_batch_group* G) {
    switch (G->d) {
        case 11: return enqueue_cycle<T, 11, DIR>(B, G);
        case 21: return enqueue_cycle<T, 21, DIR>(B, G);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t enqueue_wide(tmg_batch* B, tmg_batch_group* G, bool mixed, int dir) {
    if (mixed) return dir == 0 ? enqueue_wide_t<float, 0>(B, G) : enqueue_wide_t<float, 1>(B, G);
    return dir == 0 ? enqueue_wide_t<double, 0>(B, G) : enqueue_wide_t<double, 1>(B, G);
}

}  // namespace tmgb
