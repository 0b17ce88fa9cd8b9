// Explicit instantiation of the plain FP64 forward solver for p_t = 10
// (11 x 11 blocks).  Only the per-level kernels and the grid-wide scan of the
// coarsest level are instantiated: the two-level kernels (four interval
// blocks per lane) and the on-chip coarse solver (a stack of levels per CTA)
// would spill.  The adjoint is not built at this degree.
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f64_wide(int d, int dir) {
    if (dir != 0) return nullptr;
    switch (d) {
        case 11: return tmg::Impl<double, 11, 0>::ops();
        default: return nullptr;
    }
}
