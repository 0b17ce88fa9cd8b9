// Explicit instantiation of the plain FP64 solver for p_t = 10 (11 x 11 blocks),
// forward and adjoint.  Only the per-level kernels and the grid-wide scan of
// the coarsest level are instantiated: the two-level kernels (four interval
// blocks per lane) and the on-chip coarse solver (a stack of levels per CTA)
// would spill.  p_t = 20 is in tmg_inst_f64_w21.cu (compiled in parallel).
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f64_wide(int d, int dir) {
    switch (d) {
        case 11: return dir == 0 ? tmg::Impl<double, 11, 0>::ops() : tmg::Impl<double, 11, 1>::ops();
        default: return tmg_ops_f64_w21(d, dir);
    }
}
