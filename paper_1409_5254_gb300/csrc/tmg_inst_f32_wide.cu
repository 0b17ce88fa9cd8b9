// Explicit instantiation of the mixed-precision solver for p_t = 10 (11 x 11
// blocks), forward and adjoint: FP32 cycles, the FP64 level-0 residual
// recomputed from u in every cycle (the fused level-0 kernel with the updated
// float-pair residual would spill at this width).  Only the per-level kernels
// and the grid-wide scan of the coarsest level are instantiated: the two-level
// kernels and the on-chip coarse solver would spill.  p_t = 20 is in
// tmg_inst_f32_w21.cu (compiled in parallel).
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f32_wide(int d, int dir) {
    switch (d) {
        case 11: return dir == 0 ? tmg::Impl<float, 11, 0>::ops() : tmg::Impl<float, 11, 1>::ops();
        default: return tmg_ops_f32_w21(d, dir);
    }
}
