// Explicit instantiation of the mixed-precision forward solver for p_t = 10
// (FP32 cycles, FP64 level-0 residual recomputed from u in every cycle).  As
// for the FP64 form at this degree: per-level kernels and the grid-wide scan
// only; the fused level-0 kernel with the updated float-pair residual is not
// instantiated (its 2 x 11 float pairs per lane would spill).
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f32_wide(int d, int dir) {
    if (dir != 0) return nullptr;
    switch (d) {
        case 11: return tmg::Impl<float, 11, 0>::ops();
        default: return nullptr;
    }
}
