// Explicit instantiation of the mixed-precision solver for p_t = 20 (21 x 21
// blocks), forward and adjoint, with the same restrictions as p_t = 10:
// per-level kernels, the coarsest level by the grid-wide scan (four intervals
// per thread chunk at this width), the FP64 level-0 residual recomputed from u
// in every cycle, and k_down0 loading its inputs without shared-memory stages.
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f32_w21(int d, int dir) {
    switch (d) {
        case 21: return dir == 0 ? tmg::Impl<float, 21, 0>::ops() : tmg::Impl<float, 21, 1>::ops();
        default: return nullptr;
    }
}
