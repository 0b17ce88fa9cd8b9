// Explicit instantiation of the solver for the mixed-precision form (FP32 cycles), p_t = 0..2;
// p_t = 3..5 are instantiated in tmg_inst_f32_hi.cu (compiled in parallel).
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f32(int d, int dir) {
    switch (d) {
        case 1: return dir == 0 ? tmg::Impl<float, 1, 0>::ops() : tmg::Impl<float, 1, 1>::ops();
        case 2: return dir == 0 ? tmg::Impl<float, 2, 0>::ops() : tmg::Impl<float, 2, 1>::ops();
        case 3: return dir == 0 ? tmg::Impl<float, 3, 0>::ops() : tmg::Impl<float, 3, 1>::ops();
        default: return tmg_ops_f32_hi(d, dir);
    }
}
