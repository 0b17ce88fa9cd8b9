// Explicit instantiation of the solver for the mixed-precision form (FP32 cycles).
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f32(int d) {
    switch (d) {
        case 1: return tmg::Impl<float, 1>::ops();
        case 2: return tmg::Impl<float, 2>::ops();
        case 3: return tmg::Impl<float, 3>::ops();
        case 4: return tmg::Impl<float, 4>::ops();
        default: return nullptr;
    }
}
