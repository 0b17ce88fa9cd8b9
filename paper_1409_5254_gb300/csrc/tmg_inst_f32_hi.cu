// Explicit instantiation of the mixed-precision solver for p_t = 3..5.
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f32_hi(int d, int dir) {
    switch (d) {
        case 4: return dir == 0 ? tmg::Impl<float, 4, 0>::ops() : tmg::Impl<float, 4, 1>::ops();
        case 5: return dir == 0 ? tmg::Impl<float, 5, 0>::ops() : tmg::Impl<float, 5, 1>::ops();
        case 6: return dir == 0 ? tmg::Impl<float, 6, 0>::ops() : tmg::Impl<float, 6, 1>::ops();
        default: return tmg_ops_f32_wide(d, dir);
    }
}
