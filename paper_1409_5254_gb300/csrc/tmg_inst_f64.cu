// Explicit instantiation of the solver for the plain FP64 form, p_t = 0..2;
// p_t = 3..5 are instantiated in tmg_inst_f64_hi.cu (compiled in parallel).
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f64(int d, int dir) {
    switch (d) {
        case 1: return dir == 0 ? tmg::Impl<double, 1, 0>::ops() : tmg::Impl<double, 1, 1>::ops();
        case 2: return dir == 0 ? tmg::Impl<double, 2, 0>::ops() : tmg::Impl<double, 2, 1>::ops();
        case 3: return dir == 0 ? tmg::Impl<double, 3, 0>::ops() : tmg::Impl<double, 3, 1>::ops();
        default: return tmg_ops_f64_hi(d, dir);
    }
}
