// Explicit instantiation of the solver for the plain FP64 form.
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f64(int d, int dir) {
    switch (d) {
        case 1: return dir == 0 ? tmg::Impl<double, 1, 0>::ops() : tmg::Impl<double, 1, 1>::ops();
        case 2: return dir == 0 ? tmg::Impl<double, 2, 0>::ops() : tmg::Impl<double, 2, 1>::ops();
        case 3: return dir == 0 ? tmg::Impl<double, 3, 0>::ops() : tmg::Impl<double, 3, 1>::ops();
        case 4: return dir == 0 ? tmg::Impl<double, 4, 0>::ops() : tmg::Impl<double, 4, 1>::ops();
        default: return nullptr;
    }
}
