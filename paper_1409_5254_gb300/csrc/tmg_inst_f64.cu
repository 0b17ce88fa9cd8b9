// Explicit instantiation of the solver for the plain FP64 form.
#include "tmg_impl.cuh"

const tmg_ops* tmg_ops_f64(int d) {
    switch (d) {
        case 1: return tmg::Impl<double, 1>::ops();
        case 2: return tmg::Impl<double, 2>::ops();
        case 3: return tmg::Impl<double, 3>::ops();
        case 4: return tmg::Impl<double, 4>::ops();
        default: return nullptr;
    }
}
