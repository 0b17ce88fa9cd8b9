// Debug build with bounds checks (compiled with -DTMG_BOUNDS; build_ext
// builds it as a second library).  TMG_IN(idx, len, site) is true when
// 0 <= idx < len.  Otherwise it counts the violation, records the first
// failing site and index in this translation unit's device words, and is
// false; every caller then skips the access (a load yields 0), so a bad index
// never touches memory outside its array and the kernel runs to its end.
// tmg_debug_bounds reads and clears the words of every translation unit.
// Without TMG_BOUNDS, TMG_IN is the constant true and costs nothing.
//
// Sites: 1-9 level-vector loads and stores of the streaming kernels,
// 10-19 shared-memory layouts and indices, 20-29 batched kernels, 30-49 the
// space-time heat kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace tmg {

// One reader per translation unit built with TMG_BOUNDS: returns 0 and the
// unit's violation count and first record (site << 40 | low 40 bits of the
// index), clearing both; nonzero if the device words cannot be read.
using BoundsReader = int (*)(unsigned* count, unsigned long long* first);

inline std::vector<BoundsReader>& bounds_readers() {
    static std::vector<BoundsReader> readers;
    return readers;
}

}  // namespace tmg

#ifdef TMG_BOUNDS

// Translation-unit local (static): each unit has its own device words and
// registers its own reader.
namespace tmg {

static __device__ unsigned g_bounds_count;
static __device__ unsigned long long g_bounds_first;

static __device__ __forceinline__ bool bounds_in(long long idx, long long len, int site) {
    if (idx >= 0 && idx < len) return true;
    atomicAdd(&g_bounds_count, 1u);
    atomicCAS(&g_bounds_first, 0ull,
              ((unsigned long long)site << 40) | ((unsigned long long)idx & 0xFFFFFFFFFFull));
    return false;
}

static int read_bounds(unsigned* count, unsigned long long* first) {
    unsigned c = 0;
    unsigned long long f = 0;
    const unsigned zc = 0;
    const unsigned long long zf = 0;
    if (cudaMemcpyFromSymbol(&c, g_bounds_count, sizeof c) != cudaSuccess ||
        cudaMemcpyFromSymbol(&f, g_bounds_first, sizeof f) != cudaSuccess ||
        cudaMemcpyToSymbol(g_bounds_count, &zc, sizeof zc) != cudaSuccess ||
        cudaMemcpyToSymbol(g_bounds_first, &zf, sizeof zf) != cudaSuccess)
        return 1;
    *count = c;
    *first = f;
    return 0;
}

static const bool g_bounds_registered = (bounds_readers().push_back(&read_bounds), true);

}  // namespace tmg

#define TMG_IN(idx, len, site) (::tmg::bounds_in((long long)(idx), (long long)(len), (site)))

#else

#define TMG_IN(idx, len, site) true

#endif
