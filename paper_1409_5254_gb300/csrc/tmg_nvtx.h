// NVTX ranges around the host-side enqueue of every cycle and level (header
// only; without a profiler attached a push or pop is one indirect call).  A
// solve that runs as a CUDA graph enqueues its cycle once, at capture, so its
// ranges mark the capture; with opts.use_graph = 0 every cycle is enqueued
// anew and a profiler's timeline shows one range per cycle and level.
#pragma once

#include <stdio.h>

#include <nvtx3/nvToolsExt.h>

namespace tmg {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    NvtxRange(const char* fmt, int a) {
        char buf[64];
        snprintf(buf, sizeof(buf), fmt, a);
        nvtxRangePushA(buf);
    }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
    ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace tmg
