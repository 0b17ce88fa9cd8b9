// Host-side plan of the time-multigrid solver (shared by all translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "../../include/tmg.h"
#include "tmg_kernels.cuh"
#include "tmg_scan.cuh"

namespace tmg {

// A launch property computed once per device -- the device current at the
// call.  The shared-memory opt-in of a kernel is an attribute of the device it
// was set on, and a process may build plans on several GPUs, so neither the
// opt-in nor the occupancy it implies is cached process-wide.
constexpr int kMaxDevices = 64;

template <typename V>
struct PerDevice {
    std::mutex m;
    bool have[kMaxDevices] = {};
    V val[kMaxDevices] = {};

    template <typename F>
    V get(F compute) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return compute();
        std::lock_guard<std::mutex> lock(m);
        if (!have[dev]) {
            val[dev] = compute();
            have[dev] = true;
        }
        return val[dev];
    }
};

}  // namespace tmg

// Shared-memory ceiling of the single-CTA coarse solver.
constexpr size_t kTailSmemMax = 200 * 1024;

// FP64 constants of one level, computed once on the host.
struct tmg_level_host {
    int64_t N;          // intervals
    double z;           // lambda * tau_l
    double A[tmg::kMaxDWide * tmg::kMaxDWide];   // K + z Mhat (row-major, D x D)
    double Ainv[tmg::kMaxDWide * tmg::kMaxDWide];
    double g[tmg::kMaxDWide];                     // A^{-1} a
    double c[tmg::kMaxDWide];                     // b^T A^{-1}
    double alpha;       // b^T A^{-1} a
    double omega;
};

struct tmg_ops;

struct tmg_plan {
    int p, d;
    double tau, lambda;
    int64_t N;
    double omega_user;
    tmg_opts o;
    cudaStream_t s;
    bool own_stream;     // s was created by the plan
    int nsm;

    int nlev;            // levels 0..nlev-1
    int lt;              // first level solved on chip (tail), or the coarsest level when scanned
    bool scan_coarsest;  // the coarsest level is too large for the chip: grid-wide scan instead of the tail
    void* scan_ws;       // tile maps, incoming values and per-thread chunk maps of the scans
                         // ((3 + 2 kScanNT) x ntiles x 8 bytes)
    int64_t scan_tiles;
    size_t tail_smem;
    std::vector<tmg_level_host> lev;       // constants of L
    std::vector<tmg_level_host> lev_adj;   // constants of L^T in reversed time
    // prolongation (coarse -> fine halves)
    double P1[tmg::kMaxDWide * tmg::kMaxDWide], P2[tmg::kMaxDWide * tmg::kMaxDWide];

    // device workspace (one allocation)
    void* ws;
    size_t ws_bytes;
    tmg::DevState* st;       // device state
    tmg::DevState* st_host;  // pinned mirror
    double* partials;
    int max_blocks;
    void* fl[tmg::kMaxLevels];   // level right-hand sides (cycle precision)
    void* ul[tmg::kMaxLevels];   // level corrections
    void* ul2[tmg::kMaxLevels];  // W-cycles: the corrections of each level's second visit (levels 1..lt)
    void* rT;                    // level-0 residual (cycle precision)
    void* rl;                    // its low float parts (mixed form with an updated residual), else nullptr
    void* lk_dev;                // tail level constants of L
    void* lk_dev_adj;            // ... and of L^T in reversed time
    double* adj_buf;             // reversed g and reversed mu (adjoint solves, allocated on first use)

    // optional buffers for the host-array entry point
    double* F_dev;
    double* u_dev;

    // CUDA graphs of the whole solve (while-loop over cycles), [0] = L, [1] = L^T
    cudaGraph_t graph[2];
    cudaGraphExec_t gexec[2];
    unsigned long long cond[2];

    const tmg_ops* ops;        // kernels for L
    const tmg_ops* ops_adj;    // kernels for L^T in reversed time

    // kernels launched by the last enqueued cycle (counted by launch())
    mutable int launches_per_cycle;

    // tmg_cycle_down / tmg_cycle_up: 1 = enqueue only the way down to the
    // coarsest level (its right-hand side is exported, not solved), 2 = only
    // the way up from an imported coarsest-level correction; 0 = whole cycles
    int split;

    // statistics of the last solve
    int last_cycles;
    double last_rel;
    double last_err;               // error against the exact FP64 solve (NAN unless opts.check_fp64)
    std::vector<double> last_hist;
    double* ex_buf;                // exact FP64 solution of the error check (allocated on first use)
};

// Per-(precision, D) entry points, instantiated in tmg_inst_*.cu.
struct tmg_ops {
    size_t elem;                                   // sizeof(cycle precision)
    size_t (*tail_bytes)(int64_t Nt, int nl);
    cudaError_t (*upload)(tmg_plan*);              // per-level constants -> device
    cudaError_t (*enqueue_cycle)(tmg_plan*);       // one correction cycle
    cudaError_t (*enqueue_cycle_timed)(tmg_plan*, cudaEvent_t* ev, int* cat, int* nev);   // same, events around kernels
    cudaError_t (*enqueue_normF)(tmg_plan*);       // ||F|| for a caller-given start
    cudaError_t (*enqueue_residual)(tmg_plan*, const double* f, double u0, const double* u, double* r);
    cudaError_t (*enqueue_direct)(tmg_plan*, const double* f, double u0, double* u);   // FP64 exact scan solve
    // the coarsest level's right-hand side out to, and its correction in from, FP64 arrays
    cudaError_t (*enqueue_coarse_io)(tmg_plan*, double* fc_out, const double* uc_in);
};

const tmg_ops* tmg_ops_f32(int d, int dir);
const tmg_ops* tmg_ops_f64(int d, int dir);
const tmg_ops* tmg_ops_f32_hi(int d, int dir);   // d = 4..6
const tmg_ops* tmg_ops_f64_hi(int d, int dir);
const tmg_ops* tmg_ops_f32_wide(int d, int dir);   // d = 11 (then tmg_ops_f32_w21)
const tmg_ops* tmg_ops_f64_wide(int d, int dir);
const tmg_ops* tmg_ops_f32_w21(int d, int dir);    // d = 21 (nullptr otherwise)
const tmg_ops* tmg_ops_f64_w21(int d, int dir);

// Adjoint helpers (tmg_adjoint.cu): reverse the interval order of an [N][d]
// array, and the gradient reductions dJ/du0 = a^T mu_0,
// dJ/dlambda = -tau sum_n mu_n^T Mhat u_n.
cudaError_t tmg_launch_reverse(const double* src, double* dst, int64_t N, int d, cudaStream_t s);
// max |u - v| and max |v| over n values (as the bits of non-negative doubles,
// out2 zeroed first), for the error of a result against the exact FP64 solve.
cudaError_t tmg_launch_maxabs2(const double* u, const double* v, int64_t n, unsigned long long* out2, int max_blocks,
                               cudaStream_t s);
cudaError_t tmg_launch_adjoint_grads(const double* mu, const double* u, int64_t N, int d, double tau,
                                     double* partials, int max_blocks, unsigned* ticket, double* dJdu0,
                                     double* dJdlambda, cudaStream_t s);
