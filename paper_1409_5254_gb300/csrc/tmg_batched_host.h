// Host side of the batched solver shared by its translation units: the plan
// structures, launch-size helpers, and the per-(precision, D, direction)
// enqueue templates (degrees 0..2 are instantiated in tmg_batched.cu,
// 3..5 in tmg_batched_hi.cu, so that the two compile in parallel).
#pragma once

#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tmg_batched.cuh"
#include "tmg_nvtx.h"
#include "tmg_setup_math.h"

using namespace tmg;

struct tmg_batch_group {
    int p, d;
    int64_t n;           // instances in the group
    int64_t Ng;          // slot length (power of two, >= 2)
    int log2Ng;
    int nlev;
    bool var;            // variable lengths: instances of the same depth s = nlev - 1, each of its own
                         // m_i 2^s intervals (m_i <= 2^log2M), tiles over real intervals only; else
                         // every instance padded at its end to Ng
    int log2M;
    bool direct;         // group arrays are the caller's arrays
    std::vector<int64_t> ids;

    void* ws;            // one allocation for everything below
    size_t ws_bytes;
    BatchState* st;
    BatchState* st_host;
    BatchInst bi;
    Res0* res;
    void* lk[2];         // LevelK table [n][nlev], per direction
    void* rT;
    void* rl;            // updated-residual form: low parts of the residual pairs (two buffers), else nullptr
    void* fl[kMaxLevels];
    void* ul[kMaxLevels];
    void* ul2[kMaxLevels];   // W-cycles: the corrections of each level's second visit (levels 1..lt_w)
    int lt_w;                // W-cycles, grid form: first level run by kb_tail (one CTA per instance)
    size_t tail_smem_w;      // its shared memory
    void* c0;
    int64_t* d_ids;
    int64_t* d_Ni;
    int64_t* d_off;
    double* Fg;          // gathered right-hand side [n][Ng][d] (allocated on first use)
    double* ug;
    double* u0g;
    cudaGraph_t graph[2];
    cudaGraphExec_t gexec[2];
    unsigned long long cond[2];
    int last_status;
    cudaStream_t s;      // the group's own stream: groups run concurrently
    cudaEvent_t done;    // recorded on s after the group's last work of a call
    bool cta_ok;         // the CTA-per-instance form fits in one CTA's shared memory
    size_t cta_smem;
    int sched;           // TMG_SCHED_GRID or TMG_SCHED_CTA
    double ms_tune[2];   // autotuner: one synthetic solve, grid form and CTA form (NAN: not timed)
    double* exk;         // error check: FP64 level-0 constants per instance, [n][D*D + 2D + 1]
                         // (A^{-1}, g, c, alpha), built on the first check
};

struct tmg_batch {
    int64_t n_inst;
    std::vector<int> p;
    std::vector<int64_t> N, off;
    std::vector<double> tau, lambda;
    int64_t total_values;
    tmg_opts o;
    double omega;
    cudaStream_t s;
    bool own_stream;
    int max_blocks;
    std::vector<tmg_batch_group*> groups;
    cudaEvent_t fork;     // recorded on s at the start of a call; every group stream waits on it
    void* table;          // device copies of off, N (int64), tau (double), p (int) for the gradient kernel
    std::vector<int> cycles;
    std::vector<double> rel;
    std::vector<double> err;  // error against the exact FP64 solve per instance (NAN unless checked)
    double* err_dev;          // its device copy (allocated on the first check)
    double ms_whole[2] = {NAN, NAN};   // autotuner: whole synthetic batch, per-group choices / all grid
};

namespace tmgb {

inline int halo(int S) { return (S + 1) / 2; }
inline int sw_down(int nu1) { return (nu1 > 0 ? nu1 - 1 : 0) + 1; }
inline int sw_up(int nu1, int nu2) { return (nu1 > 0 ? nu1 - 1 : 0) + nu2; }

inline int grid_tiles(const tmg_batch* B, int64_t nchunks, int H) {
    const int64_t per = 32 - H;
    int64_t blocks = ((nchunks + per - 1) / per + (kBNT / 32) - 1) / (kBNT / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, B->max_blocks));
}

inline int grid_flat(const tmg_batch* B, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kBNT - 1) / kBNT, B->max_blocks));
}

// Shared-memory ceiling of the CTA-per-instance form.
constexpr size_t kCtaSmemMax = 200 * 1024;

// One visit of level l >= 1 in a W-cycle over the listed instances (the
// single-problem w_visit): a first visit starts from zero and writes ul[l], a
// second (nz) starts from ul[l] and writes ul2[l]; level l+1 is visited twice
// in between.  From level lt_w on, kb_tail runs the rest of the W recursion
// in shared memory, one CTA per instance.
template <typename T, int D, int DIR>
void w_visit_b(tmg_batch* B, tmg_batch_group* G, int l, bool nz, const Xfer<T, D>& X) {
    const int nu1 = B->o.nu1, nu2 = B->o.nu2;
    const LevelK<T, D>* lk = static_cast<const LevelK<T, D>*>(G->lk[DIR]);
    const int L = G->nlev;
    T* ua = static_cast<T*>(G->ul[l]);
    T* ub = static_cast<T*>(G->ul2[l]);
    if (l == G->lt_w) {
        static PerDevice<cudaError_t> attr_c;
        attr_c.get([&] {
            return cudaFuncSetAttribute(kb_tail<DIR, T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kTailSmemMax);
        });
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(G->n, B->max_blocks / 4));
        kb_tail<DIR, T, D><<<grid, kTailNT, G->tail_smem_w, G->s>>>(
            static_cast<const T*>(G->fl[l]), nz ? ub : ua, nz ? (const T*)ua : nullptr, lk, L, l, X,
            (int)(G->Ng >> l), nu1, nu2, 2, G->st, G->bi);
        return;
    }
    const int64_t nch = G->n * (G->Ng >> l) / 2;
    if (nz) {
        const int H = halo(nu1 + 1);
        kb_down_nz<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
            static_cast<const T*>(G->fl[l]), (const T*)ua, static_cast<T*>(G->fl[l + 1]), G->log2Ng - l, lk, L, l, X,
            nu1, H, G->st, G->bi);
    } else {
        const int H = halo(sw_down(nu1));
        kb_down<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
            static_cast<const T*>(G->fl[l]), static_cast<T*>(G->fl[l + 1]), nch, G->log2Ng - l, lk, L, l, X, nu1, H,
            G->st, G->bi);
    }
    w_visit_b<T, D, DIR>(B, G, l + 1, false, X);
    w_visit_b<T, D, DIR>(B, G, l + 1, true, X);
    const T* uc = static_cast<const T*>(G->ul2[l + 1]);
    if (nz) {
        const int H = halo(nu1 + nu2);
        kb_up_nz<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
            static_cast<const T*>(G->fl[l]), (const T*)ua, uc, ub, G->log2Ng - l, lk, L, l, X, nu1, nu2, H, G->st,
            G->bi);
    } else {
        const int H = halo(sw_up(nu1, nu2));
        kb_up<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
            static_cast<const T*>(G->fl[l]), uc, ua, nch, G->log2Ng - l, lk, L, l, X, nu1, nu2, H, G->st, G->bi);
    }
}

template <typename T, int D, int DIR>
cudaError_t enqueue_cycle(tmg_batch* B, tmg_batch_group* G) {
    const NvtxRange r_cycle("tmg batch cycle, group of degree %d", G->p);
    const int nu1 = B->o.nu1, nu2 = B->o.nu2;
    Xfer<T, D> X;
    for (int i = 0; i < D * D; ++i) {   // reversed time swaps the halves
        X.P1[i] = (T)0;
        X.P2[i] = (T)0;
    }
    {
        double P1[kMaxDWide * kMaxDWide], P2[kMaxDWide * kMaxDWide];
        tmg_host::transfer_setup(D, P1, P2);
        for (int i = 0; i < D * D; ++i) {
            X.P1[i] = (T)(DIR == 0 ? P1[i] : P2[i]);
            X.P2[i] = (T)(DIR == 0 ? P2[i] : P1[i]);
        }
    }
    const LevelK<T, D>* lk = static_cast<const LevelK<T, D>*>(G->lk[DIR]);
    T* rT = static_cast<T*>(G->rT);
    const int64_t n = G->n;
    const int L = G->nlev;
    // mixed form with the level-0 residual kept as updated float pairs
    short* rl = std::is_same<T, float>::value ? static_cast<short*>(G->rl) : nullptr;
    {
        const int H = halo(1 + sw_down(nu1));
        const int64_t nch = n * G->Ng / 2;
        kb_down0<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
            rT, rl, L > 1 ? static_cast<T*>(G->fl[1]) : nullptr, nch, G->log2Ng, lk, G->res, L, X, nu1, H, G->st,
            G->bi);
    }
    kb_finalize<<<grid_flat(B, n), kBNT, 0, G->s>>>(G->st, G->bi, n, rl != nullptr ? kFinFull : kFinPlain);
    if (G->var) kb_units<<<1, kUnitsNT, 0, G->s>>>(G->st, G->bi);   // act_list changed
    if (L == 1) {
        kb_coarse<DIR, T, D><<<grid_flat(B, n * 32), kBNT, 0, G->s>>>(rT, static_cast<T*>(G->c0), n, (int)G->Ng, lk,
                                                                       L, 0, G->st, G->bi);
        // u += c; the instance of value i is i / (Ng D)
        const int64_t nv = n * G->Ng * D;
        kb_update0<T, D><<<grid_flat(B, nv), kBNT, 0, G->s>>>(static_cast<const T*>(G->c0), nv,
                                                               (int)(G->Ng * D), G->st, G->bi);
        return cudaGetLastError();
    }
    // W-cycle: level 1 is visited twice (streaming levels down to lt_w, then
    // kb_tail); the level-0 way up reads the correction of the second visit
    const bool wcycle = B->o.gamma == 2;
    if constexpr (D <= kMaxD) {   // (wider groups run V-cycles only: the set-up rejects W for them)
        if (wcycle) {
            w_visit_b<T, D, DIR>(B, G, 1, false, X);
            w_visit_b<T, D, DIR>(B, G, 1, true, X);
        }
    }
    const T* uc1 = static_cast<const T*>(wcycle ? G->ul2[1] : G->ul[1]);
    // streaming levels 1 .. L-2, two per kernel where two remain (default for
    // FP32 cycles, as in the single-problem solver)
    const bool fuse = D <= kMaxD && (B->o.fuse_levels > 0 || (B->o.fuse_levels < 0 && std::is_same<T, float>::value));
    int grp[kMaxLevels], ng = 0;
    for (int l = 1; !wcycle && l < L - 1;) {
        const bool two = fuse && l + 1 < L - 1;
        grp[ng++] = two ? -l : l;      // negative: levels l and l+1 in one kernel
        l += two ? 2 : 1;
    }
    for (int g = 0; g < ng; ++g) {
        if (grp[g] < 0) {
            if constexpr (D <= kMaxD) {
                const int l = -grp[g];
                const int H = halo(halo(sw_down(nu1)) + sw_down(nu1));
                const int64_t nq = n * (G->Ng >> l) / 4;
                kb_down2<DIR, T, D><<<grid_tiles(B, nq, H), kBNT, 0, G->s>>>(
                    static_cast<const T*>(G->fl[l]), static_cast<T*>(G->fl[l + 2]), G->log2Ng - l, lk, L, l, X, nu1,
                    H, G->st, G->bi);
            }
        } else {
            const int l = grp[g];
            const int H = halo(sw_down(nu1));
            const int64_t nch = n * (G->Ng >> l) / 2;
            kb_down<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
                static_cast<const T*>(G->fl[l]), static_cast<T*>(G->fl[l + 1]), nch, G->log2Ng - l, lk, L, l, X,
                nu1, H, G->st, G->bi);
        }
    }
    if (!wcycle)
        kb_coarse<DIR, T, D><<<grid_flat(B, n * 32), kBNT, 0, G->s>>>(static_cast<const T*>(G->fl[L - 1]),
                                                                       static_cast<T*>(G->ul[L - 1]), n,
                                                                       (int)(G->Ng >> (L - 1)), lk, L, L - 1, G->st,
                                                                       G->bi);
    for (int g = ng - 1; g >= 0; --g) {
        if (grp[g] < 0) {
            if constexpr (D <= kMaxD) {
                const int l = -grp[g];
                const int g1 = halo(sw_down(nu1)) + sw_up(nu1, nu2);
                const int H = (2 * g1 + nu2 + 3) / 4;
                const int64_t nq = n * (G->Ng >> l) / 4;
                kb_up2<DIR, T, D><<<grid_tiles(B, nq, H), kBNT, 0, G->s>>>(
                    static_cast<const T*>(G->fl[l]), static_cast<const T*>(G->ul[l + 2]), static_cast<T*>(G->ul[l]),
                    G->log2Ng - l, lk, L, l, X, nu1, nu2, H, G->st, G->bi);
            }
        } else {
            const int l = grp[g];
            const int H = halo(sw_up(nu1, nu2));
            const int64_t nch = n * (G->Ng >> l) / 2;
            kb_up<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
                static_cast<const T*>(G->fl[l]), static_cast<const T*>(G->ul[l + 1]), static_cast<T*>(G->ul[l]), nch,
                G->log2Ng - l, lk, L, l, X, nu1, nu2, H, G->st, G->bi);
        }
    }
    if constexpr (std::is_same<T, float>::value && D <= kMaxD) {
        if (rl != nullptr) {
            const int H = halo(sw_up(nu1, nu2) + 1 + sw_down(nu1));
            const int64_t nch = n * G->Ng / 2;
            kb_updown0<DIR, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(
                rT, rl, reinterpret_cast<const float*>(uc1), static_cast<float*>(G->fl[1]), nch, G->log2Ng, lk,
                G->res, L, X, nu1, nu2, H, G->st, G->bi);
            kb_finalize<<<grid_flat(B, n), kBNT, 0, G->s>>>(G->st, G->bi, n, kFinUpdated);
            if (G->var) kb_units<<<2, kUnitsNT, 0, G->s>>>(G->st, G->bi);   // both lists changed
            return cudaGetLastError();
        }
    }
    {
        const int H = halo(sw_up(nu1, nu2));
        const int64_t nch = n * G->Ng / 2;
        kb_up0<DIR, T, D><<<grid_tiles(B, nch, H), kBNT, 0, G->s>>>(rT, uc1, nch,
                                                                     G->log2Ng, lk, L, X, nu1, nu2, H, G->st, G->bi);
    }
    return cudaGetLastError();
}

template <typename T, int D, int DIR>
cudaError_t launch_cta(tmg_batch* B, tmg_batch_group* G, const double* F, double* u, const double* u0) {
    Xfer<T, D> X;
    double P1[kMaxDWide * kMaxDWide], P2[kMaxDWide * kMaxDWide];
    tmg_host::transfer_setup(D, P1, P2);
    for (int i = 0; i < D * D; ++i) {   // reversed time swaps the halves
        X.P1[i] = (T)(DIR == 0 ? P1[i] : P2[i]);
        X.P2[i] = (T)(DIR == 0 ? P2[i] : P1[i]);
    }
    static PerDevice<cudaError_t> attr_c;
    const cudaError_t attr = attr_c.get([&] {
        return cudaFuncSetAttribute(kb_cta_solve<DIR, T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kCtaSmemMax);
    });
    if (attr != cudaSuccess) return attr;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_cta_solve<DIR, T, D>, kTailNT, G->cta_smem);
    if (e != cudaSuccess) return e;
    const int64_t wave = (int64_t)(B->max_blocks / 8) * (occ > 0 ? occ : 1);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(G->n, wave));
    kb_cta_solve<DIR, T, D><<<grid, kTailNT, G->cta_smem, G->s>>>(
        F, u, u0, G->n, (int)G->Ng, G->nlev, static_cast<const LevelK<T, D>*>(G->lk[DIR]), G->res, X, B->o.nu1,
        B->o.nu2, B->o.gamma, G->st, G->bi);
    return cudaGetLastError();
}

// The same for D = 4..6 (tmg_batched_hi.cu) and for D = 11, 21 (tmg_batched_wide.cu:
// per-level kernels only, the level-0 residual recomputed from u, V-cycles).
cudaError_t enqueue_hi(tmg_batch* B, tmg_batch_group* G, bool mixed, int dir);
cudaError_t enqueue_wide(tmg_batch* B, tmg_batch_group* G, bool mixed, int dir);
cudaError_t launch_cta_hi(tmg_batch* B, tmg_batch_group* G, const double* F, double* u, const double* u0,
                          bool mixed, int dir);

}  // namespace tmgb
