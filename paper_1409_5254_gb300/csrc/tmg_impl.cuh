// Launch orchestration of one correction cycle for cycle precision T and D = p_t + 1.
#pragma once

#include <string.h>

#include "tmg_nvtx.h"
#include "tmg_plan.h"

namespace tmg {

template <typename T, int D>
LevelK<T, D> level_consts(const tmg_level_host& L) {
    LevelK<T, D> K;
    for (int i = 0; i < D * D; ++i) {
        K.A[i] = (T)L.A[i];
        K.Ainv[i] = (T)L.Ainv[i];
    }
    for (int i = 0; i < D; ++i) {
        K.g[i] = (T)L.g[i];
        K.c[i] = (T)L.c[i];
    }
    K.omega = (T)L.omega;
    K.alpha = (T)L.alpha;
    return K;
}

// Transfer matrices; in reversed time the first half of a coarse interval is
// the second half of the original one, so P1 and P2 trade places.
template <typename T, int D>
Xfer<T, D> xfer_consts(const tmg_plan* P, int dir) {
    Xfer<T, D> X;
    for (int i = 0; i < D * D; ++i) {
        X.P1[i] = (T)(dir == 0 ? P->P1[i] : P->P2[i]);
        X.P2[i] = (T)(dir == 0 ? P->P2[i] : P->P1[i]);
    }
    return X;
}

inline Res0 res0_consts(const tmg_plan* P) {
    Res0 R;
    for (int k = 0; k < kMaxDWide; ++k) {
        R.zm[k] = P->lev[0].z / (2.0 * k + 1.0);
        R.zm_hi[k] = (float)R.zm[k];
        R.zm_lo[k] = (float)(R.zm[k] - (double)R.zm_hi[k]);
    }
    return R;
}

// Groups of kernels of one cycle, for the per-kernel timing of tmg_profile_cycle.
enum : int { kCatDown0 = 0, kCatDown = 1, kCatCoarse = 2, kCatUp = 3, kCatUp0 = 4, kCatEnd = -1 };

// Halo lanes per warp tile: S sweeps that read e_{n-1} need ceil(S/2) lanes.
inline int halo_lanes(int S) { return (S + 1) / 2; }
inline int sweeps_down(int nu1) { return (nu1 > 0 ? nu1 - 1 : 0) + 1; }
inline int sweeps_up(int nu1, int nu2) { return (nu1 > 0 ? nu1 - 1 : 0) + nu2; }

// Blocks of kNT threads of a kernel that are resident on one SM at once.
template <typename Kern>
inline int resident_per_sm(Kern kernel, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kNT, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

// Grid of a warp-tile streaming kernel: one warp per tile up to one full
// wave of resident blocks (SMs x resident blocks per SM); larger levels loop
// over their tiles with that persistent grid, so no partial last wave leaves
// SMs idle.
inline int grid_for(const tmg_plan* P, int64_t nchunks, int H, int resident) {
    const int64_t per = 32 - H;
    const int64_t tiles = (nchunks + per - 1) / per;
    int64_t blocks = (tiles + (kNT / 32) - 1) / (kNT / 32);
    const int64_t wave = (int64_t)P->nsm * resident;
    if (blocks > wave) blocks = wave;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

inline int grid_flat(const tmg_plan* P, int64_t n) {
    int64_t blocks = (n + kNT - 1) / kNT;
    if (blocks > P->max_blocks) blocks = P->max_blocks;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// Launch with the programmatic-stream-serialisation attribute when the plan
// asks for it (every cycle kernel starts with pdl_enter()).
// Opt a kernel into more than 48 KB of dynamic shared memory.  Called from the
// function that launches the kernel, once per instantiation: a kernel template
// instantiated in several translation units has one registration per unit,
// and the attribute must reach the one that the launching code refers to.
template <typename... KArgs>
inline cudaError_t allow_smem(void (*kernel)(KArgs...), size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename... KArgs, typename... Args>
inline void launch(const tmg_plan* P, void (*kernel)(KArgs...), int grid, int block, size_t smem,
                   Args... args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = P->s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = P->o.use_pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
    ++P->launches_per_cycle;
}

// Element-wise copy with conversion (the coarsest level's right-hand side out
// to FP64, its correction in from FP64).
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kNT) k_convert(const Tin* __restrict__ in, Tout* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * kNT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kNT)
        out[i] = (Tout)in[i];
}

template <typename T, int D, int DIR>
struct Impl {
    static const std::vector<tmg_level_host>& L(const tmg_plan* P) { return DIR == 0 ? P->lev : P->lev_adj; }

    static size_t tail_bytes(int64_t Nt, int nl) { return tail_smem_bytes<T, D>(Nt, nl); }

    static cudaError_t upload(tmg_plan* P) {
        const int nl = P->nlev - P->lt;
        std::vector<LevelK<T, D>> lk(nl);
        for (int j = 0; j < nl; ++j) lk[j] = level_consts<T, D>(L(P)[P->lt + j]);
        return cudaMemcpyAsync(DIR == 0 ? P->lk_dev : P->lk_dev_adj, lk.data(), sizeof(LevelK<T, D>) * nl,
                               cudaMemcpyHostToDevice, P->s);
    }

    template <typename S>
    static ScanK<S, D> scan_consts(const tmg_level_host& L) {
        ScanK<S, D> K;
        for (int i = 0; i < D * D; ++i) K.Ainv[i] = (S)L.Ainv[i];
        for (int i = 0; i < D; ++i) {
            K.g[i] = (S)L.g[i];
            K.c[i] = (S)L.c[i];
        }
        K.alpha = (S)L.alpha;
        return K;
    }

    // Exact solve of level l's equation L_l x = f by the three-pass scan, in
    // precision S, from e_{-1} = e0 (or *e0p).
    template <typename S, typename TIO>
    static void enqueue_scan(tmg_plan* P, const TIO* f, TIO* x, int l, S e0, const double* e0p,
                             const DevState* st) {
        const int64_t N = P->lev[l].N;
        const int64_t nt = (N + scan_tile<D>() - 1) / scan_tile<D>();
        S* aggA = static_cast<S*>(P->scan_ws);
        S* aggB = aggA + nt;
        S* ein = aggB + nt;
        S* thrA = ein + nt;               // per-thread chunk maps, [nt][kScanNT] each
        S* thrB = thrA + nt * kScanNT;
        const ScanK<S, D> K = scan_consts<S>(L(P)[l]);
        const int grid = (int)(nt < P->max_blocks ? nt : P->max_blocks);
        // (a failed opt-in makes the launches below fail, which the caller reports)
        static PerDevice<cudaError_t> attr_t_c;
        const cudaError_t attr_t = attr_t_c.get([&] { return allow_smem(k_scan_tiles<S, D, TIO>, scan_smem_bytes<D, TIO>()); });
        static PerDevice<cudaError_t> attr_a_c;
        const cudaError_t attr_a = attr_a_c.get([&] { return allow_smem(k_scan_apply<S, D, TIO, TIO>, scan_smem_bytes<D, TIO>()); });
        (void)attr_t;
        (void)attr_a;
        launch(P, k_scan_tiles<S, D, TIO>, grid, kScanNT, scan_smem_bytes<D, TIO>(), f, N, K, aggA, aggB, thrA, thrB,
               st);
        launch(P, k_scan_prefix<S>, 1, kScanNT, 0, aggA, aggB, nt, e0, e0p, ein, st);
        launch(P, k_scan_apply<S, D, TIO, TIO>, grid, kScanNT, scan_smem_bytes<D, TIO>(), f, x, N, K, ein, thrA, thrB,
               st);
    }

    // tmg_solve_direct: the whole system by the FP64 scan (forward direction).
    static cudaError_t enqueue_direct(tmg_plan* P, const double* f, double u0, double* u) {
        if constexpr (DIR != 0 || !std::is_same<T, double>::value) {
            return cudaErrorInvalidValue;   // only the FP64 forward ops carry the direct solve
        } else {
            enqueue_scan<double, double>(P, f, u, 0, u0, nullptr, nullptr);
            return cudaGetLastError();
        }
    }

    // The on-chip coarse solver exists for p_t <= 5; a plan of a wider block
    // solves its coarsest level by the scan (checked in enqueue_cycle_timed).
    template <typename... Args>
    static void launch_tail(tmg_plan* P, Args... args) {
        if constexpr (D <= kMaxD) {
            static PerDevice<cudaError_t> attr_c;
        const cudaError_t attr = attr_c.get([&] { return allow_smem(k_tail<DIR, T, D>, kTailSmemMax); });
            (void)attr;   // a failed opt-in makes the launch fail, which the caller reports
            launch(P, k_tail<DIR, T, D>, 1, kTailNT, P->tail_smem, args...);
        }
    }

    // One visit of level l >= 1 in a W-cycle (gamma = 2): nz = the second
    // visit of the level under the same parent visit, which starts from the
    // first visit's result ul[l] and writes ul2[l]; a first visit starts from
    // zero and writes ul[l].  Levels below visit level l+1 twice; the final
    // correction of level l+1 is then in ul2[l+1].  The coarse part (level
    // lt and below) is one launch per visit: the on-chip solver (with the
    // start iterate on a second visit, and the W recursion inside) or the
    // exact scan.
    static void w_visit(tmg_plan* P, int l, bool nz, const Xfer<T, D>& X, const LevelK<T, D>* lk_tail, int nl) {
        const NvtxRange r_visit(nz ? "tmg level %d second visit" : "tmg level %d visit", l);
        const int nu1 = P->o.nu1, nu2 = P->o.nu2;
        T* ua = static_cast<T*>(P->ul[l]);
        T* ub = static_cast<T*>(P->ul2[l]);
        if (l == P->lt) {
            if (P->scan_coarsest)
                enqueue_scan<T, T>(P, static_cast<const T*>(P->fl[l]), nz ? ub : ua, l, T(0), nullptr, P->st);
            else
                launch_tail(P, static_cast<const T*>(P->fl[l]), nz ? ub : ua, lk_tail, X, nl, P->lev[l].N, nu1, nu2,
                            P->o.gamma, (const DevState*)P->st, nz ? (const T*)ua : (const T*)nullptr);
            return;
        }
        const int64_t nch = P->lev[l].N / 2;
        const LevelK<T, D> K = level_consts<T, D>(L(P)[l]);
        const CoarseTail<T, D> ct_none{nullptr, nullptr, nullptr, 0, nullptr};
        if (nz) {
            const int H = halo_lanes(nu1 + 1);
            static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_down_nz<DIR, T, D>, 0); });
            launch(P, k_down_nz<DIR, T, D>, grid_for(P, nch, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]),
                   (const T*)ua, static_cast<T*>(P->fl[l + 1]), nch, K, X, nu1, H, (const DevState*)P->st);
        } else {
            const int H = halo_lanes(sweeps_down(nu1));
            static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_down<DIR, T, D>, 0); });
            launch(P, k_down<DIR, T, D>, grid_for(P, nch, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]),
                   static_cast<T*>(P->fl[l + 1]), nch, K, X, nu1, H, (const DevState*)P->st, ct_none);
        }
        w_visit(P, l + 1, false, X, lk_tail, nl);
        w_visit(P, l + 1, true, X, lk_tail, nl);
        const T* uc = static_cast<const T*>(P->ul2[l + 1]);
        if (nz) {
            const int H = halo_lanes(nu1 + nu2);
            static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_up_nz<DIR, T, D>, 0); });
            launch(P, k_up_nz<DIR, T, D>, grid_for(P, nch, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]),
                   (const T*)ua, uc, ub, nch, K, X, nu1, nu2, H, (const DevState*)P->st);
        } else {
            const int H = halo_lanes(sweeps_up(nu1, nu2));
            static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_up<DIR, T, D>, 0); });
            launch(P, k_up<DIR, T, D>, grid_for(P, nch, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]), uc, ua,
                   nch, K, X, nu1, nu2, H, (const DevState*)P->st);
        }
    }

    static cudaError_t enqueue_cycle(tmg_plan* P) { return enqueue_cycle_timed(P, nullptr, nullptr, nullptr); }

    // tmg_cycle_down / tmg_cycle_up: the coarsest level's right-hand side out
    // (fc_out != nullptr) or its correction in (uc_in != nullptr).
    static cudaError_t enqueue_coarse_io(tmg_plan* P, double* fc_out, const double* uc_in) {
        const int64_t n = P->lev[P->lt].N * D;
        if (fc_out != nullptr)
            k_convert<T, double><<<grid_flat(P, n), kNT, 0, P->s>>>(static_cast<const T*>(P->fl[P->lt]), fc_out, n);
        if (uc_in != nullptr)
            k_convert<double, T><<<grid_flat(P, n), kNT, 0, P->s>>>(uc_in, static_cast<T*>(P->ul[P->lt]), n);
        return cudaGetLastError();
    }

    // One correction cycle.  With ev != nullptr an event is recorded before
    // every kernel group and after the last one; cat[i] receives the group
    // between ev[i] and ev[i+1] (kCat*) and *nev the number of events
    // (at most 2 * nlev + 4).
    static cudaError_t enqueue_cycle_timed(tmg_plan* P, cudaEvent_t* ev, int* cat, int* nev) {
        if constexpr (D > kMaxD) {
            if (!P->scan_coarsest) return cudaErrorInvalidValue;
        }
        const NvtxRange r_cycle(DIR == 0 ? "tmg cycle" : "tmg adjoint cycle");
        P->launches_per_cycle = 0;
        int iev = 0;
        auto mark = [&](int c) {
            if (ev) {
                cudaEventRecord(ev[iev], P->s);
                if (cat) cat[iev] = c;
                ++iev;
            }
        };
        const int nu1 = P->o.nu1, nu2 = P->o.nu2;
        const Xfer<T, D> X = xfer_consts<T, D>(P, DIR);
        const Res0 R = res0_consts(P);
        const int nl = P->nlev - P->lt;
        const LevelK<T, D>* lk = static_cast<const LevelK<T, D>*>(DIR == 0 ? P->lk_dev : P->lk_dev_adj);
        T* rT = static_cast<T*>(P->rT);
        // mixed form with the level-0 residual kept as a float pair and updated
        // by k_updown0 (the plan allocates rl only then)
        constexpr bool kMixed = std::is_same<T, float>::value;
        short* rl = kMixed && P->lt >= 1 ? static_cast<short*>(P->rl) : nullptr;
        if (P->lt == 0) {
            mark(kCatDown0);
            launch(P, k_res0<DIR, T, D>, grid_flat(P, P->N), kNT, 0, rT, P->N, R, P->partials, P->st);
            mark(kCatCoarse);
            if (P->scan_coarsest)
                enqueue_scan<T, T>(P, rT, static_cast<T*>(P->ul[0]), 0, T(0), nullptr, P->st);
            else
                launch_tail(P, rT, static_cast<T*>(P->ul[0]), lk, X, nl, P->N, nu1, nu2, P->o.gamma,
                            (const DevState*)P->st, (const T*)nullptr);
            mark(kCatUp0);
            launch(P, k_update0<T>, grid_flat(P, P->N * D), kNT, 0, static_cast<const T*>(P->ul[0]),
                   (int64_t)(P->N * D), (const DevState*)P->st);
            mark(kCatEnd);
            if (nev) *nev = iev;
            return cudaGetLastError();
        }
        const int split = P->split;   // 1: the way down only, 2: the way up only (tmg_cycle_down/up)
        if (split != 2) {
            const NvtxRange r_lev("tmg level %d down", 0);
            const int H = halo_lanes(1 + sweeps_down(nu1));
            const int64_t nch = P->N / 2;
            mark(kCatDown0);
            static PerDevice<cudaError_t> attr_c;
        const cudaError_t attr = attr_c.get([&] { return allow_smem(k_down0<DIR, T, D>, k_down0_smem_bytes<D>()); });
            if (attr != cudaSuccess) return attr;
            static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_down0<DIR, T, D>, k_down0_smem_bytes<D>()); });
            launch(P, k_down0<DIR, T, D>, grid_for(P, nch, H, occ), kNT, k_down0_smem_bytes<D>(), rT, rl,
                   static_cast<T*>(P->fl[1]), nch, R, level_consts<T, D>(L(P)[0]), X, nu1, H, P->partials, P->st);
        }
        // W-cycle: level 1 is visited twice; the level-0 way up reads the
        // correction of its second visit
        const bool wcycle = P->o.gamma == 2;
        const T* uc1 = static_cast<const T*>(wcycle ? P->ul2[1] : P->ul[1]);
        if (wcycle) {
            mark(kCatDown);
            w_visit(P, 1, false, X, lk, nl);
            w_visit(P, 1, true, X, lk, nl);
        }
        // streaming levels 1 .. lt-1, two at a time where both exist
        int grp[kMaxLevels], ng = 0;
        for (int l = 1; !wcycle && l < P->lt;) {
            // default (-1): fuse where the cycle runs in FP32; the FP64 form is
            // bound by FP64 arithmetic, which the fused way up repeats
            // (the two-level kernels exist for p_t <= 5)
            const bool fuse = D <= kMaxD && (P->o.fuse_levels > 0 || (P->o.fuse_levels < 0 && kMixed));
            const int two = fuse && l + 1 < P->lt;
            grp[ng++] = two ? -l : l;      // negative: levels l and l+1 in one kernel
            l += two ? 2 : 1;
        }
        // the coarsest level (at most 64 intervals, directly below the streaming
        // levels) is solved by the last block of the last down kernel
        const bool coarse_in_down = split == 0 && P->o.gamma == 1 && !P->scan_coarsest && P->lt == P->nlev - 1 &&
                                    ng > 0 && P->lev[P->lt].N <= 64;
        CoarseTail<T, D> ct_none{nullptr, nullptr, nullptr, 0, nullptr};
        CoarseTail<T, D> ct_last{lk, static_cast<const T*>(P->fl[P->lt]), static_cast<T*>(P->ul[P->lt]),
                                 (int)P->lev[P->lt].N, &P->st->ticket2};
        for (int g = 0; split != 2 && g < ng; ++g) {
            const NvtxRange r_lev(grp[g] < 0 ? "tmg levels %d,+1 down" : "tmg level %d down", grp[g] < 0 ? -grp[g] : grp[g]);
            const CoarseTail<T, D> ct = coarse_in_down && g == ng - 1 ? ct_last : ct_none;
            mark(kCatDown);
            if (grp[g] < 0) {
                if constexpr (D <= kMaxD) {
                    const int l = -grp[g];
                    const int g0 = sweeps_down(nu1);
                    const int H = halo_lanes(halo_lanes(g0) + sweeps_down(nu1));
                    const int64_t nq = P->lev[l].N / 4;
                    static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_down2<DIR, T, D>, 0); });
                    launch(P, k_down2<DIR, T, D>, grid_for(P, nq, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]),
                           static_cast<T*>(P->fl[l + 2]), nq, level_consts<T, D>(L(P)[l]),
                           level_consts<T, D>(L(P)[l + 1]), X, nu1, H, (const DevState*)P->st, ct);
                }
            } else {
                const int l = grp[g];
                const int H = halo_lanes(sweeps_down(nu1));
                const int64_t nch = P->lev[l].N / 2;
                static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_down<DIR, T, D>, 0); });
                launch(P, k_down<DIR, T, D>, grid_for(P, nch, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]),
                       static_cast<T*>(P->fl[l + 1]), nch, level_consts<T, D>(L(P)[l]), X, nu1, H,
                       (const DevState*)P->st, ct);
            }
        }
        if (!wcycle && split == 0) mark(kCatCoarse);
        const NvtxRange r_coarse("tmg coarsest level %d", P->lt);
        if (coarse_in_down || wcycle || split != 0) {
            // solved above, or exported / imported by tmg_cycle_down / tmg_cycle_up
        } else if (P->scan_coarsest)
            enqueue_scan<T, T>(P, static_cast<const T*>(P->fl[P->lt]), static_cast<T*>(P->ul[P->lt]), P->lt, T(0),
                               nullptr, P->st);
        else
            launch_tail(P, static_cast<const T*>(P->fl[P->lt]), static_cast<T*>(P->ul[P->lt]), lk, X, nl,
                        P->lev[P->lt].N, nu1, nu2, P->o.gamma, (const DevState*)P->st, (const T*)nullptr);
        if (split == 1) {
            mark(kCatEnd);
            if (nev) *nev = iev;
            return cudaGetLastError();
        }
        for (int g = ng - 1; g >= 0; --g) {
            const NvtxRange r_lev(grp[g] < 0 ? "tmg levels %d,+1 up" : "tmg level %d up", grp[g] < 0 ? -grp[g] : grp[g]);
            mark(kCatUp);
            if (grp[g] < 0) {
                if constexpr (D <= kMaxD) {
                    const int l = -grp[g];
                    // level-l units: the recomputed way down, then level l+1 (recomputed
                    // pre-smoothing, post-smoothing), prolongated, then level-l post-smoothing
                    const int g1 = halo_lanes(sweeps_down(nu1)) + sweeps_up(nu1, nu2);
                    const int H = (2 * g1 + nu2 + 3) / 4;
                    const int64_t nq = P->lev[l].N / 4;
                    static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_up2<DIR, T, D>, 0); });
                    launch(P, k_up2<DIR, T, D>, grid_for(P, nq, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]),
                           static_cast<const T*>(P->ul[l + 2]), static_cast<T*>(P->ul[l]), nq,
                           level_consts<T, D>(L(P)[l]), level_consts<T, D>(L(P)[l + 1]), X, nu1, nu2, H,
                           (const DevState*)P->st);
                }
            } else {
                const int l = grp[g];
                const int H = halo_lanes(sweeps_up(nu1, nu2));
                const int64_t nch = P->lev[l].N / 2;
                static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_up<DIR, T, D>, 0); });
                launch(P, k_up<DIR, T, D>, grid_for(P, nch, H, occ), kNT, 0, static_cast<const T*>(P->fl[l]),
                       static_cast<const T*>(P->ul[l + 1]), static_cast<T*>(P->ul[l]), nch,
                       level_consts<T, D>(L(P)[l]), X, nu1, nu2, H, (const DevState*)P->st);
            }
        }
        if constexpr (kMixed && D <= kMaxD) {   // (wider mixed plans recompute the residual from u)
            if (rl != nullptr) {
                const int H = halo_lanes(sweeps_up(nu1, nu2) + 1 + sweeps_down(nu1));
                const int64_t nch = P->N / 2;
                mark(kCatUp0);
                static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_updown0<DIR, D>, 0); });
                launch(P, k_updown0<DIR, D>, grid_for(P, nch, H, occ), kNT, 0, rT, rl, (const float*)uc1,
                       static_cast<float*>(P->fl[1]), nch, R, level_consts<float, D>(L(P)[0]), X, nu1, nu2, H,
                       P->partials, P->st);
                mark(kCatEnd);
                if (nev) *nev = iev;
                return cudaGetLastError();
            }
        }
        {
            const int H = halo_lanes(sweeps_up(nu1, nu2));
            const int64_t nch = P->N / 2;
            mark(kCatUp0);
            static PerDevice<int> occ_c;
            const int occ = occ_c.get([&] { return resident_per_sm(k_up0<DIR, T, D>, 0); });
            launch(P, k_up0<DIR, T, D>, grid_for(P, nch, H, occ), kNT, 0, (const T*)rT, uc1,
                   nch, level_consts<T, D>(L(P)[0]), X, nu1, nu2, H, (const DevState*)P->st);
        }
        mark(kCatEnd);
        if (nev) *nev = iev;
        return cudaGetLastError();
    }

    static cudaError_t enqueue_normF(tmg_plan* P) {
        k_normF<DIR, D><<<grid_flat(P, P->N), kNT, 0, P->s>>>(P->N, P->partials, P->st);
        return cudaGetLastError();
    }

    static cudaError_t enqueue_residual(tmg_plan* P, const double* f, double u0, const double* u, double* r) {
        k_residual_out<DIR, D><<<grid_flat(P, P->N), kNT, 0, P->s>>>(f, u, u0, r, P->N, res0_consts(P));
        return cudaGetLastError();
    }

    static const tmg_ops* ops() {
        static const tmg_ops o = {sizeof(T),        &tail_bytes,       &upload,        &enqueue_cycle,
                                  &enqueue_cycle_timed, &enqueue_normF, &enqueue_residual, &enqueue_direct,
                                  &enqueue_coarse_io};
        return &o;
    }
};

}  // namespace tmg
