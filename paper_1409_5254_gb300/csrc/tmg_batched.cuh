// Batched solves: many independent problems u' + lambda_i u = f_i with the
// same degree p_t and the same (power-of-two) number of intervals N in one
// set of launches.  Instance i occupies intervals [i N, (i+1) N) of every
// level array ([n_inst][N_l][D], N_l = N / 2^l), so a coarse pair never
// straddles two instances and each level kernel covers all instances at once.
// Differences from the single-problem kernels:
//   * the one-value halo restarts at every instance (u0_i on level 0, zero on
//     the correction levels) -- the lane whose pair opens an instance ignores
//     the shuffled value;
//   * level constants (A^{-1}, g, c, alpha, omega of z_i 2^l) come from a table
//     indexed by (instance, level);
//   * every instance has its own residual norm, stopping test and active flag;
//     the stopping test compacts the instances still iterating into a list,
//     and the level kernels tile only the listed instances' pairs (in list
//     order, as if they were contiguous), so a converged instance costs
//     nothing in later cycles;
//   * the coarsest level (at most 64 intervals) is solved exactly by one warp
//     per instance with a warp-wide scan of the affine interval maps.
#pragma once

#include "tmg_kernels.cuh"

namespace tmg {

struct BatchState {
    const double* F;          // [n_inst][N][D]
    double* u;                // [n_inst][N][D]
    const double* u0;         // [n_inst]
    double tol;
    int max_cycles;
    int cycle;                // residual evaluations done
    int done;                 // 0 running, 1 all converged, 2 some hit the cycle limit, 3 non-finite
    int use_cond;
    unsigned ticket;
    int active_count;
    int failed;               // instances stopped by the cycle limit or a non-finite norm
    int rsel;                 // updated-residual form: buffer holding the current residual pairs
    int n_act;                // instances listed in act_list
    int n_full;               // instances listed in full_list
    int cnt_full;             // kb_finalize's running count of full_list entries
    unsigned long long cond;
};

struct BatchInst {
    double* nF;       // ||F_i||
    double* norm2;    // ||r_i||^2 of the current cycle
    int* active;      // 1 while instance i iterates
    int* cycles;      // cycles applied when instance i stopped
    double* rel;      // its final relative residual
    long long nvals_per_inst;   // values per instance and level-0 vector, N * D
    int* full;        // updated-residual form, next kb_down0: 1 = confirm (norm of F - L u), 2 = recompute r from u
    float* nscale;    // power of two bringing instance i's residual near 1 (FP32 norms)
    int* act_list;    // the instances still iterating (st->n_act of them, any order)
    int* full_list;   // updated-residual form: the instances with full[i] != 0 (st->n_full of them)
    // Variable-length groups: the instances share the hierarchy depth s and
    // instance i has m_i 2^s intervals (m_i <= 2^log2M) in a slot of
    // 2^(log2M + s); the tiles cover only the real intervals.  m[i] per
    // instance; per list, the prefix of m over the listed instances (upre,
    // n_list + 1 entries) and the list position of every unit (u2p, one entry
    // per unit of m).  m == nullptr in power-of-two groups, whose instances
    // all fill their slot.
    const int* m;
    int* upre_a;
    int* u2p_a;
    int* upre_f;
    int* u2p_f;
    int log2M;
};

// Lane `lane` of virtual tile tw over the pairs of the listed instances,
// concatenated in list order (2^log2P pairs per instance): a tile owns `per`
// consecutive pairs after H halo lanes, and may straddle two instances (the
// lane that opens an instance restarts the halo).
struct ListPos {
    int64_t q;      // pair index in the level array
    int64_t inst;   // its instance
    bool inb;       // the lane maps to a listed pair
    bool first;     // the pair opens its instance
};

__device__ __forceinline__ ListPos list_pos(int64_t tw, int per, int H, int lane, const int* __restrict__ list,
                                            int n_list, int log2P, const int* __restrict__ upre = nullptr,
                                            const int* __restrict__ u2p = nullptr, int log2M = 0) {
    const int64_t qv = tw * per + lane - H;
    ListPos p;
    if (upre == nullptr) {
        const int64_t loc = qv & ((int64_t(1) << log2P) - 1);
        p.inb = qv >= 0 && qv < ((int64_t)n_list << log2P);
        p.inst = p.inb ? (int64_t)list[qv >> log2P] : 0;
        p.q = (p.inst << log2P) + loc;
        p.first = loc == 0;
        return p;
    }
    // variable lengths: instance i has m_i units of 2^sh items (pairs or
    // quads), sh = log2P - log2M; the unit's list position comes from u2p
    const int sh = log2P - log2M;
    p.inb = qv >= 0 && qv < ((int64_t)upre[n_list] << sh);
    const int pos = p.inb ? u2p[qv >> sh] : 0;
    p.inst = p.inb ? (int64_t)list[pos] : 0;
    const int64_t loc = p.inb ? qv - ((int64_t)upre[pos] << sh) : 0;
    p.q = (p.inst << log2P) + loc;
    p.first = loc == 0;
    return p;
}

// Tiles covering n_list instances of 2^log2P items (or their real items in a
// variable-length group).
__device__ __forceinline__ int64_t list_tiles(int n_list, int log2P, int per, const int* __restrict__ upre = nullptr,
                                              int log2M = 0) {
    const int64_t items = upre == nullptr ? ((int64_t)n_list << log2P) : ((int64_t)upre[n_list] << (log2P - log2M));
    return (items + per - 1) / per;
}

// Segmented warp sum of v over lanes with the same instance id (ids are
// non-decreasing along the lanes); the first lane of each run adds the run's
// total to norm2[id].
__device__ __forceinline__ void segmented_norm_add(double v, int64_t id, bool valid, double* norm2) {
    const int lane = threadIdx.x & 31;
    if (!valid) id = -1;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double vo = __shfl_down_sync(kFull, v, off);
        const long long io = __shfl_down_sync(kFull, (long long)id, off);
        if (lane + off < 32 && io == id) v += vo;
    }
    const long long ip = __shfl_up_sync(kFull, (long long)id, 1);
    if (valid && (lane == 0 || ip != id)) atomicAdd(&norm2[id], v);
}

constexpr int kBNT = 256;

// Norm contributions without an FP64 operation per value.  A warp whose
// valid lanes all belong to one instance (the common case) sums in FP32 --
// warp_sumsq for raw values, a plain warp sum for squares already scaled near
// 1 -- and adds the total with one atomic; a warp across instances falls back
// to per-lane FP64 partials and segmented_norm_add.
__device__ __forceinline__ bool one_instance(int64_t id, bool valid, unsigned& id0) {
    const unsigned lo = __reduce_min_sync(kFull, valid ? (unsigned)id : 0xFFFFFFFFu);
    const unsigned hi = __reduce_max_sync(kFull, valid ? (unsigned)id : 0u);
    id0 = lo;                 // 0xFFFFFFFF: no valid lane
    return lo >= hi;
}

template <int n>
__device__ __forceinline__ void segmented_sumsq(const float (&v)[n], int64_t id, bool valid, double* norm2) {
    unsigned id0;
    if (one_instance(id, valid, id0)) {
        float x[n];
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = valid ? v[i] : 0.f;
        const double t = warp_sumsq<n>(x);
        if ((threadIdx.x & 31) == 0 && id0 != 0xFFFFFFFFu) atomicAdd(&norm2[id0], t);
        return;
    }
    unsigned em = 0u;                       // lane-own power-of-two scale, as in warp_sumsq
#pragma unroll
    for (int i = 0; i < n; ++i) em = max(em, (__float_as_uint(v[i]) >> 23) & 0xFFu);
    int k = (int)em - 127;
    k = k < -126 ? -126 : (k > 126 ? 126 : k);
    const float s = __uint_as_float((unsigned)(127 - k) << 23);
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < n; ++i) {
        const float x = v[i] * s;
        ss = fmaf(x, x, ss);
    }
    segmented_norm_add(f2d_int(ss) * __hiloint2double((2 * k + 1023) << 20, 0), id, valid, norm2);
}

__device__ __forceinline__ void segmented_add_f(float v, int64_t id, bool valid, double* norm2) {
    unsigned id0;
    if (one_instance(id, valid, id0)) {
        float t = valid ? v : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(kFull, t, off);
        if ((threadIdx.x & 31) == 0 && id0 != 0xFFFFFFFFu) atomicAdd(&norm2[id0], f2d_int(t));
        return;
    }
    segmented_norm_add(f2d_int(v), id, valid, norm2);
}


// Level 0: residual of every active instance (float pairs for the mixed form,
// FP64 otherwise), norms, r stored in T, zero-start pre-smoothing and
// restriction onto level 1 (fc == nullptr when level 0 is the coarsest).
// In the first cycle of a solve u = 0, so u is not read and r = F (with
// u0_i a in each instance's first interval); the mixed form splits F into
// float pairs directly.
//
// Without rlo the instances of act_list are processed.  With rlo != nullptr
// (mixed form with an updated residual) only those of full_list are:
// full[i] = 2 recomputes the residual from u (the start of the solve, or
// after a failed confirmation) and stores it as a float pair (rT, rlo; low
// parts encoded by lo_encode) into buffer st->rsel of two (nchunks * 2 * D
// values each), with its restriction; full[i] = 1 only confirms an updated
// residual that met the tolerance: its norm, nothing stored.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_down0(T* __restrict__ rT, short* __restrict__ rlo, T* __restrict__ fc,
                                                 int64_t nchunks, int log2N, const LevelK<T, D>* __restrict__ lk,
                                                 const Res0* __restrict__ res, int nlev, Xfer<T, D> X, int nu1, int H,
                                                 const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    if (rlo != nullptr) {
        const int64_t nv = nchunks * 2 * D;
        rT += st->rsel * nv;
        rlo += st->rsel * nv;
    }
    const double* __restrict__ F = st->F;
    const double* __restrict__ uu = st->u;
    const bool start = st->cycle == 0;
    constexpr bool kMixed = std::is_same<T, float>::value;
    const int* __restrict__ list = rlo != nullptr ? bi.full_list : bi.act_list;
    const int n_list = rlo != nullptr ? st->n_full : st->n_act;
    const int* __restrict__ upre = bi.m == nullptr ? nullptr : rlo != nullptr ? bi.upre_f : bi.upre_a;
    const int* __restrict__ u2p = rlo != nullptr ? bi.u2p_f : bi.u2p_a;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int64_t ntiles = list_tiles(n_list, log2N - 1, per, upre, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, list, n_list, log2N - 1, upre, u2p, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const bool own = act && lane >= H;
        const bool keep = act && (rlo == nullptr || bi.full[inst] == 2);   // store r and its restriction
        const LevelK<T, D> K = lk[inst * nlev];
        const Res0 R = res[inst];
        double uv[2][D], Fv[2][D];
        short rq[2][D];
        load_pair<double, D>(uu, q, act && !start, uv);
        load_pair<double, D>(F, q, act, Fv);
        const double u0i = act ? st->u0[inst] : 0.0;
        T rt[2][D];
        if constexpr (kMixed) {
            float r0[D], r1[D], l0[D], l1[D];
            if (start) {
                if (first) {
#pragma unroll
                    for (int k = 0; k < D; ++k) Fv[0][k] += acoef<DIR>(k, u0i);
                }
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const ff s0 = split_d(Fv[0][k]), s1 = split_d(Fv[1][k]);
                    const ff n0 = two_sum(s0.hi, s0.lo), n1 = two_sum(s1.hi, s1.lo);   // rounded high parts
                    r0[k] = n0.hi;
                    l0[k] = n0.lo;
                    r1[k] = n1.hi;
                    l1[k] = n1.lo;
                }
            } else {
                ff us0[D], us1[D], sE0, sB0, sE1, sB1;
                small_sums<DIR, D>(uv[0], us0, sE0, sB0);
                small_sums<DIR, D>(uv[1], us1, sE1, sB1);
                double up0 = shfl_prev(uv[1][0]);
                ff sp{shfl_prev(sB1.hi), shfl_prev(sB1.lo)};
                if (first) {                 // the value before the instance's first interval: b^T u = u0_i
                    up0 = u0i;
                    sp = ff{0.f, 0.f};
                }
                residual0_ff<DIR, D>(Fv[0], uv[0], us0, up0, sp, sE0, R, r0, l0);
                residual0_ff<DIR, D>(Fv[1], uv[1], us1, uv[0][0], sB0, sE1, R, r1, l1);
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                rt[0][k] = act ? r0[k] : 0.f;
                rt[1][k] = act ? r1[k] : 0.f;
                rq[0][k] = lo_encode(r0[k], l0[k]);
                rq[1][k] = lo_encode(r1[k], l1[k]);
            }
            float sq[2 * D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                sq[k] = rt[0][k];
                sq[D + k] = rt[1][k];
            }
            segmented_sumsq<2 * D>(sq, inst, own, bi.norm2);
        } else {
            double r[2][D];
            const double b0 = bval<DIR, double, D>(uv[0]);
            const double b1 = bval<DIR, double, D>(uv[1]);
            double ep = shfl_prev(b1);
            if (first) ep = u0i;
            const double E0 = DIR == 0 ? b0 : endval<double, D>(uv[0]);
            const double E1 = DIR == 0 ? b1 : endval<double, D>(uv[1]);
            residual0<DIR, D>(Fv[0], uv[0], ep, E0, R, r[0]);
            residual0<DIR, D>(Fv[1], uv[1], b0, E1, R, r[1]);
            double ss = 0.0;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    rt[i][k] = act ? (T)r[i][k] : T(0);
                    ss = fma((double)rt[i][k], (double)rt[i][k], ss);
                }
            segmented_norm_add(ss, inst, own, bi.norm2);
        }
        if (own && keep) {
            store_pair<T, D>(rT, q, rt);
            if constexpr (kMixed) {
                if (rlo != nullptr) store_pair<short, D>(rlo, q, rq);
            }
        }
        if (fc != nullptr && __any_sync(kFull, keep)) {
            T h[2][D], c[2][D], w[2][D], rc[2][D], out[D];
            presmooth_zero<DIR, T, D>(K, rt, h, c, w, nu1, first);
            residual_tracked<DIR, T, D>(rt, c, w, rc, first);
            restrict_pair<T, D>(X, rc, out);
            if (own && keep) VecIO<T, D>::store(fc + q * D, out);
        }
    }
}

// Per-instance stopping test.
//   kFinPlain: after the level-0 residual of cycle k, computed from u.
//   kFinFull (updated-residual form): after kb_down0 evaluated the residual of
//     the instances flagged full -- the start of the solve, a confirmation, or
//     the recomputation after a failed one; only those instances are tested.
//   kFinUpdated: after kb_updown0 updated every active instance's residual:
//     meeting tol flags the instance for confirmation instead of stopping it;
//     the cycle counter advances and the residual buffers swap.
// Every warp appends its instances that keep iterating to act_list (and,
// after kFinUpdated, the flagged ones to full_list) with one atomic each; the
// last block publishes the counts for the next kernels.
static __global__ void __launch_bounds__(kBNT) kb_finalize(BatchState* st, BatchInst bi, int64_t n_inst,
                                                    int mode = kFinPlain) {
    if (st->done) {                          // a finished batch must also end the graph loop
        if (st->use_cond && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, 0u);
        return;
    }
    const int k = mode == kFinUpdated ? st->cycle + 1 : st->cycle;   // corrections applied
    const int lane = threadIdx.x & 31;
    int fail_local = 0;
    const int64_t stride = (int64_t)gridDim.x * kBNT;
    for (int64_t base = (int64_t)blockIdx.x * kBNT + (threadIdx.x & ~31); base < n_inst; base += stride) {
        const int64_t i = base + lane;            // the warp stays converged: lists are built by ballot
        bool keep = false;
        if (i < n_inst && bi.active[i]) {
            if (mode == kFinFull && !bi.full[i]) {
                keep = true;
            } else {
                // kb_updown0 sums squares scaled by nscale[i]^2
                const double nrm = sqrt(bi.norm2[i]) / (mode == kFinUpdated ? (double)bi.nscale[i] : 1.0);
                bi.norm2[i] = 0.0;
                if (k == 0 && mode != kFinUpdated) bi.nF[i] = nrm;
                const double nF = bi.nF[i];
                const double rel = nF > 0.0 ? nrm / nF : nrm;
                const bool bad = !(rel == rel) || rel > 1.0e300;
                if (mode != kFinPlain) {
                    // scale of the next FP32 norm of this instance
                    const double rms = nrm / sqrt((double)bi.nvals_per_inst);
                    int ex = 0;
                    if (rms > 0.0 && rms < 1.0e300) ex = -ilogb(rms);
                    ex = ex < -100 ? -100 : (ex > 100 ? 100 : ex);
                    bi.nscale[i] = ldexpf(1.0f, ex);
                }
                const bool met = rel <= st->tol;
                if (mode == kFinUpdated && !bad && met) {
                    // confirm from u at the start of the next cycle (a pending full
                    // recomputation, flag 2, confirms as well)
                    if (bi.full[i] == 0) bi.full[i] = 1;
                    keep = true;
                } else if (bad || met || k >= st->max_cycles) {
                    bi.active[i] = 0;
                    bi.cycles[i] = k;
                    bi.rel[i] = rel;
                    if (bad || !met) ++fail_local;
                } else {
                    // a failed confirmation (flag 1) recomputes the residual in the next
                    // cycle; this cycle goes on with the updated one
                    if (mode == kFinFull) bi.full[i] = bi.full[i] == 1 ? 2 : 0;
                    keep = true;
                }
            }
        }
        const bool to_full = keep && mode == kFinUpdated && bi.full[i] != 0;
        const unsigned ka = __ballot_sync(kFull, keep);
        const unsigned kf = __ballot_sync(kFull, to_full);
        int oa = 0, of = 0;
        if (lane == 0) {
            if (ka) oa = atomicAdd(&st->active_count, __popc(ka));
            if (kf) of = atomicAdd(&st->cnt_full, __popc(kf));
        }
        oa = __shfl_sync(kFull, oa, 0);
        of = __shfl_sync(kFull, of, 0);
        const unsigned below = (1u << lane) - 1u;
        if (keep) bi.act_list[oa + __popc(ka & below)] = (int)i;
        if (to_full) bi.full_list[of + __popc(kf & below)] = (int)i;
    }
    __shared__ int sf;
    __shared__ int last;
    if (threadIdx.x == 0) sf = 0;
    __syncthreads();
    if (fail_local) atomicAdd(&sf, fail_local);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sf) atomicAdd(&st->failed, sf);
        __threadfence();
        last = (atomicAdd(&st->ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const int remaining = atomicAdd(&st->active_count, 0);
    st->n_act = remaining;
    st->n_full = atomicAdd(&st->cnt_full, 0);   // zero unless kFinUpdated flagged some
    st->active_count = 0;
    st->cnt_full = 0;
    st->ticket = 0u;
    if (mode == kFinPlain) st->cycle = k + 1;
    if (mode == kFinUpdated) {
        st->cycle = k;
        st->rsel ^= 1;      // kb_updown0 wrote the other buffer
    }
    if (remaining == 0) {
        st->done = st->failed ? 2 : 1;
        if (st->use_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)st->cond, 0u);
    }
}

// Variable-length groups, after kb_finalize: the unit prefix of an instance
// list and the list position of every unit, for list_pos.  Block 0 serves
// act_list, block 1 (when launched) full_list.  Each thread takes a
// contiguous chunk of the list: sums its units, the block scans the chunk
// sums, and the thread writes its chunk's prefixes and unit positions.
constexpr int kUnitsNT = 1024;

static __global__ void __launch_bounds__(kUnitsNT) kb_units(const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    const bool act = blockIdx.x == 0;
    const int* __restrict__ list = act ? bi.act_list : bi.full_list;
    const int n = act ? st->n_act : st->n_full;
    int* __restrict__ upre = act ? bi.upre_a : bi.upre_f;
    int* __restrict__ u2p = act ? bi.u2p_a : bi.u2p_f;
    const int chunk = (n + kUnitsNT - 1) / kUnitsNT;
    const int j0 = min(n, (int)threadIdx.x * chunk), j1 = min(n, j0 + chunk);
    int own = 0;
    for (int j = j0; j < j1; ++j) own += bi.m[list[j]];
    // block-wide exclusive scan of the chunk sums
    __shared__ int wsum[kUnitsNT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    int u = (warp > 0 ? wsum[warp - 1] : 0) + x - own;
    for (int j = j0; j < j1; ++j) {
        upre[j] = u;
        const int mj = bi.m[list[j]];
        for (int k = 0; k < mj; ++k) u2p[u + k] = j;
        u += mj;
    }
    if (threadIdx.x == kUnitsNT - 1) upre[n] = wsum[kUnitsNT / 32 - 1];
}

template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_down(const T* __restrict__ f, T* __restrict__ fc, int64_t nchunks,
                                                int log2N, const LevelK<T, D>* __restrict__ lk, int nlev, int level,
                                                Xfer<T, D> X, int nu1, int H, const BatchState* __restrict__ st,
                                                BatchInst bi) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 1, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 1, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const LevelK<T, D> K = lk[inst * nlev + level];
        T fv[2][D], h[2][D], u[2][D], w[2][D], r[2][D], out[D];
        load_pair<T, D>(f, q, act, fv);
        presmooth_zero<DIR, T, D>(K, fv, h, u, w, nu1, first);
        residual_tracked<DIR, T, D>(fv, u, w, r, first);
        restrict_pair<T, D>(X, r, out);
        if (act && lane >= H) VecIO<T, D>::store(fc + q * D, out);
    }
}

template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_up(const T* __restrict__ f, const T* __restrict__ uc, T* __restrict__ u,
                                              int64_t nchunks, int log2N, const LevelK<T, D>* __restrict__ lk,
                                              int nlev, int level, Xfer<T, D> X, int nu1, int nu2, int H,
                                              const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 1, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 1, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const LevelK<T, D> K = lk[inst * nlev + level];
        T fv[2][D], h[2][D], v[2][D], w[2][D], c[D];
        load_pair<T, D>(f, q, act, fv);
        load_one<T, D>(uc, q, act, c);
        presmooth_zero<DIR, T, D>(K, fv, h, v, w, nu1, first);
        prolong_add<T, D>(X, c, v);
        postsmooth<DIR, T, D>(K, h, v, nu2, first);
        if (act && lane >= H) store_pair<T, D>(u, q, v);
    }
}

// W-cycles (gamma = 2): the second visit of level l >= 1 under the same
// parent visit starts from the first visit's result u_in (as k_down_nz /
// k_up_nz), over the listed instances, the halo restarting at each instance.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_down_nz(const T* __restrict__ f, const T* __restrict__ u_in,
                                                   T* __restrict__ fc, int log2N, const LevelK<T, D>* __restrict__ lk,
                                                   int nlev, int level, Xfer<T, D> X, int nu1, int H,
                                                   const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 1, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 1, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const LevelK<T, D> K = lk[inst * nlev + level];
        T fv[2][D], h[2][D], u[2][D], w[2][D], r[2][D], out[D];
        load_pair<T, D>(f, q, act, fv);
        load_pair<T, D>(u_in, q, act, u);
        presmooth_from<DIR, T, D>(K, fv, h, u, w, nu1, first);
        residual_tracked<DIR, T, D>(fv, u, w, r, first);
        restrict_pair<T, D>(X, r, out);
        if (act && lane >= H) VecIO<T, D>::store(fc + q * D, out);
    }
}

template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_up_nz(const T* __restrict__ f, const T* __restrict__ u_in,
                                                 const T* __restrict__ uc, T* __restrict__ u_out, int log2N,
                                                 const LevelK<T, D>* __restrict__ lk, int nlev, int level,
                                                 Xfer<T, D> X, int nu1, int nu2, int H,
                                                 const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 1, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 1, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const LevelK<T, D> K = lk[inst * nlev + level];
        T fv[2][D], h[2][D], v[2][D], w[2][D], c[D];
        load_pair<T, D>(f, q, act, fv);
        load_pair<T, D>(u_in, q, act, v);
        load_one<T, D>(uc, q, act, c);
        presmooth_from<DIR, T, D>(K, fv, h, v, w, nu1, first);
        prolong_add<T, D>(X, c, v);
        postsmooth<DIR, T, D>(K, h, v, nu2, first);
        if (act && lane >= H) store_pair<T, D>(u_out, q, v);
    }
}

// Levels l and l+1 of the way down in one kernel, over the listed
// instances (as k_down2): each lane holds four level-l intervals (a quad,
// which never straddles an instance), pre-smooths, restricts onto two level
// l+1 intervals, pre-smooths those and restricts onto one level-(l+2)
// interval; f_{l+1} is never stored.  log2N: intervals per instance at level l.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_down2(const T* __restrict__ f, T* __restrict__ fcc, int log2N,
                                                 const LevelK<T, D>* __restrict__ lk, int nlev, int level,
                                                 Xfer<T, D> X, int nu1, int H, const BatchState* __restrict__ st,
                                                 BatchInst bi) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 2, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 2, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const LevelK<T, D> K0 = lk[inst * nlev + level];
        const LevelK<T, D> K1 = lk[inst * nlev + level + 1];
        T fv[4][D], h[4][D], u[4][D], w[4][D], r[4][D];
        load_m<T, D, 4>(f, q, act, fv);
        presmooth_zero_m<DIR, T, D, 4>(K0, fv, h, u, w, nu1, first);
        residual_tracked_m<DIR, T, D, 4>(fv, u, w, r, first);
        T f1[2][D], h1[2][D], u1[2][D], w1[2][D], r1[2][D], out[D];
        restrict2<T, D>(X, r[0], r[1], f1[0]);
        restrict2<T, D>(X, r[2], r[3], f1[1]);
        presmooth_zero<DIR, T, D>(K1, f1, h1, u1, w1, nu1, first);
        residual_tracked<DIR, T, D>(f1, u1, w1, r1, first);
        restrict_pair<T, D>(X, r1, out);
        if (act && lane >= H) VecIO<T, D>::store(fcc + q * D, out);
    }
}

// Levels l+1 and l of the way up in one kernel (as k_up2): recompute level
// l's way down and level l+1's right-hand side and pre-smoothing from f_l,
// add the prolongated level-(l+2) correction ucc, post-smooth on level l+1,
// prolongate onto level l, post-smooth there and write u_l.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_up2(const T* __restrict__ f, const T* __restrict__ ucc,
                                               T* __restrict__ u, int log2N, const LevelK<T, D>* __restrict__ lk,
                                               int nlev, int level, Xfer<T, D> X, int nu1, int nu2, int H,
                                               const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 2, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 2, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const LevelK<T, D> K0 = lk[inst * nlev + level];
        const LevelK<T, D> K1 = lk[inst * nlev + level + 1];
        T fv[4][D], h[4][D], v[4][D], w[4][D], r[4][D], cc[D];
        load_m<T, D, 4>(f, q, act, fv);
        load_one<T, D>(ucc, q, act, cc);
        presmooth_zero_m<DIR, T, D, 4>(K0, fv, h, v, w, nu1, first);
        residual_tracked_m<DIR, T, D, 4>(fv, v, w, r, first);
        T f1[2][D], h1[2][D], v1[2][D], w1[2][D];
        restrict2<T, D>(X, r[0], r[1], f1[0]);
        restrict2<T, D>(X, r[2], r[3], f1[1]);
        presmooth_zero<DIR, T, D>(K1, f1, h1, v1, w1, nu1, first);
        prolong_add<T, D>(X, cc, v1);
        postsmooth<DIR, T, D>(K1, h1, v1, nu2, first);
        prolong_add2<T, D>(X, v1[0], v[0], v[1]);
        prolong_add2<T, D>(X, v1[1], v[2], v[3]);
        postsmooth_m<DIR, T, D, 4>(K0, h, v, nu2, first);
        if (act && lane >= H) store_m<T, D, 4>(u, q, v);
    }
}

template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_up0(const T* __restrict__ rT, const T* __restrict__ uc, int64_t nchunks,
                                               int log2N, const LevelK<T, D>* __restrict__ lk, int nlev, Xfer<T, D> X,
                                               int nu1, int nu2, int H, const BatchState* __restrict__ st,
                                               BatchInst bi) {
    if (st->done) return;
    double* __restrict__ uu = st->u;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 1, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 1, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const bool own = act && lane >= H;
        const LevelK<T, D> K = lk[inst * nlev];
        T rt[2][D], h[2][D], c[2][D], w[2][D], cc[D];
        double uv[2][D];
        load_pair<T, D>(rT, q, act, rt);
        load_one<T, D>(uc, q, act, cc);
        load_pair<double, D>(uu, q, own, uv);
        presmooth_zero<DIR, T, D>(K, rt, h, c, w, nu1, first);
        prolong_add<T, D>(X, cc, c);
        postsmooth<DIR, T, D>(K, h, c, nu2, first);
        if (own) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    if constexpr (std::is_same<T, float>::value) uv[i][k] += f2d_int(c[i][k]);
                    else uv[i][k] += (double)c[i][k];
                }
            store_pair<double, D>(uu, q, uv);
        }
    }
}

// Exact solve of the coarsest level (Nc <= 64 intervals per instance), one
// warp per instance: lane j holds intervals 2j and 2j+1; the affine maps
// e_n = alpha e_{n-1} + c^T f_n (e_{-1} = 0) are combined by a warp scan,
// then u_n = A^{-1} f_n + g e_{n-1}.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_coarse(const T* __restrict__ f, T* __restrict__ u, int64_t n_inst, int Nc,
                                                  const LevelK<T, D>* __restrict__ lk, int nlev, int level,
                                                  const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * kBNT) >> 5;
    const int n_list = st->n_act;
    const int slot = Nc;
    for (int64_t j = wid; j < n_list; j += nw) {
        const int64_t inst = bi.act_list[j];
        const LevelK<T, D> K = lk[inst * nlev + level];
        if (bi.m != nullptr) Nc = bi.m[inst];    // variable lengths: the instance's own coarsest level
        const int n0 = 2 * lane, n1 = 2 * lane + 1;
        T f0[D], f1[D];
        load_one<T, D>(f + inst * (int64_t)slot * D, n0, n0 < Nc, f0);
        load_one<T, D>(f + inst * (int64_t)slot * D, n1, n1 < Nc, f1);
        const T b0 = dotc<T, D>(K.c, f0), b1 = dotc<T, D>(K.c, f1);
        T A = n1 < Nc ? K.alpha * K.alpha : (n0 < Nc ? K.alpha : T(1));
        T B = n1 < Nc ? fma(K.alpha, b0, b1) : (n0 < Nc ? b0 : T(0));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const T Ap = __shfl_up_sync(kFull, A, off);
            const T Bp = __shfl_up_sync(kFull, B, off);
            if (lane >= off) {
                B = fma(A, Bp, B);
                A = A * Ap;
            }
        }
        T ein = __shfl_up_sync(kFull, B, 1);        // e before interval 2j (inclusive prefix of lane j-1)
        if (lane == 0) ein = T(0);
        T x0[D], x1[D];
        matvec<T, D>(K.Ainv, f0, x0);
        matvec<T, D>(K.Ainv, f1, x1);
        const T emid = fma(K.alpha, ein, b0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            x0[k] = fma(K.g[k], ein, x0[k]);
            x1[k] = fma(K.g[k], emid, x1[k]);
        }
        T* ub = u + inst * (int64_t)slot * D;
        if (n0 < Nc) VecIO<T, D>::store(ub + n0 * D, x0);
        if (n1 < Nc) VecIO<T, D>::store(ub + n1 * D, x1);
    }
}

// Level 0 of the mixed form with an updated residual (see k_updown0): the way
// up of one cycle fused with the way down of the next, for every active
// instance; r -= L c on the residual pairs (read from buffer st->rsel, written
// to the other), u += c in FP64, per-instance FP32 norms scaled by nscale[i].
template <int DIR, int D>
__global__ void __launch_bounds__(kBNT, D <= 2 ? 4 : 2) kb_updown0(float* __restrict__ rh, short* __restrict__ rl,
                                                                   const float* __restrict__ uc,
                                                                   float* __restrict__ fc, int64_t nchunks,
                                                                   int log2N,
                                                                   const LevelK<float, D>* __restrict__ lk,
                                                                   const Res0* __restrict__ res, int nlev,
                                                                   Xfer<float, D> X, int nu1, int nu2, int H,
                                                                   const BatchState* __restrict__ st,
                                                                   BatchInst bi) {
    if (st->done) return;
    double* __restrict__ uu = st->u;
    const int64_t nv = nchunks * 2 * D;
    const int sel = st->rsel;
    const float* __restrict__ rh_in = rh + sel * nv;
    const short* __restrict__ rl_in = rl + sel * nv;
    float* __restrict__ rh_out = rh + (1 - sel) * nv;
    short* __restrict__ rl_out = rl + (1 - sel) * nv;
    const int lane = threadIdx.x & 31;
    const int per = 32 - H;
    const int n_list = st->n_act;
    const int64_t ntiles = list_tiles(n_list, log2N - 1, per, bi.m ? bi.upre_a : nullptr, bi.log2M);
    const int64_t nwarps = ((int64_t)gridDim.x * kBNT) >> 5;
    for (int64_t tw = ((int64_t)blockIdx.x * kBNT + threadIdx.x) >> 5; tw < ntiles; tw += nwarps) {
        const ListPos P = list_pos(tw, per, H, lane, bi.act_list, n_list, log2N - 1, bi.m ? bi.upre_a : nullptr, bi.u2p_a, bi.log2M);
        const int64_t q = P.q, inst = P.inst;
        const bool act = P.inb, first = P.first;
        const bool own = act && lane >= H;
        const LevelK<float, D> K = lk[inst * nlev];
        const Res0 R = res[inst];
        const float nsc = bi.nscale[inst];
        float r[2][D], rlo[2][D], cc[D];
        short rq[2][D];
        double uv[2][D];
        load_pair<float, D>(rh_in, q, act, r);
        load_pair<short, D>(rl_in, q, act, rq);
        load_one<float, D>(uc, q, act, cc);
        load_pair<double, D>(uu, q, own, uv);
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int k = 0; k < D; ++k) rlo[i][k] = lo_decode(r[i][k], rq[i][k]);
        float h[2][D], c[2][D], w[2][D];
        presmooth_zero<DIR, float, D>(K, r, h, c, w, nu1, first);
        prolong_add<float, D>(X, cc, c);
        postsmooth<DIR, float, D>(K, h, c, nu2, first);
        if (!act) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) c[i][k] = 0.f;
        }
        const ff b0 = bsum_ff<DIR, D>(c[0]);
        const ff b1 = bsum_ff<DIR, D>(c[1]);
        ff bp{shfl_prev(b1.hi), shfl_prev(b1.lo)};
        if (first) bp = ff{0.f, 0.f};            // the correction starts from zero at every instance
        residual_update_ff<DIR, D>(r[0], rlo[0], c[0], bp, R);
        residual_update_ff<DIR, D>(r[1], rlo[1], c[1], b0, R);
        float ssf = 0.f;
        if (own) {
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    uv[i][k] += f2d_int(c[i][k]);
                    const float v = r[i][k] * nsc;
                    ssf = fmaf(v, v, ssf);
                    rq[i][k] = lo_encode(r[i][k], rlo[i][k]);
                }
            store_pair<double, D>(uu, q, uv);
            store_pair<float, D>(rh_out, q, r);
            store_pair<short, D>(rl_out, q, rq);
        }
        segmented_add_f(ssf, inst, own, bi.norm2);   // in units of nscale^2 (kb_finalize)
        // the next cycle's way down on L c' = r
        float rc[2][D], out[D];
        presmooth_zero<DIR, float, D>(K, r, h, c, w, nu1, first);
        residual_tracked<DIR, float, D>(r, c, w, rc, first);
        restrict_pair<float, D>(X, rc, out);
        if (own) VecIO<float, D>::store(fc + q * D, out);
    }
}

// u += c on level 0 when level 0 is itself the coarsest level.
template <typename T, int D>
__global__ void __launch_bounds__(kBNT) kb_update0(const T* __restrict__ c, int64_t n_values, int values_per_inst,
                                                   const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    double* __restrict__ uu = st->u;
    for (int64_t i = (int64_t)blockIdx.x * kBNT + threadIdx.x; i < n_values; i += (int64_t)gridDim.x * kBNT) {
        if (!bi.active[i / values_per_inst]) continue;
        if constexpr (std::is_same<T, float>::value) uu[i] += f2d_int(c[i]);
        else uu[i] += (double)c[i];
    }
}

}  // namespace tmg

namespace tmg {

// ------------------------------------------- one CTA per small instance --
//
// The whole solve of one instance in one CTA's shared memory: F and u in
// FP64, the cycle's level hierarchy in the cycle precision (the on-chip
// solver's layout, tail_view), every cycle in the same launch.  Per cycle:
// r = F - L u in FP64 and its norm (block reduction), the stopping test, one
// cycle on L c = r from a zero start (tail_cycle), u += c in FP64.  Blocks
// loop over the instances; the last block to finish sets the group's state.

// Shared memory of the CTA form for a padded length Ng and nlev levels.
template <typename T, int D>
inline size_t cta_smem_bytes(int64_t Ng, int nlev) {
    return (size_t)2 * Ng * D * sizeof(double) + 32 * sizeof(double) + tail_smem_bytes<T, D>(Ng, nlev);
}

// Sum of v over the block, returned to every thread.
__device__ __forceinline__ double block_sum_all(double v, double* red) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();   // red may still be read from the previous call
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kTailNT) kb_cta_solve(const double* __restrict__ F, double* __restrict__ u,
                                                        const double* __restrict__ u0, int64_t n_inst, int Ng,
                                                        int nlev, const LevelK<T, D>* __restrict__ lk,
                                                        const Res0* __restrict__ res, Xfer<T, D> X, int nu1, int nu2,
                                                        int gamma, BatchState* st, BatchInst bi) {
    extern __shared__ __align__(16) unsigned char cta_smem[];
    double* Fs = reinterpret_cast<double*>(cta_smem);
    double* us = Fs + (int64_t)Ng * D;
    double* red = us + (int64_t)Ng * D;
    const int64_t slot = (int64_t)Ng * D;
    const double tol = st->tol;
    const int max_cycles = st->max_cycles;
    int failed = 0;
    for (int64_t inst = blockIdx.x; inst < n_inst; inst += gridDim.x) {
        // variable lengths: the instance's own intervals (its hierarchy has
        // the group's nlev levels down to m_i intervals)
        const int Ni = bi.m != nullptr ? bi.m[inst] << (nlev - 1) : Ng;
        const TailView<T, D> V = tail_view<T, D>(reinterpret_cast<T*>(red + 32), Ni, nlev);
        if (!tail_view_fits<T, D>(V, cta_smem)) continue;   // debug build: layout outside shared memory
        const int64_t nv = (int64_t)Ni * D;
        const LevelK<T, D>* lki = lk + inst * nlev;
        const Res0 R = res[inst];
        const double u0i = u0[inst];
        for (int64_t i = threadIdx.x; i < nv; i += kTailNT) {
            Fs[i] = F[inst * slot + i];
            us[i] = 0.0;
        }
        __syncthreads();
        double nF = 0.0, rel = 0.0;
        int k = 0;
        while (true) {
            double ss = 0.0;
            for (int64_t n = threadIdx.x; n < Ni; n += kTailNT) {
                double uv[D], Fv[D], r[D];
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    uv[q] = us[n * D + q];
                    Fv[q] = Fs[n * D + q];
                }
                double ep = u0i;
                if (n > 0) {
                    double up[D];
#pragma unroll
                    for (int q = 0; q < D; ++q) up[q] = us[(n - 1) * D + q];
                    ep = bval<DIR, double, D>(up);
                }
                residual0<DIR, D>(Fv, uv, ep, endval<double, D>(uv), R, r);
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    V.f[0][n * D + q] = (T)r[q];
                    ss = fma(r[q], r[q], ss);
                }
            }
            const double nrm = sqrt(block_sum_all(ss, red));   // ends synchronised: V.f[0] complete
            if (k == 0) nF = nrm;
            rel = nF > 0.0 ? nrm / nF : nrm;
            if (!(rel == rel) || rel > 1.0e300 || rel <= tol || k >= max_cycles) break;
            tail_cycle<DIR, T, D>(V, lki, X, nlev, nu1, nu2, gamma);
            for (int64_t i = threadIdx.x; i < nv; i += kTailNT) us[i] += (double)V.u[0][i];
            __syncthreads();
            ++k;
        }
        for (int64_t i = threadIdx.x; i < nv; i += kTailNT) u[inst * slot + i] = us[i];
        if (threadIdx.x == 0) {
            bi.cycles[inst] = k;
            bi.rel[inst] = rel;
            bi.active[inst] = 0;
            if (!(rel <= tol)) ++failed;
        }
        __syncthreads();
    }
    // the last block to finish records the outcome of the group
    __shared__ int last;
    if (threadIdx.x == 0) {
        if (failed) atomicAdd(&st->failed, failed);
        __threadfence();
        last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        st->ticket = 0u;
        st->done = atomicAdd(&st->failed, 0) ? 2 : 1;
    }
}

// W-cycles over the grid schedule: the levels from lt down of every listed
// instance in one CTA's shared memory (the on-chip solver's tail_cycle, whose
// W recursion runs in place), one CTA per instance at a time.  f: level-lt
// right-hand sides [n][Nt][D]; u_out receives the corrections; u_init (or
// nullptr for a zero start) holds the first visit's result on a second visit.
template <int DIR, typename T, int D>
__global__ void __launch_bounds__(kTailNT) kb_tail(const T* __restrict__ f, T* __restrict__ u_out,
                                                   const T* __restrict__ u_init, const LevelK<T, D>* __restrict__ lk,
                                                   int nlev, int lt, Xfer<T, D> X, int Nt, int nu1, int nu2,
                                                   int gamma, const BatchState* __restrict__ st, BatchInst bi) {
    if (st->done) return;
    extern __shared__ __align__(16) unsigned char kb_tail_smem[];
    const int nl = nlev - lt;
    const int64_t slot = (int64_t)Nt * D;
    const int n_list = st->n_act;
    for (int64_t j = blockIdx.x; j < n_list; j += gridDim.x) {
        const int64_t inst = bi.act_list[j];
        // variable lengths: the instance's own intervals on level lt
        const int Ni = bi.m != nullptr ? bi.m[inst] << (nl - 1) : Nt;
        const TailView<T, D> V = tail_view<T, D>(reinterpret_cast<T*>(kb_tail_smem), Ni, nl);
        if (!tail_view_fits<T, D>(V, kb_tail_smem)) continue;   // debug build: layout outside shared memory
        const int64_t nv = (int64_t)Ni * D;
        const int64_t off = inst * slot;
        for (int64_t i = threadIdx.x; i < nv; i += kTailNT) {
            V.f[0][i] = f[off + i];
            if (u_init != nullptr) V.u[0][i] = u_init[off + i];
        }
        __syncthreads();
        tail_cycle<DIR, T, D>(V, lk + inst * nlev + lt, X, nl, nu1, nu2, gamma, u_init != nullptr);
        for (int64_t i = threadIdx.x; i < nv; i += kTailNT) u_out[off + i] = V.u[0][i];
        __syncthreads();
    }
}

}  // namespace tmg
