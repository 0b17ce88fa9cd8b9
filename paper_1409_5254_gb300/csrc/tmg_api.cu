// C ABI of the time-multigrid library: plan set-up (FP64 host arithmetic),
// workspaces, the CUDA-graph solve loop, and the public entry points.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "tmg_bounds.h"
#include "tmg_nvtx.h"
#include "tmg_plan.h"
#include "tmg_setup_math.h"

namespace {

using namespace tmg_host;

thread_local int g_last_cuda = 0;

tmg_status cuda_fail(cudaError_t e) {
    g_last_cuda = (int)e;
    return TMG_ECUDA;
}

#define TMG_CUDA(call)                                  \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) return cuda_fail(_e);    \
    } while (0)

// Same hierarchy rule as the textbook cycle: coarsen while the level has an
// even number of intervals, more than n_min of them, and the level cap allows.
int count_levels(int64_t N, int64_t n_min, int max_levels) {
    int L = 1;
    int64_t n = N;
    while ((max_levels <= 0 || L < max_levels) && n % 2 == 0 && n > n_min && L < tmg::kMaxLevels) {
        n /= 2;
        ++L;
    }
    return L;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Degrees accepted as arguments (larger ones are rejected as invalid; those
// between the built ones as unsupported).
const int kMaxDegree = 20;

const int64_t kTailNmax = 8192;
// Default largest level of the on-chip coarse solver: small, because inside
// a graph with programmatic dependent launch a streaming kernel on a small
// level costs less than a level of the single-CTA solver; W-cycles need the
// on-chip solver from level 1 and take the largest one.
const int64_t kTailDefaultV = 64;

// Argument checks shared by tmg_setup and tmg_plan_shape; fixes the options
// a degree implies (p_t = 10 recomputes the mixed form's level-0 residual).
tmg_status check_setup(int p_t, double tau, double lambda, int64_t N, double omega, tmg_opts* o) {
    if (p_t < 0 || p_t > kMaxDegree || !(tau > 0.0) || !isfinite(tau) || !(lambda >= 0.0) || !isfinite(lambda) ||
        N < 1 || !(omega < 2.0) || !isfinite(omega) || o->nu1 < 0 || o->nu1 > 8 || o->nu2 < 0 || o->nu2 > 8 ||
        o->nu1 + o->nu2 < 1 || o->gamma < 1 || o->gamma > 2 || (o->precision != TMG_FP64 && o->precision != TMG_MIXED) ||
        o->n_min < 1 || o->max_cycles < 0 || o->max_cycles >= tmg::kHist || !(o->tol >= 0.0) ||
        o->check_fp64 < 0 || o->check_fp64 > 1)
        return TMG_EINVAL;
    // p_t <= 5, and p_t = 10, 20 (in the mixed form the level-0 residual is
    // recomputed from u in every cycle: no updated float pair)
    if (!tmg::built_width(p_t + 1)) return TMG_EUNSUPPORTED;
    if (p_t + 1 > tmg::kMaxD) o->update_residual = 0;
    return TMG_OK;
}

// Hierarchy of a plan (host arithmetic only): the number of levels, and the
// first level handed to the on-chip coarse solver -- the largest that fits --
// or, when none fits or the blocks are wider than that solver takes, the
// coarsest level solved by the grid-wide scan.
struct Shape {
    int nlev;
    int lt;
    bool scan;
    size_t tail_smem;
};

Shape plan_shape(const tmg_ops* ops, int d, int64_t N, int levels, const tmg_opts& o) {
    Shape sh{count_levels(N, o.n_min, levels), -1, false, 0};
    const bool wide = d > tmg::kMaxD;
    for (int l = 0; !wide && l < sh.nlev; ++l) {
        const int64_t Nl = N >> l;
        const size_t b = ops->tail_bytes(Nl, sh.nlev - l);
        const int64_t cap = o.tail_cap > 0 ? (o.tail_cap < kTailNmax ? o.tail_cap : kTailNmax)
                                           : (o.gamma == 2 ? kTailNmax : kTailDefaultV);
        if ((Nl <= cap || l == sh.nlev - 1) && Nl <= kTailNmax && b <= kTailSmemMax &&
            sh.nlev - l <= tmg::kTailLevels) {
            sh.lt = l;
            sh.tail_smem = b;
            break;
        }
    }
    if (sh.lt < 0) {
        sh.lt = sh.nlev - 1;
        sh.scan = true;
        sh.tail_smem = 0;
    }
    return sh;
}

const tmg_ops* forward_ops(const tmg_opts& o, int d) {
    return o.precision == TMG_MIXED ? tmg_ops_f32(d, 0) : tmg_ops_f64(d, 0);
}

tmg_status build_graph(tmg_plan* P, int dir) {
    cudaGraph_t g = nullptr;
    TMG_CUDA(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    // cudaGraphNodeParams has no default constructor: zero a raw buffer instead
    alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)];
    memset(np_buf, 0, sizeof(np_buf));
    cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_buf);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(P->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    cudaError_t ek = (dir == 0 ? P->ops : P->ops_adj)->enqueue_cycle(P);
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(P->s, &captured);
    if (ek != cudaSuccess || e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(ek != cudaSuccess ? ek : e);
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    P->graph[dir] = g;
    P->gexec[dir] = ex;
    P->cond[dir] = (unsigned long long)h;
    return TMG_OK;
}

// Start-of-solve state: written through the pinned mirror with one copy.
tmg_status stage_state(tmg_plan* P, const double* f, double u0, double* u, double tol, int max_cycles,
                       int use_cond, int nF_from_first, int dir = 0, int u_zero = 0) {
    tmg::DevState* h = P->st_host;
    TMG_CUDA(cudaStreamSynchronize(P->s));    // the mirror may still be read by a previous copy
    h->F = f;
    h->u = u;
    h->u0 = u0;
    h->nF = 0.0;
    h->tol = tol;
    h->max_cycles = max_cycles;
    h->cycle = 0;
    h->done = 0;
    h->nF_from_first = nF_from_first;
    h->use_cond = use_cond;
    h->full = 2;
    h->rsel = 0;
    h->u_zero = u_zero;
    h->ticket = 0u;
    h->nscale = 1.0f;
    h->nvals = (long long)P->N * P->d;
    h->cond = P->cond[dir];
    TMG_CUDA(cudaMemcpyAsync(P->st, h, offsetof(tmg::DevState, hist), cudaMemcpyHostToDevice, P->s));
    return TMG_OK;
}

tmg_status check_ptr(const void* p) {
    if (p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) != 0) return TMG_EINVAL;
    return TMG_OK;
}

tmg_status run_solve(tmg_plan* P, const double* f, double u0, double* u, int dir = 0, int initial_guess = -1) {
    if (check_ptr(f) != TMG_OK || check_ptr(u) != TMG_OK) return TMG_EINVAL;
    const tmg::NvtxRange r_solve(dir == 0 ? "tmg_solve" : "tmg_adjoint solve");
    const tmg_ops* ops = dir == 0 ? P->ops : P->ops_adj;
    if (initial_guess < 0) initial_guess = P->o.initial_guess;
    const int use_graph = P->o.use_graph != 0;
    if (use_graph && P->gexec[dir] == nullptr) {
        tmg_status s = build_graph(P, dir);
        if (s != TMG_OK) return s;
    }
    tmg_status s =
        stage_state(P, f, u0, u, P->o.tol, P->o.max_cycles, use_graph, initial_guess ? 0 : 1, dir, initial_guess ? 0 : 1);
    if (s != TMG_OK) return s;
    if (initial_guess) {
        TMG_CUDA(ops->enqueue_normF(P));
    } else {
        TMG_CUDA(cudaMemsetAsync(u, 0, sizeof(double) * P->N * P->d, P->s));
    }
    if (use_graph) {
        TMG_CUDA(cudaGraphLaunch(P->gexec[dir], P->s));
    } else {
        // eager loop: a few cycles per host check; kernels after convergence return at once
        for (int k = 0; k <= P->o.max_cycles;) {
            const int batch = 4;
            for (int i = 0; i < batch && k <= P->o.max_cycles; ++i, ++k) TMG_CUDA(ops->enqueue_cycle(P));
            TMG_CUDA(cudaMemcpyAsync(&P->st_host->done, &P->st->done, sizeof(int), cudaMemcpyDeviceToHost, P->s));
            TMG_CUDA(cudaStreamSynchronize(P->s));
            if (P->st_host->done) break;
        }
    }
    TMG_CUDA(cudaMemcpyAsync(P->st_host, P->st, sizeof(tmg::DevState), cudaMemcpyDeviceToHost, P->s));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    const tmg::DevState* h = P->st_host;
    const int nres = h->cycle;    // residual evaluations
    P->last_cycles = nres > 0 ? nres - 1 : 0;
    const int nh = nres < tmg::kHist ? nres : tmg::kHist;
    P->last_hist.assign(h->hist, h->hist + nh);
    P->last_rel = nh > 0 ? h->hist[nh - 1] : NAN;
    switch (h->done) {
        case 1: return TMG_OK;
        case 2: return TMG_ENOTCONV;
        case 3: return TMG_ENUMERIC;
        default: return TMG_ETIMEOUT;
    }
}

}  // namespace

extern "C" {

void tmg_opts_default(tmg_opts* o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_cycles = 100;
    o->nu1 = 1;
    o->nu2 = 1;
    o->gamma = 1;
    o->precision = TMG_MIXED;
    o->n_min = 64;
    o->use_graph = 1;
    o->initial_guess = 0;
    o->tail_cap = 0;
    o->use_pdl = 1;
    o->update_residual = 1;
    o->fuse_levels = -1;
    o->schedule = TMG_SCHED_AUTO;
    o->check_fp64 = 0;
}

tmg_status tmg_setup(tmg_plan** plan, int p_t, double tau, double lambda, int64_t N, int levels, double omega,
                     const tmg_opts* opts, void* stream) {
    if (plan == nullptr) return TMG_EINVAL;
    *plan = nullptr;
    tmg_opts o;
    tmg_opts_default(&o);
    if (opts) o = *opts;
    const tmg_status cs = check_setup(p_t, tau, lambda, N, omega, &o);
    if (cs != TMG_OK) return cs;

    tmg_plan* P = new (std::nothrow) tmg_plan();
    if (!P) return TMG_ENOMEM;
    P->p = p_t;
    P->d = p_t + 1;
    P->tau = tau;
    P->lambda = lambda;
    P->N = N;
    P->omega_user = omega;
    P->o = o;
    P->last_err = NAN;
    P->s = static_cast<cudaStream_t>(stream);
    P->own_stream = false;
    if (P->s == nullptr) {
        // The legacy default stream cannot be captured into a graph; a blocking
        // stream created here is implicitly ordered with it.
        cudaError_t se = cudaStreamCreate(&P->s);
        if (se != cudaSuccess) {
            delete P;
            return cuda_fail(se);
        }
        P->own_stream = true;
    }
    P->ops = forward_ops(o, P->d);
    P->ops_adj = o.precision == TMG_MIXED ? tmg_ops_f32(P->d, 1) : tmg_ops_f64(P->d, 1);

    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) {
        tmg_destroy(P);
        return cuda_fail(ce);
    }
    P->max_blocks = P->nsm * 8;

    // hierarchy and FP64 constants
    const Shape sh = plan_shape(P->ops, P->d, N, levels, o);
    P->nlev = sh.nlev;
    P->lev.resize(P->nlev);
    for (int l = 0; l < P->nlev; ++l) {
        P->lev[l].N = N >> l;
        level_setup(P->d, lambda * ldexp(tau, l), omega, &P->lev[l]);
    }
    transfer_setup(P->d, P->P1, P->P2);
    P->lev_adj.resize(P->nlev);
    for (int l = 0; l < P->nlev; ++l) level_setup_adjoint(P->d, P->lev[l], &P->lev_adj[l]);

    // first level handled on chip, or the coarsest level by the grid-wide scan
    P->lt = sh.lt;
    P->scan_coarsest = sh.scan;
    P->tail_smem = sh.tail_smem;

    // workspace: level vectors in the cycle precision, level-0 residual,
    // tail constants, block partials, device state
    const size_t el = P->ops->elem;
    const size_t A = 256;
    size_t off = 0;
    size_t off_f[tmg::kMaxLevels], off_u[tmg::kMaxLevels], off_u2[tmg::kMaxLevels];
    const bool wcycle = o.gamma == 2 && P->lt >= 1;   // levels 1..lt are visited twice per visit of their parent
    for (int l = 0; l <= P->lt; ++l) {
        off_f[l] = off;
        off = align_up(off + el * P->lev[l].N * P->d, A);
        off_u[l] = off;
        off = align_up(off + el * P->lev[l].N * P->d, A);
        off_u2[l] = off;
        if (wcycle && l >= 1) off = align_up(off + el * P->lev[l].N * P->d, A);
    }
    // level-0 residual; the mixed form that keeps r as a float pair updated
    // between cycles (k_updown0) needs two buffers of high and of low parts
    const bool updated_res = o.precision == TMG_MIXED && o.update_residual != 0 && P->lt >= 1;
    const size_t off_r = off;
    off = align_up(off + el * N * P->d * (updated_res ? 2 : 1), A);
    const size_t off_rl = off;
    if (updated_res) off = align_up(off + sizeof(short) * N * P->d * 2, A);
    const size_t off_lk = off;
    off = align_up(off + sizeof(tmg::LevelK<double, tmg::kMaxDWide>) * (P->nlev - P->lt), A);
    const size_t off_lk_adj = off;
    off = align_up(off + sizeof(tmg::LevelK<double, tmg::kMaxDWide>) * (P->nlev - P->lt), A);
    const size_t off_p = off;
    off = align_up(off + sizeof(double) * P->max_blocks, A);
    P->scan_tiles = (N + tmg::kScanTileMin - 1) / tmg::kScanTileMin;   // enough for every block width
    const size_t off_scan = off;
    off = align_up(off + sizeof(double) * (3 + 2 * tmg::kScanNT) * P->scan_tiles, A);
    const size_t off_st = off;
    off = align_up(off + sizeof(tmg::DevState), A);
    P->ws_bytes = off;
    ce = cudaMalloc(&P->ws, P->ws_bytes);
    if (ce != cudaSuccess) {
        P->ws = nullptr;
        tmg_destroy(P);
        g_last_cuda = (int)ce;
        return TMG_ENOMEM;
    }
    char* base = static_cast<char*>(P->ws);
    for (int l = 0; l <= P->lt; ++l) {
        P->fl[l] = base + off_f[l];
        P->ul[l] = base + off_u[l];
        P->ul2[l] = wcycle && l >= 1 ? base + off_u2[l] : nullptr;
    }
    P->rT = base + off_r;
    P->rl = updated_res ? base + off_rl : nullptr;
    P->lk_dev = base + off_lk;
    P->lk_dev_adj = base + off_lk_adj;
    P->partials = reinterpret_cast<double*>(base + off_p);
    P->scan_ws = base + off_scan;
    P->st = reinterpret_cast<tmg::DevState*>(base + off_st);
    ce = cudaMallocHost(&P->st_host, sizeof(tmg::DevState));
    if (ce != cudaSuccess) {
        P->st_host = nullptr;
        tmg_destroy(P);
        g_last_cuda = (int)ce;
        return TMG_ENOMEM;
    }
    memset(P->st_host, 0, sizeof(tmg::DevState));
    ce = cudaMemsetAsync(P->ws, 0, P->ws_bytes, P->s);
    // the attribute is per kernel, shared by every plan: set the common ceiling
    if (ce == cudaSuccess) ce = P->ops->upload(P);
    if (ce == cudaSuccess && P->ops_adj) ce = P->ops_adj->upload(P);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(P->s);
    if (ce != cudaSuccess) {
        tmg_destroy(P);
        return cuda_fail(ce);
    }
    *plan = P;
    return TMG_OK;
}

// Error of u against the exact FP64 solve of the same system (opts.check_fp64):
// the FP64 parallel scan into the plan's buffer, then max|u - u_exact| and
// max|u_exact| on the device.
tmg_status error_vs_fp64(tmg_plan* P, const double* f, double u0, const double* u) {
    const size_t nv = (size_t)P->N * P->d;
    if (!P->ex_buf) {
        cudaError_t e = cudaMalloc(&P->ex_buf, nv * sizeof(double));
        if (e != cudaSuccess) {
            P->ex_buf = nullptr;
            g_last_cuda = (int)e;
            return TMG_ENOMEM;
        }
    }
    TMG_CUDA(tmg_ops_f64(P->d, 0)->enqueue_direct(P, f, u0, P->ex_buf));
    unsigned long long* out2 = reinterpret_cast<unsigned long long*>(P->partials);
    TMG_CUDA(tmg_launch_maxabs2(u, P->ex_buf, (int64_t)nv, out2, P->max_blocks, P->s));
    unsigned long long h[2] = {0, 0};
    TMG_CUDA(cudaMemcpyAsync(h, out2, sizeof(h), cudaMemcpyDeviceToHost, P->s));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    double md, mv;
    memcpy(&md, &h[0], sizeof(double));
    memcpy(&mv, &h[1], sizeof(double));
    P->last_err = mv > 0.0 ? md / mv : md;
    return TMG_OK;
}

tmg_status tmg_solve(tmg_plan* P, const double* f, double u0, double* u) {
    if (!P || !isfinite(u0)) return TMG_EINVAL;
    P->last_err = NAN;
    tmg_status s = run_solve(P, f, u0, u);
    if ((s == TMG_OK || s == TMG_ENOTCONV) && P->o.check_fp64) {
        const tmg_status se = error_vs_fp64(P, f, u0, u);
        if (se != TMG_OK) return se;
    }
    return s;
}

tmg_status tmg_solve_host(tmg_plan* P, const double* f_host, double u0, double* u_host) {
    if (!P || !f_host || !u_host || !isfinite(u0)) return TMG_EINVAL;
    const size_t bytes = sizeof(double) * P->N * P->d;
    if (!P->F_dev) {
        cudaError_t e = cudaMalloc(&P->F_dev, bytes);
        if (e == cudaSuccess) e = cudaMalloc(&P->u_dev, bytes);
        if (e != cudaSuccess) {
            g_last_cuda = (int)e;
            return TMG_ENOMEM;
        }
    }
    TMG_CUDA(cudaMemcpyAsync(P->F_dev, f_host, bytes, cudaMemcpyHostToDevice, P->s));
    if (P->o.initial_guess) TMG_CUDA(cudaMemcpyAsync(P->u_dev, u_host, bytes, cudaMemcpyHostToDevice, P->s));
    P->last_err = NAN;
    tmg_status s = run_solve(P, P->F_dev, u0, P->u_dev);
    if (s != TMG_OK && s != TMG_ENOTCONV) return s;
    if (P->o.check_fp64) {
        const tmg_status se = error_vs_fp64(P, P->F_dev, u0, P->u_dev);
        if (se != TMG_OK) return se;
    }
    TMG_CUDA(cudaMemcpyAsync(u_host, P->u_dev, bytes, cudaMemcpyDeviceToHost, P->s));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return s;
}

tmg_status tmg_adjoint(tmg_plan* P, const double* g, const double* u, double* dJdf, double* dJdu0,
                       double* dJdlambda) {
    if (!P || check_ptr(g) != TMG_OK || check_ptr(u) != TMG_OK || check_ptr(dJdf) != TMG_OK || !dJdu0 ||
        !dJdlambda || (reinterpret_cast<uintptr_t>(dJdu0) & 7u) || (reinterpret_cast<uintptr_t>(dJdlambda) & 7u))
        return TMG_EINVAL;
    if (!P->ops_adj) return TMG_EUNSUPPORTED;   // no adjoint kernels at this degree
    const size_t nv = (size_t)P->N * P->d;
    if (!P->adj_buf) {
        cudaError_t e = cudaMalloc(&P->adj_buf, 2 * nv * sizeof(double));
        if (e != cudaSuccess) {
            P->adj_buf = nullptr;
            g_last_cuda = (int)e;
            return TMG_ENOMEM;
        }
    }
    double* g_rev = P->adj_buf;
    double* mu_rev = P->adj_buf + nv;
    // L^T mu = g is, in reversed time, the forward structure with A^T and (a', b') = (b, a)
    TMG_CUDA(tmg_launch_reverse(g, g_rev, P->N, P->d, P->s));
    tmg_status s = run_solve(P, g_rev, 0.0, mu_rev, 1, 0);
    if (s != TMG_OK && s != TMG_ENOTCONV) return s;
    TMG_CUDA(tmg_launch_reverse(mu_rev, dJdf, P->N, P->d, P->s));
    TMG_CUDA(cudaMemsetAsync(&P->st->ticket, 0, sizeof(unsigned), P->s));
    TMG_CUDA(tmg_launch_adjoint_grads(dJdf, u, P->N, P->d, P->tau, P->partials, P->max_blocks, &P->st->ticket,
                                      dJdu0, dJdlambda, P->s));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return s;
}

tmg_status tmg_error_vs_fp64(tmg_plan* P, const double* f, double u0, const double* u, double* err) {
    if (!P || !err || !isfinite(u0) || check_ptr(f) != TMG_OK || check_ptr(u) != TMG_OK) return TMG_EINVAL;
    const tmg_status s = error_vs_fp64(P, f, u0, u);
    if (s != TMG_OK) return s;
    *err = P->last_err;
    return TMG_OK;
}

tmg_status tmg_solve_direct(tmg_plan* P, const double* f, double u0, double* u) {
    if (!P || !isfinite(u0) || check_ptr(f) != TMG_OK || check_ptr(u) != TMG_OK) return TMG_EINVAL;
    TMG_CUDA(tmg_ops_f64(P->d, 0)->enqueue_direct(P, f, u0, u));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return TMG_OK;
}

tmg_status tmg_cycle(tmg_plan* P, const double* f, double u0, double* u) {
    if (!P || !isfinite(u0) || check_ptr(f) != TMG_OK || check_ptr(u) != TMG_OK) return TMG_EINVAL;
    tmg_status s = stage_state(P, f, u0, u, -1.0, 1 << 30, 0, 1);
    if (s != TMG_OK) return s;
    TMG_CUDA(P->ops->enqueue_cycle(P));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return TMG_OK;
}

// A plan whose cycle can be split at its coarsest level: V-cycles, the
// coarsest level below at least one streaming level and not part of an
// on-chip multi-level solver, and no updated level-0 residual (whose fused
// kernel joins the way up of one cycle to the way down of the next).
static bool splittable(const tmg_plan* P) {
    return P->o.gamma == 1 && P->lt >= 1 && P->lt == P->nlev - 1 && P->rl == nullptr;
}

tmg_status tmg_cycle_down(tmg_plan* P, const double* f, double u0, double* u, double* fc) {
    if (!P || !isfinite(u0) || check_ptr(f) != TMG_OK || check_ptr(u) != TMG_OK || !fc ||
        (reinterpret_cast<uintptr_t>(fc) & 7u))
        return TMG_EINVAL;
    if (!splittable(P)) return TMG_EUNSUPPORTED;
    tmg_status s = stage_state(P, f, u0, u, -1.0, 1 << 30, 0, 1);
    if (s != TMG_OK) return s;
    P->split = 1;
    const cudaError_t e = P->ops->enqueue_cycle(P);
    P->split = 0;
    TMG_CUDA(e);
    TMG_CUDA(P->ops->enqueue_coarse_io(P, fc, nullptr));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return TMG_OK;
}

tmg_status tmg_cycle_up(tmg_plan* P, const double* uc, double* u) {
    if (!P || !uc || (reinterpret_cast<uintptr_t>(uc) & 7u) || check_ptr(u) != TMG_OK) return TMG_EINVAL;
    if (!splittable(P)) return TMG_EUNSUPPORTED;
    if (P->st_host->u != u) return TMG_EINVAL;   // the u of the tmg_cycle_down call this completes
    TMG_CUDA(P->ops->enqueue_coarse_io(P, nullptr, uc));
    P->split = 2;
    const cudaError_t e = P->ops->enqueue_cycle(P);
    P->split = 0;
    TMG_CUDA(e);
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return TMG_OK;
}

tmg_status tmg_residual(tmg_plan* P, const double* f, double u0, const double* u, double* r) {
    if (!P || !isfinite(u0) || check_ptr(f) != TMG_OK || check_ptr(u) != TMG_OK || check_ptr(r) != TMG_OK)
        return TMG_EINVAL;
    TMG_CUDA(P->ops->enqueue_residual(P, f, u0, u, r));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return TMG_OK;
}

tmg_status tmg_stats(const tmg_plan* P, int* cycles, double* rel_res, double* err_vs_fp64, double* hist,
                     int hist_len) {
    if (!P) return TMG_EINVAL;
    if (cycles) *cycles = P->last_cycles;
    if (rel_res) *rel_res = P->last_rel;
    if (err_vs_fp64) *err_vs_fp64 = P->last_err;
    if (hist)
        for (int i = 0; i < hist_len; ++i) hist[i] = i < (int)P->last_hist.size() ? P->last_hist[i] : NAN;
    return TMG_OK;
}

tmg_status tmg_plan_shape(int p_t, double tau, double lambda, int64_t N, int levels, double omega,
                          const tmg_opts* opts, int* num_levels, int* tail_level, int64_t* tail_intervals,
                          int* scan_coarsest) {
    tmg_opts o;
    tmg_opts_default(&o);
    if (opts) o = *opts;
    const tmg_status cs = check_setup(p_t, tau, lambda, N, omega, &o);
    if (cs != TMG_OK) return cs;
    const Shape sh = plan_shape(forward_ops(o, p_t + 1), p_t + 1, N, levels, o);
    if (num_levels) *num_levels = sh.nlev;
    if (tail_level) *tail_level = sh.lt;
    if (tail_intervals) *tail_intervals = N >> sh.lt;
    if (scan_coarsest) *scan_coarsest = sh.scan ? 1 : 0;
    return TMG_OK;
}

tmg_status tmg_level_constants(int p_t, double z, double omega_user, double* A, double* Ainv, double* g, double* c,
                               double* alpha, double* omega) {
    if (p_t < 0 || p_t > kMaxDegree || !(z >= 0.0) || !isfinite(z) || !(omega_user < 2.0) || !isfinite(omega_user))
        return TMG_EINVAL;
    if (!tmg::built_width(p_t + 1)) return TMG_EUNSUPPORTED;
    const int d = p_t + 1;
    tmg_level_host L;
    level_setup(d, z, omega_user, &L);
    for (int i = 0; i < d * d; ++i) {
        if (A) A[i] = L.A[i];
        if (Ainv) Ainv[i] = L.Ainv[i];
    }
    for (int k = 0; k < d; ++k) {
        if (g) g[k] = L.g[k];
        if (c) c[k] = L.c[k];
    }
    if (alpha) *alpha = L.alpha;
    if (omega) *omega = L.omega;
    return TMG_OK;
}

tmg_status tmg_transfer_matrices(int p_t, double* P1, double* P2) {
    if (p_t < 0 || p_t > kMaxDegree || !P1 || !P2) return TMG_EINVAL;
    if (!tmg::built_width(p_t + 1)) return TMG_EUNSUPPORTED;
    transfer_setup(p_t + 1, P1, P2);
    return TMG_OK;
}

tmg_status tmg_plan_info(const tmg_plan* P, int* num_levels, int* tail_level, int64_t* tail_intervals,
                         double* omega_per_level, int omega_len) {
    if (!P) return TMG_EINVAL;
    if (num_levels) *num_levels = P->nlev;
    if (tail_level) *tail_level = P->lt;
    if (tail_intervals) *tail_intervals = P->lev[P->lt].N;
    if (omega_per_level)
        for (int i = 0; i < omega_len; ++i) omega_per_level[i] = i < P->nlev ? P->lev[i].omega : NAN;
    return TMG_OK;
}

tmg_status tmg_profile_cycle(tmg_plan* P, const double* f, double u0, double* u, int reps, double* ms, int n_ms) {
    if (!P || reps < 1 || !ms || n_ms < 6 || !isfinite(u0) || check_ptr(f) != TMG_OK || check_ptr(u) != TMG_OK)
        return TMG_EINVAL;
    const int max_ev = 2 * P->nlev + 4;    // kernel groups per cycle + 1
    std::vector<cudaEvent_t> ev(max_ev);
    std::vector<int> cat(max_ev, -1);
    for (auto& e : ev) TMG_CUDA(cudaEventCreate(&e));
    double acc[6] = {0, 0, 0, 0, 0, 0};
    tmg_status status = TMG_OK;
    for (int r = 0; r < reps && status == TMG_OK; ++r) {
        status = stage_state(P, f, u0, u, -1.0, 1 << 30, 0, 1);
        if (status != TMG_OK) break;
        int nev = 0;
        cudaError_t e = P->ops->enqueue_cycle_timed(P, ev.data(), cat.data(), &nev);
        if (e == cudaSuccess) e = cudaStreamSynchronize(P->s);
        if (e != cudaSuccess) {
            status = cuda_fail(e);
            break;
        }
        for (int k = 0; k + 1 < nev; ++k) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            if (cat[k] >= 0 && cat[k] < 5) acc[cat[k]] += t;
        }
        float tot = 0.f;
        cudaEventElapsedTime(&tot, ev[0], ev[nev - 1]);
        acc[5] += tot;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    for (int i = 0; i < 6; ++i) ms[i] = acc[i] / reps;
    for (int i = 6; i < n_ms; ++i) ms[i] = 0.0;
    return status;
}

tmg_status tmg_plan_launches(const tmg_plan* P, int* per_cycle) {
    if (!P || !per_cycle) return TMG_EINVAL;
    *per_cycle = P->launches_per_cycle;
    return TMG_OK;
}

tmg_status tmg_inspect(const tmg_plan* P, int which, int level, void* host_dst, size_t bytes) {
    if (!P || !host_dst || which < 0 || which > 3) return TMG_EINVAL;
    const void* src = nullptr;
    int64_t n = P->N;
    size_t elem = P->ops->elem;
    if (which == 2 || which == 3) {
        // the current one of the two residual buffers of the updated form
        int sel = 0;
        if (P->rl != nullptr) {
            TMG_CUDA(cudaMemcpyAsync(&P->st_host->rsel, &P->st->rsel, sizeof(int), cudaMemcpyDeviceToHost, P->s));
            TMG_CUDA(cudaStreamSynchronize(P->s));
            sel = P->st_host->rsel;
        }
        const size_t nv = (size_t)P->N * P->d;
        if (which == 2) {
            src = static_cast<const char*>(P->rT) + sel * nv * elem;
        } else {
            // the low parts are stored as 16-bit codes relative to ulp(hi): decode here
            if (P->rl == nullptr) return TMG_EINVAL;
            if (bytes < nv * sizeof(float)) return TMG_EINVAL;
            std::vector<float> hi(nv);
            std::vector<short> code(nv);
            TMG_CUDA(cudaMemcpyAsync(hi.data(), static_cast<const float*>(P->rT) + sel * nv, nv * sizeof(float),
                                     cudaMemcpyDeviceToHost, P->s));
            TMG_CUDA(cudaMemcpyAsync(code.data(), static_cast<const short*>(P->rl) + sel * nv, nv * sizeof(short),
                                     cudaMemcpyDeviceToHost, P->s));
            TMG_CUDA(cudaStreamSynchronize(P->s));
            float* out = static_cast<float*>(host_dst);
            for (size_t i = 0; i < nv; ++i) {
                uint32_t b;
                memcpy(&b, &hi[i], sizeof(b));
                const int E = (int)((b >> 23) & 0xFFu);
                out[i] = E < 39 ? 0.f : ldexpf((float)code[i], E - 165);
            }
            return TMG_OK;
        }
    } else {
        if (level < 0 || level > P->lt || (level == 0 && which == 0)) return TMG_EINVAL;
        // the final correction of a level: in a W-cycle that of its second visit
        src = which == 0 ? P->fl[level] : (P->ul2[level] != nullptr ? P->ul2[level] : P->ul[level]);
        n = P->lev[level].N;
    }
    const size_t need = (size_t)n * P->d * elem;
    if (bytes < need) return TMG_EINVAL;
    TMG_CUDA(cudaMemcpyAsync(host_dst, src, need, cudaMemcpyDeviceToHost, P->s));
    TMG_CUDA(cudaStreamSynchronize(P->s));
    return TMG_OK;
}

void tmg_destroy(tmg_plan* P) {
    if (!P) return;
    cudaStreamSynchronize(P->s);
    for (int dir = 0; dir < 2; ++dir) {
        if (P->gexec[dir]) cudaGraphExecDestroy(P->gexec[dir]);
        if (P->graph[dir]) cudaGraphDestroy(P->graph[dir]);
    }
    if (P->adj_buf) cudaFree(P->adj_buf);
    if (P->ws) cudaFree(P->ws);
    if (P->st_host) cudaFreeHost(P->st_host);
    if (P->F_dev) cudaFree(P->F_dev);
    if (P->ex_buf) cudaFree(P->ex_buf);
    if (P->u_dev) cudaFree(P->u_dev);
    if (P->own_stream) cudaStreamDestroy(P->s);
    delete P;
}

const char* tmg_strerror(tmg_status s) {
    switch (s) {
        case TMG_OK: return "ok";
        case TMG_EINVAL: return "invalid argument";
        case TMG_ENOMEM: return "out of memory";
        case TMG_ECUDA: return "CUDA error";
        case TMG_ENOTCONV: return "cycle limit reached before the tolerance";
        case TMG_ENUMERIC: return "non-finite residual";
        case TMG_ETIMEOUT: return "device-side wait timed out";
        case TMG_EUNSUPPORTED: return "unsupported configuration";
        default: return "unknown status";
    }
}

int tmg_last_cuda_error(void) { return g_last_cuda; }

tmg_status tmg_debug_bounds(unsigned* violations, unsigned long long* first) {
    if (!violations || !first) return TMG_EINVAL;
    *violations = 0;
    *first = 0;
    if (tmg::bounds_readers().empty()) return TMG_EUNSUPPORTED;
    for (tmg::BoundsReader rd : tmg::bounds_readers()) {
        unsigned c = 0;
        unsigned long long f = 0;
        if (rd(&c, &f) != 0) return TMG_ECUDA;
        *violations += c;
        if (*first == 0) *first = f;
    }
    return TMG_OK;
}

}  // extern "C"
