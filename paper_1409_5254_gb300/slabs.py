"""Time-slab partition of one long horizon over several ranks.

The paper parallelises its multigrid in time by giving every core a slab of
time steps (Section 5).  Here a rank (one GPU) owns the slab [a, b) of the
fine intervals, S = N / R of them, and runs the cycle's levels 0 .. L_s - 1 on
its slab; the coarse part of the cycle (level L_s and below) is a small global
problem of N / 2^L_s intervals that every rank solves from the gathered
right-hand sides.  The result is exactly the single-rank cycle:

* Each level operation of the cycle reads, to the left, a bounded number of
  intervals (the one-value halo e_{n-1} per smoothing sweep).  A rank
  therefore runs its levels on the *extended* slab [a - M, b), the margin M
  recomputing what its left neighbour's slab would feed in.  Garbage from the
  extended slab's truncated start moves right by at most nu1 + 1 intervals per
  level on the way down (so the own coarse right-hand sides stay exact) and by
  at most (2 nu1 + nu2 + 1) 2^(L_s - l) fine intervals on the way up from
  level l; M = 2^L_s (2 nu1 + nu2 + 1) covers it.
* The level-0 residual on the margin needs the current iterate there and the
  endpoint value e before the margin: the left neighbour sends them once per
  cycle (M (p_t + 1) values and one scalar) -- the only point-to-point
  exchange.
* The coarse right-hand sides of the own part of every slab are all-gathered
  (N / 2^L_s (p_t + 1) values in all); every rank applies the coarse part of
  the cycle to the gathered problem (one cycle from zero on it, the same
  hierarchy below L_s as the single-rank solve) and takes the corrections of
  its extended slab.

The per-rank arithmetic comes from a backend: on GPUs the library's plans
(tmg_cycle_down / tmg_cycle_up on the extended slab, tmg_cycle on the coarse
problem); any object with the same four methods works.  Two drivers: ranks of
torch.distributed (point-to-point margin, all_gather of the coarse problem),
and all ranks in one process one after the other (``run_in_process``), which
exchanges the same data by copies.
"""
from __future__ import annotations

from dataclasses import dataclass


def _levels(N: int, n_min: int) -> int:
    """Levels of the hierarchy of N intervals: coarsen while even and longer
    than n_min (the paper's nested meshes)."""
    L, n = 1, N
    while n % 2 == 0 and n > n_min:
        n //= 2
        L += 1
    return L


@dataclass(frozen=True)
class SlabLayout:
    """Where one rank's slab sits.  Global fine intervals [a, b) are owned;
    the rank computes on [start, b) with start = a - margin.  The coarse
    problem has N >> slab_levels intervals, of which the own part is
    [a, b) >> slab_levels."""
    N: int
    ranks: int
    rank: int
    slab_levels: int
    margin: int
    a: int
    b: int
    nu1: int = 1
    nu2: int = 1

    def margin_of(self, rank: int) -> int:
        """The margin of another rank of the same partition."""
        return min(margin_for(self.slab_levels, self.nu1, self.nu2), rank * (self.N // self.ranks))

    @property
    def start(self) -> int:
        return self.a - self.margin

    @property
    def n_ext(self) -> int:
        return self.b - self.start

    @property
    def coarse_n(self) -> int:
        return self.N >> self.slab_levels


def margin_for(slab_levels: int, nu1: int, nu2: int) -> int:
    """Fine intervals of recomputation in front of a slab: the reach of the
    way up's garbage, 2^L_s (2 nu1 + nu2 + 1) (see the module text)."""
    return (1 << slab_levels) * (2 * nu1 + nu2 + 1)


def slab_layout(N: int, ranks: int, rank: int, nu1: int = 1, nu2: int = 1, n_min: int = 64,
                coarse_per_slab: int = 256) -> SlabLayout:
    """Equal slabs; L_s is the most slab levels that leave at least
    coarse_per_slab coarse intervals per slab, keep the slab boundaries on
    the coarse mesh, stay above the global coarsest level, and let the margin
    fit inside the left neighbour's slab."""
    if ranks < 1 or not 0 <= rank < ranks or N % ranks:
        raise ValueError("N must split into equal slabs over the ranks")
    S = N // ranks
    levels = _levels(N, n_min)
    Ls = 0
    while (Ls + 1 < levels - 1 and S % (1 << (Ls + 1)) == 0 and (S >> (Ls + 1)) >= coarse_per_slab
           and margin_for(Ls + 1, nu1, nu2) + 1 <= S):
        Ls += 1
    if Ls < 1:
        raise ValueError("slabs too short for a slab level above the coarse problem")
    a, b = rank * S, (rank + 1) * S
    margin = min(margin_for(Ls, nu1, nu2), a)
    return SlabLayout(N, ranks, rank, Ls, margin, a, b, nu1, nu2)


class GpuSlabBackend:
    """The library's plans for one rank: the extended slab (levels 0..L_s,
    split at L_s: tmg_cycle_down / tmg_cycle_up) and the coarse problem
    (tmg_cycle from zero)."""

    def __init__(self, lay: SlabLayout, p: int, tau: float, lam: float, *, precision="fp64", nu1: int = 1,
                 nu2: int = 1, n_min: int = 64, stream=None):
        from . import tmg
        self.lay = lay
        self.ext = tmg.Plan(p, tau, lam, lay.n_ext, lay.slab_levels + 1, precision=precision, nu1=nu1, nu2=nu2,
                            n_min=1, tail_cap=1, update_residual=False, stream=stream)
        self.coarse = tmg.Plan(p, tau * (1 << lay.slab_levels), lam, lay.coarse_n, precision=precision, nu1=nu1,
                               nu2=nu2, n_min=n_min, stream=stream)
        self.d = p + 1

    def down(self, F_ext, e_before, u_ext):
        return self.ext.cycle_down(F_ext, e_before, u_ext)

    def up(self, uc_ext, u_ext):
        self.ext.cycle_up(uc_ext.contiguous(), u_ext)

    def coarse_cycle(self, fc):
        import torch
        uc = torch.zeros_like(fc)
        self.coarse.cycle(fc, 0.0, uc)
        return uc

    def close(self):
        self.ext.close()
        self.coarse.close()


class SlabRank:
    """One rank's state: the extended slab's load vector and iterate, and the
    steps of a cycle between which the drivers exchange data.  Arrays are
    torch tensors on the backend's device (CPU for host backends)."""

    def __init__(self, lay: SlabLayout, backend, F_ext, u0: float, b_vec):
        import torch
        self.lay, self.be = lay, backend
        self.F = F_ext
        self.u = torch.zeros_like(F_ext)
        self.u0 = float(u0)          # the true initial value (rank 0) -- others get e from the left
        self.b = b_vec               # b_l = psi_l(1): e = b^T u_n
        self.e_before = self.u0 if lay.a == 0 else 0.0

    def margin_out(self, next_margin: int):
        """What this rank sends right: its last next_margin own intervals of
        u and the endpoint value e = b^T u of the own interval before them
        (the layout keeps every margin shorter than a slab)."""
        m = next_margin
        own = self.u[self.lay.margin:]
        return own[own.shape[0] - m:].clone(), float(own[-m - 1] @ self.b)

    def margin_in(self, u_margin, e_before: float):
        self.u[:self.lay.margin] = u_margin
        self.e_before = e_before

    def down(self):
        """The way down on the extended slab; the own part of the coarse
        right-hand side."""
        fc = self.be.down(self.F, self.e_before, self.u)
        return fc[self.lay.margin >> self.lay.slab_levels:]

    def up(self, uc_global):
        s = self.lay.slab_levels
        self.be.up(uc_global[self.lay.start >> s:self.lay.b >> s], self.u)

    def own(self):
        return self.u[self.lay.margin:]


def _exchange_in_process(ranks):
    for r in range(len(ranks) - 1, 0, -1):
        m = ranks[r].lay.margin
        um, e = ranks[r - 1].margin_out(m)
        ranks[r].margin_in(um, e)


def run_in_process(ranks, cycles: int, backend_coarse):
    """All ranks in one process, one after the other: the same exchanges as
    ranks of a process group, as copies.  backend_coarse applies the coarse
    part of the cycle to the gathered coarse problem."""
    import torch
    for _ in range(cycles):
        _exchange_in_process(ranks)
        fc = torch.cat([rk.down() for rk in ranks])
        uc = backend_coarse(fc)
        for rk in ranks:
            rk.up(uc)


def run_distributed(rk: SlabRank, cycles: int, dist, group=None):
    """One rank of a torch.distributed group: per cycle one point-to-point
    exchange of the margin (iterate and endpoint value, left to right) and one
    all_gather of the coarse right-hand sides."""
    import torch
    lay = rk.lay
    R, r = lay.ranks, lay.rank
    next_margin = lay.margin_of(r + 1) if r + 1 < R else 0
    d = rk.F.shape[1]
    for _ in range(cycles):
        reqs = []
        if r + 1 < R:
            um, e = rk.margin_out(next_margin)
            buf = torch.cat([um.reshape(-1), torch.tensor([e], dtype=um.dtype, device=um.device)])
            reqs.append(dist.isend(buf.contiguous(), r + 1, group=group))
        if r > 0:
            buf = torch.empty(lay.margin * d + 1, dtype=rk.F.dtype, device=rk.F.device)
            dist.recv(buf, r - 1, group=group)
            rk.margin_in(buf[:-1].reshape(lay.margin, d), float(buf[-1]))
        for q in reqs:
            q.wait()
        fc_own = rk.down().contiguous()
        parts = [torch.empty_like(fc_own) for _ in range(R)]
        dist.all_gather(parts, fc_own, group=group)
        uc = rk.be.coarse_cycle(torch.cat(parts))
        rk.up(uc)
