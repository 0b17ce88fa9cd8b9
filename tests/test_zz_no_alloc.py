"""The residual entry point that allocates nothing (tmg_residual_norm_noalloc).

It serves callers that may not allocate device memory at the point of the
check: real-time loops that cannot take the device synchronisation an
allocation may cause, and applications whose device memory all belongs to
their own pool.  It must give the oracle's residual F - L u, the same residual
as the plan-based entry point tmg_residual, and a norm equal to ||r||_2, on two
calls in a row (the second call reuses the shared scratch array the first one
left behind).  Every degree is covered: p_t = 4 and 5 take the generic
Legendre loop of the residual.  This file is collected last so that a run
stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1409_5254_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5254_gb300 import build_ext
    build_ext.build()
    return torch.device("cuda:0")


@pytest.mark.parametrize("p,N", [(1, 1 << 16), (3, 12352), (0, 1), (2, 4097), (4, 3000), (5, 2049)])
def test_noalloc_residual_matches_plan_residual_twice(dev, p, N):
    from paper_1409_5254_gb300 import tmg
    lam = 2.0
    prob = inputs.scalar_problem(7, N, p, lam=lam, T=1.0, u0=0.6)
    F = torch.from_numpy(prob["F"]).to(dev)
    rng = np.random.default_rng(3)
    with tmg.Plan(p, prob["tau"], lam, N) as plan:
        for call in range(2):
            u = torch.from_numpy(rng.standard_normal((N, p + 1)) * (call + 1)).to(dev)
            r_ref = plan.residual(F, prob["u0"], u)
            r = torch.full_like(u, float("nan"))
            norm = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            tmg.residual_norm_noalloc(p, prob["tau"], lam, F, prob["u0"], u, r, norm)
            torch.cuda.synchronize()
            np.testing.assert_allclose(r.cpu().numpy(), r_ref.cpu().numpy(), rtol=1e-13, atol=1e-13)
            # and against the oracle directly: rounding of |r| + |L||u| scale
            u_h = u.cpu().numpy()
            r_or = O.residual(p, lam * prob["tau"], prob["F"], prob["u0"], u_h)
            scale = np.abs(u_h).max() * (3.0 + lam * prob["tau"]) * (p + 1) + np.abs(prob["F"]).max()
            assert np.abs(r.cpu().numpy() - r_or).max() <= 1e-14 * scale
            ref_norm = float(torch.linalg.vector_norm(r_ref))
            assert float(norm.item()) == pytest.approx(ref_norm, rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch(dev):
    from paper_1409_5254_gb300 import tmg
    lib = tmg._lib()
    st = lib.tmg_residual_norm_noalloc(1, 1e-3, 1.0, (1 << 21) + 2, ctypes.c_void_p(16), 0.0, ctypes.c_void_p(16),
                                       ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == tmg.TMG_EUNSUPPORTED
