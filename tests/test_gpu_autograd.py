"""The torch.autograd.Function over the batched solve: gradients of a nodal
least-squares loss with respect to f, u0 and lambda against the oracle's
adjoint formulas, with and without keeping the forward solution."""
import numpy as np
import pytest

import oracle as O
from paper_1409_5254_gb300 import inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("save", [True, False])
def test_autograd_gradients(save):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1409_5254_gb300 import autograd, build_ext, tmg
    build_ext.build()
    dev = torch.device("cuda:0")
    n, N, p = 6, 1024, 2
    rng = np.random.default_rng(21)
    lam_np = 10.0 ** rng.uniform(0, 3, n)
    tau = np.full(n, 1.0 / N)
    Fs = [inputs.load_vector(p, N, 1.0, inputs.Forcing.draw(rng, 1.0)) for _ in range(n)]
    y = rng.standard_normal((n, N))
    u0_np = rng.standard_normal(n)
    with tmg.Batch([p] * n, tau, lam_np, [N] * n, precision="fp64", tol=1e-12, max_cycles=300) as B:
        f = torch.from_numpy(np.concatenate([F.reshape(-1) for F in Fs])).to(dev).requires_grad_(True)
        u0 = torch.from_numpy(u0_np).to(dev).requires_grad_(True)
        lam = torch.from_numpy(lam_np).to(dev).requires_grad_(True)
        u = autograd.solve(f, u0, lam, B, save_solution=save)
        e = u.view(n, N, p + 1).sum(dim=2)                        # nodal values b^T u_n (b = 1)
        loss = 0.5 * ((e - torch.from_numpy(y).to(dev)) ** 2).sum()
        loss.backward()
    gf = f.grad.cpu().numpy()
    for i in range(n):
        z = lam_np[i] * tau[i]
        ui = O.fsub(p, z, Fs[i], u0_np[i])
        g = np.outer(O.nodal_values(p, ui) - y[i], np.ones(p + 1))
        dJdf, d0, dl = O.adjoint_grads(p, lam_np[i], tau[i], g, ui)
        gi = gf[i * N * (p + 1):(i + 1) * N * (p + 1)].reshape(N, p + 1)
        assert np.abs(gi - dJdf).max() <= 1e-8 * np.abs(dJdf).max()
        assert float(u0.grad[i]) == pytest.approx(d0, rel=1e-8, abs=1e-12)
        assert float(lam.grad[i]) == pytest.approx(dl, rel=1e-8, abs=1e-12)
