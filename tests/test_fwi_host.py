"""Host logic of the FWI autograd wrapper (no GPU): Misfit.apply passes the
model to the library call and its backward returns grad_output times the
library's gradient. The library call is replaced by a quadratic misfit whose
gradient is known in closed form, and torch.autograd.gradcheck confirms the
wiring."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2004_07930_gb300 import fwi


@pytest.fixture
def quadratic(monkeypatch):
    rng = np.random.Generator(np.random.PCG64(3))
    c = rng.standard_normal(7)
    W = np.diag(rng.uniform(1.0, 2.0, 7))

    def fake(prob, m, src, rec, d_obs=None, options=None):
        r = np.asarray(m) - c
        return 0.5 * float(r @ W @ r), W @ r, None, {"converged": 1}

    monkeypatch.setattr(fwi, "misfit_and_gradient", fake)
    return c, W


def test_backward_is_grad_output_times_gradient(quadratic):
    c, W = quadratic
    m = torch.tensor(np.linspace(0.1, 0.7, 7), dtype=torch.float64, requires_grad=True)
    chi = fwi.Misfit.apply(m, None, None, None, None)
    (3.0 * chi).backward()
    expect = 3.0 * W @ (m.detach().numpy() - c)
    np.testing.assert_allclose(m.grad.numpy(), expect, rtol=1e-14, atol=0)


def test_gradcheck(quadratic):
    m = torch.tensor(np.linspace(-0.3, 0.4, 7), dtype=torch.float64, requires_grad=True)
    assert torch.autograd.gradcheck(lambda x: fwi.Misfit.apply(x, None, None, None, None), (m,))
