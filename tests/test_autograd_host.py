"""Host glue of autograd.PolarizationLoss, with a stand-in for the library
run: the gradients pic_adjoint returns per slot come back to the caller in
the caller's particle order, scaled by the upstream gradient."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2002_02211_gb300.autograd import PolarizationLoss  # noqa: E402


class _Sim:
    """What PolarizationLoss reads from a context: the loss and dL/da0, and
    per-slot gradients with the particle ids (slots in a permuted order)."""

    def __init__(self, n, perm):
        self.n, self.perm = n, perm

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def adjoint(self, nsteps, checkpoint_every, species, **loss):
        return 0.37, -2.5

    def adjoint_particle_grads(self, s):
        ids = 100 + self.perm                       # caller ids 100, 101, ... in slot order
        return {"id": ids, "w": 10.0 * self.perm, "sx": 1.0 * self.perm, "sy": -1.0 * self.perm,
                "sz": 0.5 * self.perm}


class _Run:
    def __init__(self, n):
        self.species, self.nsteps, self.checkpoint_every, self.loss = 0, 3, 2, {}
        self.perm = np.random.default_rng(1).permutation(n)
        self.particles = [{"id": np.arange(100, 100 + n, dtype=np.int32)}]
        self.n = n

    def start(self, a0, weights, spins):
        assert len(weights) == self.n and spins.shape == (self.n, 3)
        return _Sim(self.n, self.perm)


def test_gradients_come_back_in_particle_order():
    n = 7
    run = _Run(n)
    a0 = torch.tensor(2.0, dtype=torch.float64, requires_grad=True)
    w = torch.rand(n, dtype=torch.float64, requires_grad=True)
    sp = torch.rand(n, 3, dtype=torch.float64, requires_grad=True)
    L = PolarizationLoss(a0, w, sp, run)
    assert L.detach().item() == pytest.approx(0.37)
    (3.0 * L).backward()
    assert float(a0.grad) == pytest.approx(3.0 * -2.5)
    # particle i (id 100 + i) has gradient 10 i in w and (i, -i, i/2) in s
    i = np.arange(n)
    np.testing.assert_allclose(w.grad.numpy(), 3.0 * 10.0 * i)
    np.testing.assert_allclose(sp.grad.numpy(), 3.0 * np.stack([i, -i, 0.5 * i], axis=1))
    assert w.grad.device == w.device and sp.grad.device == sp.device
