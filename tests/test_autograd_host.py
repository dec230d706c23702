"""Host logic of the checkpointed differentiable rollout (autograd.py) on the CPU:
the solver is replaced by a small nonlinear stand-in with a known Jacobian, so
that the segment bookkeeping (checkpoints every K steps, recomputation inside a
segment, each adjoint step applied about the state it linearises) is checked
against central differences of the same map, for several segment lengths."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_12915_gb300 import autograd as AG  # noqa: E402
from workloads import inputs as I  # noqa: E402

SHAPE = (16, 2, 3)
N = int(np.prod(SHAPE))
_rng = np.random.default_rng(11)
B = torch.from_numpy(_rng.normal(size=(N, N)) / np.sqrt(N))


def _map(x, dt):
    """x + dt sin(B x): nonlinear, so every adjoint step depends on its state."""
    return x + dt * torch.sin(B @ x)


class FakeSolver:
    calls = []

    def __init__(self, grid, gamma, x, precision="fp64", variant="tai", stream=None):
        self.x = x.detach().reshape(-1).clone().cpu()

    def step(self, dt, n=1):
        for _ in range(n):
            self.x = _map(self.x, dt)

    def state(self, out=None):
        out.copy_(self.x.reshape(SHAPE))
        return out

    def set_state(self, s):
        self.x = s.detach().reshape(-1).clone()

    def adjoint(self, dt, lam, out=None):
        FakeSolver.calls.append(self.x.clone())
        J = torch.eye(N, dtype=torch.float64) + dt * torch.cos(B @ self.x)[:, None] * B
        return (J.T @ lam.reshape(-1)).reshape(SHAPE)

    def sync(self):
        pass

    def close(self):
        pass


@pytest.fixture
def fake(monkeypatch):
    monkeypatch.setattr(AG, "Solver", FakeSolver)
    monkeypatch.setattr(AG.torch.cuda, "current_stream", lambda: None)
    FakeSolver.calls = []
    return FakeSolver


@pytest.mark.parametrize("n_steps,every", [(13, 5), (10, 5), (7, 50), (6, 1)])
def test_rollout_gradient_matches_central_differences(fake, n_steps, every):
    grid = I.Grid(3, 2, 0.0, 0.0, 0.1)
    dt = 0.3
    x0 = torch.from_numpy(_rng.normal(size=SHAPE)).requires_grad_(True)
    xn = AG.rollout(x0, grid, 1.4, dt, n_steps, every)
    J = (xn ** 2).sum()
    J.backward()
    g = x0.grad.numpy().reshape(-1)

    def Jof(x):
        x = torch.from_numpy(x)
        for _ in range(n_steps):
            x = _map(x, dt)
        return float((x ** 2).sum())

    base = x0.detach().numpy().reshape(-1)
    for k in range(0, N, 7):
        e = np.zeros(N)
        e[k] = 1e-6
        fd = (Jof(base + e) - Jof(base - e)) / 2e-6
        assert abs(g[k] - fd) <= 1e-7 * max(1.0, abs(fd)), (k, g[k], fd)
    # one adjoint step per forward step, about the states n-1, ..., 0 in turn
    assert len(fake.calls) == n_steps
    x = torch.from_numpy(base)
    states = []
    for _ in range(n_steps):
        states.append(x)
        x = _map(x, dt)
    for got, want in zip(fake.calls, reversed(states)):
        assert torch.equal(got, want)


def test_second_backward_raises_a_clear_error(fake):
    """The first backward releases the solver and the checkpoints."""
    grid = I.Grid(3, 2, 0.0, 0.0, 0.1)
    x0 = torch.from_numpy(_rng.normal(size=SHAPE)).requires_grad_(True)
    xn = AG.rollout(x0, grid, 1.4, 0.3, 4, 2)
    J = (xn ** 2).sum()
    J.backward(retain_graph=True)
    with pytest.raises(RuntimeError, match="one backward pass"):
        J.backward()
