"""The torch.autograd wrapper of the film-solve gradient, on the CPU with a stand-in problem
(the wrapper only marshals: it sets the parameters, calls the solve gradient once and scales the
stored gradient by the incoming one)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1801_04869_gb300.adjoint import film_solve_loss  # noqa: E402


class StandIn:
    """Quadratic loss 1/2 |jc - a|^2 + 1/2 |v - b|^2 with its exact gradient."""

    def __init__(self, a, b):
        self.a, self.b = a, b
        self.jc = None
        self.kv = None
        self.calls = 0
        self.grads = 0

    def mf_set_jc_map(self, jc):
        self.jc = jc.clone()

    def mf_set_knot_values(self, values):
        self.kv = torch.tensor(values, dtype=torch.float64)

    def mf_film_solve_gradient(self, g0, target, steps, iters, ckpt_every=20, warm0=None,
                               grad=True, warm0_grad=False):
        self.calls += 1
        self.grads += int(grad)
        assert len(iters) == 3 * len(steps)
        loss = 0.5 * float(((self.jc - self.a) ** 2).sum() + ((self.kv - self.b) ** 2).sum())
        if not grad:
            return loss, None, None, None
        return loss, (self.jc - self.a).reshape(-1), (self.kv - self.b).tolist(), None


def test_gradients_flow_and_are_scaled():
    a = torch.randn(4, 6, dtype=torch.float64)
    b = torch.tensor([0.0, 0.2, 0.4], dtype=torch.float64)
    p = StandIn(a, b)
    jc = torch.ones(4, 6, dtype=torch.float64, requires_grad=True)
    kv = torch.tensor([0.1, 0.1, 0.1], dtype=torch.float64, requires_grad=True)
    loss = film_solve_loss(jc, kv, p, None, None, [(0.0, 0.1)], [3, 3, 3])
    (3.0 * loss).backward()
    assert p.calls == 1
    assert torch.allclose(jc.grad, 3.0 * (jc.detach() - a))
    assert torch.allclose(kv.grad, 3.0 * (kv.detach() - b))
    assert loss.item() == pytest.approx(0.5 * float(((1 - a) ** 2).sum() + ((kv.detach() - b) ** 2).sum()))


def test_parameters_are_set_before_the_solve():
    p = StandIn(torch.zeros(2, 2, dtype=torch.float64), torch.zeros(2, dtype=torch.float64))
    jc = torch.full((2, 2), 2.0, dtype=torch.float64)
    kv = torch.tensor([1.0, 3.0], dtype=torch.float64)
    with torch.no_grad():
        film_solve_loss(jc, kv, p, None, None, [(0.0, 0.1)], [1, 1, 1])
    assert torch.equal(p.jc, jc) and torch.equal(p.kv, kv)


def test_no_grad_forward_computes_the_loss_alone():
    p = StandIn(torch.zeros(2, 2, dtype=torch.float64), torch.zeros(2, dtype=torch.float64))
    jc = torch.full((2, 2), 2.0, dtype=torch.float64, requires_grad=True)
    kv = torch.tensor([1.0, 3.0], dtype=torch.float64, requires_grad=True)
    with torch.no_grad():
        loss = film_solve_loss(jc, kv, p, None, None, [(0.0, 0.1)], [1, 1, 1])
    assert p.calls == 1 and p.grads == 0
    assert loss.item() == pytest.approx(0.5 * (4 * 4.0 + 1.0 + 9.0))


def test_gradient_comes_back_on_the_parameter_device():
    """The problem's tensors may live elsewhere (a stand-in returns them as they are): the
    gradients are moved to the devices of jc and knots."""
    a = torch.zeros(3, 3, dtype=torch.float64)
    p = StandIn(a, torch.zeros(2, dtype=torch.float64))
    jc = torch.ones(3, 3, dtype=torch.float64, requires_grad=True)
    kv = torch.tensor([0.5, 0.5], dtype=torch.float64, requires_grad=True)
    film_solve_loss(jc, kv, p, None, None, [(0.0, 0.1)], [2, 2, 2]).backward()
    assert jc.grad.device == jc.device and kv.grad.device == kv.device
    assert torch.allclose(jc.grad, jc.detach() - a)
