"""Host logic of the autograd wrapper (ThermalObjective) on CPU: with the library's adjoint
sweep replaced by a stand-in that returns known J and dJ/d(P, s), the Function returns J per
instance and its backward pass delivers the incoming gradient times the stored one, for P and
s separately and on their own devices and dtypes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_backward_scales_the_stored_gradient(monkeypatch):
    from paper_2302_05164_gb300 import autograd as A
    batch, n_seg = 3, 4
    grad = np.arange(batch * (n_seg + 1), dtype=np.float64).reshape(batch, n_seg + 1) + 1.0
    J = np.array([2.0, 3.0, 5.0])
    seen = {}

    def fake_sweep(h, T0, ls, t0, dt, nsteps, ncp, T_target=2300.0, p_exp=16.0, batch=1):
        seen.update(power=np.array(ls["power"]), batch=batch, nsteps=nsteps, ncp=ncp)
        return J.copy(), grad.copy(), nsteps

    monkeypatch.setattr(A.pbf, "pbf_adjoint_sweep", fake_sweep)
    monkeypatch.setattr(A.pbf, "pbf_ctx_set_k_scale", lambda h, s: seen.update(s=np.array(s)))
    P = torch.tensor(np.full((batch, n_seg), 200.0), requires_grad=True)
    s = torch.tensor([0.9, 1.0, 1.1], requires_grad=True)
    laser = dict(seg=np.zeros((n_seg, 6)), power=np.zeros((1, n_seg)), eta=0.35, radius=40e-6)
    out = A.ThermalObjective.apply(P, s, None, None, laser, 0.0, 1e-8, 7, 3)
    assert np.array_equal(out.detach().numpy(), J)
    assert np.array_equal(seen["power"], P.detach().numpy()) and np.array_equal(seen["s"], s.detach().numpy())
    assert seen["batch"] == batch and seen["nsteps"] == 7 and seen["ncp"] == 3
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64)
    (w * out).sum().backward()
    assert np.allclose(P.grad.numpy(), w.numpy()[:, None] * grad[:, :-1], rtol=0, atol=0)
    assert np.allclose(s.grad.numpy(), w.numpy() * grad[:, -1], rtol=0, atol=0)


def test_shape_mismatch_is_rejected(monkeypatch):
    from paper_2302_05164_gb300 import autograd as A
    P = torch.zeros((2, 3), dtype=torch.float64, requires_grad=True)
    s = torch.zeros(3, dtype=torch.float64, requires_grad=True)
    with pytest.raises(ValueError):
        A.ThermalObjective.apply(P, s, None, None, {}, 0.0, 1e-8, 1, 1)
