"""The torch.autograd.Function over the C ABI (sph_density_force): a
backward through the hand-written adjoint kernels against the FP64 oracle
gradient, every element of dL/dx, dL/dm and dL/du within
1e-3 (rms(g) + |g_i|); the guards against a context whose forward state was
replaced before backward, and against velocities that require grad (they
are constants of the adjoint)."""
import numpy as np
import pytest
import torch

from oracle import sph_oracle as O
import synth.configs as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _t(a, **kw):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").clone().requires_grad_(
        kw.get("grad", False))


@pytest.mark.parametrize("case", ["sinusoid16", "clumped4000"])
def test_backward_matches_oracle_gradient(case):
    from paper_1404_2303_gb300 import SPH, sph_density_force
    d = C.sinusoid(16, seed=4) if case == "sinusoid16" else C.random_box(4000, 29, "clumped",
                                                                       v_sigma=0.1)
    pos = _t(d["x"], grad=True)
    m = _t(d["m"], grad=True)
    u = _t(d["u"], grad=True)
    vel = _t(d["v"])
    rho, acc, dudt, h = sph_density_force(pos, m, u, vel, sph=SPH())
    w = torch.as_tensor(np.random.default_rng(3).normal(size=d["x"].shape[0]).astype(np.float32),
                        device="cuda")
    loss = ((rho - 1.0) ** 2).sum() + (acc ** 2).sum() + (w * dudt).sum()
    loss.backward()
    assert pos.grad.dtype == torch.float64
    ref = O.evaluate(d["x"], d["m"], d["u"], v=d["v"], h_guess=0.1)
    gref = O.gradient(ref, d["x"], d["m"], d["u"], d["v"].astype(np.float64),
                      2.0 * (rho.detach().double().cpu().numpy() - 1.0),
                      2.0 * acc.detach().double().cpu().numpy(),
                      w.double().cpu().numpy())
    for got, want in ((pos.grad, gref["g_x"]), (m.grad, gref["g_m"]), (u.grad, gref["g_u"])):
        gg = got.detach().double().cpu().numpy().reshape(want.shape)
        rms = np.sqrt(np.mean(want ** 2))
        err = np.abs(gg - want) / (rms + np.abs(want))
        assert err.max() <= 1e-3, (case, float(err.max()))


def test_backward_refuses_a_replaced_forward_state():
    from paper_1404_2303_gb300 import SPH, sph_density_force
    d = C.random_box(3000, 5, "uniform")
    s = SPH()
    pos = _t(d["x"], grad=True)
    rho, acc, _, _ = sph_density_force(pos, _t(d["m"]), _t(d["u"]), sph=s)
    sph_density_force(_t(d["x"]), _t(d["m"]), _t(d["u"]), sph=s)  # a second forward, same context
    with pytest.raises(RuntimeError):
        (acc ** 2).sum().backward()


def test_velocities_that_require_grad_are_refused():
    from paper_1404_2303_gb300 import SPH, sph_density_force
    d = C.random_box(3000, 5, "uniform", v_sigma=0.1)
    with pytest.raises(ValueError):
        sph_density_force(_t(d["x"]), _t(d["m"]), _t(d["u"]), _t(d["v"], grad=True), sph=SPH())
