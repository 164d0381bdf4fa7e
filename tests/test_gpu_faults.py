"""Robustness of the C ABI against bad inputs, and run-to-run determinism.
Every failure here is made on the host side of the interface or by an
input that the library's own checks turn into an error status: non-finite
positions, non-positive or non-finite h guesses, an empty set, a box too
small for the smoothing lengths, and an h iteration cut short
(max_newton = 1).  Nothing faults, traps or hangs the GPU."""
import numpy as np
import pytest
import torch

import synth.configs as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _code(fn):
    from paper_1404_2303_gb300._lib import SphError
    with pytest.raises(SphError) as e:
        fn()
    return e.value.code


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
def test_non_finite_positions_are_rejected(bad):
    from paper_1404_2303_gb300 import SPH
    d = C.random_box(4000, 3, "uniform")
    x = d["x"].copy()
    x[1234, 1] = bad
    s = SPH()
    assert _code(lambda: s.build(_t(x))) == -1
    with pytest.raises(Exception):
        s.density(_t(d["m"]))  # nothing usable was built
    s.build(_t(d["x"]))  # the context recovers with good input
    s.density(_t(d["m"]))


@pytest.mark.parametrize("bad", [0.0, -0.01, np.nan, np.inf])
def test_bad_h_guesses_are_rejected(bad):
    from paper_1404_2303_gb300 import SPH
    d = C.random_box(4000, 3, "uniform")
    hg = np.full(4000, 0.05, np.float32)
    hg[17] = bad
    assert _code(lambda: SPH().build(_t(d["x"]), h_guess=_t(hg))) == -1


def test_empty_set_and_too_small_box():
    from paper_1404_2303_gb300 import SPH
    s = SPH()
    assert _code(lambda: s.build(torch.zeros((0, 3), device="cuda", dtype=torch.float64))) == -1
    d = C.random_box(4000, 3, "uniform")
    # an h guess above a quarter of the box admits no top grid of at least 4 cells per axis
    assert _code(lambda: s.build(_t(d["x"]), box=1.0,
                                 h_guess=_t(np.full(4000, 0.3, np.float32)))) == -1


def test_h_iteration_cut_short_reports_not_converged():
    from paper_1404_2303_gb300 import SPH
    d = C.random_box(20000, 7, "clumped")
    s = SPH(max_newton=1)
    s.build(_t(d["x"]))
    assert _code(lambda: s.density(_t(d["m"]))) == -4
    assert s.stats()["unconverged"] > 0


def test_full_step_is_bitwise_deterministic():
    from paper_1404_2303_gb300 import SPH
    d = C.random_box(30000, 19, "clumped", v_sigma=0.1)
    outs = []
    for _ in range(2):
        s = SPH()
        s.build(_t(d["x"]))
        den = s.density(_t(d["m"]))
        acc, dudt, _ = s.force(_t(d["u"]), _t(d["v"]))
        g = s.adjoint(2.0 * (den["rho"] - 1.0), 2.0 * acc, dudt)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in (den["h"], den["rho"], acc, dudt, *g)])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
