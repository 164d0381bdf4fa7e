"""The allocation-free entry point (sph_density_small_noalloc) against the
regular one (sph_build + sph_density) on the same small boxes.

sph_density_small_noalloc exists for callers that cannot call cudaMalloc
(code inside a framework that owns all device memory, real-time paths,
applications with a fixed device footprint); it keeps its solver scratch in
a file-scope device array.  This file is collected last so that a failure
here cannot hide another test; it also passes alone in a fresh process.
Both calls of a pair must agree with the regular path within the density /
smoothing-length tolerance of the parity tests (1e-5 relative): the second
call checks that what the shared array keeps from the first call does not
leak into the next result.  The first call is also held to the FP64 oracle
(the definition both paths approximate) at the same tolerance."""
import numpy as np
import pytest
import torch

import synth.configs as C
from oracle import sph_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("make", [lambda: C.uniform_lattice(16, seed=1),
                                  lambda: C.random_box(3000, 23, "clumped")],
                         ids=["lattice16", "clumped3000"])
def test_noalloc_matches_regular_entry_point_twice(make):
    from paper_1404_2303_gb300 import SPH
    from paper_1404_2303_gb300.sph import density_small_noalloc
    d = make()
    pos, m = _t(d["x"]), _t(d["m"])
    hg = None if d["h_guess"] is None else _t(d["h_guess"])
    s = SPH()
    s.build(pos, h_guess=hg)
    ref = s.density(m)
    h_ref = ref["h"].cpu().numpy().astype(np.float64)
    rho_ref = ref["rho"].cpu().numpy().astype(np.float64)
    orc = O.evaluate(d["x"], d["m"], np.ones(len(d["m"])),
                     h_guess=None if d["h_guess"] is None else d["h_guess"].astype(np.float64))
    for call in range(2):
        h, rho, iters = density_small_noalloc(pos, m, h_guess=hg)
        torch.cuda.synchronize()
        h = h.cpu().numpy().astype(np.float64)
        rho = rho.cpu().numpy().astype(np.float64)
        assert iters >= 1
        assert np.max(np.abs(h - h_ref) / h_ref) <= TOL, call
        assert np.max(np.abs(rho - rho_ref) / rho_ref) <= TOL, call
        if call == 0:
            assert np.max(np.abs(h - orc["h"]) / orc["h"]) <= TOL
            assert np.max(np.abs(rho - orc["rho"]) / orc["rho"]) <= TOL


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_1404_2303_gb300._lib import NOALLOC_MAX_N, SphError
    from paper_1404_2303_gb300.sph import density_small_noalloc
    n = NOALLOC_MAX_N + 1
    pos = torch.zeros((n, 3), device="cuda", dtype=torch.float64)
    m = torch.ones(n, device="cuda")
    with pytest.raises(SphError) as e:
        density_small_noalloc(pos, m)
    assert e.value.code == -1
