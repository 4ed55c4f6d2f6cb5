"""Fragment count on the device (cem_get_fragments; needs a GPU) against the
host definition in metrics.fragments, which the CPU tests check against
brute force and against pre-cut meshes whose count geometry fixes."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs, metrics

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode,steps", [("neumann", 600), ("dirichlet", 400)])
def test_fragments_match_the_host_definition(precision, mode, steps):
    from paper_2509_01827_gb300.cem import Solver
    p = inputs.fragmentation(96, mode=mode, r=0.012, p0=150e6, v0=15.0, steps=0,
                             phantom_cap=60000, crack_cap=9216)
    g = Solver(p, precision=precision)
    n0, _ = g.fragments()
    assert n0 == 1
    g.step(steps)
    n, lab = g.fragments()
    want, want_lab = metrics.fragments(g.cracks(), p.nx, p.ny, p.active)
    assert n == want
    np.testing.assert_array_equal(lab, want_lab)
    assert n > 1  # the plate did break up
    print(f"{mode} fp{64 if precision == 0 else 32}: {n} fragments after {steps} steps")


def test_fragments_of_pre_cut_plate():
    """A full-width row of pre-cracks cuts the plate in two; the lower half's
    pieces take fragment 0 (it holds element 0)."""
    from paper_2509_01827_gb300.cem import Solver
    nx, ny = 30, 12
    p = inputs.Problem(name="cut", nx=nx, ny=ny, hx=1e-3, hy=1e-3)
    p.precracks = np.array([[5 * nx + i, 3, 1] for i in range(nx)], np.int32)
    g = Solver(p)
    n, lab = g.fragments()
    assert n == 2
    assert lab[0, 0] == 0 and lab[(ny - 1) * nx, 0] == 1
