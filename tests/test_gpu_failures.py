"""Failure detection (needs a GPU; no GPU fault is made).

The device kernels report capacity overflows and non-finite states in a
status word that cem_step reads back after its steps; these tests provoke
both with valid inputs (tiny capacities, a NaN initial velocity) and check
that the host gets the right error, with the handle still usable."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def test_capacity_overflow_is_reported():
    from paper_2509_01827_gb300.cem import CEM_ERR_CAPACITY, CemError, Solver
    p = inputs.notched_plate(100, 40, traction=3e6, steps=0, phantom_cap=210, crack_cap=4000)
    s = Solver(p)  # the 50 pre-cracks need ~100 phantoms; growth needs more
    with pytest.raises(CemError) as ei:
        s.step(2000)
    assert ei.value.code == CEM_ERR_CAPACITY
    assert "phantoms" in str(ei.value)
    c = s.counts()  # the handle still answers
    assert c["n_phantoms"] <= 210


def test_nonfinite_state_is_reported():
    from paper_2509_01827_gb300.cem import CEM_ERR_NONFINITE, CemError, Solver
    p = inputs.notched_plate(37, 19, steps=0)
    for prec in (0, 1):
        s = Solver(p, precision=prec)
        n = s.n_total()
        vx = np.zeros(n)
        vx[5] = np.nan
        s.set_state(vx=vx)
        with pytest.raises(CemError) as ei:
            s.step(3)
        assert ei.value.code == CEM_ERR_NONFINITE
        s.close()


def test_batch_names_the_failing_member():
    from paper_2509_01827_gb300.cem import Batch, CEM_ERR_CAPACITY, CemError, Solver
    good = inputs.notched_plate(60, 24, steps=0, phantom_cap=20000, crack_cap=5000)
    bad = inputs.notched_plate(100, 40, traction=3e6, steps=0, phantom_cap=210, crack_cap=4000)
    members = [Solver(good), Solver(bad)]
    b = Batch(members)
    with pytest.raises(CemError) as ei:
        b.step(2000)
    assert ei.value.code == CEM_ERR_CAPACITY
    assert "member 1" in str(ei.value)
    b.close()


def test_argument_errors():
    from paper_2509_01827_gb300 import cem
    from paper_2509_01827_gb300.cem import CEM_ERR_ARG, CEM_ERR_STATE, CemError, Solver
    s = Solver(inputs.notched_plate(20, 8, steps=0))
    with pytest.raises(CemError) as ei:
        s.step(-1)
    assert ei.value.code == CEM_ERR_ARG
    s.step(1)
    with pytest.raises(CemError) as ei:
        s.set_state(vx=np.zeros(s.n_total()))  # only before the first step
    assert ei.value.code == CEM_ERR_STATE
