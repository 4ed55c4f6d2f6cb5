"""Replaying steps in graphs of several steps (needs a GPU).

cem_step replays groups of consecutive steps as one CUDA graph, with single
steps wherever an energy record would fall inside a group.  The kernels and
their order are the same either way, so a run taken in one call must be
bit-identical to the same run taken one step per call (fields, masses,
splits, energy records), in both precisions."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_one_call_equals_single_steps(precision):
    from paper_2509_01827_gb300.cem import Solver
    p = inputs.notched_plate(100, 40, traction=3e6, steps=0, phantom_cap=20000, crack_cap=4000)
    p.energy_every = 10  # records at steps 0, 10, 20, ...: groups and single steps mix
    a, b = Solver(p, precision=precision), Solver(p, precision=precision)
    n = 237
    a.step(n)
    for _ in range(n):
        b.step(1)
    na, nb = a.nodes(), b.nodes()
    for k in ("ux", "uy", "vx", "vy", "m"):
        np.testing.assert_array_equal(na[k], nb[k], err_msg=k)
    ca, cb = a.cracks(), b.cracks()
    assert len(ca["elem"]) > 0  # the run splits elements
    for k in ("elem", "ka", "kb", "step", "ud", "nodes"):
        np.testing.assert_array_equal(ca[k], cb[k], err_msg=k)
    ea, eb = a.energy(), b.energy()
    for k in ("step", "KE", "SE", "W_ext", "W_dir", "U_d"):
        np.testing.assert_array_equal(ea[k], eb[k], err_msg=k)
    assert a.counts()["step"] == b.counts()["step"] == n
    a.close()
    b.close()


@pytest.mark.parametrize("precision,calls", [(0, "ones"), (1, "ones"), (0, "mixed"), (1, "mixed")])
def test_async_steps_equal_blocking_steps(precision, calls):
    """cem_step_async, each call collecting the previous call's status (and,
    for calls of at most 32 steps, every step's status word from the ring),
    then cem_sync, ends bit-identical to cem_step: one step per call, or a
    mix of 1-, 3-, 8-, 16- and 40-step calls (eight-step graphs with and
    without the per-step words, energy records inside them)."""
    from paper_2509_01827_gb300.cem import Solver
    p = inputs.notched_plate(100, 40, traction=3e6, steps=0, phantom_cap=20000, crack_cap=4000)
    p.energy_every = 10
    a, b = Solver(p, precision=precision), Solver(p, precision=precision)
    n = 237
    a.step(n)
    pattern = [1] if calls == "ones" else [1, 1, 8, 8, 3, 40, 8, 16, 1, 8]
    done, q = 0, 0
    while done < n:
        k = min(pattern[q % len(pattern)], n - done)
        b.step_async(k)
        done += k
        q += 1
    b.sync()
    na, nb = a.nodes(), b.nodes()
    for k in ("ux", "uy", "vx", "vy", "m"):
        np.testing.assert_array_equal(na[k], nb[k], err_msg=k)
    ca, cb = a.cracks(), b.cracks()
    assert len(ca["elem"]) > 0
    for k in ("elem", "ka", "kb", "step", "nodes"):
        np.testing.assert_array_equal(ca[k], cb[k], err_msg=k)
    ea, eb = a.energy(), b.energy()
    for k in ("step", "KE", "SE", "W_ext", "W_dir", "U_d"):
        np.testing.assert_array_equal(ea[k], eb[k], err_msg=k)
    assert b.counts()["step"] == n
    a.close()
    b.close()


def test_async_errors_come_one_call_late():
    """A non-finite state makes the steps of one cem_step_async call fail:
    that call returns, and the next call (or cem_sync) reports the error,
    from the per-step status words (3-step calls) or from the word copied
    after the call (40-step calls)."""
    from paper_2509_01827_gb300.cem import CEM_ERR_NONFINITE, CemError, Solver
    p = inputs.notched_plate(37, 19, steps=0)
    s = Solver(p, precision=1)
    vx = np.zeros(s.n_total())
    vx[5] = np.nan
    s.set_state(vx=vx)
    s.step_async(3)
    with pytest.raises(CemError) as ei:
        s.sync()
    assert ei.value.code == CEM_ERR_NONFINITE
    s.close()
    s = Solver(p, precision=1)
    s.set_state(vx=vx)
    s.step_async(3)
    with pytest.raises(CemError) as ei:
        s.step_async(1)
    assert ei.value.code == CEM_ERR_NONFINITE
    s.close()
    s = Solver(p, precision=1)
    s.set_state(vx=vx)
    s.step_async(40)
    with pytest.raises(CemError) as ei:
        s.step_async(40)
    assert ei.value.code == CEM_ERR_NONFINITE
    s.close()
