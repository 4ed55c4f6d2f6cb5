"""Checkpoint and restart (cem_save_state / cem_load_state; needs a GPU).

A run of 2N steps and a run of N steps, saved, loaded into a fresh handle
and run N more steps must end bit-identical -- fields, masses, split and
phantom tables, surface list and energy records -- in both precisions, with
splits happening on both sides of the checkpoint."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def _plate():
    p = inputs.notched_plate(60, 24, lx=0.06, ly=0.024, notch_len=0.02, traction=3e6, steps=0,
                             phantom_cap=20000, crack_cap=1440)
    p.energy_every = 20
    return p


def _snapshot(s):
    n = s.nodes()
    return (n, s.cracks(), s.phantoms(), s.surface(), s.energy(), s.counts())


def _assert_same(a, b):
    (na, ca, pa, sa, ea, ka), (nb, cb, pb, sb, eb, kb) = a, b
    for k in ("ux", "uy", "vx", "vy", "m"):
        np.testing.assert_array_equal(na[k], nb[k], err_msg=k)
    for k in ("elem", "ka", "kb", "step", "ud", "nodes"):
        np.testing.assert_array_equal(ca[k], cb[k], err_msg=k)
    for k in ("owner", "creator_e", "creator_a", "nuser", "users"):
        np.testing.assert_array_equal(pa[k], pb[k], err_msg=k)
    for k in ("edge", "ahead", "is_tip"):
        np.testing.assert_array_equal(sa[k], sb[k], err_msg=k)
    for k in ("step", "t", "KE", "SE", "W_ext", "W_dir", "U_d"):
        np.testing.assert_array_equal(ea[k], eb[k], err_msg=k)
    for k in ("step", "n_phantoms", "n_cracked", "n_surface", "n_tips", "n_energy"):
        assert ka[k] == kb[k], k


@pytest.mark.parametrize("precision", [0, 1])
def test_save_load_resume_is_bit_identical(precision):
    from paper_2509_01827_gb300.cem import Solver
    N = 170
    a = Solver(_plate(), precision=precision)
    a.step(N)
    n_mid = a.counts()["n_cracked"]
    a.step(N)
    ref = _snapshot(a)
    assert ref[5]["n_cracked"] > n_mid > len(_plate().precracks)  # splits on both sides
    b = Solver(_plate(), precision=precision)
    b.step(N)
    blob = b.save_state()
    b.close()
    c = Solver(_plate(), precision=precision)
    c.load_state(blob)
    assert c.counts()["step"] == N and c.counts()["n_cracked"] == n_mid
    c.step(N)
    _assert_same(_snapshot(c), ref)
    a.close()
    c.close()


def test_load_checks_mesh_precision_and_capacity():
    from paper_2509_01827_gb300.cem import (CEM_ERR_ARG, CEM_ERR_CAPACITY, CEM_FP32_MIXED,
                                            CemError, Solver)
    s = Solver(_plate())
    s.step(300)
    blob = s.save_state()
    with pytest.raises(CemError) as ei:
        Solver(_plate(), precision=CEM_FP32_MIXED).load_state(blob)
    assert ei.value.code == CEM_ERR_ARG
    other = inputs.notched_plate(61, 24, lx=0.061, ly=0.024, notch_len=0.02, traction=3e6, steps=0)
    with pytest.raises(CemError) as ei:
        Solver(other).load_state(blob)
    assert ei.value.code == CEM_ERR_ARG
    small = _plate()
    small.phantom_cap = 200
    small.crack_cap = 40
    with pytest.raises(CemError) as ei:
        Solver(small).load_state(blob)
    assert ei.value.code == CEM_ERR_CAPACITY
    with pytest.raises(CemError) as ei:
        Solver(_plate()).load_state(blob[:100])
    assert ei.value.code == CEM_ERR_ARG
