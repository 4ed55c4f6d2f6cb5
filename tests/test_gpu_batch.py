"""Batched stepping of independent meshes (needs a GPU).

A batch runs one launch per kernel kind for all its members.  Each member
must end exactly where it ends when stepped alone: bit-identical in FP64
(fields, masses, cracks, energy records); in the FP32-mixed mode fields,
masses and cracks are bit-identical too (a node's arithmetic does not depend
on the tiling), while the energy records sum FP32 partials per tile, and the
tile height of a mesh stepped alone is sized to the GPU, so they agree to
1e-6; members stop at their own step limits."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def _specimens():
    """Three notched plates of different sizes, notches and tractions."""
    out = []
    for (nx, ny, notch, trac) in [(60, 24, 0.025, 2.5e6), (100, 40, 0.05, 1e6), (37, 19, 0.02, 3e6)]:
        p = inputs.notched_plate(nx, ny, notch_len=notch, traction=trac, steps=0,
                                 phantom_cap=4000, crack_cap=2000)
        p.energy_every = 10
        out.append(p)
    return out


def _state(s):
    n = s.nodes()
    c = s.cracks()
    e = s.energy()
    return n, c, e


def _assert_same(a, b, energy_rtol=0.0):
    (na, ca, ea), (nb, cb, eb) = a, b
    for k in ("ux", "uy", "vx", "vy", "m"):
        np.testing.assert_array_equal(na[k], nb[k], err_msg=k)
    for k in ("elem", "ka", "kb", "step", "ud", "nodes"):
        np.testing.assert_array_equal(ca[k], cb[k], err_msg=k)
    np.testing.assert_array_equal(ea["step"], eb["step"])
    for k in ("KE", "SE", "W_ext", "W_dir", "U_d"):
        if energy_rtol:
            scale = max(np.max(np.abs(eb[k])), 1e-300)
            np.testing.assert_allclose(ea[k], eb[k], rtol=0, atol=energy_rtol * scale, err_msg=k)
        else:
            np.testing.assert_array_equal(ea[k], eb[k], err_msg=k)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_solo_runs(precision):
    from paper_2509_01827_gb300.cem import Batch, Solver
    probs = _specimens()
    limits = [250, 400, 180]
    solo = []
    for p, lim in zip(probs, limits):
        s = Solver(p, precision=precision)
        s.step(lim)
        solo.append(_state(s))
        s.close()
    members = [Solver(p, precision=precision) for p in probs]
    b = Batch(members, step_end=limits)
    b.step(150)
    b.step(300)  # beyond every limit: members stop at theirs
    assert b.counts()["step"] == 450
    for m, lim, ref in zip(members, limits, solo):
        assert m.counts()["step"] == lim
        _assert_same(_state(m), ref, energy_rtol=1e-6 if precision == 1 else 0.0)
    assert sum(len(r[1]["elem"]) for r in solo) > 3 * 50  # the notches grew
    b.close()


def test_batch_members_equal_the_oracle_fp64():
    """Each FP64 member of a batch against the CPU oracle directly (not only
    against its own solo run): fields, masses, crack and phantom tables and
    energies identical.  One member is drawn at the 400 x 160 end of the
    64-specimen batch's size range (the largest mesh that batch holds)."""
    from tests._parity import compare_energy, compare_fp64
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import Batch, Solver
    probs = _specimens()[:2]
    big = inputs.notched_plate(400, 160, notch_len=0.04, traction=2.5e6, steps=0,
                               phantom_cap=40000, crack_cap=16000)
    big.energy_every = 10
    probs.append(big)
    limits = [300, 220, 420]
    members = [Solver(p) for p in probs]
    b = Batch(members, step_end=limits)
    b.step(max(limits))
    for p, m, lim in zip(probs, members, limits):
        o = from_problem(p)
        o.step(lim)
        compare_fp64(o, m)
        compare_energy(o, m)
    assert members[2].counts()["n_cracked"] > 170  # the notch row plus growth
    b.close()


def test_fp32_tile_rows_give_identical_fields():
    """The node update's tile height changes which warp marches a node, not
    the node's arithmetic: FP32-mixed fields are bit-identical for tile
    heights 8, 16, 32 and 64, through crack initiation."""
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, Batch, Solver
    probs = _specimens()
    runs = []
    for rows in (16, 8, 32, 64):
        members = [Solver(p, precision=CEM_FP32_MIXED) for p in probs]
        b = Batch(members)
        b.set_config(rows, 152)
        b.step(260)
        runs.append([(m.nodes(), m.cracks()) for m in members])
        b.close()
    for other in runs[1:]:
        for (a, ca), (c, cc) in zip(runs[0], other):
            for k in ("ux", "uy", "vx", "vy", "m"):
                np.testing.assert_array_equal(a[k], c[k], err_msg=k)
            np.testing.assert_array_equal(ca["elem"], cc["elem"])


def test_autotune_keeps_results_fp64():
    from paper_2509_01827_gb300.cem import Batch, Solver
    probs = _specimens()
    members = [Solver(p) for p in probs]
    b = Batch(members)
    rows, grid = b.autotune(3)
    assert rows in (8, 16) and grid >= 1
    done = b.counts()["step"]
    assert done == 4 * (1 + 3)  # FP64: four grid candidates, 1 untimed + 3 timed steps each
    b.step(100)
    total = b.counts()["step"]
    for p, m in zip(probs, members):
        s = Solver(p)
        s.step(total)
        _assert_same(_state(m), _state(s))
        s.close()
    b.close()


def test_batch_rules():
    from paper_2509_01827_gb300.cem import Batch, CemError, Solver, CEM_ERR_STATE, CEM_ERR_ARG
    probs = _specimens()
    members = [Solver(p) for p in probs]
    b = Batch(members)
    with pytest.raises(CemError) as ei:
        members[0].step(1)  # a member is stepped by its batch
    assert ei.value.code == CEM_ERR_STATE
    from paper_2509_01827_gb300 import cem
    with pytest.raises(CemError) as ei:
        cem.cem_get_cracks(b.h, 4)  # getters read members
    assert ei.value.code == CEM_ERR_STATE
    with pytest.raises(CemError) as ei:
        Batch(members[:1])  # already in a batch
    assert ei.value.code == CEM_ERR_STATE
    b.step(5)
    members[1].close()  # detaches it; the batch refuses to step
    with pytest.raises(CemError) as ei:
        b.step(1)
    assert ei.value.code == CEM_ERR_STATE
    b.close()
    members[0].step(1)  # free again once the batch is gone
    other = Solver(probs[0])
    other.step(1)
    with pytest.raises(CemError) as ei:
        Batch([members[0], other])  # different steps
    assert ei.value.code == CEM_ERR_ARG
