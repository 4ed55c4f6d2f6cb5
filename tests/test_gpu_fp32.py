"""FP32-mixed CUDA path vs the FP64 CPU oracle (needs a GPU).

Tolerances: before the first split the FP32-mixed displacement field must
agree with the FP64 oracle to 1e-5 of its maximum (FP32 element arithmetic,
compensated displacement).  After initiation the crack pattern is compared
by Jaccard index of the cracked-element sets and reported."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def _pair(p, steps, state=None):
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, Solver
    o = from_problem(p)
    g = Solver(p, precision=CEM_FP32_MIXED)
    if state:
        o.set_state(**state)
        g.set_state(**state)
    o.step(steps)
    g.step(steps)
    return o, g


def rel_err(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


@pytest.mark.parametrize("nx,ny,steps", [(100, 40, 190), (400, 160, 700), (37, 19, 150)])
def test_field_error_before_initiation(nx, ny, steps):
    p = inputs.notched_plate(nx, ny, steps=steps)
    o, g = _pair(p, steps)
    assert g.counts()["n_cracked"] == o.counts()["n_crack"]  # only the notch so far
    on, gn = o.nodes(), g.nodes()
    for k in ("ux", "uy"):
        assert rel_err(gn[k], on[k]) < 1e-5, k
    for k in ("vx", "vy"):
        assert rel_err(gn[k], on[k]) < 1e-4, k
    np.testing.assert_array_equal(gn["m"], on["m"])


def test_random_field_error_and_energy():
    nx, ny = 45, 23
    p = inputs.notched_plate(nx, ny, lx=0.045, ly=0.023, notch_len=0.01, traction=1e6, steps=200)
    p.material.gc_uniform = 1e30
    p.energy_every = 10
    rng = np.random.default_rng(3)
    from oracle.oracle import from_problem
    n = from_problem(p).counts()["nn"] + from_problem(p).counts()["n_phantom"]
    st = dict(vx=rng.standard_normal(n) * 0.05, vy=rng.standard_normal(n) * 0.05)
    o, g = _pair(p, 200, st)
    on, gn = o.nodes(), g.nodes()
    for k in ("ux", "uy"):
        assert rel_err(gn[k], on[k]) < 1e-5, k
    oe, ge = o.energy(), g.energy()
    for k in ("KE", "SE", "W_ext"):
        np.testing.assert_allclose(ge[k], oe[k], rtol=0, atol=1e-4 * np.max(np.abs(oe[k])))


def test_crack_pattern_after_initiation_reported():
    """Whole 100 x 40 notched-plate run: FP32 runs end to end and its
    cracked-element set overlaps the FP64 oracle's (Jaccard reported)."""
    p = inputs.notched_plate(100, 40, steps=400, phantom_cap=20000, crack_cap=4000)
    o, g = _pair(p, 400)
    A = set(o.cracks()["elem"].tolist())
    B = set(g.cracks()["elem"].tolist())
    jac = len(A & B) / len(A | B)
    print(f"Jaccard FP32 vs FP64 oracle at step 400: {jac:.3f} ({len(A)} vs {len(B)})")
    assert jac > 0.5


@pytest.mark.parametrize("seed", [0, 1])
def test_bookkeeping_fp32_identical(seed):
    """Selection and split are shared with the FP64 mode: scripted proposals
    give the identical crack table, phantoms and masses."""
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, Solver
    rng = np.random.default_rng(seed)
    nx, ny = 10, 8
    p = inputs.Problem(name="bk32", nx=nx, ny=ny, hx=1e-3, hy=1e-3, phantom_cap=800, crack_cap=80)
    p.precracks = np.array([[4 * nx, 3, 1]], np.int32)
    o = from_problem(p)
    g = Solver(p, precision=CEM_FP32_MIXED)
    for rnd in range(5):
        ev = o.eval_surface()
        pick = np.nonzero(rng.random(len(ev["edge"])) < 0.5)[0]
        k = np.array([rng.choice([q for q in range(4) if q != k0]) for k0 in ev["k0"][pick]])
        G = rng.integers(1, 4, len(pick)).astype(np.float64)
        o.apply_proposals(ev["edge"][pick], ev["ahead"][pick], k, G)
        g.debug_apply_proposals(ev["edge"][pick], ev["ahead"][pick], k, G)
    oc, gc = o.cracks(), g.cracks()
    for key in ("elem", "ka", "kb"):
        np.testing.assert_array_equal(oc[key], gc[key])
    np.testing.assert_array_equal(oc["nodes"], gc["nodes"])
    np.testing.assert_array_equal(o.nodes()["m"], g.nodes()["m"])
