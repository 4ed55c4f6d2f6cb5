"""FP64 CUDA path vs the CPU oracle, element by element (needs a GPU)."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs
from tests._parity import compare_energy, compare_fp64, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


@pytest.mark.parametrize("steps", [1, 2, 150, 260])
def test_notched_plate_100x40_prefix(steps):
    """Before, at and just after the first split of the notched plate."""
    p = inputs.notched_plate(100, 40, steps=steps)
    o, g = run_pair(p, steps)
    compare_fp64(o, g)


def test_notched_plate_100x40_full_run():
    """The whole 2000-step run (the mesh fractures heavily late in the run)."""
    p = inputs.notched_plate(100, 40, steps=2000, phantom_cap=20000, crack_cap=4000)
    p.energy_every = 50
    o, g = run_pair(p, 2000, chunks=[700, 600, 700])
    compare_fp64(o, g)
    compare_energy(o, g)
    assert g.counts()["n_cracked"] > 100


@pytest.mark.parametrize("nx,ny,seed", [(37, 19, 0), (70, 13, 1), (33, 9, 2), (5, 3, 3)])
def test_ragged_meshes_random_state(nx, ny, seed):
    """Tile-ragged meshes with a random initial field, a pre-crack, tractions
    and a low G_c so that many splits happen."""
    rng = np.random.default_rng(seed)
    p = inputs.notched_plate(nx, ny, lx=nx * 1e-3, ly=ny * 1e-3, notch_len=min(nx // 3, 10) * 1e-3,
                             traction=2e6, steps=300, phantom_cap=8 * nx * ny, crack_cap=nx * ny)
    p.material.gc_uniform = 0.5
    p.energy_every = 7
    nn = (nx + 1) * (ny + 1)
    st = dict(vx=rng.standard_normal(nn) * 0.3, vy=rng.standard_normal(nn) * 0.3)
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import Solver
    o = from_problem(p)
    g = Solver(p)
    n = o.counts()["nn"] + o.counts()["n_phantom"]
    st = dict(vx=rng.standard_normal(n) * 0.3, vy=rng.standard_normal(n) * 0.3)
    o.set_state(**st)
    g.set_state(**st)
    for chunk in (1, 99, 200):
        o.step(chunk)
        g.step(chunk)
        compare_fp64(o, g)
    compare_energy(o, g)


@pytest.mark.parametrize("scope", [inputs.SCOPE_GLOBAL, inputs.SCOPE_TIPS])
def test_selection_scopes(scope):
    p = inputs.notched_plate(60, 24, lx=0.06, ly=0.024, notch_len=0.02, traction=3e6, steps=400,
                             phantom_cap=20000, crack_cap=1440)
    p.material.scope = scope
    o, g = run_pair(p, 400, chunks=[200, 200])
    compare_fp64(o, g)
    assert g.counts()["n_cracked"] > 20


@pytest.mark.parametrize("mode", ["neumann", "dirichlet"])
def test_fragmentation_small(mode):
    """Square plate with a hole, Weibull G_c, pressure pulse or edge velocity."""
    p = inputs.fragmentation(96, mode=mode, r=0.012, p0=150e6, v0=15.0, steps=0,
                             phantom_cap=60000, crack_cap=9216)
    p.energy_every = 25
    o, g = run_pair(p, 500, chunks=[250, 250])
    compare_fp64(o, g)
    compare_energy(o, g)


def test_gamma_ratio_mode():
    p = inputs.notched_plate(50, 20, lx=0.05, ly=0.02, notch_len=0.02, traction=3e6, steps=300,
                             phantom_cap=10000, crack_cap=1000)
    p.material.gamma_mode = 1
    p.material.gamma = 1.05
    o, g = run_pair(p, 300)
    compare_fp64(o, g)


@pytest.mark.parametrize("nx,ny,seed,scope", [(4, 3, 0, 0), (8, 8, 2, 0), (8, 8, 3, 1),
                                              (8, 8, 4, 2), (12, 9, 5, 0)])
def test_bookkeeping_scripted_proposals(nx, ny, seed, scope):
    """Scripted proposals (with exact ties) through the test hook: identical
    winners, phantoms, masses, momenta and surface lists."""
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import Solver
    rng = np.random.default_rng(seed)
    h = 1e-3
    act = np.ones(nx * ny, np.uint8)
    if nx * ny > 30:
        act[rng.integers(nx * ny)] = 0
    p = inputs.Problem(name="bk", nx=nx, ny=ny, hx=h, hy=h, active=act,
                       phantom_cap=10 * nx * ny, crack_cap=nx * ny)
    p.material.scope = scope
    e0 = (ny // 2) * nx
    if act[e0]:
        p.precracks = np.array([[e0, 3, 1]], np.int32)
    o = from_problem(p)
    g = Solver(p)
    n = o.counts()["nn"] + o.counts()["n_phantom"]
    st = dict(vx=rng.standard_normal(n), vy=rng.standard_normal(n))
    o.set_state(**st)
    g.set_state(**st)
    for rnd in range(6):
        ev = o.eval_surface()
        m = len(ev["edge"])
        pick = np.nonzero(rng.random(m) < 0.5)[0]
        if len(pick) == 0:
            continue
        edge = ev["edge"][pick]
        elem = ev["ahead"][pick]
        k = np.array([rng.choice([q for q in range(4) if q != k0]) for k0 in ev["k0"][pick]])
        G = rng.integers(1, 4, len(pick)).astype(np.float64)
        o.apply_proposals(edge, elem, k, G)
        g.debug_apply_proposals(edge, elem, k, G)
        compare_fp64(o, g)


def test_fragmentation_full_size_first_steps():
    """2048 x 2048 fragmentation plate (the benchmark mesh), 4 FP64 steps,
    compared at every node."""
    p = inputs.fragmentation(2048, mode="neumann")
    o, g = run_pair(p, 4, chunks=[1, 3])
    compare_fp64(o, g)


def test_bookkeeping_more_proposals_than_staged():
    """A step with more proposals than the selection stages in shared memory
    (1024): the sort, winners and plans run on the global scratch and still
    match the oracle exactly.  A 64x64 mesh with a fifth of its elements
    inactive has thousands of surface points."""
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import Solver
    rng = np.random.default_rng(11)
    nx = ny = 64
    act = (rng.random(nx * ny) >= 0.2).astype(np.uint8)
    p = inputs.Problem(name="bk_many", nx=nx, ny=ny, hx=1e-3, hy=1e-3, active=act,
                       phantom_cap=20 * nx * ny, crack_cap=nx * ny)
    o = from_problem(p)
    g = Solver(p)
    n = o.counts()["nn"] + o.counts()["n_phantom"]
    st = dict(vx=rng.standard_normal(n), vy=rng.standard_normal(n))
    o.set_state(**st)
    g.set_state(**st)
    staged = 0
    for rnd in range(3):
        ev = o.eval_surface()
        pick = np.nonzero(rng.random(len(ev["edge"])) < 0.8)[0]
        staged = max(staged, len(pick))
        edge, elem = ev["edge"][pick], ev["ahead"][pick]
        k = np.array([rng.choice([q for q in range(4) if q != k0]) for k0 in ev["k0"][pick]])
        G = rng.integers(1, 6, len(pick)).astype(np.float64)
        o.apply_proposals(edge, elem, k, G)
        g.debug_apply_proposals(edge, elem, k, G)
        compare_fp64(o, g)
    assert staged > 1024


@pytest.mark.parametrize("precision,steps,tol", [(0, 260, 1e-12), (1, 150, 1e-4)])
def test_element_stress_and_sigma1(precision, steps, tol):
    """Element mean stress and its largest principal value (the stress
    contour outputs, CEM_FIELD_SIGMA / CEM_FIELD_SIGMA1) against the oracle's
    element stresses: FP64 after splits to 1e-12 of the largest stress, FP32
    before initiation to 1e-4."""
    p = inputs.notched_plate(100, 40, steps=steps)
    o, g = run_pair(p, steps, precision=precision)
    want = o.element_stress()
    got = g.element_stress()
    scale = np.max(np.abs(want))
    np.testing.assert_allclose(got, want, rtol=0, atol=tol * scale)
    h = 0.5 * (want[:, 0] - want[:, 1])
    s1 = 0.5 * (want[:, 0] + want[:, 1]) + np.sqrt(h * h + want[:, 2] ** 2)
    np.testing.assert_allclose(g.sigma1(), s1, rtol=0, atol=tol * scale)
    if precision == 0:
        assert g.counts()["n_cracked"] > len(p.precracks)  # split elements are covered


@pytest.mark.parametrize("scope", [inputs.SCOPE_NBHD, inputs.SCOPE_TIPS])
def test_kalthoff_plate(scope):
    """Upper half of the Kalthoff-Winkler plate (Sec. 4.1 steel, impact ramp
    on the left edge below the notch, symmetry line held at v_y = 0) in the
    multiple-tips (MCT) and single-tip (SCT) scopes, to 90 us on a 2 mm
    mesh: bit-identical to the oracle; the crack starts at the notch tip."""
    p = inputs.kalthoff(50, scope=scope)
    o, g = run_pair(p, p.steps, chunks=[250, p.steps - 250])
    compare_fp64(o, g)
    assert g.counts()["n_cracked"] > len(p.precracks)


@pytest.mark.parametrize("v0", [1.375, 3.993])
def test_compact_tension_plate(v0):
    """Dirichlet compact-tension plate (Sec. 4.3 velocity law on the notch
    faces, our square approximation of its geometry) at the slowest and the
    fastest loading rate of Sec. 4.3, 40 x 40 mesh to 200 us: bit-identical
    to the oracle, with the crack grown from the notch."""
    p = inputs.compact_tension(40, v0=v0)
    p.energy_every = 25
    o, g = run_pair(p, p.steps, chunks=[100, p.steps - 100])
    compare_fp64(o, g)
    assert g.counts()["n_cracked"] > len(p.precracks)
