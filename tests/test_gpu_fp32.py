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


def test_crack_pattern_after_initiation_100x40():
    """Whole 100 x 40 notched-plate run to step 400 against the FP64 oracle:
    the cracked-element sets agree to the stated crack-pattern tolerance
    (Jaccard >= 0.9; crack counts within 10%)."""
    p = inputs.notched_plate(100, 40, steps=400, phantom_cap=20000, crack_cap=4000)
    o, g = _pair(p, 400)
    from paper_2509_01827_gb300 import metrics
    A, B = o.cracks()["elem"], g.cracks()["elem"]
    jac = metrics.jaccard(A, B)
    print(f"Jaccard FP32 vs FP64 oracle at step 400: {jac:.3f} ({len(A)} vs {len(B)})")
    assert jac >= 0.9
    assert abs(len(A) - len(B)) <= 0.1 * len(A)


def test_crack_pattern_notched_400x160_to_80us():
    """The 0.25 mm notched plate to 80 us: FP32-mixed against the FP64 mode
    (bit-identical to the oracle in the parity tests).  Stated tolerance:
    Jaccard >= 0.95, branching time within 2%, branch angle within 5
    degrees."""
    from paper_2509_01827_gb300 import metrics
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, CEM_FP64, Solver
    p = inputs.CONFIGS["notched_plate_400x160"]()
    tabs = {}
    for prec in (CEM_FP64, CEM_FP32_MIXED):
        g = Solver(p, precision=prec)
        g.step(p.steps)
        tabs[prec] = g.cracks()
        g.close()
    a, b = tabs[CEM_FP64], tabs[CEM_FP32_MIXED]
    jac = metrics.jaccard(a["elem"], b["elem"])
    sa = metrics.branching_step(a, p.nx, p.ny, p.hx, p.hy)
    sb = metrics.branching_step(b, p.nx, p.ny, p.hx, p.hy)
    aa, _ = metrics.branch_angle(a, p.nx, p.ny, p.hx, p.hy)
    ab, _ = metrics.branch_angle(b, p.nx, p.ny, p.hx, p.hy)
    print(f"400x160: Jaccard {jac:.4f}, branching step {sa} vs {sb}, angle {aa} vs {ab}")
    assert jac >= 0.95
    assert sa is not None and sb is not None and abs(sa - sb) <= 0.02 * sa
    assert aa is not None and ab is not None and abs(aa - ab) <= 5.0


@pytest.mark.parametrize("mode", ["neumann", "dirichlet"])
def test_fragmentation_fields_fp32(mode):
    """The benchmarked workload's ingredients in FP32-mixed mode -- hole rim
    loaded by the pressure pulse, or outer edges driven by the velocity ramp,
    Weibull G_c field (scaled up so that nothing splits in the window) --
    against the FP64 oracle over 400 steps: displacement within 1e-5 of its
    maximum, energies within 1e-4."""
    p = inputs.fragmentation(128, mode=mode, gc_mean=3e4, steps=400)
    p.energy_every = 20
    o, g = _pair(p, 400)
    assert o.counts()["n_crack"] == 0 and g.counts()["n_cracked"] == 0
    on, gn = o.nodes(), g.nodes()
    for k in ("ux", "uy"):
        assert rel_err(gn[k], on[k]) < 1e-5, k
    oe, ge = o.energy(), g.energy()
    for k in ("KE", "SE", "W_ext", "W_dir"):
        np.testing.assert_allclose(ge[k], oe[k], rtol=0, atol=1e-4 * max(np.max(np.abs(oe[k])), 1e-30),
                                   err_msg=k)


@pytest.mark.parametrize("mode", ["neumann", "dirichlet"])
def test_fragmentation_initiation_fp32(mode):
    """Weibull G_c field of the benchmark (mean 3 J/m^2): the first splits
    (chosen where G crosses the per-element G_c) are the oracle's up to the
    square plate's symmetries -- the hole and the loads are symmetric, so
    mirrored elements release the same G up to rounding and a neighbourhood
    maximum between them is a tie that rounding breaks -- and
    the cracked sets stay within Jaccard 0.95 over the next 100 steps (on a
    coarser 128 x 128 plate such ties are frequent enough that the patterns
    drift to Jaccard 0.6-0.8 in 100 steps; at 256 x 256 they agree)."""
    from paper_2509_01827_gb300 import metrics
    p = inputs.fragmentation(256, mode=mode, steps=0, phantom_cap=200000, crack_cap=60000)
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, Solver
    o = from_problem(p)
    g = Solver(p, precision=CEM_FP32_MIXED)
    s = 0
    while o.counts()["n_crack"] == 0 and s < 400:
        o.step(1)
        g.step(1)
        s += 1
    assert o.counts()["n_crack"] > 0
    A, B = set(o.cracks()["elem"].tolist()), set(g.cracks()["elem"].tolist())
    assert len(A) == len(B)
    n = p.nx

    def images(e):  # the element's images under the square's eight symmetries
        i, j = e % n, e // n
        out = set()
        for a, b in ((i, j), (j, i)):
            for x in (a, n - 1 - a):
                for y in (b, n - 1 - b):
                    out.add(y * n + x)
        return out
    assert all(images(e) & (B - A) for e in A - B), (sorted(A - B), sorted(B - A))
    o.step(100)
    g.step(100)
    jac = metrics.jaccard(o.cracks()["elem"], g.cracks()["elem"])
    print(f"{mode}: first split at step {s} ({len(A - B)} of {len(A)} mirrored); "
          f"Jaccard after 100 more steps {jac:.4f}")
    assert jac >= 0.95


@pytest.mark.parametrize("where", ["below_1e-6", "above_1e-6", "below_ulp", "above_ulp"])
def test_fp64_recheck_near_threshold(where):
    """One element under uniform eps_yy: the straight paths from the left and
    right edge points release G = 1/2 D11 e^2 hy exactly.  With G_c within
    1e-6 of G, or the FP32 neighbour of G on either side (6e-8 away), FP32
    arithmetic alone cannot order them; the FP64 re-check within 1e-3 of G_c
    makes the oracle's decision."""
    from oracle.oracle import from_problem
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, Solver
    h, e = 1e-3, 2e-4
    E, nu = 32e9, 0.2
    D11 = E * (1 - nu) / ((1 + nu) * (1 - 2 * nu))
    G = 0.5 * D11 * e * e * h
    p = inputs.Problem(name="recheck", nx=1, ny=1, hx=h, hy=h, phantom_cap=64, crack_cap=8)
    g32 = np.float32(G)
    gc = {"below_1e-6": np.float32(G * (1 - 1e-6)), "above_1e-6": np.float32(G * (1 + 1e-6)),
          "below_ulp": np.nextafter(g32, np.float32(0)) if g32 >= G else g32,
          "above_ulp": np.nextafter(g32, np.float32(1)) if g32 <= G else g32}[where]
    p.gc = np.array([gc], np.float32)
    uy = np.array([0.0, 0.0, e * h, e * h])
    o = from_problem(p)
    g = Solver(p, precision=CEM_FP32_MIXED)
    o.set_state(uy=uy)
    g.set_state(uy=uy)
    o.step(1)
    g.step(1)
    want = o.counts()["n_crack"]
    assert want == (1 if G > float(p.gc[0]) else 0)
    assert g.counts()["n_cracked"] == want


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
