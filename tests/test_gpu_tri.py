"""Constant-strain triangles on unstructured meshes (Sec. 2.1, Eqs. 1, 3, 5):
the CUDA path (cem_tri_mesh_create) against the CST oracle, FP64, bit for
bit on the fields, energies within 1e-12 (needs a GPU)."""
import numpy as np
import pytest

from paper_2509_01827_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def _pair(p, chunks):
    from oracle.cst_oracle import from_problem
    from paper_2509_01827_gb300.cem import TriSolver
    o = from_problem(p)
    g = TriSolver(p)
    for n in chunks:
        o.step(n)
        g.step(n)
    return o, g


def _compare(o, g):
    a, b = o.nodes(), g.nodes()
    for k in ("ux", "uy", "vx", "vy", "m"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    ea, eb = o.energy(), g.energy()
    np.testing.assert_array_equal(ea["step"], eb["step"])
    for k in ("KE", "SE", "W_ext", "W_dir"):
        scale = max(1e-300, np.max(np.abs(ea[k])))
        np.testing.assert_allclose(eb[k], ea[k], rtol=0, atol=1e-12 * scale, err_msg=k)


def test_jittered_plate_traction_and_random_state():
    """A 30 x 12 plate of 720 jittered triangles, tractions on top and
    bottom, a random initial displacement and velocity (every term of the
    stiffness active), 400 steps in three calls."""
    p = inputs.tri_plate(30, 12, jitter=0.2, traction=1e6, random_state=1e-3, steps=400)
    p.energy_every = 20
    o, g = _pair(p, [1, 150, 249])
    _compare(o, g)
    assert np.max(np.abs(g.nodes()["uy"])) > 0


def test_prescribed_velocity_and_ramp():
    """Left edge driven along x with a ramp, tractions on top and bottom."""
    p = inputs.tri_plate(24, 10, jitter=0.2, traction=2e6, v0=0.5, t0=2e-6, steps=300)
    p.energy_every = 10
    o, g = _pair(p, [300])
    _compare(o, g)
    assert np.max(g.energy()["W_dir"]) != 0


def _delaunay_plate(npts, seed):
    """A Delaunay mesh of the unit-square corners, its edges' points and
    seeded interior points (Philox streams 0, 1), counter-clockwise."""
    spatial = pytest.importorskip("scipy.spatial")
    m = 8
    t = np.linspace(0.0, 1.0, m + 1)
    bnd = np.concatenate([np.stack([t, 0 * t], 1), np.stack([t, 1 + 0 * t], 1),
                          np.stack([0 * t[1:-1], t[1:-1]], 1), np.stack([1 + 0 * t[1:-1], t[1:-1]], 1)])
    inner = np.stack([0.05 + 0.9 * inputs.uniform01(npts, seed, 0),
                      0.05 + 0.9 * inputs.uniform01(npts, seed, 1)], 1)
    X = np.concatenate([bnd, inner]) * 0.02
    tri = spatial.Delaunay(X).simplices.astype(np.int32)
    a, b, c = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    cw = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]) < 0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    return X, tri


def test_delaunay_mesh_with_pressure():
    """An unstructured Delaunay mesh (varying node degrees and triangle
    shapes), pressure on the top edge, random initial state."""
    X, conn = _delaunay_plate(150, 7)
    ed = inputs.tri_edges(conn)
    y = X[:, 1]
    top = np.flatnonzero((ed["e2"] < 0) & (y[ed["n1"]] > 0.0199) & (y[ed["n2"]] > 0.0199))
    n = len(X)
    r = [(inputs.uniform01(n, 9, q) - 0.5) for q in range(4)]
    p = inputs.TriProblem(name="delaunay", X=X, conn=conn,
                          bcs=[inputs.BC(inputs.PRESSURE, top.astype(np.int32), 0,
                                         inputs.LAW_RAMP_EXP, 5e6, 1e-6, 5e-6)],
                          energy_every=25, init=(r[0] * 1e-6, r[1] * 1e-6, r[2], r[3]))
    o, g = _pair(p, [200, 100])
    _compare(o, g)


def test_argument_and_state_errors():
    from paper_2509_01827_gb300.cem import (CEM_ERR_ARG, CEM_ERR_STATE, CemError, TriSolver,
                                            cem_get_cracks)
    bad = inputs.TriProblem(name="cw", X=np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]]),
                            conn=np.array([[0, 1, 2]], np.int32))
    with pytest.raises(CemError) as ei:
        TriSolver(bad)
    assert ei.value.code == CEM_ERR_ARG
    p = inputs.tri_plate(4, 2, traction=0)
    g = TriSolver(p)
    with pytest.raises(CemError) as ei:
        cem_get_cracks(g.h, 4)
    assert ei.value.code == CEM_ERR_STATE
    interior = np.flatnonzero(inputs.tri_edges(p.conn)["e2"] >= 0)[:1].astype(np.int32)
    from paper_2509_01827_gb300.cem import cem_set_bc
    with pytest.raises(CemError) as ei:
        cem_set_bc(g.h, inputs.TRACTION, interior, 2, inputs.LAW_CONST, 1.0, 0.0, 0.0)
    assert ei.value.code == CEM_ERR_ARG
    g.close()


@pytest.mark.parametrize("case", ["traction_random_state", "velocity"])
def test_fp32_mixed_against_the_oracle(case):
    """FP32-mixed triangles (FP32 element arithmetic, compensated float-pair
    displacement) against the FP64 oracle: displacement error
    max|u32 - u64| / max|u64| below 1e-5 and energy records within 1e-4 of
    the largest, over 400 steps."""
    from oracle.cst_oracle import from_problem
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, TriSolver
    if case == "traction_random_state":
        p = inputs.tri_plate(30, 12, jitter=0.2, traction=1e6, random_state=1e-3, steps=400)
    else:
        p = inputs.tri_plate(24, 10, jitter=0.2, traction=2e6, v0=0.5, t0=2e-6, steps=400)
    p.energy_every = 20
    o = from_problem(p)
    g = TriSolver(p, precision=CEM_FP32_MIXED)
    o.step(p.steps)
    g.step(p.steps)
    a, b = o.nodes(), g.nodes()
    for k in ("ux", "uy"):
        err = np.max(np.abs(b[k] - a[k])) / np.max(np.abs(a[k]))
        assert err < 1e-5, (k, err)
    np.testing.assert_array_equal(a["m"], b["m"])
    ea, eb = o.energy(), g.energy()
    for k in ("KE", "SE", "W_ext", "W_dir"):
        scale = max(1e-300, np.max(np.abs(ea[k])))
        np.testing.assert_allclose(eb[k], ea[k], rtol=0, atol=1e-4 * scale, err_msg=k)


@pytest.mark.parametrize("precision", [0, 1])
def test_crack_evaluation_against_the_oracle(precision):
    """G of the two candidate paths and the CST decision rule (Sec. 2.2) at
    every boundary edge and a set of interior (edge, element) points after
    120 steps, with a per-element G_c field around the median G: FP64
    bit-identical to the oracle; FP32-mixed G within 1e-4 of the largest and
    the same decisions wherever G is not within 1e-3 of G_c."""
    from oracle.cst_oracle import from_problem
    from paper_2509_01827_gb300.cem import TriSolver
    p = inputs.tri_plate(30, 12, jitter=0.2, traction=5e6, random_state=1e-3, steps=120)
    ed = inputs.tri_edges(p.conn)
    bnd = np.flatnonzero(ed["e2"] < 0)
    inner = np.flatnonzero(ed["e2"] >= 0)[::7]
    edge = np.concatenate([bnd, inner, inner]).astype(np.int32)
    elem = np.concatenate([ed["e1"][bnd], ed["e1"][inner], ed["e2"][inner]]).astype(np.int32)
    pre = from_problem(p)
    pre.step(p.steps)
    Gpre, _ = pre.eval_surface(edge, elem)
    scale = float(np.median(np.abs(Gpre[Gpre != 0]))) if np.any(Gpre != 0) else 1.0
    p.gc = (scale * (0.5 + inputs.uniform01(len(p.conn), 5))).astype(np.float32)
    o = from_problem(p)
    g = TriSolver(p, precision=precision)
    o.step(p.steps)
    g.step(p.steps)
    Go, co = o.eval_surface(edge, elem)
    Gg, cg = g.eval_surface(edge, elem)
    assert np.any(co >= 0) and np.any(co < 0)
    if precision == 0:
        np.testing.assert_array_equal(Gg, Go)
        np.testing.assert_array_equal(cg, co)
    else:
        np.testing.assert_allclose(Gg, Go, rtol=0, atol=1e-4 * np.max(np.abs(Go)))
        gce = p.gc[elem].astype(np.float64)[:, None]
        near = np.any(np.abs(Go / gce - 1.0) < 1e-3, axis=1)
        np.testing.assert_array_equal(cg[~near], co[~near])
