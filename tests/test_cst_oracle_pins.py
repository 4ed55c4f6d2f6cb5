"""Pins of the FP64 CST oracle (ES-FEM constant-strain triangles, Sec. 2.1,
Eqs. 1, 3, 5) against facts fixed by mathematics (CPU only).

None of these re-types the oracle's loops: each checks a hand-derived value,
a closed form, an invariant or a special case, so that a dropped term, a
wrong sign or index, or a missing average in the oracle fails one."""
import numpy as np
import pytest

from oracle.cst_oracle import CstOracle, from_problem
from paper_2509_01827_gb300 import inputs


def _unit_triangle(E=1.0, nu=0.0):
    s = CstOracle(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[0, 1, 2]]))
    s.set_material(E, nu, 1.0, plane_strain=False)
    return s


def _stiffness(s, nn):
    """Columns of K from unit displacements (f = K u)."""
    K = np.zeros((2 * nn, 2 * nn))
    for q in range(2 * nn):
        u = np.zeros(2 * nn)
        u[q] = 1.0
        s.set_state(ux=u[0::2], uy=u[1::2])
        fx, fy = s.internal_force()
        K[0::2, q], K[1::2, q] = fx, fy
    return K


def test_single_triangle_is_the_textbook_cst():
    """A lone triangle: every edge is a boundary edge, its smoothed strain is
    the triangle's own, and the three thirds add up to the textbook CST
    stiffness K = A B^T D B.  For the triangle (0,0), (1,0), (0,1), plane
    stress, E = 1, nu = 0 (D = diag(1, 1, 1/2)), A = 1/2 and, in the dof order
    (u0, v0, u1, v1, u2, v2), the strain rows are
        eps_xx = -u0 + u1,  eps_yy = -v0 + v2,  gamma = -u0 - v0 + v1 + u2,
    so K = 1/2 (r_xx r_xx^T + r_yy r_yy^T + 1/2 r_g r_g^T) with the matrix M
    below written out by hand."""
    M = np.array([[1.5, 0.5, -1.0, -0.5, -0.5, 0.0],
                  [0.5, 1.5, 0.0, -0.5, -0.5, -1.0],
                  [-1.0, 0.0, 1.0, 0.0, 0.0, 0.0],
                  [-0.5, -0.5, 0.0, 0.5, 0.5, 0.0],
                  [-0.5, -0.5, 0.0, 0.5, 0.5, 0.0],
                  [0.0, -1.0, 0.0, 0.0, 0.0, 1.0]])
    K = _stiffness(_unit_triangle(), 3)
    np.testing.assert_allclose(K, 0.5 * M, rtol=0, atol=1e-15)


def _square_two_triangles():
    # nodes 0 (0,0), 1 (1,0), 2 (1,1), 3 (0,1); diagonal 0-2
    X = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    conn = np.array([[0, 1, 2], [0, 2, 3]])
    s = CstOracle(X, conn)
    s.set_material(1.0, 0.0, 1.0, plane_strain=False)
    return s


def test_edge_smoothing_couples_the_far_nodes():
    """Two triangles sharing the diagonal of the unit square, T1 = (0, 1, 2),
    T2 = (0, 2, 3), plane stress E = 1, nu = 0.  Move node 3 (only in T2) by
    one unit along x.  T2's strain is (b, 0, c) of node 3 in T2: b = y0 - y2
    = -1, c = x2 - x0 = 1 (2A = 1), so eps_T2 = (-1, 0, 1) and eps_T1 = 0.
    On the shared edge the strain is the area-weighted average (Eq. 1), here
    (-1/2, 0, 1/2), stress (-1/2, 0, 1/4).  Node 1 belongs to T1 only, whose
    other two edges carry T1's zero strain, so its whole force comes from the
    shared edge: B^T sigma A_1/3 with node 1's b = y2 - y0 = 1, c = x0 - x2
    = -1: f_1 = ((1)(-1/2) + (-1)(1/4), (-1)(0) + (1)(1/4)) / 6 = (-1/8, 1/24).
    Without the average (each triangle its own strain) f_1 would be 0."""
    s = _square_two_triangles()
    s.set_state(ux=np.array([0.0, 0.0, 0.0, 1.0]))
    fx, fy = s.internal_force()
    assert fx[1] == pytest.approx(-1.0 / 8.0, abs=1e-15)
    assert fy[1] == pytest.approx(1.0 / 24.0, abs=1e-15)
    assert abs(fx.sum()) < 1e-15 and abs(fy.sum()) < 1e-15


def test_edges_and_masses():
    """Edge list: distinct node pairs in increasing (min, max), boundary edges
    with one element; lumped masses rho A / 3 per node sum to rho x area."""
    s = _square_two_triangles()
    e = s.edges()
    assert e["n1"].tolist() == [0, 0, 0, 1, 2]
    assert e["n2"].tolist() == [1, 2, 3, 2, 3]
    assert e["e1"].tolist() == [0, 0, 1, 0, 1]
    assert e["e2"].tolist() == [-1, 1, -1, -1, -1]
    m = s.nodes()["m"]
    np.testing.assert_allclose(m, [1 / 3, 1 / 6, 1 / 3, 1 / 6], rtol=1e-15)
    p = inputs.tri_plate(12, 6, jitter=0.2)
    o = from_problem(p)
    assert abs(o.nodes()["m"].sum() - p.material.rho * 0.1 * 0.04) < 1e-12 * p.material.rho * 4e-3


def test_rejects_bad_meshes():
    with pytest.raises(ValueError):   # clockwise
        CstOracle(np.array([[0.0, 0.0], [0.0, 1.0], [1.0, 0.0]]), np.array([[0, 1, 2]]))
    with pytest.raises(ValueError):   # an edge with three triangles
        CstOracle(np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0], [0.5, -1.0], [0.6, 2.0]]),
                  np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]]))


def test_rigid_body_and_patch_test():
    """On a jittered mesh: a rigid motion (translation plus infinitesimal
    rotation) gives zero force; a linear field gives the same strain in
    every triangle, zero force at every interior node, the boundary force of
    the constant stress (f_N = sum over N's two boundary edges of
    sigma n L/2) and strain energy 1/2 eps.D eps x area."""
    p = inputs.tri_plate(10, 6, jitter=0.2, traction=0)
    s = from_problem(p)
    x, y = p.X[:, 0], p.X[:, 1]
    w = 1e-3
    s.set_state(ux=2e-4 - w * y, uy=-1e-4 + w * x)
    fx, fy = s.internal_force()
    m = p.material
    scale = m.E * 1e-3 * 0.01
    assert np.max(np.abs(fx)) < 1e-10 * scale and np.max(np.abs(fy)) < 1e-10 * scale
    a, b, c, d = 1e-4, -3e-5, 2e-5, -6e-5
    s.set_state(ux=a * x + b * y, uy=c * x + d * y)
    fx, fy = s.internal_force()
    k = m.E / ((1 + m.nu) * (1 - 2 * m.nu))
    D11, D12, D33 = k * (1 - m.nu), k * m.nu, k * (1 - 2 * m.nu) / 2
    eps = np.array([a, d, b + c])
    sig = np.array([D11 * eps[0] + D12 * eps[1], D12 * eps[0] + D11 * eps[1], D33 * eps[2]])
    ed = inputs.tri_edges(p.conn)
    expect = np.zeros((len(x), 2))
    for g in np.flatnonzero(ed["e2"] < 0):
        e = ed["e1"][g]
        tri = p.conn[e].tolist()
        n1, n2 = ed["n1"][g], ed["n2"][g]
        k0 = [q for q in range(3) if {tri[q], tri[(q + 1) % 3]} == {n1, n2}][0]
        pa, pb = p.X[tri[k0]], p.X[tri[(k0 + 1) % 3]]
        t = pb - pa
        L = np.hypot(*t)
        nvec = np.array([t[1], -t[0]]) / L
        trac = np.array([sig[0] * nvec[0] + sig[2] * nvec[1], sig[2] * nvec[0] + sig[1] * nvec[1]])
        expect[n1] += 0.5 * L * trac
        expect[n2] += 0.5 * L * trac
    fs = np.max(np.abs(expect))
    np.testing.assert_allclose(fx, expect[:, 0], rtol=0, atol=1e-9 * fs)
    np.testing.assert_allclose(fy, expect[:, 1], rtol=0, atol=1e-9 * fs)
    se = s.strain_energy()
    assert se == pytest.approx(0.5 * eps.dot(sig) * 0.1 * 0.04, rel=1e-12)


def test_stiffness_is_symmetric():
    """u . K w = w . K u on a jittered mesh (ES-FEM forces are the gradient of
    a quadratic energy)."""
    p = inputs.tri_plate(9, 5, jitter=0.2, traction=0)
    s = from_problem(p)
    rng = np.random.default_rng(4)
    n = len(p.X)
    u, w = rng.normal(size=(2, n)), rng.normal(size=(2, n))
    s.set_state(ux=u[0], uy=u[1])
    fu = s.internal_force()
    s.set_state(ux=w[0], uy=w[1])
    fw = s.internal_force()
    a = np.dot(w[0], fu[0]) + np.dot(w[1], fu[1])
    b = np.dot(u[0], fw[0]) + np.dot(u[1], fw[1])
    assert abs(a - b) < 1e-12 * abs(a)


def test_energy_conserved_free_plate():
    """Central differences conserve 1/2 v^{n+1/2}.M v^{n+1/2} +
    1/2 u^n.K u^{n+1} exactly for a symmetric K: on a free jittered plate with
    a random initial state it must hold to roundoff (K u from a second,
    never-stepped oracle)."""
    p = inputs.tri_plate(10, 5, jitter=0.2, traction=0, random_state=1e-3)
    s = from_problem(p)
    k = from_problem(p)
    m = s.nodes()["m"]
    u_prev, inv = None, []
    for n in range(400):
        s.step(1)
        st = s.nodes()
        if u_prev is not None:
            k.set_state(ux=st["ux"], uy=st["uy"])
            fx, fy = k.internal_force()
            ke = 0.5 * np.sum(m * (st["vx"] ** 2 + st["vy"] ** 2))
            inv.append(ke + 0.5 * (np.dot(u_prev[0], fx) + np.dot(u_prev[1], fy)))
        u_prev = (st["ux"], st["uy"])
    inv = np.array(inv)
    assert np.max(np.abs(inv - inv[0])) < 1e-11 * inv[0]


def test_work_balance_with_traction_and_velocity():
    """With tractions and a prescribed velocity, the kinetic plus strain
    energy change equals the external work plus the work of the reaction
    forces, both recorded by the oracle (integer-step measure, within the
    O(dt^2) offset of the discrete energy)."""
    p = inputs.tri_plate(12, 6, jitter=0.2, traction=2e6, v0=0.5, t0=2e-6, steps=300)
    p.energy_every = 10
    s = from_problem(p)
    s.step(p.steps)
    e = s.energy()
    tot = e["KE"] + e["SE"]
    work = e["W_ext"] + e["W_dir"]
    assert work[-1] > 0
    assert np.max(np.abs(tot - work)) < 2e-2 * np.max(np.abs(work))


def _eyy_triangle(e, gc, gamma=1.0, gamma_mode=0, nu=0.25):
    """The triangle (0,0), (1,0), (0,1) under u_y = e y (uniform eps_yy = e),
    plane strain E = 1."""
    s = CstOracle(np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]), np.array([[0, 1, 2]]))
    s.set_material(1.0, nu, 1.0, plane_strain=True)
    s.set_fracture(None, gc, gamma, gamma_mode)
    s.set_state(uy=np.array([0.0, 0.0, e]))
    D11 = (1 - nu) / ((1 + nu) * (1 - 2 * nu))
    return s, D11


def test_G_hand_computation_uniform_eyy():
    """Sec. 2.2, CST.  The point is the midpoint (0, 1/2) of the left edge
    (local edge 2, N1 = node 2 at (0,1), N2 = node 0 at (0,0); edge id 1 of
    the pairs (0,1), (0,2), (1,2)).  delta_d = u_N2 - u_N1 = (0, -e), the edge
    stretches (H = 1).  Candidate local edge 0 (midpoint (1/2, 0)): the
    segment's normal along X_N2 - X_N1 = (0, -1) is n = -(1, 1)/sqrt 2, the
    stress (D12 e, D11 e, 0) gives sigma n = -(D12, D11) e/sqrt 2, so
    G = D11 e^2 / (2 sqrt 2).  Candidate local edge 1 (midpoint (1/2, 1/2)):
    the segment is horizontal, n = (0, -1), sigma n = (0, -D11 e), so
    G = D11 e^2 / 2.  Both above G_c: the larger (local edge 1) wins."""
    e = 1e-3
    s, D11 = _eyy_triangle(e, gc=1e-9)
    G, ch = s.eval_surface([1], [0])
    assert G[0, 0] == pytest.approx(D11 * e * e / (2 * np.sqrt(2)), rel=1e-12)
    assert G[0, 1] == pytest.approx(D11 * e * e / 2, rel=1e-12)
    assert ch[0] == 1
    # G_c between the two: only local edge 1 qualifies; above both: none
    s.set_fracture(None, 0.4 * D11 * e * e, 1.0, 0)
    assert s.eval_surface([1], [0])[1][0] == 1
    s.set_fracture(None, 0.6 * D11 * e * e, 1.0, 0)
    assert s.eval_surface([1], [0])[1][0] == -1


def test_G_ratio_mode_and_compression():
    """Ratio mode (G_p > gamma G_q): G_1 / G_0 = sqrt 2, so gamma = 1.2 picks
    local edge 1 and gamma = 2 picks none.  Under compression (e < 0) the
    edge shortens, H = 0 and both G vanish."""
    e = 1e-3
    s, D11 = _eyy_triangle(e, gc=1e-9, gamma=1.2, gamma_mode=1)
    assert s.eval_surface([1], [0])[1][0] == 1
    s.set_fracture(None, 1e-9, 2.0, 1)
    assert s.eval_surface([1], [0])[1][0] == -1
    s2, _ = _eyy_triangle(-e, gc=1e-12)
    G, ch = s2.eval_surface([1], [0])
    assert np.all(G == 0.0) and ch[0] == -1
