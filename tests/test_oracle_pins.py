"""Pins of the FP64 CPU oracle against facts fixed by mathematics or the paper.

None of these re-types the oracle's own loops: each checks a closed form, an
invariant, a special case or a brute-force enumeration, so that a dropped
term, a wrong sign or index, or a transposed operand in the oracle fails one.
"""
import math
import os

import numpy as np
import pytest

from oracle.oracle import (LAW_CONST, LAW_RAMP, LAW_RAMP_EXP, PRESSURE, SCOPE_GLOBAL,
                           SCOPE_NBHD, SCOPE_TIPS, TRACTION, VELOCITY, OracleSim)
from paper_2509_01827_gb300 import inputs

E, NU, RHO = 32e9, 0.2, 2450.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def d_plane_strain(E=E, nu=NU):
    c = E / ((1 + nu) * (1 - 2 * nu))
    return c * (1 - nu), c * nu, c * (1 - 2 * nu) / 2


def node_xy(nx, ny, hx, hy):
    i = np.tile(np.arange(nx + 1), ny + 1)
    j = np.repeat(np.arange(ny + 1), nx + 1)
    return i * hx, j * hy


def make(nx, ny, hx, hy, active=None, gc=3.0, scope=SCOPE_NBHD, pc=4096, cc=4096, **kw):
    s = OracleSim(nx, ny, hx, hy, active, pc, cc)
    s.set_material(E, NU, RHO, None, gc, True, kw.get("gamma", 1.0), kw.get("gamma_mode", 0),
                   scope)
    return s


# ------------------------------------------------------------ input generators
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    for r in rows:
        w = [int(x, 16) for x in r]
        ctr, key, out = w[:4], w[4:6], w[6:]
        got = inputs.philox4x32_10(np.array([ctr], np.uint32), key)[0]
        assert [int(x) for x in got] == out


def test_weibull_mean_and_shape():
    g = inputs.weibull_gc(200000, 3.0, 10.0, seed=7).astype(np.float64)
    assert abs(g.mean() - 3.0) < 0.01
    # Weibull CDF check at the scale parameter: P(G <= lam) = 1 - 1/e
    lam = 3.0 / math.gamma(1.1)
    assert abs(np.mean(g <= lam) - (1 - math.exp(-1))) < 0.005


# ------------------------------------------------------------ a1-a3 intact mesh
def test_rigid_body_gives_zero_force():
    nx, ny, hx, hy = 6, 4, 0.3e-3, 0.2e-3
    s = make(nx, ny, hx, hy)
    x, y = node_xy(nx, ny, hx, hy)
    w, cx, cy = 1e-3, 2e-6, -3e-6
    s.set_state(ux=cx - w * y, uy=cy + w * x)
    fx, fy = s.internal_force()
    # force scale of a strain of the same size as the rotation
    D11, _, _ = d_plane_strain()
    fscale = D11 * w * hx
    assert np.max(np.abs(fx)) < 1e-12 * fscale and np.max(np.abs(fy)) < 1e-12 * fscale


@pytest.mark.parametrize("hx,hy", [(1e-3, 1e-3), (0.3e-3, 0.17e-3)])
def test_patch_test_linear_field(hx, hy):
    nx, ny = 7, 5
    s = make(nx, ny, hx, hy)
    x, y = node_xy(nx, ny, hx, hy)
    a, b, c, d = 1.0e-4, -0.4e-4, 0.7e-4, -2.0e-4
    s.set_state(ux=a * x + b * y, uy=c * x + d * y)
    fx, fy = s.internal_force()
    D11, D12, D33 = d_plane_strain()
    sxx, syy, sxy = D11 * a + D12 * d, D12 * a + D11 * d, D33 * (b + c)
    scale = abs(sxx) * hx
    F = np.stack([fx, fy], 1).reshape(ny + 1, nx + 1, 2)
    # interior nodes: zero force
    assert np.max(np.abs(F[1:-1, 1:-1])) < 1e-10 * scale
    # boundary: f_int = integral of N * sigma.n over the boundary (divergence theorem)
    for i in range(1, nx):
        np.testing.assert_allclose(F[0, i], [-sxy * hx, -syy * hx], rtol=1e-11, atol=1e-10 * scale)
        np.testing.assert_allclose(F[ny, i], [sxy * hx, syy * hx], rtol=1e-11, atol=1e-10 * scale)
    for j in range(1, ny):
        np.testing.assert_allclose(F[j, 0], [-sxx * hy, -sxy * hy], rtol=1e-11, atol=1e-10 * scale)
        np.testing.assert_allclose(F[j, nx], [sxx * hy, sxy * hy], rtol=1e-11, atol=1e-10 * scale)
    np.testing.assert_allclose(F[0, 0], [-(sxy * hx + sxx * hy) / 2, -(syy * hx + sxy * hy) / 2],
                               rtol=1e-11, atol=1e-10 * scale)
    # strain energy = 1/2 sigma:eps * area
    se = s.strain_energy()
    exact = 0.5 * (sxx * a + syy * d + sxy * (b + c)) * nx * ny * hx * hy
    assert abs(se - exact) < 1e-12 * abs(exact)


def _random_cracked_mesh(seed):
    rng = np.random.default_rng(seed)
    nx, ny, h = 8, 6, 1e-3
    act = np.ones(nx * ny, np.uint8)
    act[3 * nx + 5] = 0
    s = make(nx, ny, h, h, act)
    s.precrack([[2 * nx + 1, 3, 1], [2 * nx + 2, 3, 0], [4 * nx + 3, 0, 2], [1 * nx + 6, 1, 2]])
    return s, rng


def test_stiffness_is_symmetric_with_cracks_and_holes():
    s, rng = _random_cracked_mesh(1)
    n = s.counts()["nn"] + s.counts()["n_phantom"]
    u = rng.standard_normal((2, n)) * 1e-6
    w = rng.standard_normal((2, n)) * 1e-6
    s.set_state(ux=u[0], uy=u[1])
    fu = np.array(s.internal_force())
    s.set_state(ux=w[0], uy=w[1])
    fw = np.array(s.internal_force())
    lhs, rhs = np.sum(w * fu), np.sum(u * fw)
    assert abs(lhs - rhs) < 1e-12 * (np.sum(np.abs(w * fu)))
    # forces are the gradient of the strain energy: SE(u) = 1/2 u.K u
    s.set_state(ux=u[0], uy=u[1])
    se = s.strain_energy()
    assert abs(se - 0.5 * np.sum(u * fu)) < 1e-12 * abs(se)


def test_internal_forces_sum_to_zero():
    s, rng = _random_cracked_mesh(2)
    n = s.counts()["nn"] + s.counts()["n_phantom"]
    u = rng.standard_normal((2, n)) * 1e-6
    s.set_state(ux=u[0], uy=u[1])
    fx, fy = s.internal_force()
    assert abs(fx.sum()) < 1e-12 * np.abs(fx).sum()
    assert abs(fy.sum()) < 1e-12 * np.abs(fy).sum()


# ------------------------------------------------------------ a1-a3 quadrature and smoothing
# Natural-coordinate derivatives of the bilinear shape functions
# N_a = (1 + xi_a xi)(1 + eta_a eta)/4 at the four edge midpoints
# k = 0 (0,-1), 1 (1,0), 2 (0,1), 3 (-1,0); rows a = 0..3, columns k.
# dN/dxi_a = xi_a (1 + eta_a eta)/4, dN/deta_a = eta_a (1 + xi_a xi)/4.
_P = np.array([[-0.5, -0.25, 0.0, -0.25], [0.5, 0.25, 0.0, 0.25],
               [0.0, 0.25, 0.5, 0.25], [0.0, -0.25, -0.5, -0.25]])
_Q = np.array([[-0.25, 0.0, -0.25, -0.5], [-0.25, -0.5, -0.25, 0.0],
               [0.25, 0.5, 0.25, 0.0], [0.25, 0.0, 0.25, 0.5]])


def _isolated_column_node1(hx, hy, dx, dy):
    """Forces on the four nodes of one isolated hx x hy element when its local
    node 1 moves by (dx, dy), from Eq. 6 with the four edge-midpoint points
    each weighted A/4 (reading C1).

    With dN/dx = 2P/hx, dN/dy = 2Q/hy and A/4 = hx hy/4, the 2x2 block
    K_a1 = sum_k (A/4) B_a^T D B_1 reduces to sums of products of the tables
    above, worked out by hand (r = hy/hx):
      sum_k P_a P_1 = (-3/8, 3/8, 1/8, -1/8)   sum_k Q_a Q_1 = (1/8, 3/8, -3/8, -1/8)
      sum_k Q_a P_1 = (-1/4, -1/4, 1/4, 1/4)   sum_k P_a Q_1 = (1/4, -1/4, -1/4, 1/4)
      f_ax = (D11 r S_PP + D33/r S_QQ) dx + (D12 S_PQ + D33 S_QP) dy
      f_ay = (D12 S_QP + D33 S_PQ) dx + (D11/r S_QQ + D33 r S_PP) dy
    (2x2 Gauss quadrature would give S_PP(1,1) = 1/3 instead of 3/8.)"""
    D11, D12, D33 = d_plane_strain()
    r = hy / hx
    spp = np.array([-3, 3, 1, -1]) / 8.0
    sqq = np.array([1, 3, -3, -1]) / 8.0
    sqp = np.array([-1, -1, 1, 1]) / 4.0
    spq = np.array([1, -1, -1, 1]) / 4.0
    fx = (D11 * r * spp + D33 / r * sqq) * dx + (D12 * spq + D33 * sqp) * dy
    fy = (D12 * sqp + D33 * spq) * dx + (D11 / r * sqq + D33 * r * spp) * dy
    return np.stack([fx, fy], 1)


def test_shape_derivative_tables_are_the_bilinear_ones():
    """The tables above are the bilinear derivatives (checked by central
    differences of N_a at the edge midpoints), so the pins below rest on the
    element's definition, not on a retyped table."""
    xa = np.array([-1, 1, 1, -1.0])
    ya = np.array([-1, -1, 1, 1.0])
    pts = [(0, -1), (1, 0), (0, 1), (-1, 0)]
    N = lambda a, x, y: (1 + xa[a] * x) * (1 + ya[a] * y) / 4
    d = 1e-6
    for a in range(4):
        for k, (x, y) in enumerate(pts):
            assert abs((N(a, x + d, y) - N(a, x - d, y)) / (2 * d) - _P[a, k]) < 1e-9
            assert abs((N(a, x, y + d) - N(a, x, y - d)) / (2 * d) - _Q[a, k]) < 1e-9
    # the closed-form sums of the column helper
    assert np.allclose(_P @ _P[1], [-3 / 8, 3 / 8, 1 / 8, -1 / 8])
    assert np.allclose(_Q @ _Q[1], [1 / 8, 3 / 8, -3 / 8, -1 / 8])
    assert np.allclose(_Q @ _P[1], [-1 / 4, -1 / 4, 1 / 4, 1 / 4])
    assert np.allclose(_P @ _Q[1], [1 / 4, -1 / 4, -1 / 4, 1 / 4])


@pytest.mark.parametrize("hx,hy", [(1e-3, 1e-3), (0.7e-3, 0.3e-3)])
@pytest.mark.parametrize("dx,dy", [(1e-6, 0.0), (0.0, 1e-6), (0.4e-6, -0.9e-6)])
def test_single_element_stiffness_column(hx, hy, dx, dy):
    """One element alone: every edge is a boundary edge (own strain), so the
    nodal forces are the element stiffness column of the moved node under the
    edge-midpoint rule (a non-linear field: the hourglass parts of a single
    moved node are resisted, Sec. 2.1 Eq. 4 at the edge points)."""
    s = make(1, 1, hx, hy)
    ux, uy = np.zeros(4), np.zeros(4)
    ux[1], uy[1] = dx, dy
    s.set_state(ux=ux, uy=uy)
    fx, fy = s.internal_force()
    want = _isolated_column_node1(hx, hy, dx, dy)
    glob = [0, 1, 3, 2]                                 # local node -> global node
    scale = np.max(np.abs(want))
    np.testing.assert_allclose(np.stack([fx[glob], fy[glob]], 1), want, rtol=0,
                               atol=1e-13 * scale)


@pytest.mark.parametrize("hx,hy", [(1e-3, 1e-3), (0.6e-3, 0.25e-3)])
def test_edge_smoothing_couples_far_nodes_horizontal(hx, hy):
    """2 x 1 mesh, node 0 (a corner of the left element only) moves by
    (dx, dy).  The right element's own strain is zero everywhere, so its far
    nodes (2 and 5) feel the move only through the area-weighted edge strain
    of Eqs. 1-2 at the shared edge:
      left element, right-edge point (xi = 1, eta = 0): dN_0/dx = -1/(2hx),
        dN_0/dy = 0, so eps_own = (-dx/(2hx), 0, -dy/(2hx));
      equal areas: eps_g = eps_own / 2, sigma_g = D eps_g
        = (-D11 dx, -D12 dx, -D33 dy) / (4hx);
      right element, left-edge point (xi = -1, eta = 0): its local nodes 1, 2
        have dN/dx = 1/(2hx), dN/dy = 0, so f = (A/4)(1/(2hx)) (sxx, sxy)
        = hy/8 (sxx, sxy) = (-D11 dx, -D33 dy) hy / (32 hx).
    Using each element's own strain (no averaging) would give exactly zero
    there, and pairing the wrong edge of the neighbour another value."""
    D11, D12, D33 = d_plane_strain()
    dx, dy = 1e-6, -0.7e-6
    s = make(2, 1, hx, hy)
    ux, uy = np.zeros(6), np.zeros(6)
    ux[0], uy[0] = dx, dy
    s.set_state(ux=ux, uy=uy)
    fx, fy = s.internal_force()
    want = np.array([-D11 * dx, -D33 * dy]) * hy / (32 * hx)
    for n in (2, 5):
        np.testing.assert_allclose([fx[n], fy[n]], want, rtol=1e-12)


@pytest.mark.parametrize("hx,hy", [(1e-3, 1e-3), (0.25e-3, 0.6e-3)])
def test_edge_smoothing_couples_far_nodes_vertical(hx, hy):
    """1 x 2 mesh (elements stacked), node 0 moves by (dx, dy).  Bottom
    element, top-edge point (xi = 0, eta = 1): dN_0/dx = 0, dN_0/dy =
    -1/(2hy), so eps_own = (0, -dy/(2hy), -dx/(2hy)); halved by the averaging;
    sigma_g = (-D12 dy, -D11 dy, -D33 dx)/(4hy).  Top element, bottom-edge
    point: its local nodes 2, 3 (global 5, 4) have dN/dx = 0, dN/dy = 1/(2hy):
    f = (A/4)(1/(2hy)) (sxy, syy) = (-D33 dx, -D11 dy) hx / (32 hy)."""
    D11, D12, D33 = d_plane_strain()
    dx, dy = -0.8e-6, 1.1e-6
    s = make(1, 2, hx, hy)
    ux, uy = np.zeros(6), np.zeros(6)
    ux[0], uy[0] = dx, dy
    s.set_state(ux=ux, uy=uy)
    fx, fy = s.internal_force()
    want = np.array([-D33 * dx, -D11 * dy]) * hx / (32 * hy)
    for n in (4, 5):
        np.testing.assert_allclose([fx[n], fy[n]], want, rtol=1e-12)


@pytest.mark.parametrize("hx,hy", [(1e-3, 1e-3), (0.5e-3, 0.8e-3)])
def test_no_smoothing_beside_a_split_element(hx, hy):
    """Reading C4: smoothing is off on every edge touching a split element.
    2 x 1 mesh with the left element pre-cut (left to right edge midpoint);
    the right element's far node 2 (its local node 1) moves.  The left
    element's pieces do not move, so the right element must act exactly as
    if it were alone: its four nodes carry the isolated-element column
    (hand form above).  With the left element intact the shared edge
    averages the strains and the forces differ (control)."""
    dx, dy = 0.9e-6, 0.5e-6
    want = _isolated_column_node1(hx, hy, dx, dy)      # rows: e1 local 0..3
    glob = [1, 2, 5, 4]                                 # e1 local -> global node
    s = make(2, 1, hx, hy)
    s.precrack([[0, 3, 1]])
    n = s.counts()["nn"] + s.counts()["n_phantom"]
    ux, uy = np.zeros(n), np.zeros(n)
    ux[2], uy[2] = dx, dy
    s.set_state(ux=ux, uy=uy)
    fx, fy = s.internal_force()
    scale = np.max(np.abs(want))
    got = np.array([[fx[g], fy[g]] for g in glob])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * scale)
    # phantoms and the left element's own real nodes feel nothing
    assert np.all(fx[[0, 3]] == 0) and np.all(fx[6:] == 0) and np.all(fy[6:] == 0)
    c = make(2, 1, hx, hy)
    c.set_state(ux=ux[:6], uy=uy[:6])
    cx, cy = c.internal_force()
    assert np.max(np.abs(np.array([[cx[g], cy[g]] for g in glob]) - want)) > 1e-3 * scale


def test_element_stress_of_a_linear_field_and_a_rotation():
    """Element mean stress (the contour output): a linear field gives
    D eps_exact in every element -- intact or split (phantoms carry the
    field at their real node's position) -- and a rigid rotation gives 0."""
    nx, ny, hx, hy = 7, 5, 1e-3, 0.6e-3
    s = make(nx, ny, hx, hy)
    s.precrack([[2 * nx + i, 3, 1] for i in range(4)] + [[4 * nx + 5, 3, 0]])
    c = s.counts()
    nn = c["nn"]
    x, y = node_xy(nx, ny, hx, hy)
    owner = s.phantoms()["owner"]
    X = np.concatenate([x, x[owner]])
    Y = np.concatenate([y, y[owner]])
    a, b, cc, d = 1.0e-4, -0.4e-4, 0.7e-4, -2.0e-4
    s.set_state(ux=a * X + b * Y, uy=cc * X + d * Y)
    D11, D12, D33 = d_plane_strain()
    want = np.array([D11 * a + D12 * d, D12 * a + D11 * d, D33 * (b + cc)])
    got = s.element_stress()
    np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=1e-11,
                               atol=1e-11 * np.max(np.abs(want)))
    w = 1e-3
    s2 = make(nx, ny, hx, hy)
    s2.set_state(ux=-w * y, uy=w * x)
    assert np.max(np.abs(s2.element_stress())) < 1e-12 * D11 * w
    del nn


def test_element_stress_uses_the_smoothed_edge_stress():
    """2 x 1 mesh, node 0 moved by dx: the right element's own strain is 0;
    at the shared edge the smoothing gives half of the left element's
    eps_xx = -dx/(2hx) there, so its mean stress over four edge points is
    (D11, D12) * (-dx/(4hx)) / 4."""
    hx, hy, dx = 1e-3, 0.5e-3, 1e-6
    s = make(2, 1, hx, hy)
    ux = np.zeros(6)
    ux[0] = dx
    s.set_state(ux=ux)
    D11, D12, _ = d_plane_strain()
    got = s.element_stress()[1]
    np.testing.assert_allclose(got[:2], np.array([D11, D12]) * (-dx / (4 * hx)) / 4, rtol=1e-13)
    assert got[2] == 0.0


# ------------------------------------------------------------ a5 dynamics
def test_total_mass_equals_density_times_area():
    s, _ = _random_cracked_mesh(3)
    m = s.nodes()["m"]
    nact = 8 * 6 - 1
    assert abs(m.sum() - RHO * nact * 1e-6) < 1e-13 * RHO * nact * 1e-6


def test_energy_conserved_free_plate():
    """Uncracked free plate with a smooth initial velocity field.

    Central differences conserve the discrete energy
    E_{n+1/2} = 1/2 v^{n+1/2}.M v^{n+1/2} + 1/2 u^n.K u^{n+1} exactly (K
    symmetric): it must hold to roundoff.  K u is taken from a second,
    never-stepped oracle instance.  The integer-step measure KE(vbar)+SE(u)
    recorded by the oracle stays within O(dt^2) of it without drift."""
    nx, ny, h = 16, 8, 1e-3
    s = make(nx, ny, h, h, gc=1e30)
    k = make(nx, ny, h, h, gc=1e30)
    x, y = node_xy(nx, ny, h, h)
    Lx, Ly = nx * h, ny * h
    vx = 0.5 * np.sin(np.pi * x / Lx) * np.cos(np.pi * y / Ly)
    vy = 0.3 * np.cos(np.pi * x / Lx) * np.sin(2 * np.pi * y / Ly)
    s.set_state(vx=vx, vy=vy)
    s.set_energy_every(5)
    m = s.nodes()["m"]
    u_prev = None
    inv = []
    for n in range(1500):
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
    e = s.energy()
    tot = e["KE"] + e["SE"]
    # integer-step measure: offset by O((omega dt / 2)^2), no secular drift
    assert np.max(np.abs(tot[1:] - inv[0])) < 3e-2 * inv[0]
    q = len(tot) // 4
    assert abs(tot[-q:].mean() - tot[1:q].mean()) < 2e-3 * inv[0]
    assert e["SE"].max() > 0.3 * inv[0]


def test_work_balance_with_traction():
    """With Neumann loads the discrete balance
    1/2 v^{n+1/2}.M v^{n+1/2} + 1/2 u^n.K u^{n+1} - W^{n+1} = const holds to
    roundoff, where W is the oracle's own external-work record
    (sum of f_ext^m . (u^{m+1} - u^{m-1}) / 2)."""
    nx, ny, h = 12, 6, 1e-3
    s = make(nx, ny, h, h, gc=1e30)
    k = make(nx, ny, h, h, gc=1e30)
    s.add_bc(TRACTION, inputs.boundary_edges(nx, ny, "top"), 2, LAW_RAMP, 1e6, 2e-6)
    s.add_bc(TRACTION, inputs.boundary_edges(nx, ny, "bottom"), 2, LAW_RAMP, -1e6, 2e-6)
    s.set_energy_every(1)
    m = s.nodes()["m"]
    hist = []
    N = 800
    for n in range(N):
        s.step(1)
        st = s.nodes()
        hist.append((st["ux"].copy(), st["uy"].copy(), st["vx"].copy(), st["vy"].copy()))
    W = s.energy()["W_ext"]
    inv = []
    for n in range(1, N - 1):
        ux1, uy1, vx, vy = hist[n]          # u^{n+1}, v^{n+1/2}
        ux0, uy0 = hist[n - 1][:2]          # u^n
        k.set_state(ux=ux1, uy=uy1)
        fx, fy = k.internal_force()
        ke = 0.5 * np.sum(m * (vx ** 2 + vy ** 2))
        inv.append(ke + 0.5 * (np.dot(ux0, fx) + np.dot(uy0, fy)) - W[n + 1])
    inv = np.array(inv)
    assert np.max(np.abs(inv - inv[0])) < 1e-10 * np.max(np.abs(W))
    assert np.max(W) > 0


def test_momentum_equals_impulse_of_traction():
    """Internal forces cancel, so total momentum = integral of the applied load.
    Each node of a loaded edge of length L takes L/2 of the traction; the
    ramp/exponential pulse is the shape of the paper's pressure law."""
    nx, ny, h = 10, 4, 1e-3
    s = make(nx, ny, h, h, gc=1e30)
    T, t0, tau = 2e6, 1e-6, 3e-6
    s.add_bc(TRACTION, inputs.boundary_edges(nx, ny, "top"), 2, LAW_RAMP_EXP, T, t0, tau)
    dt = s.dt
    n = 200
    s.step(n)
    st = s.nodes()
    p = np.sum(st["m"] * st["vy"])
    t = np.arange(n) * dt
    lam = np.where(t <= t0, t / t0, np.exp(-(t - t0) / tau))
    w = np.full(n, dt)
    w[0] = dt / 2
    impulse = T * nx * h * np.sum(w * lam)
    assert abs(p - impulse) < 1e-10 * abs(impulse)
    assert abs(np.sum(st["m"] * st["vx"])) < 1e-10 * abs(impulse)


@pytest.mark.parametrize("law", [LAW_RAMP, LAW_RAMP_EXP])
def test_dirichlet_time_law(law):
    """Nodes with prescribed velocity follow v(t_{n+1/2}) = lambda(t) v0 exactly."""
    s = make(2, 1, 1e-3, 1e-3, gc=1e30)
    v0, t0, tau = 2.0, 1e-6, 4e-6
    allnodes = np.arange(6)
    s.add_bc(VELOCITY, allnodes, 3, law, v0, t0, tau)
    dt = s.dt
    n = 300
    s.step(n)
    ux = s.nodes()["ux"]
    t = (np.arange(n) + 0.5) * dt
    if law == LAW_RAMP:
        lam = np.minimum(t / t0, 1.0)
    else:
        lam = np.where(t <= t0, t / t0, np.exp(-(t - t0) / tau))
    np.testing.assert_allclose(ux, dt * v0 * lam.sum(), rtol=1e-12)


def test_bar_wave_speed_and_stress():
    """Uniaxial strain strip: v_y = 0 everywhere and a step velocity v0 at
    x = 0.  The front travels at c_d and carries sigma_xx = -rho c_d v0."""
    nx, ny, h = 400, 1, 0.25e-3
    s = make(nx, ny, h, h, gc=1e30)
    nn = (nx + 1) * (ny + 1)
    s.add_bc(VELOCITY, np.arange(nn), 2, LAW_CONST, 0.0)
    v0 = 1.0
    s.add_bc(VELOCITY, inputs.boundary_nodes(nx, ny, "left"), 1, LAW_CONST, v0)
    D11, _, _ = d_plane_strain()
    cd = math.sqrt(D11 / RHO)
    dt = s.dt
    L = nx * h
    probe = nx // 2                      # node index along the bottom row
    t_arr = None
    vx_hist = []
    nsteps = int(0.8 * L / cd / dt)
    for q in range(nsteps):
        s.step(1)
        vx = s.nodes()["vx"][probe]
        vx_hist.append(vx)
        if t_arr is None and vx >= 0.5 * v0:
            t_arr = (q + 1) * dt
    expect = probe * h / cd
    assert t_arr is not None and abs(t_arr - expect) < 0.02 * expect
    ux = s.nodes()["ux"][: nx + 1]
    # strain behind the front, between x = L/8 and L/4
    i1, i2 = nx // 8, nx // 4
    eps = (ux[i2] - ux[i1]) / ((i2 - i1) * h)
    sig = D11 * eps
    assert abs(sig - (-RHO * cd * v0)) < 0.02 * RHO * cd * v0


def test_time_step_is_half_the_cfl_limit_and_stable():
    """dt = 0.5 h / c_d; a random initial field stays bounded for 20k steps."""
    nx, ny, h = 10, 6, 1e-3
    s = make(nx, ny, h, h, gc=1e30)
    D11, _, _ = d_plane_strain()
    assert abs(s.dt - 0.5 * h / math.sqrt(D11 / RHO)) < 1e-15 * s.dt
    rng = np.random.default_rng(5)
    nn = (nx + 1) * (ny + 1)
    s.set_state(vx=rng.standard_normal(nn), vy=rng.standard_normal(nn))
    s.set_energy_every(500)
    s.step(20000)
    e = s.energy()
    tot = e["KE"] + e["SE"]
    assert np.all(np.isfinite(tot)) and tot.max() < 1.5 * tot[0]


# ------------------------------------------------------------ a6 release rate
def _single_element(hx, hy, exx=0.0, eyy=0.0):
    s = make(1, 1, hx, hy)
    x, y = node_xy(1, 1, hx, hy)
    s.set_state(ux=exx * x, uy=eyy * y)
    ev = s.eval_surface()
    return {int(k0): G for k0, G in zip(ev["k0"], ev["G"])}, ev


@pytest.mark.parametrize("hx,hy", [(1e-3, 1e-3), (1e-3, 0.6e-3)])
def test_G_hand_computation_uniform_eyy(hx, hy):
    """Uniform eps_yy = e; surface point at the left edge midpoint.
    delta_d = (0, e*hy) stretch of the left edge; the straight (pattern II)
    path has n = (0, 1): G = 1/2 e hy * D11 e.  The pattern-I paths to the
    bottom/top midpoints have unit normal (hy, hx)/l: G = 1/2 D11 e^2 hx hy / l."""
    e = 2e-4
    G, _ = _single_element(hx, hy, eyy=e)
    D11, _, _ = d_plane_strain()
    l = math.hypot(hx, hy)
    g2 = 0.5 * D11 * e * e * hy
    g1 = 0.5 * D11 * e * e * hx * hy / l
    np.testing.assert_allclose(G[3][[0, 1, 2]], [g1, g2, g1], rtol=1e-12)
    np.testing.assert_allclose(G[1][[0, 2, 3]], [g1, g1, g2], rtol=1e-12)
    # bottom and top edges are not stretched (eps_xx = 0): H = 0
    assert np.all(G[0][[1, 2, 3]] == 0.0) and np.all(G[2][[0, 1, 3]] == 0.0)


def test_G_label_invariance_and_compression():
    """Uniform eps_xx = e: bottom and top surface points (opposite N1->N2
    orientation) give the same G; compression gives G = 0."""
    e, h = 1.5e-4, 1e-3
    G, _ = _single_element(h, h, exx=e)
    D11, _, _ = d_plane_strain()
    np.testing.assert_allclose(G[0][2], 0.5 * D11 * e * e * h, rtol=1e-12)
    np.testing.assert_allclose(G[2][0], G[0][2], rtol=1e-15)
    Gc, _ = _single_element(h, h, exx=-e)
    assert all(np.all(Gc[k][np.arange(4) != k] == 0.0) for k in range(4))


def test_q4_rule_thresholds():
    """One candidate above G_c -> that path; several -> the largest; none -> none."""
    e, h = 2e-4, 1e-3
    D11, _, _ = d_plane_strain()
    g2 = 0.5 * D11 * e * e * h
    g1 = g2 / math.sqrt(2)
    for gc, want in [(1.01 * g2, -1), (0.5 * (g1 + g2), 1), (0.9 * g1, 1)]:
        s = make(1, 1, h, h, gc=gc)
        x, y = node_xy(1, 1, h, h)
        s.set_state(uy=e * y)
        ev = s.eval_surface()
        k = {int(k0): int(p) for k0, p in zip(ev["k0"], ev["prop_k"])}
        assert k[3] == want
    # ratio-mode split test with gamma = 1.5: G_p = 1.414 G_q < 1.5 G_q -> waits
    s = make(1, 1, h, h, gc=0.9 * g1, gamma=1.5, gamma_mode=1)
    s.set_state(uy=e * node_xy(1, 1, h, h)[1])
    ev = s.eval_surface()
    assert dict(zip(ev["k0"], ev["prop_k"]))[3] == -1


# ------------------------------------------------------------ a7 bookkeeping
def _surface_brute(nx, ny, active, cracked):
    """Edges with exactly one intact neighbour, by direct enumeration."""
    nh = nx * (ny + 1)
    st = {}
    for e in range(nx * ny):
        st[e] = 0 if not active[e] else (2 if e in cracked else 1)
    out = {}
    for g in range(nh + (nx + 1) * ny):
        if g < nh:
            j, i = divmod(g, nx)
            lo = (j - 1) * nx + i if j > 0 else None
            hi = j * nx + i if j < ny else None
            klo, khi = 2, 0
        else:
            j, i = divmod(g - nh, nx + 1)
            lo = j * nx + i - 1 if i > 0 else None
            hi = j * nx + i if i < nx else None
            klo, khi = 1, 3
        slo = st.get(lo, 0) if lo is not None else 0
        shi = st.get(hi, 0) if hi is not None else 0
        if (slo == 1) != (shi == 1):
            ahead, other, kother = (lo, hi, khi) if slo == 1 else (hi, lo, klo)
            tip = other is not None and other in cracked and kother in cracked[other]
            out[g] = (ahead, tip)
    return out


def _brute_winners(props, nx, scope):
    def key(p):
        return (p[3], -p[0])
    if scope == SCOPE_GLOBAL:
        return [max(props, key=key)] if props else []
    win = []
    for p in props:
        ok = True
        for q in props:
            if q is p:
                continue
            di = abs(p[1] % nx - q[1] % nx)
            dj = abs(p[1] // nx - q[1] // nx)
            if di <= 1 and dj <= 1 and not key(p) > key(q):
                ok = False
        if ok:
            win.append(p)
    return win


@pytest.mark.parametrize("nx,ny,seed,scope", [(4, 3, 0, SCOPE_NBHD), (6, 4, 1, SCOPE_NBHD),
                                              (8, 8, 2, SCOPE_NBHD), (8, 8, 3, SCOPE_GLOBAL),
                                              (8, 8, 4, SCOPE_TIPS), (6, 6, 5, SCOPE_NBHD)])
def test_tracking_bookkeeping_brute_force(nx, ny, seed, scope):
    rng = np.random.default_rng(seed)
    h = 1e-3
    act = np.ones(nx * ny, np.uint8)
    if nx * ny > 30:
        act[rng.integers(nx * ny)] = 0
    s = make(nx, ny, h, h, act, scope=scope, pc=10 * nx * ny, cc=nx * ny)
    cracked = {}
    e0 = (ny // 2) * nx
    if act[e0]:
        s.precrack([[e0, 3, 1]])
        cracked[e0] = (3, 1)
    n = s.counts()["nn"] + s.counts()["n_phantom"]
    s.set_state(vx=rng.standard_normal(n), vy=rng.standard_normal(n))
    for rnd in range(6):
        surf = s.surface()
        brute = _surface_brute(nx, ny, act, cracked)
        assert sorted(brute) == list(surf["edge"])
        assert [brute[g][0] for g in surf["edge"]] == list(surf["ahead"])
        assert [brute[g][1] for g in surf["edge"]] == list(surf["is_tip"])
        # scripted proposals on a random subset of surface points, with ties
        ev = s.eval_surface()
        m = len(ev["edge"])
        pick = rng.random(m) < 0.5
        props = []
        for q in np.nonzero(pick)[0]:
            k0 = int(ev["k0"][q])
            k = int(rng.choice([k for k in range(4) if k != k0]))
            G = float(rng.integers(1, 4))          # small integers: many exact ties
            props.append((int(ev["edge"][q]), int(ev["ahead"][q]), k, G))
        if scope == SCOPE_TIPS:
            tips = set(int(g) for g, t in zip(surf["edge"], surf["is_tip"]) if t)
            eligible = [p for p in props if p[0] in tips]
        else:
            eligible = props
        winners = _brute_winners(eligible, nx, scope)
        want = set(p[1] for p in winners)
        assert len(want) == len(winners)
        nodes0 = s.nodes()
        m0 = nodes0["m"].sum()
        px0 = np.sum(nodes0["m"] * nodes0["vx"])
        py0 = np.sum(nodes0["m"] * nodes0["vy"])
        before = set(int(e) for e in s.cracks()["elem"])
        if props:
            s.apply_proposals([p[0] for p in props], [p[1] for p in props],
                              [p[2] for p in props], [p[3] for p in props])
        cr = s.cracks()
        after = set(int(e) for e in cr["elem"])
        assert after - before == want
        for p in winners:
            idx = list(cr["elem"]).index(p[1])
            # the exit edge is the winning proposal's chosen path
            assert int(cr["kb"][idx]) == p[2]
            cracked[p[1]] = (int(cr["ka"][idx]), int(cr["kb"][idx]))
        nodes1 = s.nodes()
        assert abs(nodes1["m"].sum() - m0) < 1e-14 * m0
        sc = np.sum(nodes1["m"] * np.abs(nodes1["vx"])) + 1e-30
        assert abs(np.sum(nodes1["m"] * nodes1["vx"]) - px0) < 1e-13 * sc
        assert abs(np.sum(nodes1["m"] * nodes1["vy"]) - py0) < 1e-13 * sc
    _check_phantom_consistency(s, nx, ny)


def _check_phantom_consistency(s, nx, ny):
    nn = (nx + 1) * (ny + 1)
    cr = s.cracks()
    ph = s.phantoms()
    for q, e in enumerate(cr["elem"]):
        i, j = e % nx, e // nx
        real = [j * (nx + 1) + i, j * (nx + 1) + i + 1, (j + 1) * (nx + 1) + i + 1,
                (j + 1) * (nx + 1) + i]
        for a in range(4):
            ids = cr["nodes"][q, :, a]
            # exactly one piece holds the real node, the other a phantom of it
            assert sorted([int(ids[0] < nn), int(ids[1] < nn)]) == [0, 1]
            r = ids[0] if ids[0] < nn else ids[1]
            p = ids[1] if ids[0] < nn else ids[0]
            assert r == real[a] and ph["owner"][p - nn] == real[a]
    for P in range(len(ph["owner"])):
        us = ph["users"][P][: ph["nuser"][P]]
        assert list(us[:, 0]) == sorted(us[:, 0])
        for (e, piece, a) in us:
            q = list(cr["elem"]).index(e)
            assert cr["nodes"][q, piece, a] == nn + P


def test_precrack_row_shares_phantoms():
    """A straight row of n pattern-II splits: consecutive elements share the
    phantoms of the nodes on their common cut edge, so 2(n+1) phantoms."""
    nx, ny, h = 12, 6, 1e-3
    s = make(nx, ny, h, h)
    n = 7
    s.precrack([[2 * nx + i, 3, 1] for i in range(n)])
    assert s.counts()["n_phantom"] == 2 * (n + 1)
    m = s.nodes()["m"]
    nn = (nx + 1) * (ny + 1)
    # mass of an interior shared phantom: two half pieces -> 2 * rho*(A/2)/4
    np.testing.assert_allclose(m[nn + 2], RHO * h * h / 4, rtol=1e-15)
    _check_phantom_consistency(s, nx, ny)
    tips = s.surface()
    assert int(np.sum(tips["is_tip"])) == 1


def test_pattern_I_area_fractions_and_dissipation():
    """Element (1,1) of a 3x3 mesh is cut from its left to its bottom midpoint
    (pattern I) after its left neighbour was cut straight through.  The
    corner piece has 1/8 of the area; the phantom of the corner node is the
    one the upper piece of the left neighbour already uses."""
    nx, ny, h = 3, 3, 1e-3
    A = h * h
    s = make(nx, ny, h, h, gc=3.0)
    s.precrack([[3, 3, 1]])                     # element (0,1), pattern II
    g = inputs.v_edge(nx, ny, 1, 1)             # its right edge = tip
    s.apply_proposals([g], [4], [0], [10.0])    # into element (1,1): left -> bottom
    cr = s.cracks()
    q = list(cr["elem"]).index(4)
    assert cr["ka"][q] == 3 and cr["kb"][q] == 0
    np.testing.assert_allclose(cr["ud"][q], 3.0 * h / math.sqrt(2), rtol=1e-15)
    m = s.nodes()["m"]
    nn = (nx + 1) * (ny + 1)
    corner = 1 * (nx + 1) + 1                   # node (1,1) = local node 0 of element 4
    # real corner node: two intact elements, half of (0,1), 1/8 of (1,1)
    np.testing.assert_allclose(m[corner], RHO * A / 4 * (1 + 1 + 0.5 + 0.125), rtol=1e-15)
    ph_corner = int(cr["nodes"][q, :, 0].max())
    assert ph_corner >= nn
    q3 = list(cr["elem"]).index(3)
    assert ph_corner in set(int(x) for x in cr["nodes"][q3].reshape(-1))
    # the shared phantom carries the upper half of (0,1) and 7/8 of (1,1)
    np.testing.assert_allclose(m[ph_corner], RHO * A / 4 * (0.5 + 0.875), rtol=1e-15)
    assert abs(m.sum() - RHO * 9 * A) < 1e-14 * RHO * 9 * A
