"""Seeded synthetic problem generators (meshes, masks, loads, G_c fields).

This module holds no arithmetic of the crack-element method itself: it only
describes problems -- structured Q4 grid sizes, which elements are active,
which edges are loaded and by what time law, which elements are pre-cracked,
and the per-element critical energy release rate G_c.  Both the CUDA library
binding and the CPU oracle read the same ``Problem``.

Numbering (also stated in ``include/cem.h``):
  node (i, j)      -> j*(nx+1) + i
  element (i, j)   -> j*nx + i
  horizontal edge (i, j), nodes (i,j)-(i+1,j), 0 <= j <= ny -> j*nx + i
  vertical edge (i, j),   nodes (i,j)-(i,j+1), 0 <= j < ny  -> nx*(ny+1) + j*(nx+1) + i
  element local edges: 0 bottom, 1 right, 2 top, 3 left.

Workloads (materials from the paper's Sec. 4.2 Neumann branching example:
E = 32 GPa, nu = 0.2, rho = 2450 kg/m^3, G_c = 3 J/m^2):
  * ``notched_plate``: 0.1 x 0.04 m plate, pre-notch along mid-height from
    the left edge, constant normal traction on top and bottom (Sec. 4.2).
  * ``fragmentation``: square plate with a central hole under an internal
    pressure pulse (shape of the Sec. 4.4 law) or an outward edge velocity,
    Weibull G_c field.
  * ``batch_specimens``: notched plates of random size, notch and traction.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

TRACTION, PRESSURE, VELOCITY = 0, 1, 2
LAW_CONST, LAW_RAMP, LAW_RAMP_EXP = 0, 1, 2
SCOPE_NBHD, SCOPE_GLOBAL, SCOPE_TIPS = 0, 1, 2


# ----------------------------------------------------------------- Philox
_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(counter: np.ndarray, key) -> np.ndarray:
    """Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), vectorised.

    counter: (n, 4) uint32 array; key: two uint32 words.  Returns (n, 4) uint32.
    """
    c = np.asarray(counter, dtype=np.uint64).reshape(-1, 4)
    c0, c1, c2, c3 = (np.ascontiguousarray(c[:, i]) for i in range(4))
    k0, k1 = np.uint64(int(key[0]) & _MASK), np.uint64(int(key[1]) & _MASK)
    m0, m1, mask, sh = np.uint64(_M0), np.uint64(_M1), np.uint64(_MASK), np.uint64(32)
    for r in range(10):
        if r:
            k0 = np.uint64((int(k0) + _W0) & _MASK)
            k1 = np.uint64((int(k1) + _W1) & _MASK)
        p0 = m0 * c0
        p1 = m1 * c2
        # (hi(p1) ^ c1 ^ k0, lo(p1), hi(p0) ^ c3 ^ k1, lo(p0))
        c0, c1, c2, c3 = (p1 >> sh) ^ c1 ^ k0, p1 & mask, (p0 >> sh) ^ c3 ^ k1, p0 & mask
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def uniform01(n: int, seed: int, stream: int = 0) -> np.ndarray:
    """n uniforms in (0, 1): U_e = (x_e + 0.5) / 2^32, x_e = first Philox word
    of counter (e, stream, 0, 0) under key (seed, 0)."""
    ctr = np.zeros((n, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(n, dtype=np.uint64)
    ctr[:, 1] = stream
    x = philox4x32_10(ctr, (seed, 0))[:, 0].astype(np.float64)
    return (x + 0.5) / 4294967296.0


def weibull_gc(n: int, mean: float, shape: float, seed: int) -> np.ndarray:
    """Per-element G_c = lam * (-ln U)^(1/k), lam = mean / Gamma(1 + 1/k), FP32."""
    lam = mean / math.gamma(1.0 + 1.0 / shape)
    u = uniform01(n, seed)
    return (lam * (-np.log(u)) ** (1.0 / shape)).astype(np.float32)


# ---------------------------------------------------------------- records
@dataclass
class Material:
    E: float = 32e9
    nu: float = 0.2
    rho: float = 2450.0
    gc_uniform: float = 3.0
    plane_strain: bool = True
    gamma: float = 1.0
    gamma_mode: int = 0
    scope: int = SCOPE_NBHD


@dataclass
class BC:
    kind: int
    items: np.ndarray
    comp_mask: int = 0
    law: int = LAW_CONST
    a0: float = 0.0
    t0: float = 0.0
    tau: float = 0.0


@dataclass
class Problem:
    name: str
    nx: int
    ny: int
    hx: float
    hy: float
    material: Material = field(default_factory=Material)
    active: Optional[np.ndarray] = None      # uint8 per element, None = all
    gc: Optional[np.ndarray] = None          # float32 per element, None = uniform
    bcs: List[BC] = field(default_factory=list)
    precracks: np.ndarray = field(default_factory=lambda: np.zeros((0, 3), np.int32))
    dt_factor: float = 0.5
    dt: Optional[float] = None
    steps: int = 0
    energy_every: int = 0
    phantom_cap: int = 4096
    crack_cap: int = 4096

    @property
    def n_nodes(self):
        return (self.nx + 1) * (self.ny + 1)

    @property
    def n_elems(self):
        return self.nx * self.ny

    @property
    def n_active(self):
        return self.n_elems if self.active is None else int(np.count_nonzero(self.active))


# ---------------------------------------------------------------- topology
def h_edge(nx, i, j):
    return j * nx + i


def v_edge(nx, ny, i, j):
    return nx * (ny + 1) + j * (nx + 1) + i


def node_id(nx, i, j):
    return j * (nx + 1) + i


def boundary_edges(nx, ny, side):
    """Edge ids of one side of the outer rectangle: 'bottom', 'top', 'left', 'right'."""
    if side == "bottom":
        return np.array([h_edge(nx, i, 0) for i in range(nx)], np.int32)
    if side == "top":
        return np.array([h_edge(nx, i, ny) for i in range(nx)], np.int32)
    if side == "left":
        return np.array([v_edge(nx, ny, 0, j) for j in range(ny)], np.int32)
    if side == "right":
        return np.array([v_edge(nx, ny, nx, j) for j in range(ny)], np.int32)
    raise ValueError(side)


def boundary_nodes(nx, ny, side):
    if side == "bottom":
        return np.array([node_id(nx, i, 0) for i in range(nx + 1)], np.int32)
    if side == "top":
        return np.array([node_id(nx, i, ny) for i in range(nx + 1)], np.int32)
    if side == "left":
        return np.array([node_id(nx, 0, j) for j in range(ny + 1)], np.int32)
    if side == "right":
        return np.array([node_id(nx, nx, j) for j in range(ny + 1)], np.int32)
    raise ValueError(side)


def interface_edges(nx, ny, active):
    """Edges between an active and an inactive element (the rim of a hole)."""
    act = np.asarray(active, bool).reshape(ny, nx)
    out = []
    # horizontal edges 1..ny-1 separate rows j-1 and j
    for j in range(1, ny):
        diff = act[j - 1, :] != act[j, :]
        for i in np.nonzero(diff)[0]:
            out.append(h_edge(nx, int(i), j))
    for j in range(ny):
        diff = act[j, :-1] != act[j, 1:]
        for i in np.nonzero(diff)[0]:
            out.append(v_edge(nx, ny, int(i) + 1, j))
    return np.array(sorted(out), np.int32)


# ---------------------------------------------------------------- workloads
def notched_plate(nx=100, ny=40, lx=0.1, ly=0.04, notch_len=0.05, traction=1e6,
                  steps=2000, material: Optional[Material] = None, name=None,
                  dt_factor=0.5, energy_every=0, phantom_cap=None, crack_cap=None):
    """Pre-notched plate under constant opposite normal tractions on the top
    and bottom edges (Sec. 4.2 setting).  The notch runs from the left edge
    through the element row just below mid-height (mid-height is a node
    line), as a row of pattern-II pre-cracks from left to right edge points."""
    hx, hy = lx / nx, ly / ny
    jn = ny // 2 - 1
    nn = int(round(notch_len / hx))
    pre = np.array([[jn * nx + i, 3, 1] for i in range(nn)], np.int32).reshape(-1, 3)
    bcs = [BC(TRACTION, boundary_edges(nx, ny, "top"), 2, LAW_CONST, +traction),
           BC(TRACTION, boundary_edges(nx, ny, "bottom"), 2, LAW_CONST, -traction)]
    ne = nx * ny
    return Problem(name=name or f"notched_plate_{nx}x{ny}", nx=nx, ny=ny, hx=hx, hy=hy,
                   material=material or Material(), bcs=bcs, precracks=pre, steps=steps,
                   dt_factor=dt_factor, energy_every=energy_every,
                   phantom_cap=phantom_cap or max(4096, ne // 4),
                   crack_cap=crack_cap or max(4096, ne // 4))


def hole_mask(n, L, r):
    """Element inactive iff its centroid lies strictly within r of the centre."""
    h = L / n
    c = (np.arange(n) + 0.5) * h - 0.5 * L
    X, Y = np.meshgrid(c, c)
    return (X * X + Y * Y >= r * r).astype(np.uint8).reshape(-1)


def fragmentation(n=2048, L=0.1, r=0.005, mode="neumann", p0=50e6, v0=2.0, seed=2509,
                  gc_mean=3.0, gc_shape=10.0, steps=None, t_end=60e-6,
                  material: Optional[Material] = None, energy_every=0, name=None,
                  phantom_cap=None, crack_cap=None):
    """Square plate with a central hole; Weibull G_c; internal pressure pulse
    p(t) = p0 t/t0 (t <= t0), p0 exp(-(t-t0)/tau) after, t0 = 1 us,
    tau = 100 us (Sec. 4.4 law shape) or outward edge velocity ramped over
    t0 = 1 us (Sec. 4.1 ramp shape)."""
    h = L / n
    active = hole_mask(n, L, r)
    gc = weibull_gc(n * n, gc_mean, gc_shape, seed)
    mat = material or Material()
    if mode == "neumann":
        bcs = [BC(PRESSURE, interface_edges(n, n, active), 0, LAW_RAMP_EXP, p0, 1e-6, 100e-6)]
    elif mode == "dirichlet":
        bcs = [BC(VELOCITY, boundary_nodes(n, n, "left"), 1, LAW_RAMP, -v0, 1e-6),
               BC(VELOCITY, boundary_nodes(n, n, "right"), 1, LAW_RAMP, +v0, 1e-6),
               BC(VELOCITY, boundary_nodes(n, n, "bottom"), 2, LAW_RAMP, -v0, 1e-6),
               BC(VELOCITY, boundary_nodes(n, n, "top"), 2, LAW_RAMP, +v0, 1e-6)]
    else:
        raise ValueError(mode)
    ne = n * n
    prob = Problem(name=name or f"fragmentation_{n}x{n}_{mode}", nx=n, ny=n, hx=h, hy=h,
                   material=mat, active=active, gc=gc, bcs=bcs, energy_every=energy_every,
                   phantom_cap=phantom_cap or max(8192, ne // 4),
                   crack_cap=crack_cap or max(8192, ne // 8))
    if steps is None:
        steps = int(math.ceil(t_end / estimate_dt(prob)))
    prob.steps = steps
    return prob


def kalthoff(n=200, L=0.1, notch_y=0.025, notch_len=0.05, v0=16.5, t0=1e-6, t_end=90e-6,
             scope=SCOPE_NBHD, steps=None, name=None, phantom_cap=None, crack_cap=None):
    """Upper half of the Kalthoff-Winkler plate (Sec. 4.1): an L x L square
    (the plate's symmetry line is the bottom edge, held at v_y = 0), a notch
    from the left edge along y = notch_y of length notch_len, and the impact
    on the left edge below the notch: v_x = v0 t/t0 (t <= t0), v0 after.
    Steel of Sec. 4.1: E = 190 GPa, nu = 0.3, rho = 8000 kg/m^3,
    G_c = 2.213e4 J/m^2, plane strain.  The notch is a row of pattern-II
    pre-cracks in the element row just below y = notch_y (a node line); the
    tracking scope is MCT (node neighbourhoods) or SCT (tips only)."""
    h = L / n
    mat = Material(E=190e9, nu=0.3, rho=8000.0, gc_uniform=2.213e4, scope=scope)
    jn = int(round(notch_y / h)) - 1
    nnotch = int(round(notch_len / h))
    pre = np.array([[jn * n + i, 3, 1] for i in range(nnotch)], np.int32).reshape(-1, 3)
    left = [node_id(n, 0, j) for j in range(jn + 1)]  # left-edge nodes below the notch
    bcs = [BC(VELOCITY, np.array(left, np.int32), 1, LAW_RAMP, v0, t0),
           BC(VELOCITY, boundary_nodes(n, n, "bottom"), 2, LAW_RAMP, 0.0, t0)]
    prob = Problem(name=name or f"kalthoff_{n}x{n}_{'sct' if scope == SCOPE_TIPS else 'mct'}",
                   nx=n, ny=n, hx=h, hy=h, material=mat, bcs=bcs, precracks=pre,
                   phantom_cap=phantom_cap or max(8192, n * n), crack_cap=crack_cap or max(4096, n * n // 2))
    if steps is None:
        steps = int(math.ceil(t_end / estimate_dt(prob)))
    prob.steps = steps
    return prob


def compact_tension(n=100, L=0.25, notch_len=0.125, v0=3.993, t0=100e-6, t_end=200e-6, gc=100.0,
                    scope=SCOPE_NBHD, steps=None, name=None, phantom_cap=None, crack_cap=None):
    """Dirichlet compact-tension plate (our approximation of Sec. 4.3, whose
    dimensions are given only in a figure): an L x L square, a vertical
    notch from the middle of the top edge down to depth notch_len, driven by
    velocities on the notch faces: the nodes of the right face get
    v_x = v0 t/t0 (t <= t0), v0 after (the ramp-then-constant law of Sec.
    4.3; v0 = 1.375, 3.318 or 3.993 m/s there, t0 = 100 us), the nodes of the
    left face are held at v_x = 0.  The notch is a column of pattern-II
    pre-cracks (bottom-edge midpoint to top-edge midpoint) in element column
    n/2; the face nodes are those of its elements above the tip element's
    lower edge.  The material is the concrete-like one of Sec. 4.2
    (E = 32 GPa, nu = 0.2, rho = 2450 kg/m^3, G_c = 3 J/m^2), plane strain."""
    h = L / n
    mat = Material(E=32e9, nu=0.2, rho=2450.0, gc_uniform=gc, scope=scope)
    i0 = n // 2
    nnotch = max(1, int(round(notch_len / h)))
    rows = range(n - nnotch, n)
    pre = np.array([[j * n + i0, 0, 2] for j in reversed(rows)], np.int32).reshape(-1, 3)
    face = range(n - nnotch + 1, n + 1)
    left = np.array([node_id(n, i0, j) for j in face], np.int32)
    right = np.array([node_id(n, i0 + 1, j) for j in face], np.int32)
    bcs = [BC(VELOCITY, right, 1, LAW_RAMP, v0, t0),
           BC(VELOCITY, left, 1, LAW_RAMP, 0.0, t0)]
    prob = Problem(name=name or f"compact_tension_{n}x{n}_v{v0:g}", nx=n, ny=n, hx=h, hy=h,
                   material=mat, bcs=bcs, precracks=pre,
                   phantom_cap=phantom_cap or max(8192, 2 * n * n),
                   crack_cap=crack_cap or max(4096, n * n // 2))
    if steps is None:
        steps = int(math.ceil(t_end / estimate_dt(prob)))
    prob.steps = steps
    return prob


def estimate_dt(prob: Problem) -> float:
    """Half the plane-strain CFL limit, for sizing step counts only."""
    m = prob.material
    E, nu, rho = m.E, m.nu, m.rho
    cd = math.sqrt(E * (1 - nu) / (rho * (1 + nu) * (1 - 2 * nu)))
    return prob.dt_factor * min(prob.hx, prob.hy) / cd


def batch_specimens(count=64, seed=1827, t_end=80e-6, smin=1.0, smax=4.0):
    """Notched plates with s ~ U(smin, smax): nx = round(100 s), ny = round(40 s),
    notch length ~ U(30, 60) mm, traction ~ U(0.5, 3) MPa, each run to t_end."""
    u = np.stack([uniform01(count, seed, stream=q) for q in range(3)], axis=1)
    out = []
    for b in range(count):
        s = smin + (smax - smin) * u[b, 0]
        nx, ny = int(round(100 * s)), int(round(40 * s))
        notch = 0.030 + 0.030 * u[b, 1]
        trac = 0.5e6 + 2.5e6 * u[b, 2]
        p = notched_plate(nx=nx, ny=ny, notch_len=notch, traction=trac, steps=0,
                          name=f"specimen_{b}", phantom_cap=max(8192, 4 * nx * ny),
                          crack_cap=max(4096, nx * ny))
        p.steps = int(math.ceil(t_end / estimate_dt(p)))
        out.append(p)
    return out


def surrogate_run(seed, nx=400, ny=160, t_end=80e-6, gc_mean=3.0, gc_shape=10.0):
    """One run of the surrogate's data set: the 400 x 160 notched plate with
    traction ~ U(0.5, 3) MPa (Philox stream 1), notch length ~ U(30, 60) mm
    (stream 2) and a Weibull G_c field (mean 3 J/m^2, shape 10, stream 0),
    all drawn from `seed`, run to t_end.  Returns the problem and the drawn
    scalars."""
    trac = 0.5e6 + 2.5e6 * float(uniform01(1, seed, stream=1)[0])
    notch = 0.030 + 0.030 * float(uniform01(1, seed, stream=2)[0])
    ne = nx * ny
    p = notched_plate(nx=nx, ny=ny, notch_len=notch, traction=trac, steps=0,
                      name=f"surrogate_run_{seed}", phantom_cap=4 * ne, crack_cap=ne)
    p.gc = weibull_gc(ne, gc_mean, gc_shape, seed)
    p.steps = int(math.ceil(t_end / estimate_dt(p)))
    return p, {"traction": trac, "notch_len": notch, "seed": int(seed)}


CONFIGS = {
    "notched_plate_100x40": lambda: notched_plate(100, 40, steps=2000),
    "notched_plate_400x160": lambda: notched_plate(400, 160, steps=int(math.ceil(80e-6 / estimate_dt(notched_plate(400, 160, steps=0))))),
    "fragmentation_2048_neumann": lambda: fragmentation(2048, mode="neumann"),
    "fragmentation_2048_dirichlet": lambda: fragmentation(2048, mode="dirichlet"),
}


# ------------------------------------------------ unstructured triangles
@dataclass
class TriProblem:
    """An unstructured mesh of constant-strain triangles (the paper's own
    element, Sec. 2.1): node coordinates X (nn, 2), counter-clockwise
    connectivity conn (ne, 3); loads as for Problem, with Neumann items given
    as edge ids of ``tri_edges`` and Dirichlet items as node ids; an optional
    initial state init = (ux, uy, vx, vy)."""
    name: str
    X: np.ndarray
    conn: np.ndarray
    material: Material = field(default_factory=Material)
    bcs: List[BC] = field(default_factory=list)
    dt_factor: float = 0.5
    dt: Optional[float] = None
    steps: int = 0
    energy_every: int = 0
    init: Optional[tuple] = None
    gc: Optional[np.ndarray] = None          # float32 per element, None = uniform

    @property
    def n_nodes(self):
        return len(self.X)

    @property
    def n_elems(self):
        return len(self.conn)


def tri_edges(conn):
    """The edges of a triangle mesh: the distinct node pairs {a, b} of the
    elements' sides, numbered in increasing (min, max); for each, its nodes
    n1 < n2 and its elements e1 < e2 (e2 = -1 on the boundary)."""
    conn = np.asarray(conn, np.int64)
    ne = len(conn)
    a = conn.reshape(-1)
    b = conn[:, [1, 2, 0]].reshape(-1)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    el = np.repeat(np.arange(ne), 3)
    order = np.lexsort((el, hi, lo))
    lo, hi, el = lo[order], hi[order], el[order]
    first = np.ones(len(lo), bool)
    first[1:] = (lo[1:] != lo[:-1]) | (hi[1:] != hi[:-1])
    idx = np.flatnonzero(first)
    n1, n2, e1 = lo[idx], hi[idx], el[idx]
    e2 = np.full(len(idx), -1, np.int64)
    two = np.append(idx[1:], len(lo)) - idx == 2
    e2[two] = el[idx[two] + 1]
    return dict(n1=n1.astype(np.int32), n2=n2.astype(np.int32), e1=e1.astype(np.int32),
                e2=e2.astype(np.int32))


def tri_plate(nx=40, ny=16, lx=0.1, ly=0.04, jitter=0.2, seed=11, traction=1e6, v0=0.0,
              t0=1e-6, t_end=20e-6, random_state=0.0, steps=None, name=None,
              material=None):
    """A rectangular plate meshed by triangles: an (nx+1) x (ny+1) grid whose
    interior nodes are moved by up to jitter x the cell size (Philox streams
    0 and 1 of seed; jitter <= 0.2 keeps every triangle counter-clockwise:
    two nodes then move at most 0.57 of the 0.71 cell-size altitude towards
    each other), each cell split along a diagonal that alternates with the
    cell's parity.  Loads: normal traction on the top and bottom edges
    (top +y, bottom -y, from t = 0) and, if v0 != 0, a prescribed
    x-velocity ramped to v0 over t0 on the left edge.  random_state > 0 adds
    a seeded initial displacement and velocity field of that amplitude
    (streams 2-5), to exercise every term of the stiffness."""
    if not 0 <= jitter <= 0.2:
        raise ValueError("jitter must be in [0, 0.2]")
    hx, hy = lx / nx, ly / ny
    ii, jj = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1))
    x = ii.reshape(-1) * hx
    y = jj.reshape(-1) * hy
    nn = (nx + 1) * (ny + 1)
    interior = ((ii > 0) & (ii < nx) & (jj > 0) & (jj < ny)).reshape(-1)
    if jitter:
        dx = (uniform01(nn, seed, stream=0) - 0.5) * 2.0 * jitter * hx
        dy = (uniform01(nn, seed, stream=1) - 0.5) * 2.0 * jitter * hy
        x = np.where(interior, x + dx, x)
        y = np.where(interior, y + dy, y)
    X = np.stack([x, y], axis=1)
    tris = []
    for j in range(ny):
        for i in range(nx):
            n00, n10 = j * (nx + 1) + i, j * (nx + 1) + i + 1
            n01, n11 = n00 + nx + 1, n10 + nx + 1
            if (i + j) % 2 == 0:
                tris += [(n00, n10, n11), (n00, n11, n01)]
            else:
                tris += [(n00, n10, n01), (n10, n11, n01)]
    conn = np.array(tris, np.int32)
    ed = tri_edges(conn)
    yb = ed["e2"] < 0
    top = np.flatnonzero(yb & (np.abs(y[ed["n1"]] - ly) < 1e-12 * ly) & (np.abs(y[ed["n2"]] - ly) < 1e-12 * ly))
    bot = np.flatnonzero(yb & (np.abs(y[ed["n1"]]) < 1e-12 * ly) & (np.abs(y[ed["n2"]]) < 1e-12 * ly))
    bcs = []
    if traction:
        bcs += [BC(TRACTION, top.astype(np.int32), 2, LAW_CONST, traction),
                BC(TRACTION, bot.astype(np.int32), 2, LAW_CONST, -traction)]
    if v0:
        left = np.flatnonzero(np.abs(x) < 1e-12 * lx).astype(np.int32)
        bcs.append(BC(VELOCITY, left, 1, LAW_RAMP, v0, t0))
    init = None
    if random_state:
        r = [(uniform01(nn, seed, stream=q) - 0.5) * random_state for q in (2, 3, 4, 5)]
        init = (r[0] * hx, r[1] * hy, r[2], r[3])
    prob = TriProblem(name=name or f"tri_plate_{nx}x{ny}", X=X, conn=conn,
                      material=material or Material(), bcs=bcs, init=init)
    if steps is None:
        m = prob.material
        cd = math.sqrt(m.E * (1 - m.nu) / (m.rho * (1 + m.nu) * (1 - 2 * m.nu)))
        steps = int(math.ceil(t_end / (0.5 * 0.5 * min(hx, hy) / cd)))
    prob.steps = steps
    return prob
