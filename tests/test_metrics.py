"""Crack-pattern metrics (Jaccard, tips, branching, branch angle, fragments)
against brute force, the oracle's own tip list, and constructed patterns
whose answer is known geometrically (CPU only)."""
import math

import numpy as np
import pytest

from oracle.oracle import OracleSim, from_problem
from paper_2509_01827_gb300 import inputs, metrics

E, NU, RHO = 32e9, 0.2, 2450.0


def test_jaccard():
    assert metrics.jaccard([], []) == 1.0
    assert metrics.jaccard([1, 2, 3], [3, 4]) == pytest.approx(1 / 4)
    assert metrics.jaccard(np.array([5, 6]), [6, 5]) == 1.0


def _edge_id(e, k, nx, ny):
    i, j = e % nx, e // nx
    return [inputs.h_edge(nx, i, j), inputs.v_edge(nx, ny, i + 1, j),
            inputs.h_edge(nx, i, j + 1), inputs.v_edge(nx, ny, i, j)][k]


def test_tips_match_the_oracle_tip_list_through_a_run():
    """Tip sets reconstructed from the final crack table at earlier steps
    equal the oracle's own surface/tip list recorded at those steps."""
    p = inputs.notched_plate(60, 24, lx=0.06, ly=0.024, notch_len=0.02, traction=3e6, steps=0,
                             phantom_cap=20000, crack_cap=1440)
    o = from_problem(p)
    seen = {}
    for _ in range(16):
        o.step(25)
        sf = o.surface()
        seen[o.counts()["step"]] = sorted(int(g) for g, t in zip(sf["edge"], sf["is_tip"]) if t)
    cr = o.cracks()
    assert len(cr["elem"]) > 40 and len(set(cr["step"].tolist())) > 5
    for step, want in seen.items():
        # splits are recorded with the step that made them; the list after
        # `step` completed steps holds the splits of steps < step
        got = sorted(_edge_id(e, k, p.nx, p.ny)
                     for e, k, _, _ in metrics.tips_at(cr, step - 1, p.nx, p.ny, p.hx, p.hy))
        assert got == want, step


def _branch(start, k_in, moves, nx):
    """Cracked elements of a staircase path: from element `start` entered
    through local edge k_in, one move per element ('R', 'U', 'D')."""
    exit_of = {"R": 1, "U": 2, "D": 0}
    entry_of = {"R": 3, "U": 0, "D": 2}
    step = {"R": (1, 0), "U": (0, 1), "D": (0, -1)}
    i, j = start
    out = []
    for m in moves:
        out.append((j * nx + i, k_in, exit_of[m]))
        k_in = entry_of[m]
        i, j = i + step[m][0], j + step[m][1]
    return out


def _v_table(nx, ny, ib, j0, up, down):
    elem, ka, kb, st = [], [], [], []
    for i in range(ib + 1):                     # trunk, one element per step
        elem.append(j0 * nx + i), ka.append(3), kb.append(1), st.append(i)
    for q, (e, a, b) in enumerate(_branch((ib + 1, j0), 3, up, nx)):
        elem.append(e), ka.append(a), kb.append(b), st.append(ib + 1 + q)
    for q, (e, a, b) in enumerate(_branch((ib, j0 - 1), 2, down, nx)):
        elem.append(e), ka.append(a), kb.append(b), st.append(ib + 1 + q)
    order = np.argsort(np.array(st), kind="stable")
    return {k: np.array(v)[order] for k, v in
            dict(elem=elem, ka=ka, kb=kb, step=st).items()}


@pytest.mark.parametrize("up,down,angle", [
    ("UR" * 30, "RD" * 30, 90.0),
    ("RRU" * 20, "RRD" * 20, 2 * math.degrees(math.atan(0.5))),
    ("RRRU" * 15, "RRRD" * 15, 2 * math.degrees(math.atan(1 / 3))),
])
def test_branch_angle_of_constructed_v(up, down, angle):
    """A straight trunk along a row, then two staircase branches that leave
    its last element at slopes +-s (one from the tip, one from a face point
    below it).  The tips separate by >= 3h a few steps after the fork, the
    branch element is the trunk's last element, and the angle is 2 atan(s)
    up to the staircase's discretisation."""
    nx, ny, h = 120, 80, 0.25e-3
    ib, j0 = 40, 40
    cr = _v_table(nx, ny, ib, j0, up, down)
    s = metrics.branching_step(cr, nx, ny, h, h)
    assert s is not None and ib + 1 <= s <= ib + 6
    a, b = metrics.branch_angle(cr, nx, ny, h, h, radius=5e-3)
    assert b == j0 * nx + ib
    assert abs(a - angle) < 6.0, (a, angle)


def test_straight_crack_never_branches():
    """A crack grown from the left boundary, one element per step, has one
    tip at every step.  (A crack that starts inside the mesh has two ends,
    and the definition counts them as two tips.)"""
    nx, ny, h = 50, 20, 1e-3
    cr = dict(elem=np.arange(0, 40) + 10 * nx, ka=np.full(40, 3), kb=np.full(40, 1),
              step=np.arange(40))
    assert metrics.branching_step(cr, nx, ny, h, h) is None
    assert metrics.branch_angle(cr, nx, ny, h, h) == (None, None)


def _oracle_cracks(nx, ny, triples, active=None):
    s = OracleSim(nx, ny, 1e-3, 1e-3, active, 10 * nx * ny, nx * ny)
    s.set_material(E, NU, RHO, None, 3.0, True, 1.0, 0, 0)
    if triples:
        s.precrack(triples)
    return s.cracks()


@pytest.mark.parametrize("case,want", [
    ("intact", 1), ("partial_row", 1), ("full_row", 2), ("two_rows", 3), ("cross", 2),
    ("hole_column", 2), ("notch_around_corner", 2),
])
def test_fragment_counts(case, want):
    """Fragments of pre-cut meshes whose count is fixed by their geometry."""
    nx, ny = 9, 7
    act = None
    if case == "intact":
        t = []
    elif case == "partial_row":
        t = [[3 * nx + i, 3, 1] for i in range(nx - 1)]
    elif case == "full_row":
        t = [[3 * nx + i, 3, 1] for i in range(nx)]
    elif case == "two_rows":
        t = [[2 * nx + i, 3, 1] for i in range(nx)] + [[5 * nx + i, 3, 1] for i in range(nx)]
    elif case == "cross":
        # a full column cut from bottom to top, and a row cut that stops at
        # both sides of the crossing element (an element is cut once): that
        # element's left and right pieces still join the upper and lower
        # quarters on their side, so the cuts leave two fragments
        col = 4
        t = [[3 * nx + i, 3, 1] for i in range(nx) if i != col]
        t += [[j * nx + col, 0, 2] for j in range(ny)]
    elif case == "hole_column":
        act = np.ones(nx * ny, np.uint8)
        act[[j * nx + 4 for j in range(ny)]] = 0
        t = []
    elif case == "notch_around_corner":
        # cut from the left edge along row 3 to column 4, then down to the
        # bottom edge: the lower-left block separates
        t = [[3 * nx + i, 3, 1] for i in range(4)] + [[3 * nx + 4, 3, 0]]
        t += [[j * nx + 4, 2, 0] for j in range(2, -1, -1)]
    cr = _oracle_cracks(nx, ny, t, act)
    n, labels = metrics.fragments(cr, nx, ny, act)
    assert n == want
    assert n == _brute_fragments(cr, nx, ny, act)


def _brute_fragments(cr, nx, ny, active):
    """Flood fill over pieces: two pieces touch when they hold a common node
    id (dense piece-by-piece comparison, no union-find)."""
    pieces = []
    split = {int(e): q for q, e in enumerate(cr["elem"])}
    for e in range(nx * ny):
        if active is not None and not active[e]:
            continue
        i, j = e % nx, e // nx
        if e in split:
            for p in (0, 1):
                pieces.append(set(int(x) for x in cr["nodes"][split[e]][p]))
        else:
            pieces.append({j * (nx + 1) + i, j * (nx + 1) + i + 1,
                           (j + 1) * (nx + 1) + i + 1, (j + 1) * (nx + 1) + i})
    seen = [False] * len(pieces)
    count = 0
    for s0 in range(len(pieces)):
        if seen[s0]:
            continue
        count += 1
        stack = [s0]
        seen[s0] = True
        while stack:
            a = stack.pop()
            for b in range(len(pieces)):
                if not seen[b] and pieces[a] & pieces[b]:
                    seen[b] = True
                    stack.append(b)
    return count


def test_fragments_of_random_scripted_cracking_match_brute_force():
    rng = np.random.default_rng(11)
    nx, ny = 10, 8
    s = OracleSim(nx, ny, 1e-3, 1e-3, None, 10 * nx * ny, nx * ny)
    s.set_material(E, NU, RHO, None, 3.0, True, 1.0, 0, 0)
    s.precrack([[4 * nx, 3, 1]])
    for _ in range(12):
        ev = s.eval_surface()
        pick = np.nonzero(rng.random(len(ev["edge"])) < 0.6)[0]
        k = [int(rng.choice([q for q in range(4) if q != k0])) for k0 in ev["k0"][pick]]
        s.apply_proposals(ev["edge"][pick], ev["ahead"][pick], k,
                          rng.integers(1, 5, len(pick)).astype(float))
    cr = s.cracks()
    assert len(cr["elem"]) > 30
    n, _ = metrics.fragments(cr, nx, ny)
    assert n == _brute_fragments(cr, nx, ny, None)
    assert n > 1


@pytest.mark.parametrize("slope_deg", [70.0, 45.0, 20.0])
def test_crack_angle_of_a_staircase(slope_deg):
    """Elements along a straight line from the origin at a known angle (their
    centroids within half an element of it) give that angle back."""
    nx, ny, h = 300, 300, 0.5e-3
    ox, oy = 50e-3, 25e-3
    t = math.radians(slope_deg)
    elems = []
    for q in range(1, 2000):
        x, y = ox + q * 0.1 * h * math.cos(t), oy + q * 0.1 * h * math.sin(t)
        e = int(y // h) * nx + int(x // h)
        if e not in elems:
            elems.append(e)
    cr = dict(elem=np.array(elems), step=np.arange(len(elems)))
    a = metrics.crack_angle(cr, nx, h, h, (ox, oy), 5e-3, 40e-3)
    assert abs(a - slope_deg) < 1.5, a
    assert metrics.crack_angle(cr, nx, h, h, (ox, oy), 200e-3, 300e-3) is None
