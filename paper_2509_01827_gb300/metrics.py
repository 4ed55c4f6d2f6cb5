"""Crack-pattern metrics over the library's crack tables (host-side analysis).

These compare two runs of the same problem (for example the FP32-mixed mode
against the FP64 mode) after crack initiation.  The paper prints none of
them; the definitions are this library's own:

* Jaccard index of the cracked-element sets, |A & B| / |A | B| (1 when both
  are empty).
* Tip set at step s: every cut edge (element e split at a step <= s, local
  edge k in {ka, kb}) whose neighbour across k is an active element that is
  still intact at step s.  A tip's position is its edge midpoint (the crack
  front of Sec. 3's multiple-tip tracking).
* Branching step: the first step at which the tip set holds two tips at least
  3h apart (h = the element size).
* Branch angle: at the branching step, the branch element b is the split
  element that is closest, along the graph of split elements that share an
  edge cut in at least one of them (a crack that starts at a face point of
  another crack enters through an edge the other element does not cut), to
  both of the two tips that are furthest apart (it minimises the larger of
  its two graph distances).  The trunk direction d points from the mean
  centroid of the other elements split no later than b within `radius` of b
  to b.  The split elements of the final table that lie within
  `radius` of b and ahead of it ((c - b) . d > 0) form two branches, one on
  each side of d; the angle is the one between the vectors from b's centroid
  to each branch's mean centroid.
* Crack angle: the direction, from a crack's origin (a notch tip), of the
  mean offset of the elements split within a ring of radii r_min .. r_max
  around it.
* Fragments: connected pieces of material after splitting.  Every intact
  element is one piece and every split element two (the pieces on each side
  of its cut); pieces that share a node, real or phantom, are joined (they
  share its degrees of freedom).  This is the count of Sec. 4.4 (Table 1
  lists the fragments of the pressurised cylinder).

Every function takes plain arrays (numpy) from ``cem.Solver.cracks()``, the
oracle's ``cracks()``, or any caller holding the same table.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np

# element local edge k joins local nodes k and (k + 1) % 4;
# local node a of element (i, j) sits at (i + di[a], j + dj[a])
_DI = (0, 1, 1, 0)
_DJ = (0, 0, 1, 1)
# neighbour across local edge k: (di, dj) of the element, and the edge it shares
_NB = ((0, -1, 2), (1, 0, 3), (0, 1, 0), (-1, 0, 1))


def jaccard(a, b) -> float:
    """|A & B| / |A | B| of two element-id collections (1.0 if both empty)."""
    A, B = set(int(x) for x in a), set(int(x) for x in b)
    if not A and not B:
        return 1.0
    return len(A & B) / len(A | B)


def _centroid(e, nx, hx, hy):
    return ((e % nx) + 0.5) * hx, ((e // nx) + 0.5) * hy


def _edge_mid(e, k, nx, hx, hy):
    i, j = e % nx, e // nx
    a, b = k, (k + 1) % 4
    return (i + 0.5 * (_DI[a] + _DI[b])) * hx, (j + 0.5 * (_DJ[a] + _DJ[b])) * hy


def _neighbour(e, k, nx, ny):
    i, j = e % nx, e // nx
    di, dj, kf = _NB[k]
    ii, jj = i + di, j + dj
    if ii < 0 or jj < 0 or ii >= nx or jj >= ny:
        return -1, -1
    return jj * nx + ii, kf


def tips_at(cracks, step, nx, ny, hx, hy, active=None):
    """Tip set after the splits of `step`: list of (element, local edge, x, y)."""
    elem = np.asarray(cracks["elem"])
    st = np.asarray(cracks["step"])
    ka, kb = np.asarray(cracks["ka"]), np.asarray(cracks["kb"])
    split_at = {int(e): int(s) for e, s in zip(elem, st)}
    out = []
    for e, s, a, b in zip(elem, st, ka, kb):
        if s > step:
            continue
        for k in (int(a), int(b)):
            f, _ = _neighbour(int(e), k, nx, ny)
            if f < 0 or (active is not None and not active[f]):
                continue
            if split_at.get(f, step + 1) <= step:
                continue
            x, y = _edge_mid(int(e), k, nx, hx, hy)
            out.append((int(e), k, x, y))
    return out


def _far_pair(tips):
    best, pair = -1.0, None
    P = np.array([(t[2], t[3]) for t in tips])
    for p in range(len(tips)):
        d2 = np.sum((P[p + 1:] - P[p]) ** 2, axis=1)
        if len(d2):
            q = int(np.argmax(d2))
            if d2[q] > best:
                best, pair = float(d2[q]), (p, p + 1 + q)
    return math.sqrt(max(best, 0.0)), pair


def branching_step(cracks, nx, ny, hx, hy, active=None, min_sep=3.0):
    """First step whose tip set holds two tips >= min_sep * h apart, or None.

    Only steps at which some element split can change the tip set, so those
    are the steps examined."""
    h = max(hx, hy)
    for s in sorted(set(int(x) for x in np.asarray(cracks["step"]))):
        tips = tips_at(cracks, s, nx, ny, hx, hy, active)
        if len(tips) < 2:
            continue
        d, _ = _far_pair(tips)
        if d >= min_sep * h - 1e-12 * h:
            return s
    return None


def _split_graph(cracks, step, nx, ny):
    """Adjacency of elements split at or before `step` that share an edge cut
    in at least one of them."""
    elem = np.asarray(cracks["elem"])
    st = np.asarray(cracks["step"])
    ka, kb = np.asarray(cracks["ka"]), np.asarray(cracks["kb"])
    cuts = {}
    for e, s, a, b in zip(elem, st, ka, kb):
        if s <= step:
            cuts[int(e)] = (int(a), int(b))
    adj = {e: [] for e in cuts}
    for e, (a, b) in cuts.items():
        for k in (a, b):
            f, _ = _neighbour(e, k, nx, ny)
            if f in cuts and f not in adj[e]:
                adj[e].append(f)
                adj[f].append(e)
    return adj


def _bfs(adj, src):
    dist = {src: 0}
    q = deque([src])
    while q:
        e = q.popleft()
        for f in adj[e]:
            if f not in dist:
                dist[f] = dist[e] + 1
                q.append(f)
    return dist


def branch_angle(cracks, nx, ny, hx, hy, active=None, radius=5e-3, min_sep=3.0):
    """Branch angle in degrees (definition in the module docstring) and the
    branch element, or (None, None) when the run never branches or a branch
    is empty."""
    s = branching_step(cracks, nx, ny, hx, hy, active, min_sep)
    if s is None:
        return None, None
    tips = tips_at(cracks, s, nx, ny, hx, hy, active)
    _, (p, q) = _far_pair(tips)
    adj = _split_graph(cracks, s, nx, ny)
    d1, d2 = _bfs(adj, tips[p][0]), _bfs(adj, tips[q][0])
    common = [e for e in d1 if e in d2]
    if not common:
        return None, None
    b = min(common, key=lambda e: (max(d1[e], d2[e]), d1[e] + d2[e], e))
    bx, by = _centroid(b, nx, hx, hy)
    elem = np.asarray(cracks["elem"])
    st = np.asarray(cracks["step"])
    sb = int(st[np.nonzero(elem == b)[0][0]])
    trunk = [e for e, t in zip(elem, st) if t <= sb and e != b]
    trunk = [_centroid(int(e), nx, hx, hy) for e in trunk]
    trunk = [(x, y) for x, y in trunk if (x - bx) ** 2 + (y - by) ** 2 <= radius * radius]
    if not trunk:
        return None, b
    tx, ty = np.mean(trunk, axis=0)
    d = np.array([bx - tx, by - ty])
    nd = np.linalg.norm(d)
    if nd == 0.0:
        return None, b
    d /= nd
    left, right = [], []
    for e in elem:
        cx, cy = _centroid(int(e), nx, hx, hy)
        r = np.array([cx - bx, cy - by])
        if r @ r > radius * radius or r @ d <= 0.0:
            continue
        side = d[0] * r[1] - d[1] * r[0]
        if side > 0:
            left.append(r)
        elif side < 0:
            right.append(r)
    if not left or not right:
        return None, b
    u, v = np.mean(left, axis=0), np.mean(right, axis=0)
    c = float(u @ v / (np.linalg.norm(u) * np.linalg.norm(v)))
    return math.degrees(math.acos(max(-1.0, min(1.0, c)))), b


def crack_angle(cracks, nx, hx, hy, origin, r_min, r_max, grown_only=True):
    """Direction (degrees from +x) of the crack grown from `origin`: the
    angle of the mean offset from origin of the split elements whose
    centroids lie between r_min and r_max from it (split during the run,
    not pre-cracks, when grown_only).  None when no element qualifies."""
    elem = np.asarray(cracks["elem"])
    st = np.asarray(cracks["step"])
    sel = st >= 0 if grown_only else np.ones(len(elem), bool)
    e = elem[sel]
    cx = (e % nx + 0.5) * hx - origin[0]
    cy = (e // nx + 0.5) * hy - origin[1]
    r = np.hypot(cx, cy)
    m = (r >= r_min) & (r <= r_max)
    if not np.any(m):
        return None
    return math.degrees(math.atan2(float(np.mean(cy[m])), float(np.mean(cx[m]))))


def fragments(cracks, nx, ny, active=None):
    """Number of fragments, and the fragment id of every piece.

    Pieces: an active intact element e is one piece, (e, 0), on its four real
    nodes; a split element is two, (e, p) on ``cracks["nodes"][c][p]`` (the
    real nodes on side p and phantom copies of the others).  Two pieces
    belong to one fragment when a chain of pieces joins them in which each
    consecutive pair shares a node, real or phantom: shared nodes are shared
    degrees of freedom, so such pieces move together.  Returns (count,
    labels): labels is an int array of shape (nx*ny, 2), the fragment id of
    piece (e, p) or -1 where there is no such piece; ids are numbered in
    increasing order of each fragment's lowest (element, piece)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    ne = nx * ny
    nn = (nx + 1) * (ny + 1)
    elem = np.asarray(cracks["elem"], np.int64)
    nodes = np.asarray(cracks["nodes"], np.int64).reshape(len(elem), 2, 4)
    act = np.ones(ne, bool) if active is None else np.asarray(active, bool)
    is_split = np.zeros(ne, bool)
    is_split[elem] = True
    e = np.arange(ne)
    i, j = e % nx, e // nx
    real = np.stack([j * (nx + 1) + i, j * (nx + 1) + i + 1, (j + 1) * (nx + 1) + i + 1,
                     (j + 1) * (nx + 1) + i], 1)
    # piece (e, p) -> vertex 2e + p; node n -> vertex 2 ne + n
    intact = np.nonzero(act & ~is_split)[0]
    rows = [np.repeat(2 * intact, 4)]
    cols = [real[intact].reshape(-1)]
    live = act[elem]
    for p in (0, 1):
        rows.append(np.repeat(2 * elem[live] + p, 4))
        cols.append(nodes[live, p].reshape(-1))
    r = np.concatenate(rows)
    c = 2 * ne + np.concatenate(cols)
    nv = 2 * ne + max(nn, int(c.max()) - 2 * ne + 1 if len(c) else nn)
    g = coo_matrix((np.ones(len(r), np.int8), (r, c)), shape=(nv, nv))
    _, comp = connected_components(g, directed=False)
    has = np.zeros(2 * ne, bool)
    has[2 * intact] = True
    has[2 * elem[live]] = True
    has[2 * elem[live] + 1] = True
    pv = np.nonzero(has)[0]                      # piece vertices in (e, p) order
    ids = np.full(2 * ne, -1, np.int64)
    _, inv = np.unique(comp[pv], return_inverse=True)
    # renumber components in order of their lowest piece
    _, first = np.unique(inv, return_index=True)
    rank = np.empty(len(first), np.int64)
    rank[np.argsort(first)] = np.arange(len(first))
    ids[pv] = rank[inv]
    return int(len(first)), ids.reshape(ne, 2)
