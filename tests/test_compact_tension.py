"""The Dirichlet compact-tension input (Sec. 4.3) and its run on the oracle
(CPU only)."""
import numpy as np

from paper_2509_01827_gb300 import inputs


def test_notch_and_face_velocities():
    """The notch is a column of bottom-to-top pre-cracks from the top edge in
    element column n/2; the right face is driven along x with the ramp law,
    the left face held along x; nodes of the tip element's lower edge carry
    no prescribed velocity."""
    n = 20
    p = inputs.compact_tension(n, L=0.2, notch_len=0.05)
    i0, nn = n // 2, 5
    pre = np.asarray(p.precracks)
    assert sorted(pre[:, 0].tolist()) == [j * n + i0 for j in range(n - nn, n)]
    assert set(pre[:, 1].tolist()) == {0} and set(pre[:, 2].tolist()) == {2}
    right, left = p.bcs
    assert right.kind == inputs.VELOCITY and right.comp_mask == 1 and right.a0 == 3.993
    assert right.law == inputs.LAW_RAMP and right.t0 == 100e-6
    assert left.kind == inputs.VELOCITY and left.comp_mask == 1 and left.a0 == 0.0
    rows = range(n - nn + 1, n + 1)
    assert sorted(right.items.tolist()) == [j * (n + 1) + i0 + 1 for j in rows]
    assert sorted(left.items.tolist()) == [j * (n + 1) + i0 for j in rows]


def test_faster_loading_dissipates_more():
    """On the oracle, the dissipated energy at 200 us and the number of
    grown splits increase with the loading rate of Sec. 4.3 (1.375, 3.318,
    3.993 m/s): more energy goes into cracking, and the crack branches."""
    from oracle.oracle import from_problem
    out = []
    for v0 in (1.375, 3.318, 3.993):
        p = inputs.compact_tension(30, v0=v0)
        o = from_problem(p)
        o.step(p.steps)
        c = o.cracks()  # U_d is the sum of the splits' G_c L (pre-cracks add 0)
        out.append((float(np.sum(c["ud"])), int(np.sum(c["step"] >= 0))))
        o.close()
    assert out[0][0] < out[1][0] < out[2][0]
    assert out[0][1] < out[1][1] < out[2][1]
