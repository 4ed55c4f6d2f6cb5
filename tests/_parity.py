"""Helpers that run one problem through the CUDA library and the CPU oracle
and compare them (test infrastructure)."""
import numpy as np

from oracle.oracle import from_problem


def run_pair(prob, steps, precision=0, state=None, chunks=None):
    """Builds both simulations, optionally sets an initial state, steps both."""
    from paper_2509_01827_gb300.cem import Solver
    o = from_problem(prob)
    g = Solver(prob, precision=precision)
    if state is not None:
        o.set_state(**state)
        g.set_state(**state)
    for n in (chunks or [steps]):
        o.step(n)
        g.step(n)
    return o, g


def compare_fp64(o, g, exact=True, rtol=1e-12):
    """FP64 mode vs oracle: identical cracked sets, crack table, phantoms,
    surface/tip sets; fields bit-identical (exact) or within rtol."""
    oc, gc = o.counts(), g.counts()
    assert oc["n_crack"] == gc["n_cracked"], (oc, gc)
    assert oc["n_phantom"] == gc["n_phantoms"], (oc, gc)
    assert oc["step"] == gc["step"]
    ocr, gcr = o.cracks(), g.cracks()
    for k in ("elem", "ka", "kb", "step"):
        np.testing.assert_array_equal(ocr[k], gcr[k], err_msg=k)
    np.testing.assert_array_equal(ocr["nodes"], gcr["nodes"])
    np.testing.assert_array_equal(ocr["ud"], gcr["ud"])
    oph, gph = o.phantoms(), g.phantoms()
    for k in ("owner", "creator_e", "creator_a", "nuser"):
        np.testing.assert_array_equal(oph[k], gph[k], err_msg=k)
    np.testing.assert_array_equal(oph["users"], gph["users"])
    osf, gsf = o.surface(), g.surface()
    np.testing.assert_array_equal(osf["edge"], gsf["edge"])
    np.testing.assert_array_equal(osf["ahead"], gsf["ahead"])
    np.testing.assert_array_equal(osf["is_tip"], gsf["is_tip"])
    on, gn = o.nodes(), g.nodes()
    for k in ("ux", "uy", "vx", "vy", "m"):
        if exact:
            bad = np.nonzero(on[k] != gn[k])[0]
            assert len(bad) == 0, f"{k}: {len(bad)} differ, first {bad[:5]} " \
                                  f"{on[k][bad[:3]]} vs {gn[k][bad[:3]]}"
        else:
            scale = np.max(np.abs(on[k])) + 1e-300
            np.testing.assert_allclose(gn[k], on[k], rtol=0, atol=rtol * scale, err_msg=k)


def compare_energy(o, g, rtol=1e-12):
    oe, ge = o.energy(), g.energy()
    np.testing.assert_array_equal(oe["step"], ge["step"])
    for k in ("KE", "SE", "W_ext", "W_dir", "U_d"):
        scale = max(np.max(np.abs(oe[k])), 1e-300)
        np.testing.assert_allclose(ge[k], oe[k], rtol=0, atol=rtol * scale, err_msg=k)
