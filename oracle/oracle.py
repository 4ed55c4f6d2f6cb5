"""ctypes wrapper of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

It takes a problem description from the seeded input generators
(``paper_2509_01827_gb300.inputs``) and runs the oracle's explicit steps.
Nothing here imports or calls the CUDA library.
"""
import ctypes as C

import numpy as np

from . import build as _build

_LIB = None

TRACTION, PRESSURE, VELOCITY = 0, 1, 2
LAW_CONST, LAW_RAMP, LAW_RAMP_EXP = 0, 1, 2
SCOPE_NBHD, SCOPE_GLOBAL, SCOPE_TIPS = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_fp = C.POINTER(C.c_float)
_bp = C.POINTER(C.c_ubyte)


def lib():
    global _LIB
    if _LIB is None:
        L = C.CDLL(_build.build())
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _bp, C.c_int, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_error.restype = C.c_char_p
        L.orc_error.argtypes = [C.c_void_p]
        L.orc_set_material.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, _fp,
                                       C.c_double, C.c_int, C.c_double, C.c_int, C.c_int]
        L.orc_set_dt.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.orc_dt.restype = C.c_double
        L.orc_dt.argtypes = [C.c_void_p]
        L.orc_add_bc.argtypes = [C.c_void_p, C.c_int, C.c_int, _ip, C.c_int, C.c_int,
                                 C.c_double, C.c_double, C.c_double]
        L.orc_precrack.argtypes = [C.c_void_p, C.c_int, _ip]
        L.orc_set_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_set_energy_every.argtypes = [C.c_void_p, C.c_int]
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_counts.argtypes = [C.c_void_p, C.POINTER(C.c_long)]
        L.orc_get_nodes.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp]
        L.orc_get_phantoms.argtypes = [C.c_void_p, _ip, _ip, _ip, _ip, _ip]
        L.orc_get_cracks.argtypes = [C.c_void_p, _ip, _ip, _ip, _ip, _dp, _ip]
        L.orc_get_surface.argtypes = [C.c_void_p, _ip, _ip, _ip]
        L.orc_get_energy.argtypes = [C.c_void_p, _dp]
        L.orc_internal_force.argtypes = [C.c_void_p, _dp, _dp]
        L.orc_strain_energy.argtypes = [C.c_void_p, _dp]
        L.orc_element_stress.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.orc_eval_surface.argtypes = [C.c_void_p, _ip, _ip, _ip, _dp, _ip]
        L.orc_apply_proposals.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _ip, _dp]
        _LIB = L
    return _LIB


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


class OracleError(RuntimeError):
    pass


class OracleSim:
    """One oracle simulation on a structured nx*ny Q4 mesh."""

    def __init__(self, nx, ny, hx, hy, active=None, phantom_cap=4096, crack_cap=4096):
        L = lib()
        self.nx, self.ny, self.hx, self.hy = int(nx), int(ny), float(hx), float(hy)
        act = None if active is None else np.ascontiguousarray(active, dtype=np.uint8)
        self._h = L.orc_create(self.nx, self.ny, self.hx, self.hy, _p(act, _bp),
                               int(phantom_cap), int(crack_cap))
        if not self._h:
            raise OracleError("orc_create failed")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc != 0:
            raise OracleError(f"oracle error {rc}: {lib().orc_error(self._h).decode()}")

    # --- set-up -----------------------------------------------------------
    def set_material(self, E, nu, rho, gc=None, gc_uniform=3.0, plane_strain=True,
                     gamma=1.0, gamma_mode=0, scope=SCOPE_NBHD):
        g = None if gc is None else np.ascontiguousarray(gc, dtype=np.float32)
        self._gc_keep = g
        self._chk(lib().orc_set_material(self._h, E, nu, rho, _p(g, _fp), gc_uniform,
                                         int(bool(plane_strain)), gamma, gamma_mode, scope))

    def set_dt(self, dt_factor=0.5, dt=0.0):
        self._chk(lib().orc_set_dt(self._h, dt_factor, dt))

    @property
    def dt(self):
        return lib().orc_dt(self._h)

    def add_bc(self, kind, items, comp_mask=0, law=LAW_CONST, a0=0.0, t0=0.0, tau=0.0):
        it = np.ascontiguousarray(items, dtype=np.int32)
        self._chk(lib().orc_add_bc(self._h, kind, len(it), _p(it, _ip), comp_mask, law,
                                   a0, t0, tau))

    def precrack(self, triples):
        t = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1))
        self._chk(lib().orc_precrack(self._h, len(t) // 3, _p(t, _ip)))

    def set_state(self, ux=None, uy=None, vx=None, vy=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64)
                for a in (ux, uy, vx, vy)]
        self._chk(lib().orc_set_state(self._h, *[_p(a, _dp) for a in arrs]))

    def set_energy_every(self, K):
        self._chk(lib().orc_set_energy_every(self._h, int(K)))

    def step(self, n=1):
        self._chk(lib().orc_step(self._h, int(n)))

    # --- queries ----------------------------------------------------------
    def counts(self):
        out = (C.c_long * 9)()
        lib().orc_counts(self._h, out)
        keys = ["nn", "ne", "nedge", "n_phantom", "n_crack", "step", "n_surface",
                "n_tips", "n_energy"]
        return dict(zip(keys, [int(v) for v in out]))

    def nodes(self):
        c = self.counts()
        n = c["nn"] + c["n_phantom"]
        a = [np.zeros(n) for _ in range(5)]
        lib().orc_get_nodes(self._h, *[_p(x, _dp) for x in a])
        return dict(zip(["ux", "uy", "vx", "vy", "m"], a))

    def phantoms(self):
        n = self.counts()["n_phantom"]
        owner, ce, ca, nu = (np.zeros(n, np.int32) for _ in range(4))
        users = np.zeros(n * 12, np.int32)
        lib().orc_get_phantoms(self._h, _p(owner, _ip), _p(ce, _ip), _p(ca, _ip), _p(nu, _ip),
                               _p(users, _ip))
        return dict(owner=owner, creator_e=ce, creator_a=ca, nuser=nu,
                    users=users.reshape(n, 4, 3))

    def cracks(self):
        n = self.counts()["n_crack"]
        elem, ka, kb, st = (np.zeros(n, np.int32) for _ in range(4))
        ud = np.zeros(n)
        nodes = np.zeros(n * 8, np.int32)
        lib().orc_get_cracks(self._h, _p(elem, _ip), _p(ka, _ip), _p(kb, _ip), _p(st, _ip),
                             _p(ud, _dp), _p(nodes, _ip))
        return dict(elem=elem, ka=ka, kb=kb, step=st, ud=ud, nodes=nodes.reshape(n, 2, 4))

    def surface(self):
        n = self.counts()["n_surface"]
        edge, ahead, tip = (np.zeros(n, np.int32) for _ in range(3))
        lib().orc_get_surface(self._h, _p(edge, _ip), _p(ahead, _ip), _p(tip, _ip))
        return dict(edge=edge, ahead=ahead, is_tip=tip.astype(bool))

    def energy(self):
        n = self.counts()["n_energy"]
        rec = np.zeros(n * 7)
        lib().orc_get_energy(self._h, _p(rec, _dp))
        rec = rec.reshape(n, 7)
        return dict(step=rec[:, 0].astype(np.int64), t=rec[:, 1], KE=rec[:, 2], SE=rec[:, 3],
                    W_ext=rec[:, 4], W_dir=rec[:, 5], U_d=rec[:, 6])

    def internal_force(self):
        c = self.counts()
        n = c["nn"] + c["n_phantom"]
        fx, fy = np.zeros(n), np.zeros(n)
        lib().orc_internal_force(self._h, _p(fx, _dp), _p(fy, _dp))
        return fx, fy

    def strain_energy(self):
        se = np.zeros(1)
        self._chk(lib().orc_strain_energy(self._h, _p(se, _dp)))
        return float(se[0])

    def element_stress(self):
        """Mean stress (sxx, syy, sxy) of every element, shape (ne, 3)."""
        ne = self.nx * self.ny
        out = [np.zeros(ne) for _ in range(3)]
        self._chk(lib().orc_element_stress(self._h, *[_p(a, _dp) for a in out]))
        return np.stack(out, 1)

    def eval_surface(self):
        n = self.counts()["n_surface"]
        edge, ahead, k0, pk = (np.zeros(n, np.int32) for _ in range(4))
        G = np.zeros(n * 4)
        lib().orc_eval_surface(self._h, _p(edge, _ip), _p(ahead, _ip), _p(k0, _ip), _p(G, _dp),
                               _p(pk, _ip))
        return dict(edge=edge, ahead=ahead, k0=k0, G=G.reshape(n, 4), prop_k=pk)

    def apply_proposals(self, edge, elem, k, G):
        e = np.ascontiguousarray(edge, np.int32)
        el = np.ascontiguousarray(elem, np.int32)
        kk = np.ascontiguousarray(k, np.int32)
        g = np.ascontiguousarray(G, np.float64)
        self._chk(lib().orc_apply_proposals(self._h, len(e), _p(e, _ip), _p(el, _ip),
                                            _p(kk, _ip), _p(g, _dp)))


def from_problem(prob, phantom_cap=None, crack_cap=None):
    """Builds an oracle simulation from a ``paper_2509_01827_gb300.inputs.Problem``."""
    ne = prob.nx * prob.ny
    pc = phantom_cap if phantom_cap is not None else prob.phantom_cap
    cc = crack_cap if crack_cap is not None else prob.crack_cap
    s = OracleSim(prob.nx, prob.ny, prob.hx, prob.hy, prob.active, pc, cc)
    m = prob.material
    s.set_material(m.E, m.nu, m.rho, prob.gc, m.gc_uniform, m.plane_strain, m.gamma,
                   m.gamma_mode, m.scope)
    if prob.dt is not None:
        s.set_dt(0.0, prob.dt)
    else:
        s.set_dt(prob.dt_factor, 0.0)
    for bc in prob.bcs:
        s.add_bc(bc.kind, bc.items, bc.comp_mask, bc.law, bc.a0, bc.t0, bc.tau)
    if len(prob.precracks):
        s.precrack(prob.precracks)
    if prob.energy_every:
        s.set_energy_every(prob.energy_every)
    del ne
    return s
