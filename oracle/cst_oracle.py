"""ctypes wrapper of the FP64 CST oracle -- TEST INFRASTRUCTURE ONLY.

ES-FEM constant-strain triangles on an unstructured mesh (Sec. 2.1, Eqs. 1,
3, 5), no cracking.  Takes a ``paper_2509_01827_gb300.inputs.TriProblem``.
Nothing here imports or calls the CUDA library.
"""
import ctypes as C

import numpy as np

from .oracle import lib as _lib

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_READY = False


def lib():
    global _READY
    L = _lib()
    if not _READY:
        L.ocst_create.restype = C.c_void_p
        L.ocst_create.argtypes = [C.c_int, C.c_int, _dp, _ip]
        L.ocst_create_error.restype = C.c_char_p
        L.ocst_error.restype = C.c_char_p
        L.ocst_error.argtypes = [C.c_void_p]
        L.ocst_destroy.argtypes = [C.c_void_p]
        L.ocst_n_edges.argtypes = [C.c_void_p]
        L.ocst_edges.argtypes = [C.c_void_p, _ip, _ip, _ip, _ip]
        L.ocst_set_material.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int]
        L.ocst_set_dt.argtypes = [C.c_void_p, C.c_double, C.c_double]
        L.ocst_dt.restype = C.c_double
        L.ocst_dt.argtypes = [C.c_void_p]
        L.ocst_add_bc.argtypes = [C.c_void_p, C.c_int, C.c_int, _ip, C.c_int, C.c_int, C.c_double,
                                  C.c_double, C.c_double]
        L.ocst_set_state.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.ocst_set_energy_every.argtypes = [C.c_void_p, C.c_int]
        L.ocst_step.argtypes = [C.c_void_p, C.c_int]
        L.ocst_get_nodes.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp]
        L.ocst_n_energy.argtypes = [C.c_void_p]
        L.ocst_get_energy.argtypes = [C.c_void_p, _dp]
        L.ocst_internal_force.argtypes = [C.c_void_p, _dp, _dp]
        L.ocst_strain_energy.argtypes = [C.c_void_p, _dp]
        L.ocst_set_fracture.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.c_double, C.c_double,
                                        C.c_int]
        L.ocst_eval_surface.argtypes = [C.c_void_p, C.c_int, _ip, _ip, _dp, _ip]
        _READY = True
    return L


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


class CstOracle:
    def __init__(self, X, conn):
        X = np.ascontiguousarray(X, np.float64).reshape(-1)
        conn = np.ascontiguousarray(conn, np.int32).reshape(-1)
        self.nn, self.ne = len(X) // 2, len(conn) // 3
        self._h = lib().ocst_create(self.nn, self.ne, _p(X, _dp), _p(conn, _ip))
        if not self._h:
            raise ValueError(lib().ocst_create_error().decode())

    def close(self):
        if self._h:
            lib().ocst_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, rc):
        if rc:
            raise RuntimeError(f"cst oracle error {rc}: {lib().ocst_error(self._h).decode()}")

    def edges(self):
        n = lib().ocst_n_edges(self._h)
        a = [np.zeros(n, np.int32) for _ in range(4)]
        lib().ocst_edges(self._h, *(_p(x, _ip) for x in a))
        return dict(n1=a[0], n2=a[1], e1=a[2], e2=a[3])

    def set_material(self, E, nu, rho, plane_strain=True):
        self._chk(lib().ocst_set_material(self._h, E, nu, rho, int(bool(plane_strain))))

    def set_dt(self, dt_factor=0.5, dt=0.0):
        self._chk(lib().ocst_set_dt(self._h, dt_factor, dt))

    @property
    def dt(self):
        return lib().ocst_dt(self._h)

    def add_bc(self, kind, items, comp_mask=0, law=0, a0=0.0, t0=0.0, tau=0.0):
        it = np.ascontiguousarray(items, np.int32)
        self._chk(lib().ocst_add_bc(self._h, kind, len(it), _p(it, _ip), comp_mask, law, a0, t0, tau))

    def set_state(self, ux=None, uy=None, vx=None, vy=None):
        f = lambda a: None if a is None else np.ascontiguousarray(a, np.float64)
        ux, uy, vx, vy = f(ux), f(uy), f(vx), f(vy)
        self._chk(lib().ocst_set_state(self._h, _p(ux, _dp), _p(uy, _dp), _p(vx, _dp), _p(vy, _dp)))

    def set_energy_every(self, K):
        self._chk(lib().ocst_set_energy_every(self._h, K))

    def step(self, n=1):
        self._chk(lib().ocst_step(self._h, int(n)))

    def nodes(self):
        a = [np.zeros(self.nn) for _ in range(5)]
        lib().ocst_get_nodes(self._h, *(_p(x, _dp) for x in a))
        return dict(ux=a[0], uy=a[1], vx=a[2], vy=a[3], m=a[4])

    def energy(self):
        n = lib().ocst_n_energy(self._h)
        rec = np.zeros((max(n, 1), 7))
        lib().ocst_get_energy(self._h, _p(rec, _dp))
        rec = rec[:n]
        return dict(step=rec[:, 0].astype(np.int64), t=rec[:, 1], KE=rec[:, 2], SE=rec[:, 3],
                    W_ext=rec[:, 4], W_dir=rec[:, 5], U_d=rec[:, 6])

    def internal_force(self):
        fx, fy = np.zeros(self.nn), np.zeros(self.nn)
        self._chk(lib().ocst_internal_force(self._h, _p(fx, _dp), _p(fy, _dp)))
        return fx, fy

    def set_fracture(self, gc=None, gc_uniform=3.0, gamma=1.0, gamma_mode=0):
        g = None if gc is None else np.ascontiguousarray(gc, np.float32)
        self._chk(lib().ocst_set_fracture(self._h, None if g is None else g.ctypes.data_as(
            C.POINTER(C.c_float)), gc_uniform, gamma, gamma_mode))

    def eval_surface(self, edge, elem):
        e = np.ascontiguousarray(edge, np.int32)
        el = np.ascontiguousarray(elem, np.int32)
        G = np.zeros(2 * len(e))
        ch = np.zeros(len(e), np.int32)
        self._chk(lib().ocst_eval_surface(self._h, len(e), _p(e, _ip), _p(el, _ip), _p(G, _dp),
                                          _p(ch, _ip)))
        return G.reshape(-1, 2), ch

    def strain_energy(self):
        se = np.zeros(1)
        self._chk(lib().ocst_strain_energy(self._h, _p(se, _dp)))
        return float(se[0])


def from_problem(prob):
    """Builds a CST oracle run from a ``TriProblem``."""
    s = CstOracle(prob.X, prob.conn)
    m = prob.material
    s.set_material(m.E, m.nu, m.rho, m.plane_strain)
    s.set_fracture(getattr(prob, "gc", None), m.gc_uniform, m.gamma, m.gamma_mode)
    if prob.dt is not None:
        s.set_dt(0.0, prob.dt)
    else:
        s.set_dt(prob.dt_factor, 0.0)
    for bc in prob.bcs:
        s.add_bc(bc.kind, bc.items, bc.comp_mask, bc.law, bc.a0, bc.t0, bc.tau)
    if prob.energy_every:
        s.set_energy_every(prob.energy_every)
    if prob.init is not None:
        s.set_state(*prob.init)
    return s
