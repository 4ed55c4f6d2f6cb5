"""Thin ctypes binding of libcem.so (include/cem.h), same names as the C ABI.

Only argument marshalling happens here: every step of the method runs in the
library's CUDA kernels.  PyTorch supplies device memory (through the
library's allocator callbacks) and the CUDA stream.  If libcem.so has not
been built, ``lib()`` raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import inputs as _inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libcem.so")

CEM_OK, CEM_ERR_ARG, CEM_ERR_CUDA, CEM_ERR_CAPACITY = 0, -1, -2, -3
CEM_ERR_NONFINITE, CEM_ERR_TIMEOUT, CEM_ERR_STATE = -4, -5, -6
CEM_FP64, CEM_FP32_MIXED = 0, 1
(CEM_FIELD_U, CEM_FIELD_V, CEM_FIELD_MASS, CEM_FIELD_STATE, CEM_FIELD_ENERGY, CEM_FIELD_GC,
 CEM_FIELD_SIGMA, CEM_FIELD_SIGMA1) = range(8)

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class cem_mesh_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("hx", C.c_double), ("hy", C.c_double),
                ("elem_active", C.POINTER(C.c_ubyte)), ("n_precracks", C.c_int),
                ("precrack", C.POINTER(C.c_int)), ("phantom_capacity", C.c_int),
                ("crack_capacity", C.c_int), ("list_capacity", C.c_int), ("precision", C.c_int),
                ("dt_factor", C.c_double), ("dt", C.c_double), ("energy_every", C.c_int),
                ("cuda_stream", C.c_void_p), ("device", C.c_int), ("alloc", _ALLOC_FN),
                ("free", _FREE_FN), ("alloc_ctx", C.c_void_p)]


class cem_tri_mesh_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("n_elems", C.c_int), ("X", C.POINTER(C.c_double)),
                ("conn", C.POINTER(C.c_int)), ("precision", C.c_int), ("dt_factor", C.c_double),
                ("dt", C.c_double),
                ("energy_every", C.c_int), ("cuda_stream", C.c_void_p), ("device", C.c_int),
                ("alloc", _ALLOC_FN), ("free", _FREE_FN), ("alloc_ctx", C.c_void_p)]


class cem_counts(C.Structure):
    _fields_ = [("n_nodes", C.c_long), ("n_phantoms", C.c_long), ("n_elems", C.c_long),
                ("n_active", C.c_long), ("n_cracked", C.c_long), ("n_surface", C.c_long),
                ("n_tips", C.c_long), ("n_energy", C.c_long), ("step", C.c_long),
                ("dt", C.c_double), ("t", C.c_double), ("kernel_launches", C.c_long),
                ("last_proposals", C.c_long), ("last_winners", C.c_long)]


class cem_tip(C.Structure):
    _fields_ = [("edge_id", C.c_int), ("ahead_elem", C.c_int), ("x", C.c_double),
                ("y", C.c_double), ("G_last", C.c_double), ("birth_step", C.c_int),
                ("parent", C.c_int)]


class cem_crack(C.Structure):
    _fields_ = [("elem", C.c_int), ("ka", C.c_int), ("kb", C.c_int), ("step", C.c_int),
                ("node", (C.c_int * 4) * 2), ("Ap", C.c_double * 2), ("ud", C.c_double)]


class cem_phantom(C.Structure):
    _fields_ = [("id", C.c_int), ("owner", C.c_int), ("creator_elem", C.c_int),
                ("creator_local", C.c_int), ("n_users", C.c_int), ("users", (C.c_int * 3) * 4)]


_LIB = None
_ip = C.POINTER(C.c_int)
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_h = C.c_void_p

# name -> (restype, argtypes); every entry point of include/cem.h
SIGNATURES = {
    "cem_mesh_create": (C.c_int, [C.POINTER(cem_mesh_desc), C.POINTER(C.c_void_p)]),
    "cem_tri_mesh_create": (C.c_int, [C.POINTER(cem_tri_mesh_desc), C.POINTER(C.c_void_p)]),
    "cem_tri_eval_surface": (C.c_int, [_h, C.c_int, _ip, _ip, _dp, _ip]),
    "cem_set_material": (C.c_int, [_h, C.c_double, C.c_double, C.c_double, _fp, C.c_double,
                                   C.c_int, C.c_double, C.c_int, C.c_int]),
    "cem_set_bc": (C.c_int, [_h, C.c_int, C.c_int, _ip, C.c_int, C.c_int, C.c_double,
                             C.c_double, C.c_double]),
    "cem_set_fields": (C.c_int, [_h, C.c_int, C.c_void_p, C.c_long, C.c_int]),
    "cem_step": (C.c_int, [_h, C.c_int]),
    "cem_step_async": (C.c_int, [_h, C.c_int]),
    "cem_sync": (C.c_int, [_h]),
    "cem_get_fields": (C.c_int, [_h, C.c_int, C.c_void_p, C.c_long, C.c_int]),
    "cem_get_counts": (C.c_int, [_h, C.POINTER(cem_counts)]),
    "cem_get_crack_tips": (C.c_int, [_h, C.POINTER(cem_tip), C.c_int, _ip]),
    "cem_get_cracks": (C.c_int, [_h, C.POINTER(cem_crack), C.c_int, _ip]),
    "cem_get_phantoms": (C.c_int, [_h, C.POINTER(cem_phantom), C.c_int, _ip]),
    "cem_get_surface": (C.c_int, [_h, _ip, _ip, _ip, C.c_int, _ip]),
    "cem_debug_apply_proposals": (C.c_int, [_h, C.c_int, _ip, _ip, _ip, _dp]),
    "cem_profile_steps": (C.c_int, [_h, C.c_int, _dp]),
    "cem_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_long),
                                   C.c_void_p, C.POINTER(C.c_void_p)]),
    "cem_batch_set_config": (C.c_int, [_h, C.c_int, C.c_int]),
    "cem_batch_autotune": (C.c_int, [_h, C.c_int, _ip, _ip]),
    "cem_state_energy_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_void_p,
                                           C.c_double, C.c_double, C.c_double, C.c_int,
                                           C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_char_p, C.c_int]),
    "cem_get_fragments": (C.c_int, [_h, _ip, _ip, C.c_long]),
    "cem_state_size": (C.c_int, [_h, C.POINTER(C.c_long)]),
    "cem_save_state": (C.c_int, [_h, C.c_void_p, C.c_long]),
    "cem_load_state": (C.c_int, [_h, C.c_void_p, C.c_long]),
    "cem_last_error": (C.c_char_p, [_h]),
    "cem_mesh_destroy": (None, [_h]),
}


def lib():
    """Loads libcem.so; raises if it has not been built (no fallback)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2509_01827_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class CemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"cem error {code}: {msg}")
        self.code = code


def _p(a, t):
    return None if a is None else a.ctypes.data_as(t)


# ---------------------------------------------------------------- raw names
def cem_mesh_create(desc: cem_mesh_desc) -> int:
    h = C.c_void_p()
    rc = lib().cem_mesh_create(C.byref(desc), C.byref(h))
    if rc != CEM_OK:
        raise CemError(rc, lib().cem_last_error(None).decode())
    return h.value


def cem_tri_mesh_create(desc: cem_tri_mesh_desc) -> int:
    h = C.c_void_p()
    rc = lib().cem_tri_mesh_create(C.byref(desc), C.byref(h))
    if rc != CEM_OK:
        raise CemError(rc, lib().cem_last_error(None).decode())
    return h.value


def cem_step_async(h, n):
    _chk(h, lib().cem_step_async(h, int(n)))


def cem_sync(h):
    _chk(h, lib().cem_sync(h))


def cem_last_error(h) -> str:
    return lib().cem_last_error(h).decode()


def _chk(h, rc):
    if rc != CEM_OK:
        raise CemError(rc, cem_last_error(h))


def cem_set_material(h, E, nu, rho, gc=None, gc_uniform=3.0, plane_strain=True, gamma=1.0,
                     gamma_mode=0, scope=0):
    g = None if gc is None else np.ascontiguousarray(gc, dtype=np.float32)
    _chk(h, lib().cem_set_material(h, E, nu, rho, _p(g, _fp), gc_uniform, int(bool(plane_strain)),
                                   gamma, gamma_mode, scope))


def cem_set_bc(h, kind, items, comp_mask=0, law=0, a0=0.0, t0=0.0, tau=0.0):
    it = np.ascontiguousarray(items, dtype=np.int32)
    _chk(h, lib().cem_set_bc(h, kind, len(it), _p(it, _ip), comp_mask, law, a0, t0, tau))


def cem_set_fields(h, which, data: np.ndarray):
    a = np.ascontiguousarray(data, dtype=np.float64)
    _chk(h, lib().cem_set_fields(h, which, a.ctypes.data, a.nbytes, 0))


def cem_step(h, n: int):
    _chk(h, lib().cem_step(h, int(n)))


def cem_get_counts(h) -> dict:
    c = cem_counts()
    _chk(h, lib().cem_get_counts(h, C.byref(c)))
    return {k: getattr(c, k) for k, _ in cem_counts._fields_}


def cem_get_fields(h, which, n_nodes_total=None, n_elems=None, n_energy=None):
    if which in (CEM_FIELD_U, CEM_FIELD_V):
        out = np.empty(2 * n_nodes_total)
    elif which == CEM_FIELD_MASS:
        out = np.empty(n_nodes_total)
    elif which == CEM_FIELD_STATE:
        out = np.empty(n_elems, np.uint8)
    elif which == CEM_FIELD_ENERGY:
        out = np.empty(7 * n_energy)
    elif which == CEM_FIELD_GC:
        out = np.empty(n_elems, np.float32)
    elif which == CEM_FIELD_SIGMA:
        out = np.empty(3 * n_elems)
    elif which == CEM_FIELD_SIGMA1:
        out = np.empty(n_elems)
    else:
        raise ValueError(which)
    _chk(h, lib().cem_get_fields(h, which, out.ctypes.data, out.nbytes, 0))
    return out


def cem_get_crack_tips(h, cap):
    arr = (cem_tip * max(cap, 1))()
    n = C.c_int()
    _chk(h, lib().cem_get_crack_tips(h, arr, cap, C.byref(n)))
    return [arr[q] for q in range(n.value)]


def cem_get_cracks(h, cap):
    arr = (cem_crack * max(cap, 1))()
    n = C.c_int()
    _chk(h, lib().cem_get_cracks(h, arr, cap, C.byref(n)))
    return [arr[q] for q in range(n.value)]


def cem_get_phantoms(h, cap):
    arr = (cem_phantom * max(cap, 1))()
    n = C.c_int()
    _chk(h, lib().cem_get_phantoms(h, arr, cap, C.byref(n)))
    return [arr[q] for q in range(n.value)]


def cem_get_surface(h, cap):
    e, a, t = (np.empty(max(cap, 1), np.int32) for _ in range(3))
    n = C.c_int()
    _chk(h, lib().cem_get_surface(h, _p(e, _ip), _p(a, _ip), _p(t, _ip), cap, C.byref(n)))
    n = n.value
    return e[:n], a[:n], t[:n].astype(bool)


def cem_debug_apply_proposals(h, edge, elem, k, G):
    e = np.ascontiguousarray(edge, np.int32)
    el = np.ascontiguousarray(elem, np.int32)
    kk = np.ascontiguousarray(k, np.int32)
    g = np.ascontiguousarray(G, np.float64)
    _chk(h, lib().cem_debug_apply_proposals(h, len(e), _p(e, _ip), _p(el, _ip), _p(kk, _ip),
                                            _p(g, _dp)))


def cem_profile_steps(h, n):
    ms = np.zeros(9)
    _chk(h, lib().cem_profile_steps(h, int(n), _p(ms, _dp)))
    keys = ["total", "pieces", "main", "phantom", "eval", "select", "energy", "kernels", "apply"]
    return dict(zip(keys, ms.tolist()))


def cem_batch_create(handles, step_end=None, stream_ptr=0) -> int:
    n = len(handles)
    arr = (C.c_void_p * n)(*handles)
    lim = None if step_end is None else (C.c_long * n)(*[int(x) for x in step_end])
    out = C.c_void_p()
    rc = lib().cem_batch_create(arr, n, lim, stream_ptr or None, C.byref(out))
    if rc != CEM_OK:
        raise CemError(rc, lib().cem_last_error(None).decode())
    return out.value


def cem_batch_set_config(b, tile_rows, grid_main):
    _chk(b, lib().cem_batch_set_config(b, int(tile_rows), int(grid_main)))


def cem_batch_autotune(b, steps_per_candidate):
    r, g = C.c_int(), C.c_int()
    _chk(b, lib().cem_batch_autotune(b, int(steps_per_candidate), C.byref(r), C.byref(g)))
    return r.value, g.value


def cem_state_energy_noalloc(nx, ny, hx, hy, elem_active_ptr, E, nu, rho, plane_strain,
                             u_ptr, v_ptr, out_ptr, stream_ptr=0):
    """Allocation-free energy check on device pointers (integers): enqueues
    KE and SE of one uncracked state into out_ptr (double[2]) on the stream.
    For callers that cannot allocate device memory; the library's scratch is a
    fixed device array, so calls that overlap on the GPU must be ordered."""
    err = C.create_string_buffer(256)
    rc = lib().cem_state_energy_noalloc(int(nx), int(ny), float(hx), float(hy),
                                        elem_active_ptr or None, float(E), float(nu), float(rho),
                                        int(bool(plane_strain)), u_ptr, v_ptr, out_ptr,
                                        stream_ptr or None, err, len(err))
    if rc != CEM_OK:
        raise CemError(rc, err.value.decode())


def cem_get_fragments(h, n_elems, labels=True):
    """(number of fragments, labels of the pieces 2 e + p or None)."""
    n = C.c_int()
    lab = np.empty(2 * n_elems, np.int32) if labels else None
    _chk(h, lib().cem_get_fragments(h, C.byref(n), _p(lab, _ip), 0 if lab is None else len(lab)))
    return n.value, lab


def cem_state_size(h) -> int:
    n = C.c_long()
    _chk(h, lib().cem_state_size(h, C.byref(n)))
    return n.value


def cem_save_state(h) -> bytes:
    """The run's state blob (include/cem.h: cem_save_state)."""
    n = cem_state_size(h)
    buf = (C.c_char * n)()
    _chk(h, lib().cem_save_state(h, buf, n))
    return bytes(buf)


def cem_load_state(h, blob: bytes):
    buf = C.create_string_buffer(blob, len(blob))
    _chk(h, lib().cem_load_state(h, buf, len(blob)))


def cem_mesh_destroy(h):
    if h:
        lib().cem_mesh_destroy(h)


# ---------------------------------------------------------------- allocator
class TorchDeviceMemory:
    """Device memory for libcem from PyTorch's caching allocator."""

    def __init__(self, device: int):
        import torch
        self._torch = torch
        self.device = torch.device("cuda", device)
        self.live = {}
        self.alloc_cb = _ALLOC_FN(self._alloc)
        self.free_cb = _FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


# ---------------------------------------------------------------- solver
class Solver:
    """One simulation of a ``paper_2509_01827_gb300.inputs.Problem`` on a GPU."""

    def __init__(self, prob: _inputs.Problem, precision: int = CEM_FP64, device: int = 0,
                 use_torch: bool = True, stream=None, phantom_cap: Optional[int] = None,
                 crack_cap: Optional[int] = None, energy_every: Optional[int] = None,
                 list_cap: int = 0):
        self.prob = prob
        self.h = None
        self._mem = None
        self._keep = []
        if use_torch:
            import torch
            self._mem = TorchDeviceMemory(device)
            if stream is None:
                stream = torch.cuda.Stream(device=device)
            self._stream = stream
            stream_ptr = stream.cuda_stream
        else:
            self._stream = None
            stream_ptr = 0 if stream is None else int(stream)
        act = None if prob.active is None else np.ascontiguousarray(prob.active, np.uint8)
        pre = np.ascontiguousarray(np.asarray(prob.precracks, np.int32).reshape(-1))
        self._keep += [act, pre]
        d = cem_mesh_desc()
        d.nx, d.ny, d.hx, d.hy = prob.nx, prob.ny, prob.hx, prob.hy
        d.elem_active = _p(act, C.POINTER(C.c_ubyte))
        d.n_precracks = len(pre) // 3
        d.precrack = pre.ctypes.data_as(_ip) if len(pre) else None
        d.phantom_capacity = phantom_cap if phantom_cap is not None else prob.phantom_cap
        d.crack_capacity = crack_cap if crack_cap is not None else prob.crack_cap
        d.list_capacity = list_cap
        d.precision = precision
        d.dt_factor = prob.dt_factor
        d.dt = prob.dt if prob.dt is not None else 0.0
        d.energy_every = prob.energy_every if energy_every is None else energy_every
        d.cuda_stream = stream_ptr
        d.device = device
        if self._mem is not None:
            d.alloc = self._mem.alloc_cb
            d.free = self._mem.free_cb
        else:
            d.alloc = _ALLOC_FN()
            d.free = _FREE_FN()
        self.h = cem_mesh_create(d)
        m = prob.material
        cem_set_material(self.h, m.E, m.nu, m.rho, prob.gc, m.gc_uniform, m.plane_strain,
                         m.gamma, m.gamma_mode, m.scope)
        for bc in prob.bcs:
            cem_set_bc(self.h, bc.kind, bc.items, bc.comp_mask, bc.law, bc.a0, bc.t0, bc.tau)

    def close(self):
        if self.h:
            cem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        cem_step(self.h, n)

    def step_async(self, n=1):
        """Enqueues n steps; raises the previous call's error, if any."""
        cem_step_async(self.h, n)

    def sync(self):
        cem_sync(self.h)

    def counts(self):
        return cem_get_counts(self.h)

    def n_total(self):
        c = self.counts()
        return c["n_nodes"] + c["n_phantoms"]

    def set_state(self, ux=None, uy=None, vx=None, vy=None):
        n = self.n_total()
        if ux is not None or uy is not None:
            u = np.zeros(2 * n)
            if ux is not None:
                u[:n] = ux
            if uy is not None:
                u[n:] = uy
            cem_set_fields(self.h, CEM_FIELD_U, u)
        if vx is not None or vy is not None:
            v = np.zeros(2 * n)
            if vx is not None:
                v[:n] = vx
            if vy is not None:
                v[n:] = vy
            cem_set_fields(self.h, CEM_FIELD_V, v)

    def nodes(self):
        n = self.n_total()
        u = cem_get_fields(self.h, CEM_FIELD_U, n)
        v = cem_get_fields(self.h, CEM_FIELD_V, n)
        m = cem_get_fields(self.h, CEM_FIELD_MASS, n)
        return dict(ux=u[:n], uy=u[n:], vx=v[:n], vy=v[n:], m=m)

    def state(self):
        return cem_get_fields(self.h, CEM_FIELD_STATE, n_elems=self.prob.nx * self.prob.ny)

    def element_stress(self):
        """Element mean stress, shape (ne, 3): sxx, syy, sxy."""
        ne = self.prob.nx * self.prob.ny
        return cem_get_fields(self.h, CEM_FIELD_SIGMA, n_elems=ne).reshape(3, ne).T.copy()

    def sigma1(self):
        """Largest principal value of the element mean stress, shape (ne,)."""
        return cem_get_fields(self.h, CEM_FIELD_SIGMA1, n_elems=self.prob.nx * self.prob.ny)

    def energy(self):
        n = self.counts()["n_energy"]
        rec = cem_get_fields(self.h, CEM_FIELD_ENERGY, n_energy=n).reshape(n, 7)
        return dict(step=rec[:, 0].astype(np.int64), t=rec[:, 1], KE=rec[:, 2], SE=rec[:, 3],
                    W_ext=rec[:, 4], W_dir=rec[:, 5], U_d=rec[:, 6])

    def cracks(self):
        cr = cem_get_cracks(self.h, self.counts()["n_cracked"])
        n = len(cr)
        out = dict(elem=np.array([c.elem for c in cr], np.int32),
                   ka=np.array([c.ka for c in cr], np.int32),
                   kb=np.array([c.kb for c in cr], np.int32),
                   step=np.array([c.step for c in cr], np.int32),
                   ud=np.array([c.ud for c in cr]),
                   Ap=np.array([[c.Ap[0], c.Ap[1]] for c in cr]).reshape(n, 2),
                   nodes=np.array([[list(c.node[0]), list(c.node[1])] for c in cr],
                                  np.int32).reshape(n, 2, 4))
        return out

    def phantoms(self):
        ph = cem_get_phantoms(self.h, self.counts()["n_phantoms"])
        n = len(ph)
        return dict(id=np.array([p.id for p in ph], np.int32),
                    owner=np.array([p.owner for p in ph], np.int32),
                    creator_e=np.array([p.creator_elem for p in ph], np.int32),
                    creator_a=np.array([p.creator_local for p in ph], np.int32),
                    nuser=np.array([p.n_users for p in ph], np.int32),
                    users=np.array([[list(u) for u in p.users] for p in ph],
                                   np.int32).reshape(n, 4, 3))

    def surface(self):
        e, a, t = cem_get_surface(self.h, self.counts()["n_surface"])
        return dict(edge=e, ahead=a, is_tip=t)

    def tips(self):
        return cem_get_crack_tips(self.h, self.counts()["n_tips"])

    def profile_steps(self, n):
        return cem_profile_steps(self.h, n)

    def fragments(self, labels=True):
        """(number of fragments, piece labels of shape (ne, 2) or None)."""
        n, lab = cem_get_fragments(self.h, self.prob.nx * self.prob.ny, labels)
        return n, None if lab is None else lab.reshape(-1, 2)

    def save_state(self) -> bytes:
        return cem_save_state(self.h)

    def load_state(self, blob: bytes):
        cem_load_state(self.h, blob)

    def debug_apply_proposals(self, edge, elem, k, G):
        cem_debug_apply_proposals(self.h, edge, elem, k, G)


# ---------------------------------------------------------------- batch
class Batch:
    """Many ``Solver`` members stepped in lock-step by one launch per kernel
    kind (cem_batch_create).  Each member stops at its own step limit."""

    def __init__(self, members, step_end=None, stream=None):
        import torch
        self.members = list(members)  # kept alive: their allocators serve the batch
        dev = self.members[0]._stream.device if self.members[0]._stream is not None else None
        self._stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.h = cem_batch_create([m.h for m in self.members], step_end,
                                  self._stream.cuda_stream)

    def close(self):
        if self.h:
            cem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        cem_step(self.h, n)

    def counts(self):
        return cem_get_counts(self.h)

    def set_config(self, tile_rows, grid_main):
        cem_batch_set_config(self.h, tile_rows, grid_main)

    def autotune(self, steps_per_candidate=5):
        return cem_batch_autotune(self.h, steps_per_candidate)


class TriSolver:
    """One run of a ``paper_2509_01827_gb300.inputs.TriProblem`` (an
    unstructured mesh of constant-strain triangles) on a GPU, FP64 or
    FP32-mixed."""

    def __init__(self, prob: _inputs.TriProblem, precision: int = CEM_FP64, device: int = 0,
                 use_torch: bool = True, stream=None, energy_every: Optional[int] = None):
        self.prob = prob
        self.h = None
        self._mem = None
        if use_torch:
            import torch
            self._mem = TorchDeviceMemory(device)
            if stream is None:
                stream = torch.cuda.Stream(device=device)
            self._stream = stream
            stream_ptr = stream.cuda_stream
        else:
            self._stream = None
            stream_ptr = 0 if stream is None else int(stream)
        X = np.ascontiguousarray(prob.X, np.float64).reshape(-1)
        conn = np.ascontiguousarray(prob.conn, np.int32).reshape(-1)
        self._keep = [X, conn]
        d = cem_tri_mesh_desc()
        d.n_nodes, d.n_elems = len(X) // 2, len(conn) // 3
        d.X = X.ctypes.data_as(_dp)
        d.conn = conn.ctypes.data_as(_ip)
        d.precision = precision
        d.dt_factor = prob.dt_factor
        d.dt = prob.dt if prob.dt is not None else 0.0
        d.energy_every = prob.energy_every if energy_every is None else energy_every
        d.cuda_stream = stream_ptr
        d.device = device
        if self._mem is not None:
            d.alloc = self._mem.alloc_cb
            d.free = self._mem.free_cb
        else:
            d.alloc = _ALLOC_FN()
            d.free = _FREE_FN()
        self.h = cem_tri_mesh_create(d)
        m = prob.material
        cem_set_material(self.h, m.E, m.nu, m.rho, getattr(prob, "gc", None), m.gc_uniform,
                         m.plane_strain, m.gamma, m.gamma_mode, m.scope)
        for bc in prob.bcs:
            cem_set_bc(self.h, bc.kind, bc.items, bc.comp_mask, bc.law, bc.a0, bc.t0, bc.tau)
        if prob.init is not None:
            self.set_state(*prob.init)

    def close(self):
        if self.h:
            cem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        cem_step(self.h, n)

    def counts(self):
        return cem_get_counts(self.h)

    def set_state(self, ux=None, uy=None, vx=None, vy=None):
        n = self.prob.n_nodes
        for which, (a, b) in ((CEM_FIELD_U, (ux, uy)), (CEM_FIELD_V, (vx, vy))):
            if a is not None or b is not None:
                f = np.zeros(2 * n)
                if a is not None:
                    f[:n] = a
                if b is not None:
                    f[n:] = b
                cem_set_fields(self.h, which, f)

    def nodes(self):
        n = self.prob.n_nodes
        u = cem_get_fields(self.h, CEM_FIELD_U, n)
        v = cem_get_fields(self.h, CEM_FIELD_V, n)
        m = cem_get_fields(self.h, CEM_FIELD_MASS, n)
        return dict(ux=u[:n], uy=u[n:], vx=v[:n], vy=v[n:], m=m)

    def energy(self):
        n = self.counts()["n_energy"]
        rec = cem_get_fields(self.h, CEM_FIELD_ENERGY, n_energy=n).reshape(n, 7)
        return dict(step=rec[:, 0].astype(np.int64), t=rec[:, 1], KE=rec[:, 2], SE=rec[:, 3],
                    W_ext=rec[:, 4], W_dir=rec[:, 5], U_d=rec[:, 6])

    def eval_surface(self, edge, elem):
        """G of the two candidate paths and the chosen local edge (-1: none)
        at surface points (edge[q] of element elem[q])."""
        e = np.ascontiguousarray(edge, np.int32)
        el = np.ascontiguousarray(elem, np.int32)
        G = np.zeros(2 * len(e))
        ch = np.zeros(len(e), np.int32)
        _chk(self.h, lib().cem_tri_eval_surface(self.h, len(e), _p(e, _ip), _p(el, _ip),
                                                _p(G, _dp), _p(ch, _ip)))
        return G.reshape(-1, 2), ch
