"""Thin Python binding of libgx.so (include/gx.h): the GB300 GL-ECSIM hot path.

Every function here only marshals arguments into the C ABI; all arithmetic
runs in the library's CUDA kernels.  There is no CPU fallback: if libgx.so is
missing or cannot be loaded, ``lib()`` raises.

Arrays may be numpy arrays (host memory, ``ptr_is_device = 0``) or CUDA torch
tensors (device memory of the context's GPU, ``ptr_is_device = 1``); the
library copies in and out during each call and keeps no pointer.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgx.so")
_lock = threading.Lock()
_lib = None

GX_OK, GX_EINVAL, GX_ENOMEM, GX_ECUDA, GX_ENOCONV, GX_ECFL, GX_ETIMEOUT, GX_ENOTIMPL, GX_EOVERFLOW, GX_ESTATE = range(10)
GX_PRECOND_NONE, GX_PRECOND_JACOBI, GX_PRECOND_NET = 0, 1, 2


class Config(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 3),
        ("comoving", C.c_int32),
        ("lf_on", C.c_int32),
        ("lf_speed_c", C.c_int32),
        ("ns_j", C.c_int32),
        ("nsmooth_u", C.c_int32),
        ("gmres_restart", C.c_int32),
        ("gmres_maxit", C.c_int32),
        ("precond", C.c_int32),
        ("track_ids", C.c_int32),
        ("dx", C.c_double * 3),
        ("c", C.c_double),
        ("theta", C.c_double),
        ("dt", C.c_double),
        ("lf_beta", C.c_double),
        ("gmres_tol", C.c_double),
        ("bin_slack", C.c_double),
        ("divb_clean", C.c_int32),
        ("nsmooth_e", C.c_int32),
        ("bc_cells", C.c_int32),
        ("bc_wall", C.c_int32),
        ("seed", C.c_uint64),
        ("lf_rhs_printed", C.c_int32),
        ("gl_gamma", C.c_double),
        ("gmres_mixed", C.c_int32),
    ]


class SolveStats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("relres", C.c_double), ("ms", C.c_double)]


class Diag(C.Structure):
    _fields_ = [
        ("energy_E", C.c_double),
        ("energy_B", C.c_double),
        ("kinetic", C.c_double),
        ("momentum", C.c_double * 3),
        ("charge", C.c_double),
        ("gauss_l2", C.c_double),
        ("divB_l2", C.c_double),
        ("n_particles", C.c_int64),
    ]


_V = C.c_void_p
_CTX = C.c_void_p
_SIGS = {
    "gx_create": (C.c_int, [C.POINTER(Config), C.POINTER(_CTX)]),
    "gx_destroy": (None, [_CTX]),
    "gx_status_string": (C.c_char_p, [C.c_int]),
    "gx_last_error": (C.c_char_p, [_CTX]),
    "gx_species_add": (C.c_int, [_CTX, C.c_double, C.c_double, C.c_int64, _V, _V, _V, _V, _V, _V, _V, C.c_int,
                                 C.POINTER(C.c_int)]),
    "gx_fields_set": (C.c_int, [_CTX, _V, _V, C.c_int]),
    "gx_boundary_source": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double), C.c_double, C.c_int]),
    "gx_species_maxwellian": (C.c_int, [_CTX, C.c_double, C.c_double, C.c_int, C.c_double, C.POINTER(C.c_double),
                                        C.c_double, C.POINTER(C.c_int)]),
    "gx_deposit": (C.c_int, [_CTX, _V]),
    "gx_field_solve": (C.c_int, [_CTX, _V, C.POINTER(SolveStats)]),
    "gx_push_and_deposit": (C.c_int, [_CTX, _V]),
    "gx_step": (C.c_int, [_CTX, C.c_int, _V, C.POINTER(SolveStats)]),
    "gx_get_fields": (C.c_int, [_CTX, _V, _V, C.c_int]),
    "gx_get_solution": (C.c_int, [_CTX, _V, C.c_int]),
    "gx_get_moments": (C.c_int, [_CTX, _V, _V, _V, _V, C.c_int]),
    "gx_species_count": (C.c_int64, [_CTX, C.c_int]),
    "gx_get_particles": (C.c_int, [_CTX, C.c_int, _V, _V, _V, _V, _V, _V, _V, _V, C.c_int]),
    "gx_diagnostics": (C.c_int, [_CTX, _V, C.POINTER(Diag)]),
    "gx_timers": (C.c_int, [_CTX, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                            C.POINTER(C.c_int64), C.c_int]),
    "gx_kernel_timer": (C.c_int, [_CTX, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int]),
    "gx_precond_param_count": (C.c_int64, []),
    "gx_precond_set_weights": (C.c_int, [_CTX, _V, C.c_int64, C.c_int]),
    "gx_precond_get_weights": (C.c_int, [_CTX, _V, C.c_int64, C.c_int]),
    "gx_precond_collect": (C.c_int, [_CTX, C.c_int]),
    "gx_precond_pairs": (C.c_int, [_CTX]),
    "gx_precond_collect_crops": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_int, C.c_uint64]),
    "gx_precond_crop": (C.c_int, [_CTX, C.c_int, _V, _V]),
    "gx_precond_train": (C.c_int, [_CTX, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_uint64, _V, _V]),
    "gx_precond_forward": (C.c_int, [_CTX, C.c_int, C.c_int, _V, _V, _V]),
    "gx_precond_loss_grad": (C.c_int, [_CTX, C.c_int, C.c_int, _V, _V, _V, _V, _V]),
    "gx_precond_apply": (C.c_int, [_CTX, _V, _V, _V]),
    "gx_noalloc_max_cells": (C.c_int, []),
    "gx_get_particles_noalloc": (C.c_int, [_CTX, C.c_int, _V, _V, _V, _V, _V, _V, _V, _V, _V]),
}
EXPORTED = tuple(_SIGS)


def lib():
    """Load libgx.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libgx.so not found at {LIB_PATH}; run paper_2506_11320_gb300/build.py")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class GxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{lib().gx_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _ptr(a):
    """(pointer, is_device) of a numpy array or a torch tensor; None -> (None, 0)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(type(a))


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_config(n, dx, *, c=1.0, theta=0.5, dt=0.02, comoving=1, lf_on=1, lf_speed_c=0, lf_beta=1.0, ns_j=0,
                nsmooth_u=5, gmres_tol=1e-8, gmres_restart=50, gmres_maxit=2000, precond=GX_PRECOND_NONE,
                track_ids=0, bin_slack=1.6, divb_clean=0, nsmooth_e=0, bc_cells=0,
                bc_wall=0, seed=0, lf_rhs_printed=0, gl_gamma=0.0, gmres_mixed=0) -> Config:
    n = list(n) + [1] * (3 - len(n))
    dx = list(dx) + [1.0] * (3 - len(dx))
    cfg = Config()
    for d in range(3):
        cfg.n[d] = int(n[d])
        cfg.dx[d] = float(dx[d])
    cfg.c, cfg.theta, cfg.dt = float(c), float(theta), float(dt)
    cfg.comoving, cfg.lf_on, cfg.lf_speed_c, cfg.lf_beta = int(comoving), int(lf_on), int(lf_speed_c), float(lf_beta)
    cfg.ns_j, cfg.nsmooth_u = int(ns_j), int(nsmooth_u)
    cfg.gmres_tol, cfg.gmres_restart, cfg.gmres_maxit = float(gmres_tol), int(gmres_restart), int(gmres_maxit)
    cfg.precond, cfg.track_ids, cfg.bin_slack = int(precond), int(track_ids), float(bin_slack)
    cfg.divb_clean = int(divb_clean)
    cfg.nsmooth_e = int(nsmooth_e)
    cfg.bc_cells = int(bc_cells)
    cfg.bc_wall = int(bc_wall)
    cfg.seed = int(seed)
    cfg.lf_rhs_printed = int(lf_rhs_printed)
    cfg.gl_gamma = float(gl_gamma)
    cfg.gmres_mixed = int(gmres_mixed)
    return cfg


class Context:
    """Owns one gx_ctx.  Method names follow the C entry points."""

    def __init__(self, cfg: Config):
        L = lib()
        h = _CTX()
        rc = L.gx_create(C.byref(cfg), C.byref(h))
        if rc != GX_OK:
            raise GxError(rc, L.gx_last_error(None).decode())
        self.h = h
        self.cfg = cfg
        self.shape = (cfg.n[2], cfg.n[1], cfg.n[0])
        self.N = cfg.n[0] * cfg.n[1] * cfg.n[2]

    def close(self):
        if getattr(self, "h", None):
            lib().gx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != GX_OK and rc not in allow:
            raise GxError(rc, lib().gx_last_error(self.h).decode())
        return rc

    def species_add(self, q, m, x, y, z, vx, vy, vz, w):
        n = len(x)
        ptrs = [_ptr(a) for a in (x, y, z, vx, vy, vz, w)]
        dev = max(p[1] for p in ptrs)
        sid = C.c_int(-1)
        self._check(lib().gx_species_add(self.h, float(q), float(m), n, *[p[0] for p in ptrs], dev, C.byref(sid)))
        return sid.value

    def fields_set(self, E, B):
        (pe, de), (pb, db) = _ptr(E), _ptr(B)
        self._check(lib().gx_fields_set(self.h, pe, pb, max(de, db)))

    def species_maxwellian(self, q, m, ppc, n0, u, vth):
        """Add a drifting Maxwellian species drawn on the device; returns its index."""
        uu = (C.c_double * 3)(*[float(v) for v in u])
        sid = C.c_int(-1)
        self._check(lib().gx_species_maxwellian(self.h, float(q), float(m), int(ppc), float(n0), uu, float(vth),
                                                C.byref(sid)))
        return sid.value

    def boundary_source(self, side, species, n, u, vth, ppc):
        """Plasma state of open boundary `side` (0: low x, 1: high x) for a species."""
        uu = (C.c_double * 3)(*[float(v) for v in u])
        self._check(lib().gx_boundary_source(self.h, int(side), int(species), float(n), uu, float(vth), int(ppc)))

    def deposit(self, stream=None):
        self._check(lib().gx_deposit(self.h, _stream(stream)))

    def field_solve(self, stream=None, allow_noconv=False):
        st = SolveStats()
        rc = lib().gx_field_solve(self.h, _stream(stream), C.byref(st))
        self._check(rc, allow=(GX_ENOCONV,) if allow_noconv else ())
        return st

    def push_and_deposit(self, stream=None):
        self._check(lib().gx_push_and_deposit(self.h, _stream(stream)))

    def step(self, nsteps=1, stream=None, allow_noconv=False):
        st = SolveStats()
        rc = lib().gx_step(self.h, int(nsteps), _stream(stream), C.byref(st))
        self._check(rc, allow=(GX_ENOCONV,) if allow_noconv else ())
        return st

    def get_fields(self, E=None, B=None):
        if E is None and B is None:
            E = np.zeros((3,) + self.shape)
            B = np.zeros((3,) + self.shape)
        (pe, de), (pb, db) = _ptr(E), _ptr(B)
        self._check(lib().gx_get_fields(self.h, pe, pb, max(de, db)))
        return E, B

    def get_solution(self, out=None):
        out = np.zeros((3,) + self.shape) if out is None else out
        p, d = _ptr(out)
        self._check(lib().gx_get_solution(self.h, p, d))
        return out

    def get_moments(self):
        rho = np.zeros(self.shape)
        J = np.zeros((3,) + self.shape)
        M = np.zeros(self.shape + (27, 3, 3))
        u = np.zeros((3,) + self.shape)
        self._check(lib().gx_get_moments(self.h, rho.ctypes.data, J.ctypes.data, M.ctypes.data, u.ctypes.data, 0))
        return rho, J, M, u

    def species_count(self, s):
        return int(lib().gx_species_count(self.h, s))

    def get_particles(self, s, ids=False):
        n = self.species_count(s)
        x, y, z = np.zeros(n), np.zeros(n), np.zeros(n)
        vx, vy, vz, w = (np.zeros(n, np.float32) for _ in range(4))
        idv = np.zeros(n, np.int32) if ids else None
        self._check(lib().gx_get_particles(self.h, s, x.ctypes.data, y.ctypes.data, z.ctypes.data, vx.ctypes.data,
                                           vy.ctypes.data, vz.ctypes.data, w.ctypes.data,
                                           idv.ctypes.data if ids else None, 0))
        out = dict(x=x, y=y, z=z, vx=vx, vy=vy, vz=vz, w=w)
        if ids:
            out["id"] = idv
        return out

    def get_particles_noalloc(self, s, out, stream=None):
        """Gather species s into preallocated CUDA tensors (dict with keys x, y,
        z, vx, vy, vz, w and optionally id); allocates no device memory and does
        not synchronise."""
        ptr = [out[k].data_ptr() if out.get(k) is not None else None
               for k in ("x", "y", "z", "vx", "vy", "vz", "w", "id")]
        self._check(lib().gx_get_particles_noalloc(self.h, int(s), *ptr, _stream(stream)))
        return out

    def diagnostics(self, stream=None):
        d = Diag()
        self._check(lib().gx_diagnostics(self.h, _stream(stream), C.byref(d)))
        return {"energy_E": d.energy_E, "energy_B": d.energy_B, "kinetic": d.kinetic,
                "momentum": list(d.momentum), "charge": d.charge, "gauss_l2": d.gauss_l2, "divB_l2": d.divB_l2,
                "n_particles": d.n_particles, "total": d.energy_E + d.energy_B + d.kinetic}

    def timers(self, reset=False):
        a, b, s, L = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
        self._check(lib().gx_timers(self.h, C.byref(a), C.byref(b), C.byref(s), C.byref(L), int(reset)))
        return {"push_ms": a.value, "moments_ms": b.value, "solve_ms": s.value, "launches": L.value}

    def kernel_timer(self, reset=False):
        ms, n = C.c_double(), C.c_int64()
        self._check(lib().gx_kernel_timer(self.h, C.byref(ms), C.byref(n), int(reset)))
        return {"pd_kernel_ms": ms.value, "pd_launches": n.value}

    # ------------------------------------------- learned preconditioner
    @staticmethod
    def precond_param_count():
        return int(lib().gx_precond_param_count())

    def precond_set_weights(self, params):
        p, d = _ptr(params)
        self._check(lib().gx_precond_set_weights(self.h, p, len(params), d))

    def precond_get_weights(self):
        out = np.zeros(self.precond_param_count(), np.float32)
        self._check(lib().gx_precond_get_weights(self.h, out.ctypes.data, len(out), 0))
        return out

    def precond_collect(self, capacity):
        self._check(lib().gx_precond_collect(self.h, int(capacity)))

    def precond_pairs(self):
        return int(lib().gx_precond_pairs(self.h))

    def precond_collect_crops(self, capacity, crop, per_pair, seed=0):
        self._check(lib().gx_precond_collect_crops(self.h, int(capacity), int(crop), int(per_pair), int(seed)))

    def precond_crop(self, k, crop):
        S = crop + 8
        out = np.empty((2, 3, S, S), np.float32)
        sc = np.empty(1, np.float32)
        self._check(lib().gx_precond_crop(self.h, int(k), out.ctypes.data, sc.ctypes.data))
        return out, float(sc[0])

    def precond_train(self, npairs, crop, batch, epochs, lr, seed=0, stream=None):
        losses = np.zeros(epochs, np.float32)
        self._check(lib().gx_precond_train(self.h, int(npairs), int(crop), int(batch), int(epochs), float(lr),
                                           int(seed), losses.ctypes.data, _stream(stream)))
        return losses

    def precond_forward(self, x, out, stream=None):
        """x, out: CUDA float32 tensors of shape (3, H, W); out = N(x), periodic padding."""
        _, H, W = x.shape
        self._check(lib().gx_precond_forward(self.h, H, W, x.data_ptr(), out.data_ptr(), _stream(stream)))
        return out

    def precond_apply(self, v, z, stream=None):
        """v, z: CUDA float64 tensors of 3 N entries; z = the solver's preconditioner applied to v."""
        self._check(lib().gx_precond_apply(self.h, v.data_ptr(), z.data_ptr(), _stream(stream)))
        return z

    def precond_loss_grad(self, x, target, grad, stream=None):
        """Loss and parameter gradient of one (3, H, W) sample, zero padding; grad: CUDA float32."""
        _, H, W = x.shape
        L = C.c_float()
        self._check(lib().gx_precond_loss_grad(self.h, H, W, x.data_ptr(), target.data_ptr(), C.byref(L),
                                               grad.data_ptr(), _stream(stream)))
        return L.value

def from_workload(wl, *, track_ids=0, precond=GX_PRECOND_NONE, gmres_tol=None, bin_slack=1.6, gmres_restart=50,
                  divb_clean=0, gmres_mixed=0):
    """Create a context from a workloads.Workload (inputs copied from host); a
    workload with open boundaries (notes["bc"]) also gets its boundary sources."""
    cfg = make_config(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, comoving=wl.comoving, lf_on=wl.lf_on,
                      lf_speed_c=wl.lf_speed_c, lf_beta=wl.lf_beta, ns_j=wl.ns_j, nsmooth_u=wl.nsmooth_u,
                      gmres_tol=wl.gmres_tol if gmres_tol is None else gmres_tol, precond=precond,
                      track_ids=track_ids, bin_slack=bin_slack, gmres_restart=gmres_restart,
                      divb_clean=divb_clean, gmres_mixed=gmres_mixed)
    bc = wl.notes.get("bc") if isinstance(wl.notes, dict) else None
    if bc:
        cfg.bc_cells, cfg.seed, cfg.bc_wall = int(bc["cells"]), int(bc["seed"]), int(bc.get("wall", 0))
    ctx = Context(cfg)
    for s in wl.species:
        ctx.species_add(s["q"], s["m"], np.ascontiguousarray(s["x"], np.float64),
                        np.ascontiguousarray(s["y"], np.float64), np.ascontiguousarray(s["z"], np.float64),
                        np.ascontiguousarray(s["vx"], np.float32), np.ascontiguousarray(s["vy"], np.float32),
                        np.ascontiguousarray(s["vz"], np.float32), np.ascontiguousarray(s["w"], np.float32))
    ctx.fields_set(np.ascontiguousarray(wl.E0, np.float64), np.ascontiguousarray(wl.B0, np.float64))
    if bc:
        for side in range(1 if bc.get("wall", 0) else 2):
            for s, src in enumerate(bc["sources"][side]):
                ctx.boundary_source(side, s, src["n"], src["u"], src["vth"], src["ppc"])
    return ctx
