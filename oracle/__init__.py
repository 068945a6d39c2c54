"""FP64 CPU oracle of the GL-ECSIM hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm import this package.  The CUDA library never calls it and the two
share no code.  The arithmetic lives in ``gx_oracle.c`` (plain C, FP64); this
module compiles it with gcc on first use and wraps it with ctypes.

Field arrays are numpy float64 of shape ``(3, nz, ny, nx)`` (vector) or
``(nz, ny, nx)`` (scalar); E lives at nodes, B at cell centres, and node (i,j,k)
and cell (i,j,k) share the flat index ``i + nx (j + ny k)``.  The mass matrix is
``(nz, ny, nx, 27, 3, 3)``: block ``[g, o]`` couples node g to its neighbour at
offset ``o = (ox+1) + 3 (oy+1) + 9 (oz+1)``.

Parity status: every routine is pinned by ``tests/test_oracle_*.py`` except the
learned-preconditioner network's *training usefulness* (its forward pass and
gradients are pinned; what it learns is not a paper quantity).  The open-boundary
refill (``refill_boundaries``) is pinned by its generator (word for word against
numpy's Philox), the statistics of its draws and the particle counts it leaves;
the shock states themselves are the paper's printed numbers.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gx_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libgx_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gx_oracle.c into libgx_oracle.so (plain gcc, no arch flags)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Cfg(C.Structure):
    _fields_ = [
        ("n", C.c_int32 * 3),
        ("comoving", C.c_int32),
        ("lf_on", C.c_int32),
        ("lf_speed_c", C.c_int32),
        ("ns_j", C.c_int32),
        ("nsmooth_u", C.c_int32),
        ("gmres_restart", C.c_int32),
        ("gmres_maxit", C.c_int32),
        ("divb_clean", C.c_int32),
        ("nsmooth_e", C.c_int32),
        ("dx", C.c_double * 3),
        ("c", C.c_double),
        ("theta", C.c_double),
        ("dt", C.c_double),
        ("lf_beta", C.c_double),
        ("gmres_tol", C.c_double),
        ("bc_cells", C.c_int32),
        ("bc_wall", C.c_int32),
        ("lf_rhs_printed", C.c_int32),
        ("gl_gamma", C.c_double),
    ]

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def nn(self):
        return self.n[0] * self.n[1] * self.n[2]


def make_cfg(n, dx, *, c=1.0, theta=0.5, dt=0.02, comoving=0, lf_on=0, lf_speed_c=0, lf_beta=1.0,
             ns_j=0, nsmooth_u=5, gmres_tol=1e-12, gmres_restart=50, gmres_maxit=5000, divb_clean=0,
             nsmooth_e=0, bc_cells=0, bc_wall=0, lf_rhs_printed=0, gl_gamma=0.0) -> Cfg:
    n = list(n) + [1] * (3 - len(n))
    dx = list(dx) + [1.0] * (3 - len(dx))
    cfg = Cfg()
    for d in range(3):
        cfg.n[d] = int(n[d])
        cfg.dx[d] = float(dx[d])
    cfg.c, cfg.theta, cfg.dt = float(c), float(theta), float(dt)
    cfg.comoving, cfg.lf_on, cfg.lf_speed_c = int(comoving), int(lf_on), int(lf_speed_c)
    cfg.lf_beta, cfg.ns_j, cfg.nsmooth_u = float(lf_beta), int(ns_j), int(nsmooth_u)
    cfg.gmres_tol, cfg.gmres_restart, cfg.gmres_maxit = float(gmres_tol), int(gmres_restart), int(gmres_maxit)
    cfg.divb_clean = int(divb_clean)
    cfg.nsmooth_e = int(nsmooth_e)
    cfg.bc_cells = int(bc_cells)
    cfg.bc_wall = int(bc_wall)
    cfg.lf_rhs_printed = int(lf_rhs_printed)
    cfg.gl_gamma = float(gl_gamma)
    if cfg.bc_cells and cfg.gl_gamma > 0:
        raise ValueError("the Gauss's-law correction runs on periodic grids only")
    if cfg.bc_cells and (cfg.divb_clean or 2 * cfg.bc_cells >= cfg.n[0]):
        raise ValueError("open boundaries: no divergence cleaning, and 2 bc_cells < nx")
    if cfg.bc_wall and not cfg.bc_cells:
        raise ValueError("a reflecting wall needs bc_cells > 0")
    if cfg.bc_cells and cfg.nsmooth_e:
        raise ValueError("open boundaries without nsmooth_e (the filter would move the held boundary E)")
    return cfg


_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_P = C.POINTER(Cfg)

_SIGS = {
    "or_alpha": (None, [_D, _D]),
    "or_node_avg": (None, [_P, _D, _D]),
    "or_filter": (None, [_P, _D, C.c_int, C.c_int, C.c_double]),
    "or_lf_b_increment": (None, [_P, _D, _D, _D]),
    "or_philox4x64": (None, [C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "or_bc_sample": (None, [_P, C.c_uint64, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int, _D, C.c_double,
                            _D, _D, _D, _D, _D]),
    "or_bulk_moments": (None, [_P, _D, _D, C.c_int64, _I32, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
    "or_bulk_velocity": (None, [_P, _D, _D, _D]),
    "or_deposit": (None, [_P, _D, _D, C.c_int64, _I32, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
    "or_smooth_current": (None, [_P, _D, C.c_int]),
    "or_curl_C": (None, [_P, _D, _D]),
    "or_curl_N": (None, [_P, _D, _D]),
    "or_div_C": (None, [_P, _D, _D]),
    "or_div_N": (None, [_P, _D, _D]),
    "or_grad_N": (None, [_P, _D, _D]),
    "or_grad_C": (None, [_P, _D, _D]),
    "or_mc_limiter": (C.c_double, [C.c_double, C.c_double]),
    "or_lf_kappa_E": (None, [_P, _D, _D, _D]),
    "or_gl_displacement": (None, [_P, _D, C.c_int64, _I32, _D, _D, _D, _D, _D, C.c_double, _D, _D, _D, _D]),
    "or_cell_sample3": (None, [_P, C.c_uint64, C.c_int, C.c_int64, C.c_int, C.c_int, C.c_int, C.c_int, _D,
                               C.c_double, _D, _D, _D, _D, _D, _D]),
    "or_apply_A": (None, [_P, _D, _D, _D, _D]),
    "or_rhs": (None, [_P, _D, _D, _D, _D, _D, _D, _D]),
    "or_gmres": (C.c_int, [_P, _D, _D, _D, _D, _D, C.POINTER(C.c_int)]),
    "or_dense_solve": (C.c_int, [_P, _D, _D, _D, _D]),
    "or_advance_fields": (None, [_P, _D, _D, _D, _D, _D, _D]),
    "or_mover": (C.c_double, [_P, _D, _D, C.c_int64, _I32, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
    "or_energy": (None, [_P, _D, C.c_int64, _I32, _D, _D, _D, _D, _D, _D, _D]),
    "or_step": (C.c_int, [_P, _D, _D, C.c_int64, _I32, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D,
                          _D, _D, _D, _D, _D, _D]),
    "or_divb_clean": (None, [_P, _D, _D]),
    "or_net_param_count": (C.c_int64, []),
    "or_net_act_count": (C.c_int64, [C.c_int, C.c_int]),
    "or_net_forward": (None, [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D]),
    "or_net_loss_backward": (C.c_double, [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D, _D]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous, (a.dtype, a.flags)
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Plasma:
    """Particles of all species in one set of FP64 arrays (``sp`` = species id)."""

    def __init__(self, q, m, sp, x, y, z, vx, vy, vz, w):
        self.q = _f64(q)
        self.m = _f64(m)
        self.sp = np.ascontiguousarray(sp, dtype=np.int32)
        self.x, self.y, self.z = _f64(x), _f64(y), _f64(z)
        self.vx, self.vy, self.vz, self.w = _f64(vx), _f64(vy), _f64(vz), _f64(w)

    @property
    def np(self):
        return self.x.size

    def copy(self):
        return Plasma(self.q, self.m, self.sp, self.x.copy(), self.y.copy(), self.z.copy(),
                      self.vx.copy(), self.vy.copy(), self.vz.copy(), self.w.copy())

    @staticmethod
    def from_species(species):
        """species: list of dicts with q, m, x, y, z, vx, vy, vz, w (any float dtype)."""
        q = [s["q"] for s in species]
        m = [s["m"] for s in species]
        sp = np.concatenate([np.full(len(s["x"]), i, np.int32) for i, s in enumerate(species)])
        cat = lambda k: np.concatenate([np.asarray(s[k], np.float64) for s in species])
        return Plasma(q, m, sp, cat("x"), cat("y"), cat("z"), cat("vx"), cat("vy"), cat("vz"), cat("w"))

    def args(self):
        return (_d(self.q), _d(self.m), C.c_int64(self.np), self.sp.ctypes.data_as(_I32),
                _d(self.x), _d(self.y), _d(self.z), _d(self.vx), _d(self.vy), _d(self.vz))


def vec(cfg):
    return np.zeros((3,) + cfg.shape)


def scal(cfg):
    return np.zeros(cfg.shape)


def alpha(b):
    out = np.zeros(9)
    lib().or_alpha(_d(_f64(b)), _d(out))
    return out.reshape(3, 3)


def node_avg(cfg, Bc):
    out = vec(cfg)
    lib().or_node_avg(C.byref(cfg), _d(_f64(Bc)), _d(out))
    return out


def filter_pass(cfg, f, d, phi=0.5):
    f = _f64(f).copy()
    ncomp = 1 if f.ndim == 3 else f.shape[0]
    lib().or_filter(C.byref(cfg), _d(f), ncomp, d, phi)
    return f


def bulk_moments(cfg, pl: Plasma):
    rho_m, P = scal(cfg), vec(cfg)
    lib().or_bulk_moments(C.byref(cfg), *pl.args(), _d(pl.w), _d(rho_m), _d(P))
    return rho_m, P


def bulk_velocity(cfg, rho_m, P):
    u = vec(cfg)
    lib().or_bulk_velocity(C.byref(cfg), _d(_f64(rho_m)), _d(_f64(P)), _d(u))
    return u


def deposit(cfg, pl: Plasma, Bn, u=None):
    rho, J = scal(cfg), vec(cfg)
    M = np.zeros(cfg.shape + (27, 3, 3))
    lib().or_deposit(C.byref(cfg), *pl.args(), _d(pl.w), _d(_f64(Bn)),
                     None if u is None else _d(_f64(u)), _d(rho), _d(J), _d(M))
    return rho, J, M


def smooth_current(cfg, J, ns_j):
    J = _f64(J).copy()
    lib().or_smooth_current(C.byref(cfg), _d(J), ns_j)
    return J


def _op(name, cfg, inp, out_shape):
    out = np.zeros(out_shape)
    getattr(lib(), name)(C.byref(cfg), _d(_f64(inp)), _d(out))
    return out


def curl_C(cfg, E):
    return _op("or_curl_C", cfg, E, (3,) + cfg.shape)


def curl_N(cfg, B):
    return _op("or_curl_N", cfg, B, (3,) + cfg.shape)


def div_C(cfg, E):
    return _op("or_div_C", cfg, E, cfg.shape)


def div_N(cfg, B):
    return _op("or_div_N", cfg, B, cfg.shape)


def grad_N(cfg, f):
    return _op("or_grad_N", cfg, f, (3,) + cfg.shape)


def grad_C(cfg, f):
    return _op("or_grad_C", cfg, f, (3,) + cfg.shape)


def mc_limiter(r, beta):
    return lib().or_mc_limiter(float(r), float(beta))


def lf_kappa_E(cfg, En, u=None):
    kappa = np.zeros((3, 3) + cfg.shape)
    u = vec(cfg) if u is None else _f64(u)
    lib().or_lf_kappa_E(C.byref(cfg), _d(_f64(En)), _d(u), _d(kappa))
    return kappa


def apply_A(cfg, E, M=None, kappa=None):
    out = vec(cfg)
    lib().or_apply_A(C.byref(cfg), None if M is None else _d(_f64(M)),
                     None if kappa is None else _d(_f64(kappa)), _d(_f64(E)), _d(out))
    return out


def rhs(cfg, En, Bc, J, M=None, u=None, Bn=None):
    b = vec(cfg)
    u = vec(cfg) if u is None else _f64(u)
    Bn = node_avg(cfg, Bc) if Bn is None else _f64(Bn)
    lib().or_rhs(C.byref(cfg), _d(_f64(En)), _d(_f64(Bc)), _d(_f64(J)),
                 None if M is None else _d(_f64(M)), _d(u), _d(Bn), _d(b))
    return b


def gmres(cfg, b, x0, M=None, kappa=None):
    x = _f64(x0).copy()
    rel = C.c_double(0.0)
    it = C.c_int(0)
    rc = lib().or_gmres(C.byref(cfg), None if M is None else _d(_f64(M)),
                        None if kappa is None else _d(_f64(kappa)), _d(_f64(b)), _d(x), C.byref(rel), C.byref(it))
    return x, rc, rel.value, it.value


def dense_solve(cfg, b, M=None, kappa=None):
    x = vec(cfg)
    rc = lib().or_dense_solve(C.byref(cfg), None if M is None else _d(_f64(M)),
                              None if kappa is None else _d(_f64(kappa)), _d(_f64(b)), _d(x))
    return x, rc


def lf_b_increment(cfg, Bc, u=None):
    """The LF increment D that B^{n+1} receives (Eq. 17-18); zero without lf_on."""
    D = vec(cfg)
    u = vec(cfg) if u is None else _f64(u)
    lib().or_lf_b_increment(C.byref(cfg), _d(_f64(Bc)), _d(u), _d(D))
    return D


def advance_fields(cfg, En, Bc, Eth, u=None):
    Enew, Bnew = vec(cfg), vec(cfg)
    u = vec(cfg) if u is None else _f64(u)
    lib().or_advance_fields(C.byref(cfg), _d(_f64(En)), _d(_f64(Bc)), _d(_f64(Eth)), _d(u), _d(Enew), _d(Bnew))
    return Enew, Bnew


def mover(cfg, pl: Plasma, Eth, Bn, want_vbar=False):
    vbar = np.zeros(3 * pl.np) if want_vbar else None
    md = lib().or_mover(C.byref(cfg), *pl.args(), _d(_f64(Eth)), _d(_f64(Bn)), _d(vbar))
    return (md, vbar.reshape(-1, 3)) if want_vbar else md


def energy(cfg, pl: Plasma, E, Bc):
    out = np.zeros(6)
    lib().or_energy(C.byref(cfg), _d(pl.m), C.c_int64(pl.np), pl.sp.ctypes.data_as(_I32),
                    _d(pl.vx), _d(pl.vy), _d(pl.vz), _d(pl.w), _d(_f64(E)), _d(_f64(Bc)), _d(out))
    return {"W_E": out[0], "W_B": out[1], "KE": out[2], "P": out[3:6].copy(),
            "total": out[0] + out[1] + out[2]}


def divb_clean(cfg, B, phi):
    """Divergence cleaning of a cell-centred B [3][N] and phi [N], in place (Sec. 1.3)."""
    assert B.dtype == np.float64 and phi.dtype == np.float64 and B.flags.c_contiguous and phi.flags.c_contiguous
    lib().or_divb_clean(C.byref(cfg), _d(B), _d(phi))


def step(cfg, pl: Plasma, E, B, want=(), phi=None):
    """One full step, in place on pl, E and B (float64 contiguous arrays); with
    cfg.divb_clean, phi (cell-centred, float64) is the cleaning potential, in place."""
    assert E.dtype == np.float64 and B.dtype == np.float64
    if cfg.divb_clean:
        assert phi is not None and phi.dtype == np.float64 and phi.flags.c_contiguous
    outs = {
        "Eth": vec(cfg) if "Eth" in want else None,
        "J": vec(cfg) if "J" in want else None,
        "M": np.zeros(cfg.shape + (27, 3, 3)) if "M" in want else None,
        "u": vec(cfg) if "u" in want else None,
        "vbar": np.zeros((pl.np, 3)) if "vbar" in want else None,
    }
    stats = np.zeros(3)
    rc = lib().or_step(C.byref(cfg), *pl.args(), _d(pl.w), _d(E), _d(B), _d(phi),
                       _d(outs["Eth"]), _d(outs["J"]), _d(outs["M"]), _d(outs["u"]), _d(outs["vbar"]), _d(stats))
    res = {k: v for k, v in outs.items() if v is not None}
    res.update(rc=rc, iters=int(stats[0]), relres=stats[1], maxdisp=stats[2])
    return res


def gl_displacement(cfg, pl: Plasma, E, gamma):
    """Gauss's-law position correction: per-particle displacements (dx, dy, dz)
    and F = (dV/2) sum_c R_c^2 at the current positions (or_gl_displacement)."""
    d = [np.zeros(pl.np) for _ in range(3)]
    F = C.c_double(0.0)
    lib().or_gl_displacement(C.byref(cfg), _d(pl.q), pl.np, pl.sp.ctypes.data_as(_I32), _d(pl.x), _d(pl.y),
                             _d(pl.z), _d(pl.w), _d(_f64(E)), float(gamma), _d(d[0]), _d(d[1]), _d(d[2]),
                             C.byref(F))
    return d[0], d[1], d[2], F.value


def philox4x64(key, ctr):
    """Philox4x64-10 of (key[2], counter[4]) -> four uint64 words."""
    k = (C.c_uint64 * 2)(*[int(v) for v in key])
    c = (C.c_uint64 * 4)(*[int(v) for v in ctr])
    o = (C.c_uint64 * 4)()
    lib().or_philox4x64(k, c, o)
    return [int(o[i]) for i in range(4)]


def bc_sample(cfg, seed, species, step, i, j, ppc, u, vth):
    """The ppc particles that refill boundary cell (i, j) after the push of `step`."""
    x, y, vx, vy, vz = (np.zeros(ppc) for _ in range(5))
    lib().or_bc_sample(C.byref(cfg), int(seed), int(species), int(step), int(i), int(j), int(ppc),
                       _d(_f64(np.asarray(u, float))), float(vth), _d(x), _d(y), _d(vx), _d(vy), _d(vz))
    return x, y, vx, vy, vz


def maxwellian_species(cfg, seed, species, ppc, n0, u, vth):
    """The particles of a device-side drifting Maxwellian species: for every cell
    (k, then j, then i) the ppc draws of step 0 (or_bc_sample in 2D,
    or_cell_sample3 with a resolved z axis), weights n0 dV / ppc.
    Returns dict x, y, z, vx, vy, vz, w (float64)."""
    nx, ny, nz = cfg.n[0], cfg.n[1], cfg.n[2]
    if nz > 1:
        L = lib()
        uu = _f64(np.asarray(u, float))
        parts = {k: [] for k in ("x", "y", "z", "vx", "vy", "vz")}
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    a = [np.zeros(ppc) for _ in range(6)]
                    L.or_cell_sample3(C.byref(cfg), int(seed), int(species), 0, i, j, k, int(ppc), _d(uu),
                                      float(vth), *[_d(v) for v in a])
                    for key, v in zip(("x", "y", "z", "vx", "vy", "vz"), a):
                        parts[key].append(v)
        out = {key: np.concatenate(v) for key, v in parts.items()}
        out["w"] = np.full(out["x"].size, n0 * cfg.dx[0] * cfg.dx[1] * cfg.dx[2] / ppc)
        return out
    parts = {k: [] for k in ("x", "y", "vx", "vy", "vz")}
    for j in range(ny):
        for i in range(nx):
            for k, v in zip(("x", "y", "vx", "vy", "vz"), bc_sample(cfg, seed, species, 0, i, j, ppc, u, vth)):
                parts[k].append(v)
    out = {k: np.concatenate(v) for k, v in parts.items()}
    out["z"] = np.zeros_like(out["x"])
    out["w"] = np.full(out["x"].size, n0 * cfg.dx[0] * cfg.dx[1] * cfg.dx[2] / ppc)
    return out


def refill_boundaries(cfg, pl: Plasma, sources, step, seed):
    """Open x boundaries (cfg.bc_cells per end): drop every particle in a
    boundary cell and put in fresh ones from each side's plasma state.

    sources[side][s] = dict(n=density, u=(ux, uy, uz), vth=thermal speed, ppc=count) for side 0 (low x)
    and 1 (high x) and species s; weights n dV / ppc.  With cfg.bc_wall the high side is a reflecting
    wall: no particles there and no refill (sources[1] unused).  Returns the new Plasma; cells are
    visited in index order (j, then i), species in order, so the result matches the device's bins as
    a set."""
    nx, ny, G = cfg.n[0], cfg.n[1], cfg.bc_cells
    ci = np.floor(pl.x / cfg.dx[0]).astype(np.int64) % nx
    keep = ~((ci < G) | ((ci >= nx - G) & (cfg.bc_wall == 0)))
    parts = {k: [getattr(pl, k)[keep]] for k in ("x", "y", "z", "vx", "vy", "vz", "w")}
    sp = [pl.sp[keep]]
    dV = cfg.dx[0] * cfg.dx[1] * cfg.dx[2]
    for s in range(len(pl.q)):
        for j in range(ny):
            for i in list(range(G)) + ([] if cfg.bc_wall else list(range(nx - G, nx))):
                src = sources[0 if i < G else 1][s]
                x, y, vx, vy, vz = bc_sample(cfg, seed, s, step, i, j, src["ppc"], src["u"], src["vth"])
                for k, v in (("x", x), ("y", y), ("z", np.zeros_like(x)), ("vx", vx), ("vy", vy), ("vz", vz),
                             ("w", np.full(len(x), src["n"] * dV / src["ppc"]))):
                    parts[k].append(v)
                sp.append(np.full(len(x), s, np.int32))
    cat = {k: np.concatenate(v) for k, v in parts.items()}
    return Plasma(pl.q, pl.m, np.concatenate(sp), cat["x"], cat["y"], cat["z"], cat["vx"], cat["vy"], cat["vz"],
                  cat["w"])


NET_CHANNELS = (3, 32, 32, 32, 3)


def net_param_count():
    return int(lib().or_net_param_count())


def net_forward(params, x, periodic=True, want_acts=False):
    x = _f64(x)
    _, H, W = x.shape
    y = np.zeros((3, H, W))
    acts = np.zeros((3, 32, H, W)) if want_acts else None
    lib().or_net_forward(H, W, int(periodic), _d(_f64(params)), _d(x), _d(y), _d(acts))
    return (y, acts) if want_acts else y


def net_loss_backward(params, x, target, periodic=True):
    x = _f64(x)
    _, H, W = x.shape
    gp = np.zeros(net_param_count())
    gx = np.zeros_like(x)
    L = lib().or_net_loss_backward(H, W, int(periodic), _d(_f64(params)), _d(x), _d(_f64(target)), _d(gp), _d(gx))
    return L, gp, gx


def net_split(params):
    """Split a flat parameter vector into [(W[Cout,Cin,3,3], b[Cout]), ...]."""
    out, off = [], 0
    for l in range(4):
        cin, cout = NET_CHANNELS[l], NET_CHANNELS[l + 1]
        w = params[off:off + cout * cin * 9].reshape(cout, cin, 3, 3)
        off += cout * cin * 9
        b = params[off:off + cout]
        off += cout
        out.append((w, b))
    return out
