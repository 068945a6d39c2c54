"""Seeded synthetic plasma workloads (inputs only).

This module is the one piece shared by the CUDA path's tests/benchmark and the
CPU oracle: it draws particles and initial fields and holds none of the
method's arithmetic (no deposit, solve or push).  Each workload stands in for a
paper setup whose data are not available (the paper's runs need MHD-refined
initial states and a reconnection setup from another paper); the shapes, sizes
and distributions follow the configurations the project is measured on.

Units: Gaussian with explicit c.  Unless a workload says otherwise c = 1, ions
have q = 1, m = 1 and the reference density is n0 = 1/(4 pi), so that the ion
plasma frequency and the ion inertial length are 1.  Electrons have q = -1 and
m = 1 / mass_ratio.  A species of density n with ppc particles per cell gets
weights w = n dV / ppc, so the charge density it deposits is q n.

Random numbers: numpy Generator(Philox(seed + species index)).  Positions are
uniform within each cell, velocities are a drifting Maxwellian with per-
component standard deviation vth.  Positions are returned in float64 (global
coordinates), velocities and weights in float32 (the particle precision of the
GPU path; the oracle promotes the very same float32 values to float64).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

N0 = 1.0 / (4.0 * math.pi)


@dataclass
class Workload:
    name: str
    n: tuple                 # cells per axis (nx, ny, nz); nz == 1 -> 2D
    dx: tuple
    c: float
    theta: float
    dt: float
    comoving: int
    lf_on: int
    lf_beta: float
    lf_speed_c: int
    ns_j: int
    nsmooth_u: int
    gmres_tol: float
    species: list            # dicts: q, m, x, y, z (f64), vx, vy, vz, w (f32)
    E0: np.ndarray           # (3, nz, ny, nx) at nodes
    B0: np.ndarray           # (3, nz, ny, nx) at cell centres
    steps: int = 10
    notes: dict = field(default_factory=dict)

    @property
    def dim(self):
        return 3 if self.n[2] > 1 else 2

    @property
    def n_particles(self):
        return sum(len(s["x"]) for s in self.species)

    def grid_kwargs(self):
        return dict(c=self.c, theta=self.theta, dt=self.dt, comoving=self.comoving, lf_on=self.lf_on,
                    lf_beta=self.lf_beta, lf_speed_c=self.lf_speed_c, ns_j=self.ns_j,
                    nsmooth_u=self.nsmooth_u, gmres_tol=self.gmres_tol)


def _rng(seed, k):
    return np.random.Generator(np.random.Philox(seed + k))


def _uniform_positions(rng, n, dx, ppc):
    """ppc particles uniformly distributed inside every cell."""
    nx, ny, nz = n
    ncell = nx * ny * nz
    cid = np.repeat(np.arange(ncell, dtype=np.int64), ppc)
    i = cid % nx
    j = (cid // nx) % ny
    k = cid // (nx * ny)
    off = rng.random((3, cid.size), dtype=np.float32).astype(np.float64)
    x = (i + off[0]) * dx[0]
    y = (j + off[1]) * dx[1]
    z = (k + off[2]) * dx[2] if nz > 1 else np.zeros(cid.size)
    return x, y, z


def _maxwellian(rng, count, u, vth):
    v = rng.standard_normal((3, count), dtype=np.float64) * vth
    return [(v[d] + u[d]).astype(np.float32) for d in range(3)]


def drifting_species(n, dx, ppc, *, q, m, density, u, vth, seed, k):
    rng = _rng(seed, k)
    x, y, z = _uniform_positions(rng, n, dx, ppc)
    vx, vy, vz = _maxwellian(rng, x.size, u, vth)
    dV = dx[0] * dx[1] * dx[2]
    w = np.full(x.size, density * dV / ppc, np.float32)
    return dict(q=float(q), m=float(m), x=x, y=y, z=z, vx=vx, vy=vy, vz=vz, w=w)


def _uniform_fields(n, c, u, B):
    nx, ny, nz = n
    Bc = np.zeros((3, nz, ny, nx))
    E = np.zeros((3, nz, ny, nx))
    for d in range(3):
        Bc[d] = B[d]
    # initial electric field: the motional field -u x B / c of the drifting
    # plasma, with u rounded to float32 exactly as the particles carry it
    u32 = np.asarray(u, np.float32).astype(np.float64)
    Em = -np.cross(u32, np.asarray(B, float)) / c
    for d in range(3):
        E[d] = Em[d]
    return E, Bc


def uniform_drift(n=(32, 32, 1), dx=(0.1, 0.1, 1.0), ppc=64, mass_ratio=25.0, vth_e=0.05, vth_i=0.01,
                  u=(0.3, 0.0, 0.0), B=(0.0, 0.0, 0.1), dt=None, theta=0.5, comoving=1, lf_on=1,
                  lf_beta=1.0, ns_j=0, nsmooth_u=5, gmres_tol=1e-8, seed=12345, name="uniform_drift",
                  steps=10):
    """Periodic drifting Maxwellian electron-ion plasma in a uniform B.

    Defaults are the 2D 32x32 case: dx = 0.1 d_i, m_i/m_e = 25, 64 particles per
    cell per species, vth_e = 0.05 c, vth_i = 0.01 c, bulk drift 0.3 c along x,
    B = 0.1 along z, theta = 0.5, dt = 0.1 / omega_pe, comoving current and
    limited LF on, GMRES to 1e-8.  With nz > 1 it is the 3D periodic cube.
    """
    n = tuple(n)
    c = 1.0
    wpe = math.sqrt(mass_ratio)          # omega_pi = 1 at n0 = 1/(4 pi)
    if dt is None:
        dt = 0.1 / wpe
    ions = drifting_species(n, dx, ppc, q=1.0, m=1.0, density=N0, u=u, vth=vth_i, seed=seed, k=0)
    elec = drifting_species(n, dx, ppc, q=-1.0, m=1.0 / mass_ratio, density=N0, u=u, vth=vth_e, seed=seed, k=1)
    E, Bc = _uniform_fields(n, c, u, B)
    return Workload(name=name, n=n, dx=tuple(dx), c=c, theta=theta, dt=dt, comoving=comoving, lf_on=lf_on,
                    lf_beta=lf_beta, lf_speed_c=0, ns_j=ns_j, nsmooth_u=nsmooth_u, gmres_tol=gmres_tol,
                    species=[elec, ions], E0=E, B0=Bc, steps=steps,
                    notes=dict(mass_ratio=mass_ratio, ppc=ppc, u=list(u), B=list(B), vth_e=vth_e, vth_i=vth_i))


def config_small(**kw):
    """2D periodic 32x32 cells, 64 particles/cell/species, 10 steps."""
    return uniform_drift(name="periodic_32x32_ppc64", **kw)


def uniform_3d(ncell=128, ppc=64, **kw):
    """3D periodic ncell^3 drifting Maxwellian (u = 0.3 c, vth_e = 0.05 c,
    m_i/m_e = 25, B = 0.1 along z), ppc particles/cell/species."""
    kw.setdefault("name", f"periodic3d_{ncell}^3_ppc{ppc}")
    return uniform_drift(n=(ncell, ncell, ncell), dx=(0.1, 0.1, 0.1), ppc=ppc, **kw)


def harris(nx=512, ny=256, dx=0.05, ppc=100, mass_ratio=100.0, Ti_over_Te=5.0, nb=0.1, lam=0.5,
           B0=0.1, psi_frac=0.1, flow_vA=0.5, dt=0.02, theta=0.5, comoving=1, lf_on=1, lf_beta=1.0,
           ns_j=1, nsmooth_u=5, gmres_tol=1e-8, seed=12345, name=None, steps=5000):
    """Periodic double Harris sheet for reconnection (x-y plane, B along x).

    Sheet half-width lam = 0.5 d_i, background density nb = 0.1 (in units of
    n0), m_i/m_e = 100, T_i/T_e = 5 with pressure balance, psi perturbation of
    10 %, a bulk flow of 0.5 v_A along x superposed on every particle, and
    ppc particles per cell per species with weights proportional to the local
    density.  The field amplitude is taken as B0 = 0.1 in units where c = 1 and
    omega_pi(n0) = 1, i.e. v_A / c = 0.1.
    """
    n = (nx, ny, 1)
    dxs = (dx, dx, 1.0)
    c = 1.0
    Lx, Ly = nx * dx, ny * dx
    y1, y2 = 0.25 * Ly, 0.75 * Ly
    T_tot = B0 ** 2 / (8 * math.pi * N0)          # n0 (Ti + Te) = B0^2 / 8 pi
    Te = T_tot / (1.0 + Ti_over_Te)
    Ti = T_tot - Te
    vA = B0 / math.sqrt(4 * math.pi * N0 * 1.0)
    ux = flow_vA * vA
    psi0 = psi_frac * B0 * lam
    dV = dxs[0] * dxs[1] * dxs[2]

    def sech2(s):
        return 1.0 / np.cosh(s) ** 2

    species = []
    for k, (q, m, T) in enumerate(((-1.0, 1.0 / mass_ratio, Te), (1.0, 1.0, Ti))):
        rng = _rng(seed, k)
        x, y, z = _uniform_positions(rng, n, dxs, ppc)
        s1 = sech2((y - y1) / lam)
        s2 = sech2((y - y2) / lam)
        dens = nb + s1 + s2                              # in units of n0
        w = (dens * N0 * dV / ppc).astype(np.float32)
        vth = math.sqrt(T / m)
        ud = 2.0 * c * T / (q * B0 * lam)                # Harris drift of the sheet population
        pick = rng.random(x.size)
        in1 = pick < s1 / dens
        in2 = (~in1) & (pick < (s1 + s2) / dens)
        uz = np.where(in1, ud, np.where(in2, -ud, 0.0))
        v = rng.standard_normal((3, x.size)) * vth
        species.append(dict(q=q, m=m, x=x, y=y, z=z,
                            vx=(v[0] + ux).astype(np.float32), vy=v[1].astype(np.float32),
                            vz=(v[2] + uz).astype(np.float32), w=w))

    # fields: B at cell centres, E = -u x B / c at nodes (flow along x only)
    xc = (np.arange(nx) + 0.5) * dx
    yc = (np.arange(ny) + 0.5) * dx
    xn = np.arange(nx) * dx
    yn = np.arange(ny) * dx

    def bfield(X, Y):
        bx = B0 * (np.tanh((Y - y1) / lam) - np.tanh((Y - y2) / lam) - 1.0)
        kx, ky = 2 * math.pi / Lx, 4 * math.pi / Ly
        bx = bx + psi0 * ky * np.cos(kx * X) * np.sin(ky * Y)     # -d psi / dy
        by = -psi0 * kx * np.sin(kx * X) * np.cos(ky * Y)          # d psi / dx
        return bx, by

    Xc, Yc = np.meshgrid(xc, yc)
    bx, by = bfield(Xc, Yc)
    Bc = np.zeros((3, 1, ny, nx))
    Bc[0, 0], Bc[1, 0] = bx, by
    Xn, Yn = np.meshgrid(xn, yn)
    bxn, byn = bfield(Xn, Yn)
    E = np.zeros((3, 1, ny, nx))
    E[2, 0] = -(ux * byn) / c
    return Workload(name=name or f"harris_{nx}x{ny}_ppc{ppc}", n=n, dx=dxs, c=c, theta=theta, dt=dt,
                    comoving=comoving, lf_on=lf_on, lf_beta=lf_beta, lf_speed_c=0, ns_j=ns_j,
                    nsmooth_u=nsmooth_u, gmres_tol=gmres_tol, species=species, E0=E, B0=Bc, steps=steps,
                    notes=dict(mass_ratio=mass_ratio, ppc=ppc, Te=Te, Ti=Ti, vA=vA, ux=ux, lam=lam, nb=nb))


def fast_flow_1d(ppc=100, comoving=1, ns_j=1, lf_on=1, lf_beta=1.0, nsmooth_u=5, gmres_tol=1e-8, seed=12345,
                 steps=1000):
    """Uniform fast flow of Sec. 3.2 (solar wind at 1 AU) in the normalised
    units of this package (c = 1, omega_pi = 1 at the flow density, q_i = m_i = 1).

    Physical inputs as printed: n = 5 cm^-3, u = (400, 0, 0) km/s, B = (0, 0, 5)
    nT, T_i = 72,000 K, T_e = 2 T_i, m_i/m_e = 100 (proton ion mass), domain
    160 km in cells of 8 km (20 cells, periodic), dt = 0.0038 s.  Converted with
    the ion inertial length d_i = c / omega_pi (about 102 km) and 1/omega_pi:
    lengths / d_i, velocities / c, times * omega_pi, B as v_A / c (v_A = B /
    sqrt(mu0 n m_p)), per-component thermal spreads sqrt(k T / m) / c.  The
    particle count per cell is not printed (default 100 per species).  The
    cell depth along y and z is 1 d_i; it enters only the cell volume.
    """
    c_si, mp, kB, e, eps0 = 299792458.0, 1.67262192e-27, 1.380649e-23, 1.602176634e-19, 8.8541878128e-12
    mu0 = 1.0 / (eps0 * c_si ** 2)
    n_si, u_si, B_si, Ti, dx_si, L_si, dt_si = 5e6, 4.0e5, 5e-9, 72000.0, 8e3, 160e3, 0.0038
    Te, mass_ratio = 2.0 * Ti, 100.0
    wpi = math.sqrt(n_si * e * e / (eps0 * mp))
    di = c_si / wpi
    nx = int(round(L_si / dx_si))
    dx = (dx_si / di, 1.0, 1.0)
    n = (nx, 1, 1)
    u = (u_si / c_si, 0.0, 0.0)
    B = (0.0, 0.0, B_si / math.sqrt(mu0 * n_si * mp) / c_si)
    vth_i = math.sqrt(kB * Ti / mp) / c_si
    vth_e = math.sqrt(kB * Te / (mp / mass_ratio)) / c_si
    dt = dt_si * wpi
    ions = drifting_species(n, dx, ppc, q=1.0, m=1.0, density=N0, u=u, vth=vth_i, seed=seed, k=0)
    elec = drifting_species(n, dx, ppc, q=-1.0, m=1.0 / mass_ratio, density=N0, u=u, vth=vth_e, seed=seed, k=1)
    E, Bc = _uniform_fields(n, 1.0, u, B)
    return Workload(name=f"fast_flow_{nx}x1_ppc{ppc}", n=n, dx=dx, c=1.0, theta=0.5, dt=dt, comoving=comoving,
                    lf_on=lf_on, lf_beta=lf_beta, lf_speed_c=0, ns_j=ns_j, nsmooth_u=nsmooth_u,
                    gmres_tol=gmres_tol, species=[elec, ions], E0=E, B0=Bc, steps=steps,
                    notes=dict(d_i_km=di / 1e3, omega_pi=wpi, u=list(u), B=list(B), vth_e=vth_e, vth_i=vth_i,
                               v_A=B[2], mass_ratio=mass_ratio, ppc=ppc))


def _state(rho_amu_cc, u_kms, B_nT, pe_npa, pi_npa, c_kms, mass_ratio):
    """One plasma state of the shock runs in the units of this package with the
    reduced light speed c_kms as velocity unit and the upstream ion inertial
    length as length unit (density unit: the upstream density)."""
    mp, kB = 1.67262192e-27, 1.380649e-23
    n_si = rho_amu_cc * 1e6                     # protons: 1 amu each
    te = pe_npa * 1e-9 / n_si                   # k T_e in J
    ti = pi_npa * 1e-9 / n_si
    return dict(n_si=n_si, u=[v / c_kms for v in u_kms],
                vth_e=math.sqrt(te / (mp / mass_ratio)) / (c_kms * 1e3),
                vth_i=math.sqrt(ti / mp) / (c_kms * 1e3), B_nT=list(B_nT))


# The two 1D shocks of the paper as printed (Sec. 3.3 and 3.4): upstream and
# downstream (rho [amu/cc], u [km/s], B [nT], p_e, p_i [nPa]), mass ratio,
# reduced light speed [km/s], upstream ion inertial length [km], domain [km],
# default cell size [d_i].
SHOCKS = {
    "parallel": dict(up=(3.0, (-440.6, 0.0, 0.0), (4.33, 2.5, 0.0), 0.00995, 0.004975),
                     down=(10.9, (-121.3, -10.86, 0.0), (4.33, 9.47, 0.0), 0.4588, 0.2294),
                     mass_ratio=25.0, c_kms=3000.0, di_km=133.0, domain=(-1.8e4, 3.2e4), dx=0.4),
    "perpendicular": dict(up=(40.0, (-552.0, 0.0, 0.0), (20.0, 0.0, 34.6), 0.27613, 0.27613),
                          down=(119.5, (-184.9, 0.0, -31.15), (20.0, 0.0, 106.85), 5.02, 5.02),
                          mass_ratio=400.0, c_kms=10000.0, di_km=36.0, domain=(-2.0e3, 2.0e3), dx=0.2),
}


def shock_1d(kind="parallel", dx=None, length=None, ppc=100, bc_cells=8, seed=12345, cfl=0.2, steps=200,
             comoving=1, ns_j=1, lf_on=1, lf_beta=1.0, gmres_tol=1e-8, ny=1):
    """1D shock from the paper's printed upstream and downstream states:
    "parallel" (Sec. 3.3: theta_Bn = 30 deg, p_e/p_i = 2, m_i/m_e = 25, reduced
    c = 3000 km/s, domain [-1.8e4, 3.2e4] km, M_A = 7) or "perpendicular"
    (Sec. 3.4: theta_Bn = 60 deg, p_e = p_i, m_i/m_e = 400, c = 10,000 km/s,
    domain [-2e3, 2e3] km, M_A = 4), shock at x = 0, downstream on the low-x
    side, the upstream flowing in along -x.

    Units: the printed upstream ion inertial length d_i, velocities over the
    reduced c, densities over the upstream density (omega_pi = c / d_i there).
    B is v_A / c with v_A = |B| / sqrt(mu0 n m_p) per component.  dt from CFL
    0.2 on the fastest speed of the two states, |u| + 3 vth_e (the paper quotes
    CFL 0.2 without the speed it uses).  dx defaults to 0.4 d_i (parallel) and
    0.2 d_i = 4 d_e (perpendicular); `length` (in d_i) shortens the domain
    around the shock for tests, keeping the printed proportion of the two
    sides.  bc_cells cells at each end hold the two states (open boundaries,
    refilled after every push from counter-based draws keyed by seed); ppc per
    species (not printed).  ny > 1 spreads the same planar shock over ny
    periodic rows of square cells (a 2D grid of the 1D problem)."""
    P = SHOCKS[kind]
    c_kms, mass_ratio, di_km = P["c_kms"], P["mass_ratio"], P["di_km"]
    up = _state(*P["up"], c_kms, mass_ratio)
    dn = _state(*P["down"], c_kms, mass_ratio)
    mu0, mp = 4e-7 * math.pi, 1.67262192e-27
    n_up = up["n_si"]
    for st in (up, dn):
        st["n"] = st["n_si"] / n_up * N0
        st["B"] = [b * 1e-9 / math.sqrt(mu0 * n_up * mp) / (c_kms * 1e3) for b in st["B_nT"]]
    dx = P["dx"] if dx is None else float(dx)
    x0, x1 = P["domain"]
    L_full = (x1 - x0) / di_km
    L = L_full if length is None else float(length)
    nx = int(round(L / dx))
    x_shock = (-x0) / (x1 - x0) * nx * dx
    vmax = max(math.hypot(*up["u"]) + 3 * up["vth_e"], math.hypot(*dn["u"]) + 3 * dn["vth_e"])
    dt = cfl * dx / vmax
    n = (nx, int(ny), 1)
    dxs = (dx, dx if ny > 1 else 1.0, 1.0)
    rng_e, rng_i = _rng(seed, 1), _rng(seed, 0)
    xc = (np.arange(nx) + 0.5) * dx
    down_cell = xc < x_shock
    species = []
    for rng, q, m, key in ((rng_e, -1.0, 1.0 / mass_ratio, "vth_e"), (rng_i, 1.0, 1.0, "vth_i")):
        x, y, z = _uniform_positions(rng, n, dxs, ppc)
        cell = np.floor(x / dx).astype(np.int64) % nx
        v = rng.standard_normal((3, x.size))
        vel = []
        for d in range(3):
            ud = np.where(down_cell[cell], dn["u"][d], up["u"][d])
            vt = np.where(down_cell[cell], dn[key], up[key])
            vel.append((ud + vt * v[d]).astype(np.float32))
        w = (np.where(down_cell[cell], dn["n"], up["n"]) * dxs[0] * dxs[1] / ppc).astype(np.float32)
        species.append(dict(q=q, m=m, x=x, y=y if ny > 1 else np.zeros_like(x), z=z, vx=vel[0], vy=vel[1],
                            vz=vel[2], w=w))
    Bc = np.zeros((3, 1, int(ny), nx))
    E = np.zeros((3, 1, int(ny), nx))
    xn = np.arange(nx) * dx
    for d in range(3):
        Bc[d, 0, :] = np.where(down_cell, dn["B"][d], up["B"][d])[None, :]
    for st, sel in ((dn, xn < x_shock), (up, xn >= x_shock)):
        u32 = np.asarray(st["u"], np.float32).astype(np.float64)
        Em = -np.cross(u32, np.asarray(st["B"]))
        for d in range(3):
            E[d, 0][:, sel] = Em[d]
    sources = [[dict(n=st["n"], u=st["u"], vth=st[key], ppc=ppc) for key in ("vth_e", "vth_i")] for st in (dn, up)]
    return Workload(name=f"shock_{kind}_{nx}x{int(ny)}_dx{dx}_ppc{ppc}", n=n, dx=dxs, c=1.0, theta=0.5, dt=dt,
                    comoving=comoving, lf_on=lf_on, lf_beta=lf_beta, lf_speed_c=0, ns_j=ns_j, nsmooth_u=5,
                    gmres_tol=gmres_tol, species=species, E0=E, B0=Bc, steps=steps,
                    notes=dict(bc=dict(cells=bc_cells, seed=seed, sources=sources), up=up, down=dn,
                               x_shock=x_shock, mass_ratio=mass_ratio, kind=kind))


def shock_wall(nx=1024, ny=8, dx=0.1, ppc=256, u=0.2, vth_e=0.03, mass_ratio=100.0, b0=0.05, bc_cells=8,
               seed=12345, comoving=1, ns_j=1, lf_on=1, lf_beta=1.0, gmres_tol=1e-8, steps=2000):
    """Shock by reflection: a uniform plasma (density n0, bulk velocity u along
    +x, B = b0 (cos 45, 0, sin 45), T_i = T_e) streams from an open boundary at
    x = 0 onto a reflecting conducting wall at the high-x end (the last bc_cells
    cells: no particles, E = 0, B frozen).  Defaults: 1024 x 8 cells of 0.1 d_i,
    256 particles per cell and species, m_i/m_e = 100, vth_e = 0.03 c, vth_i =
    vth_e / sqrt(mass_ratio), dt = 0.2 dx / (u + 3 vth_e).  The paper's shocks
    are set up from printed Rankine-Hugoniot states instead (shock_1d); this is
    the reflecting-wall form of the same physics."""
    n = (nx, int(ny), 1)
    dxs = (dx, dx if ny > 1 else 1.0, 1.0)
    vth_i = vth_e / math.sqrt(mass_ratio)
    dt = 0.2 * dx / (u + 3 * vth_e)
    B = (b0 * math.cos(math.pi / 4), 0.0, b0 * math.sin(math.pi / 4))
    uu = (u, 0.0, 0.0)
    species = []
    for k, (q, m, vth) in enumerate(((-1.0, 1.0 / mass_ratio, vth_e), (1.0, 1.0, vth_i))):
        sp = drifting_species(n, dxs, ppc, q=q, m=m, density=N0, u=uu, vth=vth, seed=seed, k=1 - k)
        keep = sp["x"] < (nx - bc_cells) * dx                     # the wall cells hold no particles
        for key in ("x", "y", "z", "vx", "vy", "vz", "w"):
            sp[key] = sp[key][keep]
        if ny == 1:
            sp["y"] = np.zeros_like(sp["x"])
        species.append(sp)
    E, Bc = _uniform_fields(n, 1.0, uu, B)
    E[:, :, :, nx - bc_cells:] = 0.0                             # the conductor: E = 0 from the wall face on
    src = [dict(n=N0, u=uu, vth=vth_e, ppc=ppc), dict(n=N0, u=uu, vth=vth_i, ppc=ppc)]
    return Workload(name=f"shock_wall_{nx}x{int(ny)}_ppc{ppc}", n=n, dx=dxs, c=1.0, theta=0.5, dt=dt,
                    comoving=comoving, lf_on=lf_on, lf_beta=lf_beta, lf_speed_c=0, ns_j=ns_j, nsmooth_u=5,
                    gmres_tol=gmres_tol, species=species, E0=E, B0=Bc, steps=steps,
                    notes=dict(bc=dict(cells=bc_cells, seed=seed, wall=1, sources=[src, src]), u=u,
                               mass_ratio=mass_ratio))


def tophat_1d(n=80, dx=0.01, cfl=0.4, lf_on=1, lf_beta=1.0, theta=0.5):
    """Vacuum light wave with a top-hat E_y = B_z = 1 for |x| < 0.2 on
    [-0.4, 0.4) (shifted to [0, 0.8)), c = 1; the advection test of Sec. 3.1."""
    c = 1.0
    dt = cfl * dx / c
    L = n * dx
    xn = np.arange(n) * dx - 0.5 * L
    xc = (np.arange(n) + 0.5) * dx - 0.5 * L
    E = np.zeros((3, 1, 1, n))
    B = np.zeros((3, 1, 1, n))
    # B at cell centres is the cell value of the top-hat; a node sitting exactly
    # on a jump takes the mean of the two sides, so E and B describe the same
    # right-moving profile on the staggered mesh.
    E[1, 0, 0] = np.where(np.isclose(np.abs(xn), 0.2), 0.5, (np.abs(xn) < 0.2).astype(float))
    B[2, 0, 0] = (np.abs(xc) < 0.2).astype(float)
    return Workload(name="tophat", n=(n, 1, 1), dx=(dx, 1.0, 1.0), c=c, theta=theta, dt=dt, comoving=0,
                    lf_on=lf_on, lf_beta=lf_beta, lf_speed_c=1, ns_j=0, nsmooth_u=0, gmres_tol=1e-13,
                    species=[], E0=E, B0=B, steps=25, notes=dict(xn=xn, xc=xc))
