"""GPU parity of the CUDA hot path (through the C ABI) against the FP64 oracle.

Tolerances (stated up front; the particle state and deposits are FP32, the
field solve FP64):
  * moments (rho, J, M, u) after a deposit: relative L2 <= 1e-5 per field;
  * E^{n+theta}, E^{n+1}, B^{n+1} after one step: relative L2 <= 1e-6;
  * particles after one push, matched by id: |dv| <= 1e-6 max|v|,
    |dx| <= 1e-5 dx (periodic distance).
Both sides solve to a relative residual of 1e-12 here so that the comparison
measures the FP32 particle arithmetic, not solver round-off.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads

pytestmark = pytest.mark.gpu

TOL_MOM = 1e-5
TOL_FIELD = 1e-6


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def gx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    g.lib()
    return g


def oracle_cfg(wl, tol=1e-12):
    cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
    cfg.gmres_tol = tol
    return cfg


def oracle_moments(wl):
    cfg = oracle_cfg(wl)
    pl = O.Plasma.from_species(wl.species)
    Bn = O.node_avg(cfg, wl.B0)
    rm, P = O.bulk_moments(cfg, pl)
    u = O.bulk_velocity(cfg, rm, P)
    rho, J, M = O.deposit(cfg, pl, Bn, u=u if wl.comoving else None)
    J = O.smooth_current(cfg, J, wl.ns_j)
    return rho, J, M, u


WORKLOADS = {
    # several 16x8 tiles, 64 particles per cell per species, comoving + LF
    "uniform_32x32": lambda: workloads.uniform_drift(n=(32, 32, 1), ppc=64, ns_j=1),
    # ragged: cell counts vary (random positions), grid not a multiple of 16
    "ragged_36x20": lambda: _ragged(),
    # 1D line of cells (ny = 1), standard current
    "line_48x1": lambda: workloads.uniform_drift(n=(48, 1, 1), ppc=40, comoving=0, u=(0.2, 0.05, 0.0)),
    # Harris sheet: density-weighted particles, strong field gradients
    "harris_64x32": lambda: workloads.harris(nx=64, ny=32, ppc=24, steps=1),
}


def _ragged():
    wl = workloads.uniform_drift(n=(36, 20, 1), ppc=30, seed=7)
    rng = np.random.default_rng(3)
    for s in wl.species:
        n = len(s["x"])
        s["x"] = rng.random(n) * 36 * 0.1 * rng.random(n) ** 0.3      # denser toward x = 0
        s["y"] = rng.random(n) * 20 * 0.1
    # exact cell-boundary positions
    wl.species[0]["x"][:10] = np.arange(10) * 0.1
    wl.species[0]["y"][:10] = 0.1 * 3
    return wl


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_deposit_moments_match_oracle(gx, name):
    wl = WORKLOADS[name]()
    ctx = gx.from_workload(wl, gmres_tol=1e-12)
    ctx.deposit()
    rho, J, M, u = ctx.get_moments()
    orho, oJ, oM, ou = oracle_moments(wl)
    errs = {"rho": rel(rho, orho), "J": rel(J, oJ), "M": rel(M, oM), "u": rel(u, ou)}
    assert all(v <= TOL_MOM for v in errs.values()), errs
    # charge conservation of the deposit: sum rho dV = sum q_p (FP32 weights)
    dV = wl.dx[0] * wl.dx[1] * wl.dx[2]
    qtot = sum(s["q"] * np.asarray(s["w"], np.float64).sum() for s in wl.species)
    assert abs(rho.sum() * dV - qtot) <= 1e-5 * sum(abs(s["q"]) * np.asarray(s["w"], np.float64).sum() for s in wl.species)
    ctx.close()


def _oracle_index(wl):
    offs, o = [], 0
    for s in wl.species:
        offs.append(o)
        o += len(s["x"])
    return offs


@pytest.mark.parametrize("name", ["uniform_32x32", "ragged_36x20", "line_48x1", "harris_64x32"])
def test_one_step_matches_oracle(gx, name):
    wl = WORKLOADS[name]()
    ctx = gx.from_workload(wl, track_ids=1, gmres_tol=1e-12)
    st = ctx.field_solve()
    assert st.converged == 1 and st.relres <= 1e-12
    Eth = ctx.get_solution()
    ctx.push_and_deposit()
    E1, B1 = ctx.get_fields()
    rho1, J1, M1, u1 = ctx.get_moments()

    cfg = oracle_cfg(wl)
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    r = O.step(cfg, pl, E, B, want=("Eth",))
    assert r["rc"] == 0
    errs = {"Eth": rel(Eth, r["Eth"]), "E": rel(E1, E), "B": rel(B1, B)}
    assert all(v <= TOL_FIELD for v in errs.values()), errs

    # particles, matched by id
    offs = _oracle_index(wl)
    L = [wl.n[d] * wl.dx[d] for d in range(3)]
    for s in range(len(wl.species)):
        p = ctx.get_particles(s, ids=True)
        assert len(p["id"]) == len(wl.species[s]["x"])
        idx = offs[s] + p["id"]
        vmax = max(np.abs(pl.vx).max(), np.abs(pl.vy).max(), np.abs(pl.vz).max())
        for key, ref in (("vx", pl.vx), ("vy", pl.vy), ("vz", pl.vz)):
            assert np.abs(p[key] - ref[idx]).max() <= 1e-6 * vmax, key
        for key, ref, d in (("x", pl.x, 0), ("y", pl.y, 1)):
            if wl.n[d] == 1:
                continue
            dd = (p[key] - ref[idx] + 0.5 * L[d]) % L[d] - 0.5 * L[d]
            assert np.abs(dd).max() <= 1e-5 * wl.dx[d], key
    # the moments of step n+1 (deposited during the push) against the oracle
    # deposit at the moved particles with B^{n+1}
    wl1 = WORKLOADS[name]()
    for s, sp in enumerate(wl1.species):
        sel = slice(offs[s], offs[s] + len(sp["x"]))
        sp["x"], sp["y"], sp["z"] = pl.x[sel], pl.y[sel], pl.z[sel]
        sp["vx"], sp["vy"], sp["vz"] = pl.vx[sel], pl.vy[sel], pl.vz[sel]
    wl1.B0 = B
    orho, oJ, oM, ou = oracle_moments(wl1)
    errs = {"rho": rel(rho1, orho), "J": rel(J1, oJ), "M": rel(M1, oM), "u": rel(u1, ou)}
    assert all(v <= TOL_MOM for v in errs.values()), errs
    ctx.close()


def _fast_beam():
    # 0.63 cells per step along x and 0.35 along y: 76 % of the particles change
    # cell, so a warp holds more than 32 leavers at once
    return workloads.uniform_drift(n=(32, 16, 1), ppc=100, u=(0.45, 0.25, 0.0), vth_e=0.03, dt=0.14, ns_j=1)


def test_fast_beam_push_matches_oracle(gx):
    """One push of a fast drifting beam, most particles leaving their cell.
    Every particle (matched by id) against the oracle's mover; the deposit the
    push made against the oracle's deposit of the same moved particles (1e-5,
    the re-binning and the leavers' write-out included); the whole step's
    moments against the oracle's step.  For the last, J is judged against the
    beam's current scale |rho| |u|: the comoving current of a uniform beam is
    the cells' thermal residue (7 % of |rho| |u| here), and the FP32 rounding of
    the drift velocity, the same for every particle, adds coherently into it
    (measured 2.2e-5 of |J| with the comoving current, 4e-7 without it, and
    1.0e-6 for the deposit of the moved particles)."""
    wl = _fast_beam()
    ctx = gx.from_workload(wl, track_ids=1, gmres_tol=1e-12)
    st = ctx.field_solve()
    assert st.converged == 1
    ctx.push_and_deposit()
    E1, B1 = ctx.get_fields()
    rho1, J1, M1, u1 = ctx.get_moments()

    cfg = oracle_cfg(wl)
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    r = O.step(cfg, pl, E, B, want=("Eth",))
    assert r["rc"] == 0
    assert rel(E1, E) <= TOL_FIELD and rel(B1, B) <= TOL_FIELD

    offs = _oracle_index(wl)
    L = [wl.n[d] * wl.dx[d] for d in range(3)]
    moved = _fast_beam()
    left = 0
    for s in range(len(wl.species)):
        p = ctx.get_particles(s, ids=True)
        assert np.array_equal(np.sort(p["id"]), np.arange(len(wl.species[s]["x"])))
        idx = offs[s] + p["id"]
        vmax = max(np.abs(pl.vx).max(), np.abs(pl.vy).max(), np.abs(pl.vz).max())
        for key, ref in (("vx", pl.vx), ("vy", pl.vy), ("vz", pl.vz)):
            assert np.abs(p[key] - ref[idx]).max() <= 1e-6 * vmax, key
        for key, ref, d in (("x", pl.x, 0), ("y", pl.y, 1)):
            dd = (p[key] - ref[idx] + 0.5 * L[d]) % L[d] - 0.5 * L[d]
            assert np.abs(dd).max() <= 1e-5 * wl.dx[d], key
        x0 = np.floor(np.asarray(wl.species[s]["x"]) / wl.dx[0])[p["id"]]
        y0 = np.floor(np.asarray(wl.species[s]["y"]) / wl.dx[1])[p["id"]]
        left += int(np.count_nonzero((np.floor(p["x"] / wl.dx[0]) != x0) | (np.floor(p["y"] / wl.dx[1]) != y0)))
        o = np.argsort(p["id"])
        sp = moved.species[s]
        for key in ("x", "y", "vx", "vy", "vz"):
            sp[key] = np.asarray(p[key])[o]
        sp["z"] = np.zeros(len(o))
    assert left > 0.7 * sum(len(sp["x"]) for sp in wl.species)

    # the deposit of the moved particles, re-binning included
    moved.B0 = B1
    drho, dJ, dM, du = oracle_moments(moved)
    errs = {"rho": rel(rho1, drho), "J": rel(J1, dJ), "M": rel(M1, dM), "u": rel(u1, du)}
    assert all(v <= TOL_MOM for v in errs.values()), errs

    # the whole step's moments against the oracle's step
    wl1 = _fast_beam()
    for s, sp in enumerate(wl1.species):
        sel = slice(offs[s], offs[s] + len(sp["x"]))
        sp["x"], sp["y"], sp["z"] = pl.x[sel], pl.y[sel], pl.z[sel]
        sp["vx"], sp["vy"], sp["vz"] = pl.vx[sel], pl.vy[sel], pl.vz[sel]
    wl1.B0 = B
    orho, oJ, oM, ou = oracle_moments(wl1)
    errs = {"rho": rel(rho1, orho), "M": rel(M1, oM), "u": rel(u1, ou)}
    assert all(v <= TOL_MOM for v in errs.values()), errs
    ubeam = float(np.hypot(0.45, 0.25))
    assert np.linalg.norm(J1 - oJ) <= TOL_MOM * np.linalg.norm(orho) * ubeam
    ctx.close()


def test_diagnostics_match_fp64_sums(gx):
    """The kinetic energy and momentum of gx_diagnostics against FP64 sums over
    the particles read back (the device forms the per-particle terms in FP32
    and sums them in FP64 per 16 cells): within 1e-7 of the scale."""
    wl = workloads.harris(nx=64, ny=32, ppc=24, steps=1)
    ctx = gx.from_workload(wl)
    ctx.step(1)
    d = ctx.diagnostics()
    ke, P, scale = 0.0, np.zeros(3), np.zeros(3)
    for s, sp in enumerate(wl.species):
        p = ctx.get_particles(s)
        v = np.stack([p["vx"], p["vy"], p["vz"]]).astype(np.float64)
        mw = sp["m"] * p["w"].astype(np.float64)
        ke += 0.5 * (mw * (v * v).sum(0)).sum()
        P += (mw * v).sum(1)
        scale += (mw * np.abs(v)).sum(1)
    ctx.close()
    assert abs(d["kinetic"] - ke) <= 1e-7 * ke
    assert np.all(np.abs(np.array(d["momentum"]) - P) <= 1e-7 * scale)
    assert d["n_particles"] == wl.n_particles


def test_plain_ecsim_energy_conservation_on_gpu(gx):
    # theta = 0.5, standard current, no LF, no smoothing: particle + field
    # energy is conserved to the solver tolerance in exact arithmetic; the FP32
    # particle state adds round-off of order 1e-7 per particle, averaging down.
    wl = workloads.uniform_drift(n=(32, 32, 1), ppc=64, comoving=0, lf_on=0, ns_j=0, vth_e=0.2, vth_i=0.05,
                                 dt=0.05)
    ctx = gx.from_workload(wl, gmres_tol=1e-12)
    W0 = ctx.diagnostics()["total"]
    worst, Ws = 0.0, []
    for _ in range(6):
        ctx.step(1)
        W = ctx.diagnostics()["total"]
        Ws.append(W)
        worst = max(worst, abs(W - W0) / W0)
    assert worst < 1e-6, worst
    # past a transient over the first two steps (~2e-7, then ~5e-8) the total changes by a few
    # 1e-9 per step (2e-9 to 7e-9 measured on GB300): guard the per-step figure at 2e-8
    steps = [abs(b - a) / W0 for a, b in zip(Ws[:-1], Ws[1:])]
    assert max(steps[1:]) < 2e-8, steps
    ctx.close()


def test_solver_preconditioners_agree(gx):
    wl = workloads.harris(nx=64, ny=32, ppc=16, steps=1)
    sols = []
    for pc in (gx.GX_PRECOND_NONE, gx.GX_PRECOND_JACOBI):
        ctx = gx.from_workload(wl, precond=pc, gmres_tol=1e-12)
        st = ctx.field_solve()
        assert st.converged == 1
        sols.append(ctx.get_solution())
        ctx.close()
    assert rel(sols[1], sols[0]) < 1e-10


def test_cfl_violation_is_reported_not_fatal(gx):
    wl = workloads.uniform_drift(n=(16, 8, 1), ppc=4)
    wl.species[0]["vx"][:3] = 50.0          # moves ~10 cells in one step
    ctx = gx.from_workload(wl)
    ctx.field_solve()
    with pytest.raises(gx.GxError) as e:
        ctx.push_and_deposit()
    assert e.value.status == gx.GX_ECFL
    ctx.close()
    # the device is still usable
    ctx2 = gx.from_workload(workloads.uniform_drift(n=(16, 8, 1), ppc=4))
    ctx2.step(1)
    ctx2.close()


def test_empty_species_and_vacuum(gx):
    wl = workloads.tophat_1d(lf_on=1, lf_beta=1.0)
    cfg = gx.make_config(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, comoving=0, lf_on=1, lf_speed_c=1,
                         lf_beta=1.0, gmres_tol=1e-13)
    ctx = gx.Context(cfg)
    e = np.zeros(0)
    f = np.zeros(0, np.float32)
    ctx.species_add(-1.0, 0.04, e, e, e, f, f, f, f)      # an empty species
    ctx.fields_set(wl.E0, wl.B0)
    for _ in range(wl.steps):
        ctx.step(1)
    E, B = ctx.get_fields()
    ocfg = oracle_cfg(wl, 1e-13)
    Eo, Bo = wl.E0.copy(), wl.B0.copy()
    for _ in range(wl.steps):
        b = O.rhs(ocfg, Eo, Bo, np.zeros_like(Eo))
        kap = O.lf_kappa_E(ocfg, Eo)
        Eth, rc, _, _ = O.gmres(ocfg, b, Eo, kappa=kap)
        Eo, Bo = O.advance_fields(ocfg, Eo, Bo, Eth)
    # both sides solve to 1e-13; the remaining difference is the limiter's
    # ratio and switch, which the CUDA path evaluates in FP32 (about 1e-9 after
    # these 25 steps, far inside the 1e-6 per step stated for the fields)
    assert rel(E, Eo) < 1e-8 and rel(B, Bo) < 1e-8
    ctx.close()
