"""GPU parity of the 3D path (through the C ABI) against the FP64 oracle, which
is uniformly 3D: the same fused push and deposit with 8 corners and 27 pair
classes, the mass matrix over a node's 27 neighbours (Sec. 2.1), the mesh's
3D curls (Sec. 1.1), the limited LF terms along three axes (Sec. 1.2) and the
implicit solve of the assembled 27-block operator.

Tolerances (as in 2D): moments (rho, J, M, u) relative L2 <= 1e-5 per field;
E^{n+theta}, E^{n+1}, B^{n+1} after one step relative L2 <= 1e-6 with both
sides solving to 1e-12; particles matched by id |dv| <= 1e-6 max|v|,
|dx| <= 1e-5 dx.
"""
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


def _drift3(n=(12, 10, 8), ppc=8, **kw):
    return workloads.uniform_drift(n=n, dx=(0.1, 0.1, 0.1), ppc=ppc, **kw)


def _ragged3():
    wl = _drift3(n=(10, 9, 7), ppc=10, seed=11)
    rng = np.random.default_rng(5)
    for s in wl.species:
        m = len(s["x"])
        s["x"] = rng.random(m) * 1.0 * rng.random(m) ** 0.3          # denser toward x = 0
        s["y"] = rng.random(m) * 0.9
        s["z"] = rng.random(m) * 0.7
    wl.species[0]["x"][:8] = np.arange(8) * 0.1                     # exact cell faces
    wl.species[0]["z"][:8] = 0.1 * 3
    return wl


def _sheared3():
    # a non-uniform B with a curl and a varying plasma velocity: every term of the
    # mass matrix, the comoving correction and the LF terms differs from node to node
    wl = _drift3(n=(12, 8, 10), ppc=8, ns_j=1, seed=3)
    nz, ny, nx = wl.B0.shape[1:]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wl.B0[0] += 0.05 * np.sin(2 * np.pi * z / nz)
    wl.B0[1] += 0.04 * np.cos(2 * np.pi * x / nx)
    wl.B0[2] += 0.03 * np.sin(2 * np.pi * (x / nx + y / ny))
    wl.E0[1] += 0.01 * np.cos(2 * np.pi * (y / ny + z / nz))
    for s in wl.species:
        s["vy"] = (s["vy"] + 0.05 * np.sin(2 * np.pi * s["z"] / (nz * 0.1))).astype(np.float32)
    return wl


WORKLOADS = {
    "drift_12x10x8": lambda: _drift3(ns_j=1),
    "ragged_10x9x7": _ragged3,
    "sheared_12x8x10": _sheared3,
    "standard_current": lambda: _drift3(n=(8, 8, 8), comoving=0, lf_on=0),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_3d_deposit_moments_match_oracle(gx, name):
    wl = WORKLOADS[name]()
    ctx = gx.from_workload(wl, gmres_tol=1e-12)
    ctx.deposit()
    rho, J, M, u = ctx.get_moments()
    orho, oJ, oM, ou = oracle_moments(wl)
    errs = {"rho": rel(rho, orho), "J": rel(J, oJ), "M": rel(M, oM), "u": rel(u, ou)}
    assert all(v <= TOL_MOM for v in errs.values()), errs
    dV = wl.dx[0] * wl.dx[1] * wl.dx[2]
    qtot = sum(s["q"] * np.asarray(s["w"], np.float64).sum() for s in wl.species)
    qabs = sum(abs(s["q"]) * np.asarray(s["w"], np.float64).sum() for s in wl.species)
    assert abs(rho.sum() * dV - qtot) <= 1e-5 * qabs
    ctx.close()


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_3d_one_step_matches_oracle(gx, name):
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

    offs, o = [], 0
    for s in wl.species:
        offs.append(o)
        o += len(s["x"])
    L = [wl.n[d] * wl.dx[d] for d in range(3)]
    vmax = max(np.abs(pl.vx).max(), np.abs(pl.vy).max(), np.abs(pl.vz).max())
    for s in range(len(wl.species)):
        p = ctx.get_particles(s, ids=True)
        assert len(p["id"]) == len(wl.species[s]["x"])
        idx = offs[s] + p["id"]
        assert len(np.unique(idx)) == len(idx)
        for key, ref in (("vx", pl.vx), ("vy", pl.vy), ("vz", pl.vz)):
            assert np.abs(p[key] - ref[idx]).max() <= 1e-6 * vmax, key
        for key, ref, d in (("x", pl.x, 0), ("y", pl.y, 1), ("z", pl.z, 2)):
            dd = (p[key] - ref[idx] + 0.5 * L[d]) % L[d] - 0.5 * L[d]
            assert np.abs(dd).max() <= 1e-5 * wl.dx[d], key
    # the deposit of step n+1, made during the push, against the oracle's
    # deposit of the moved particles with B^{n+1}
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


def test_3d_three_steps_and_preconditioners(gx):
    # three steps against the oracle's three (the fields stay within the
    # one-step tolerance per step), and block-Jacobi FGMRES agrees with plain
    wl = _sheared3()
    ctx = gx.from_workload(wl, gmres_tol=1e-12)
    ctx.step(3)
    E1, B1 = ctx.get_fields()
    ctx.close()
    cfg = oracle_cfg(wl)
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    for _ in range(3):
        assert O.step(cfg, pl, E, B)["rc"] == 0
    assert rel(E1, E) < 3 * TOL_FIELD and rel(B1, B) < 3 * TOL_FIELD
    sols = []
    for pc in (gx.GX_PRECOND_NONE, gx.GX_PRECOND_JACOBI):
        c = gx.from_workload(wl, precond=pc, gmres_tol=1e-12)
        st = c.field_solve()
        assert st.converged == 1
        sols.append(c.get_solution())
        c.close()
    assert rel(sols[1], sols[0]) < 1e-10


def test_3d_maxwellian_species_draws_match_oracle(gx):
    n, dx = (6, 5, 4), (0.1, 0.1, 0.1)
    cfg = gx.make_config(n, dx, seed=77, track_ids=0)
    ctx = gx.Context(cfg)
    u, vth, ppc, n0 = (0.3, 0.0, -0.1), 0.05, 12, 1.0 / (4 * np.pi)
    ctx.species_maxwellian(-1.0, 0.04, ppc, n0, u, vth)
    p = ctx.get_particles(0)
    ctx.close()
    ocfg = O.make_cfg(n, dx)
    ref = O.maxwellian_species(ocfg, 77, 0, ppc, n0, u, vth)
    # the device writes cell by cell in the oracle's order (one bin per cell)
    assert len(p["x"]) == len(ref["x"]) == ppc * np.prod(n)
    for key in ("x", "y", "z"):
        assert np.abs(p[key] - ref[key]).max() <= 1e-6 * dx[0], key
    for key in ("vx", "vy", "vz"):
        assert np.abs(p[key] - ref[key]).max() <= 1e-6 * (abs(np.array(u)).max() + 6 * vth), key
    assert np.allclose(p["w"], ref["w"], rtol=1e-6)


def test_3d_plain_ecsim_energy(gx):
    # theta = 1/2, standard current, no LF, no smoothing: energy is conserved up
    # to the FP32 particle round-off (the 2D guard: < 1e-6 in total)
    wl = _drift3(n=(8, 8, 8), ppc=16, comoving=0, lf_on=0, ns_j=0, vth_e=0.2, vth_i=0.05, dt=0.05)
    ctx = gx.from_workload(wl, gmres_tol=1e-12)
    W0 = ctx.diagnostics()["total"]
    worst = 0.0
    for _ in range(5):
        ctx.step(1)
        worst = max(worst, abs(ctx.diagnostics()["total"] - W0) / W0)
    ctx.close()
    assert worst < 1e-6, worst


def test_3d_refuses_what_it_does_not_run(gx):
    for kw in (dict(divb_clean=1), dict(precond=gx.GX_PRECOND_NET), dict(bc_cells=8)):
        cfg = gx.make_config((20, 8, 8), (0.1, 0.1, 0.1), **kw)
        with pytest.raises(gx.GxError) as e:
            gx.Context(cfg)
        assert e.value.status == gx.GX_ENOTIMPL
