"""The Gauss's-law position correction (the GL of GL-ECSIM, reading stated in
the oracle and in include/gx.h: one steepest-descent step on the Gauss residual
of E^n and the deposited charge, added to the push) on the GPU, against the FP64
oracle's same step, 2D and 3D: E^{n+theta}, E^{n+1}, B^{n+1} within the 1e-6
field tolerance and the particles within the 1e-5 dx position tolerance.
Over several steps the correction keeps the Gauss residual below that of the
same run without it.
"""
import numpy as np
import pytest

import oracle as O
import workloads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def gx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    g.lib()
    return g


def _ctx(gx, wl, gl_gamma, **kw):
    cfg = gx.make_config(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, comoving=wl.comoving, lf_on=wl.lf_on,
                         lf_speed_c=wl.lf_speed_c, lf_beta=wl.lf_beta, ns_j=wl.ns_j, nsmooth_u=wl.nsmooth_u,
                         gl_gamma=gl_gamma, **kw)
    ctx = gx.Context(cfg)
    for s in wl.species:
        ctx.species_add(s["q"], s["m"], np.ascontiguousarray(s["x"]), np.ascontiguousarray(s["y"]),
                        np.ascontiguousarray(s["z"]), np.ascontiguousarray(s["vx"], np.float32),
                        np.ascontiguousarray(s["vy"], np.float32), np.ascontiguousarray(s["vz"], np.float32),
                        np.ascontiguousarray(s["w"], np.float32))
    ctx.fields_set(np.ascontiguousarray(wl.E0), np.ascontiguousarray(wl.B0))
    return ctx


def _noisy(wl, seed=5):
    # E that does not satisfy Gauss's law for the particles: the correction has work to do
    wl.E0 = wl.E0 + 0.02 * np.random.default_rng(seed).standard_normal(wl.E0.shape)
    return wl


@pytest.mark.parametrize("dim3", [False, True])
def test_gl_step_matches_oracle(gx, dim3):
    if dim3:
        wl = _noisy(workloads.uniform_drift(n=(10, 8, 6), dx=(0.1, 0.1, 0.1), ppc=8, ns_j=1))
    else:
        wl = _noisy(workloads.uniform_drift(n=(32, 24, 1), ppc=16, ns_j=1))
    gamma = 0.5
    ctx = _ctx(gx, wl, gamma, gmres_tol=1e-12, track_ids=1)
    assert ctx.field_solve().converged == 1
    Eth = ctx.get_solution()
    ctx.push_and_deposit()
    E1, B1 = ctx.get_fields()
    parts = [ctx.get_particles(s, ids=True) for s in range(len(wl.species))]
    ctx.close()
    cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs(), gl_gamma=gamma)
    cfg.gmres_tol = 1e-12
    pl = O.Plasma.from_species(wl.species)
    x0 = pl.copy()
    E, B = wl.E0.copy(), wl.B0.copy()
    r = O.step(cfg, pl, E, B, want=("Eth",))
    assert r["rc"] == 0
    errs = {"Eth": rel(Eth, r["Eth"]), "E": rel(E1, E), "B": rel(B1, B)}
    assert all(v <= 1e-6 for v in errs.values()), errs
    L = [wl.n[d] * wl.dx[d] for d in range(3)]
    off = 0
    moved = 0.0
    for s, p in enumerate(parts):
        idx = off + p["id"]
        for key, d in (("x", 0), ("y", 1), ("z", 2)):
            if wl.n[d] == 1:
                continue
            ref = getattr(pl, key)[idx]
            dd = (p[key] - ref + 0.5 * L[d]) % L[d] - 0.5 * L[d]
            assert np.abs(dd).max() <= 1e-5 * wl.dx[d], key
        off += len(wl.species[s]["x"])
    # the correction moved the particles measurably (against the same step without it)
    d = O.gl_displacement(O.make_cfg(wl.n, wl.dx), x0, wl.E0, gamma)
    moved = max(np.abs(d[0]).max() / wl.dx[0], np.abs(d[1]).max() / wl.dx[1])
    assert moved > 1e-3


def test_gl_keeps_the_gauss_residual_lower(gx):
    wl = _noisy(workloads.uniform_drift(n=(32, 24, 1), ppc=16, comoving=0, lf_on=0, ns_j=0, vth_e=0.1), seed=8)
    res = {}
    for gamma in (0.0, 1.0):
        ctx = _ctx(gx, wl, gamma)
        g = [ctx.diagnostics()["gauss_l2"]]
        for _ in range(8):
            ctx.step(1)
            g.append(ctx.diagnostics()["gauss_l2"])
        ctx.close()
        res[gamma] = np.array(g)
    print("Gauss residual without / with the correction:", res[0.0], res[1.0])
    assert res[1.0][-1] < 0.9 * res[0.0][-1]
