"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the 512 x 256 Harris workload (26.2 M particles) and the 1024 x 512 one
of the learned-preconditioner comparison (104.9 M particles), 100 particles per
cell and species, one step of the CUDA path through the C ABI.

The oracle cannot run the whole step at this size in seconds, so the check is
on sampled outputs it can compute one by one: for a few 8 x 8-cell patches the
particles the GPU holds there after the step are deposited by the oracle on a
12 x 12-cell grid that contains the patch (with the GPU's B^{n+1} and smoothed
bulk velocity u around it), and the oracle's rho, mass matrix and comoving
current (smoothed once, ns_j = 1) are compared with the GPU's at the nodes
whose stencils lie inside the patch.  One patch straddles the periodic
boundary.  Plus properties that hold at any size: the charge sum equals the
particles' charge, and no particle is lost.  Tolerance: the moments'
relative L2 <= 1e-5 (the stated bound for moments).
"""
import numpy as np
import pytest

import oracle as O
import workloads

pytestmark = pytest.mark.gpu

TOL_MOM = 1e-5
PATCH, MARGIN = 8, 2
SUB = PATCH + 2 * MARGIN


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module", params=[(512, 256), (1024, 512)], ids=["512x256", "1024x512"])
def state(request):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    g.lib()
    nx, ny = request.param
    wl = workloads.harris(nx=nx, ny=ny, ppc=100)
    ctx = g.from_workload(wl)
    st = ctx.step(1)
    assert st.converged
    E, B = ctx.get_fields()
    rho, J, M, u = ctx.get_moments()
    parts = [ctx.get_particles(s) for s in range(len(wl.species))]
    counts = [ctx.species_count(s) for s in range(len(wl.species))]
    ctx.close()
    return dict(wl=wl, E=E, B=B, rho=rho, J=J, M=M, u=u, parts=parts, counts=counts)


def patch_inputs(S, i0, j0):
    """Oracle inputs for the SUB x SUB grid whose cell (MARGIN, MARGIN) is
    global cell (i0, j0)."""
    wl = S["wl"]
    nx, ny = wl.n[0], wl.n[1]
    dx, dy = wl.dx[0], wl.dx[1]
    gi = (np.arange(SUB) + i0 - MARGIN) % nx
    gj = (np.arange(SUB) + j0 - MARGIN) % ny
    Bsub = S["B"][:, :, gj][:, :, :, gi]
    usub = S["u"][:, :, gj][:, :, :, gi]
    species = []
    for s, p in zip(wl.species, S["parts"]):
        sx, sy = p["x"] / dx, p["y"] / dy
        cx, cy = np.floor(sx).astype(np.int64), np.floor(sy).astype(np.int64)
        rx, ry = (cx - i0) % nx, (cy - j0) % ny
        sel = (rx < PATCH) & (ry < PATCH)
        x = (rx[sel] + MARGIN + (sx[sel] - cx[sel])) * dx
        y = (ry[sel] + MARGIN + (sy[sel] - cy[sel])) * dy
        species.append(dict(q=s["q"], m=s["m"], x=x, y=y, z=np.zeros(x.size),
                            vx=p["vx"][sel], vy=p["vy"][sel], vz=p["vz"][sel], w=p["w"][sel]))
    cfg = O.make_cfg((SUB, SUB, 1), wl.dx, **wl.grid_kwargs())
    return cfg, Bsub, usub, species, gi, gj


@pytest.mark.parametrize("where", ["interior", "centre", "periodic corner"])
def test_sampled_patch_moments_match_oracle(state, where):
    S = state
    wl = S["wl"]
    nx, ny = wl.n[0], wl.n[1]
    i0, j0 = {"interior": (nx // 5, ny // 4 - 4), "centre": (nx // 2 - 16, ny // 2 - 4),
              "periodic corner": (nx - 4, ny - 4)}[where]
    cfg, Bsub, usub, species, gi, gj = patch_inputs(S, i0, j0)
    assert sum(sp["x"].size for sp in species) > 8 * 8 * 100       # the patch is populated
    pl = O.Plasma.from_species(species)
    Bn = O.node_avg(cfg, Bsub)
    rho_o, J_o, M_o = O.deposit(cfg, pl, Bn, u=usub if wl.comoving else None)
    J_o = O.smooth_current(cfg, J_o, wl.ns_j)
    # nodes whose four cells lie in the patch; one node less on each side for
    # the smoothed current
    a = slice(MARGIN + 1, MARGIN + PATCH)
    b = slice(MARGIN + 1 + wl.ns_j, MARGIN + PATCH - wl.ns_j)
    rho_g = S["rho"][0][np.ix_(gj[a], gi[a])]
    M_g = S["M"][0][np.ix_(gj[a], gi[a])]
    J_g = np.stack([S["J"][k, 0][np.ix_(gj[b], gi[b])] for k in range(3)])
    assert rel(rho_g, rho_o[0][a, a]) <= TOL_MOM, rel(rho_g, rho_o[0][a, a])
    assert rel(M_g, M_o[0][a, a]) <= TOL_MOM, rel(M_g, M_o[0][a, a])
    assert rel(J_g, J_o[:, 0][:, b, b]) <= TOL_MOM, rel(J_g, J_o[:, 0][:, b, b])


def test_fullsize_conservation(state):
    S = state
    wl = S["wl"]
    for s, n in zip(wl.species, S["counts"]):
        assert n == s["x"].size                                         # no particle lost
    q_tot = sum(s["q"] * np.sum(np.asarray(s["w"], np.float64)) for s in wl.species)
    dV = wl.dx[0] * wl.dx[1] * wl.dx[2]
    q_grid = float(np.sum(S["rho"])) * dV
    scale = sum(abs(s["q"]) * np.sum(np.asarray(s["w"], np.float64)) for s in wl.species)
    assert abs(q_grid - q_tot) <= 1e-6 * scale, (q_grid, q_tot)
    assert np.all(np.isfinite(S["E"])) and np.all(np.isfinite(S["B"]))


def test_fullsize_shock_step_matches_oracle():
    """The benchmark's shock-shaped plasma at full size (the quasi-parallel shock
    on 940 x 8 cells, 256 particles per cell and species, 3.85 M particles, open
    boundaries): one step through the C ABI against one oracle step with the same
    boundary refill.  The oracle runs this whole step in seconds, so E and B are
    compared everywhere (relative L2 <= 1e-6, the one-step field tolerance) and
    the particle counts per species exactly."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    wl = workloads.shock_1d("parallel", ny=8, ppc=256)
    bc = wl.notes["bc"]
    ctx = g.from_workload(wl, gmres_tol=1e-12)
    st = ctx.step(1)
    assert st.converged == 1
    E1, B1 = ctx.get_fields()
    counts = [ctx.species_count(s) for s in range(2)]
    ctx.close()
    cfg = O.make_cfg(wl.n, wl.dx, bc_cells=bc["cells"], **wl.grid_kwargs())
    cfg.gmres_tol = 1e-12
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    assert O.step(cfg, pl, E, B)["rc"] == 0
    pl = O.refill_boundaries(cfg, pl, bc["sources"], 1, bc["seed"])
    errs = {"E": rel(E1, E), "B": rel(B1, B)}
    assert all(v <= 1e-6 for v in errs.values()), errs
    assert counts == [int((pl.sp == s).sum()) for s in range(2)]
