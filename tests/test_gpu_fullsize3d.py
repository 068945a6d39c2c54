"""Parity of the 3D path at the benchmark's full size: the 128^3 periodic
drifting plasma with 64 particles per cell and species (268 M particles, drawn
on the device), one step through the C ABI in the configuration bench.py
times.

The oracle cannot run this step in seconds, so the check is on sampled
outputs, as in 2D: the particles the GPU holds in a 6^3-cell patch after the
step (selected on the device) are deposited by the oracle on a 10^3-cell grid
that contains the patch, with the GPU's B^{n+1} and smoothed bulk velocity u
around it, and the oracle's rho, 27-block mass matrix and comoving current are
compared with the GPU's at the nodes whose 8 cells lie inside the patch.  One
patch straddles the periodic corner.  Plus properties that hold at any size:
no particle is lost and the grid charge equals the particles' charge.
Tolerance: relative L2 <= 1e-5 (the stated bound for moments).
"""
import numpy as np
import pytest

import oracle as O
import workloads

pytestmark = pytest.mark.gpu

TOL_MOM = 1e-5
N, PPC = 128, 64
PATCH, MARGIN = 6, 2
SUB = PATCH + 2 * MARGIN
DX = 0.1


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def state():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    cfg = g.make_config((N, N, N), (DX, DX, DX), dt=0.02, comoving=1, lf_on=1, gmres_tol=1e-8, seed=2024)
    ctx = g.Context(cfg)
    u, B0 = (0.3, 0.0, 0.0), (0.0, 0.0, 0.1)
    species = [(-1.0, 1.0 / 25.0, 0.05), (1.0, 1.0, 0.01)]
    for q, m, vth in species:
        ctx.species_maxwellian(q, m, PPC, workloads.N0, u, vth)
    Em = -np.cross(np.asarray(u, np.float32).astype(np.float64), np.asarray(B0))
    E = np.empty((3, N, N, N))
    B = np.empty((3, N, N, N))
    for d in range(3):
        E[d], B[d] = Em[d], B0[d]
    ctx.fields_set(E, B)
    st = ctx.step(1)
    assert st.converged == 1
    E1, B1 = ctx.get_fields()
    rho, J, M, uu = ctx.get_moments()
    counts = [ctx.species_count(s) for s in range(2)]
    parts = []
    L = g.lib()
    for s in range(2):
        n = counts[s]
        dev = {k: torch.empty(n, dtype=torch.float64, device="cuda") for k in ("x", "y", "z")}
        dev.update({k: torch.empty(n, dtype=torch.float32, device="cuda") for k in ("vx", "vy", "vz", "w")})
        rc = L.gx_get_particles(ctx.h, s, *[dev[k].data_ptr() for k in ("x", "y", "z", "vx", "vy", "vz", "w")],
                                None, 1)
        assert rc == g.GX_OK
        parts.append(dev)
    ctx.close()
    return dict(torch=torch, species=species, E=E1, B=B1, rho=rho, J=J, M=M, u=uu, parts=parts, counts=counts)


def patch_species(S, c0):
    """The GPU's particles of the patch whose first cell is c0 = (i0, j0, k0),
    moved to the SUB^3 grid whose cell (MARGIN, MARGIN, MARGIN) is c0."""
    torch = S["torch"]
    out = []
    for (q, m, _), p in zip(S["species"], S["parts"]):
        sel = torch.ones_like(p["x"], dtype=torch.bool)
        pos = []
        for d, key in enumerate(("x", "y", "z")):
            s = p[key] / DX
            c = torch.floor(s)
            r = torch.remainder(c - c0[d], N)
            sel &= r < PATCH
            pos.append((r + MARGIN + (s - c)) * DX)
        sp = dict(q=q, m=m)
        for key, v in zip(("x", "y", "z"), pos):
            sp[key] = v[sel].cpu().numpy()
        for key in ("vx", "vy", "vz", "w"):
            sp[key] = p[key][sel].cpu().numpy()
        out.append(sp)
    return out


@pytest.mark.parametrize("where", ["interior", "periodic corner"])
def test_sampled_patch_moments_match_oracle_3d(state, where):
    S = state
    c0 = {"interior": (37, 70, 101), "periodic corner": (N - 3, N - 3, N - 3)}[where]
    species = patch_species(S, c0)
    assert sum(sp["x"].size for sp in species) > PPC * PATCH ** 3          # the patch is populated
    g = [(np.arange(SUB) + c0[d] - MARGIN) % N for d in range(3)]
    ix = np.ix_(g[2], g[1], g[0])
    Bsub = np.stack([S["B"][k][ix] for k in range(3)])
    usub = np.stack([S["u"][k][ix] for k in range(3)])
    cfg = O.make_cfg((SUB, SUB, SUB), (DX, DX, DX), dt=0.02, comoving=1, lf_on=1)
    pl = O.Plasma.from_species(species)
    Bn = O.node_avg(cfg, Bsub)
    rho_o, J_o, M_o = O.deposit(cfg, pl, Bn, u=usub)
    a = slice(MARGIN + 1, MARGIN + PATCH)          # nodes whose 8 cells lie in the patch
    ia = np.ix_(g[2][a], g[1][a], g[0][a])
    rho_g = S["rho"][ia]
    M_g = S["M"][ia]
    J_g = np.stack([S["J"][k][ia] for k in range(3)])
    assert rel(rho_g, rho_o[a, a, a]) <= TOL_MOM, rel(rho_g, rho_o[a, a, a])
    assert rel(M_g, M_o[a, a, a]) <= TOL_MOM, rel(M_g, M_o[a, a, a])
    assert rel(J_g, J_o[:, a, a, a]) <= TOL_MOM, rel(J_g, J_o[:, a, a, a])


def test_fullsize_conservation_3d(state):
    S = state
    assert S["counts"] == [PPC * N ** 3] * 2                               # no particle lost
    dV = DX ** 3
    w = workloads.N0 * dV / PPC                                             # every particle's weight
    q_tot = sum(q * float(p["w"].double().sum()) for (q, _, _), p in zip(S["species"], S["parts"]))
    q_grid = float(np.sum(S["rho"])) * dV
    scale = 2 * PPC * N ** 3 * w
    assert abs(q_grid - q_tot) <= 1e-6 * scale, (q_grid, q_tot)
    assert abs(float(S["parts"][0]["w"][0]) - w) <= 1e-7 * w
    assert np.all(np.isfinite(S["E"])) and np.all(np.isfinite(S["B"]))
