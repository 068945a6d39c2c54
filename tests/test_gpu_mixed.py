"""Mixed-precision FGMRES (gmres_mixed = 1): iterative refinement whose restarts
compute the true residual and update the solution in FP64 while the Arnoldi
cycles between them run from FP32 copies of the operator with an FP32 Krylov
basis (FP64 inner products).  The solve must end where the all-FP64 solve
ends: the reported relres is the FP64 true residual, at or below gmres_tol, and
the solution agrees with the FP64 solve to that tolerance (times the
operator's conditioning) and with the FP64 oracle's step within the parity
tolerance of the FP64 path.
"""
import numpy as np
import pytest

import oracle as O
import workloads

pytestmark = pytest.mark.gpu


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


def _sheared3():
    wl = workloads.uniform_drift(n=(12, 8, 10), dx=(0.1, 0.1, 0.1), ppc=8, ns_j=1, seed=3)
    nz, ny, nx = wl.B0.shape[1:]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    wl.B0[0] += 0.05 * np.sin(2 * np.pi * z / nz)
    wl.B0[2] += 0.03 * np.sin(2 * np.pi * (x / nx + y / ny))
    return wl


WORKLOADS = {
    "harris_64x32": lambda: workloads.harris(nx=64, ny=32, ppc=16, steps=1),
    "drift_lf_48x32": lambda: workloads.uniform_drift(n=(48, 32, 1), ppc=16, ns_j=1, u=(0.4, 0.1, 0.0)),
    "sheared3d_12x8x10": _sheared3,
}


@pytest.mark.parametrize("name", list(WORKLOADS))
@pytest.mark.parametrize("pc", ["none", "jacobi"])
@pytest.mark.parametrize("tol", [1e-8, 1e-12])
def test_mixed_solve_reaches_the_fp64_tolerance(gx, name, pc, tol):
    wl = WORKLOADS[name]()
    precond = {"none": gx.GX_PRECOND_NONE, "jacobi": gx.GX_PRECOND_JACOBI}[pc]
    sols, stats = {}, {}
    for mixed in (0, 1):
        ctx = gx.from_workload(wl, precond=precond, gmres_tol=tol, gmres_mixed=mixed)
        st = ctx.field_solve()
        sols[mixed], stats[mixed] = ctx.get_solution(), st
        ctx.close()
    print(name, pc, tol, "iterations FP64", stats[0].iters, "mixed", stats[1].iters, "relres", stats[1].relres)
    assert stats[1].converged == 1 and stats[1].relres <= tol
    # both iterates are within tol (relative residual) of the same solution
    assert rel(sols[1], sols[0]) <= 1e3 * tol
    assert stats[1].iters <= 3 * stats[0].iters + 2 * 50


@pytest.mark.parametrize("name", ["harris_64x32", "sheared3d_12x8x10"])
def test_mixed_step_matches_oracle(gx, name):
    wl = WORKLOADS[name]()
    ctx = gx.from_workload(wl, gmres_tol=1e-12, gmres_mixed=1)
    st = ctx.step(1)
    assert st.converged == 1
    E1, B1 = ctx.get_fields()
    ctx.close()
    cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
    cfg.gmres_tol = 1e-12
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    assert O.step(cfg, pl, E, B)["rc"] == 0
    assert rel(E1, E) <= 1e-6 and rel(B1, B) <= 1e-6


def test_mixed_steps_track_fp64_steps(gx):
    # ten steps of the Harris sheet: the mixed solve's fields stay with the FP64 solve's
    wl = workloads.harris(nx=64, ny=32, ppc=16, steps=10)
    out = {}
    for mixed in (0, 1):
        ctx = gx.from_workload(wl, gmres_tol=1e-10, gmres_mixed=mixed)
        ctx.step(10)
        out[mixed] = ctx.get_fields()
        ctx.close()
    assert rel(out[1][0], out[0][0]) < 1e-6 and rel(out[1][1], out[0][1]) < 1e-6
