"""Cell bins at their limits (the cell sort of the hot path, through the C ABI).

Particles with negligible weight (so that the fields stay ~0 and the motion is
ballistic to FP32 accuracy) in a converging flow v_x = -a (x - x_c):
  * a slow convergence raises the largest cell count step by step; the bins
    must grow before they overflow (a step that leaves a bin above 90 % grows
    it), no particle is lost and every particle ends where ballistic motion
    puts it (matched by id; tolerance 1e-5 of a cell after the steps);
  * a convergence that packs about 73 particles into 64-slot bins within a
    single push must be reported as GX_EOVERFLOW (particles lost, said so) and
    leave the context usable.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as gx
    gx.lib()
    return gx


def converging(g, nx, ny, ppc, a_cells_per_step, slack, seed=1):
    dx, dt = 0.1, 0.01
    cfg = g.make_config((nx, ny, 1), (dx, dx, 1.0), dt=dt, comoving=0, lf_on=0, ns_j=0, track_ids=1,
                        bin_slack=slack, gmres_tol=1e-10)
    ctx = g.Context(cfg)
    rng = np.random.default_rng(seed)
    n = nx * ny * ppc
    cx = np.repeat(np.arange(nx * ny) % nx, ppc)
    cy = np.repeat(np.arange(nx * ny) // nx, ppc)
    x = (cx + rng.random(n)) * dx
    y = (cy + rng.random(n)) * dx
    xc = 0.5 * nx * dx
    # a_cells_per_step: relative compression per step of the x coordinate
    vx = (-(a_cells_per_step / dt) * (x - xc)).astype(np.float32)
    zero = np.zeros(n, np.float32)
    w = np.full(n, 1e-12, np.float32)
    ctx.species_add(1.0, 1.0, x, y, np.zeros(n), vx, zero, zero, w)
    ctx.fields_set(np.zeros((3, 1, ny, nx)), np.zeros((3, 1, ny, nx)))
    return ctx, x, y, vx, dt, dx


def test_bins_grow_before_they_overflow(g):
    nx, ny, ppc, steps = 32, 4, 40, 12
    ctx, x0, y0, vx, dt, dx = converging(g, nx, ny, ppc, a_cells_per_step=0.03, slack=1.2)
    try:
        for _ in range(steps):
            ctx.step(1)
        p = ctx.get_particles(0, ids=True)
        assert len(p["id"]) == x0.size                        # nothing lost
        idx = p["id"]
        L = nx * dx
        xe = (x0[idx] + steps * dt * vx[idx].astype(np.float64)) % L
        d = (p["x"] - xe + 0.5 * L) % L - 0.5 * L
        assert np.abs(d).max() <= 1e-5 * dx * steps
        assert np.allclose(p["y"], y0[idx], atol=1e-6 * dx)
        # the flow did pile particles up beyond the initial capacity's 90 %
        counts = np.bincount((p["x"] // dx).astype(int) % nx, minlength=nx) / ny
        assert counts.max() > 0.9 * 64
    finally:
        ctx.close()


def test_overflow_in_one_push_is_reported(g):
    nx, ny, ppc = 4, 2, 40
    # the x extent shrinks by 45 % in one step (the outermost particles move
    # 0.9 cell): 40 particles per cell become about 73, over the 64-slot bins
    ctx, x0, y0, vx, dt, dx = converging(g, nx, ny, ppc, a_cells_per_step=0.45, slack=1.2)
    try:
        with pytest.raises(g.GxError) as e:
            for _ in range(4):
                ctx.step(1)
        assert e.value.status == g.GX_EOVERFLOW
        assert "overflow" in str(e.value)
        # still usable: diagnostics and field read-back work
        d = ctx.diagnostics()
        assert np.isfinite(d["energy_E"])
        ctx.get_fields()
    finally:
        ctx.close()
