"""Failure paths of the C ABI on the GPU: statuses come back, nothing crashes,
and the context stays usable afterwards.

  * a solve cut off by gmres_maxit returns GX_ENOCONV and keeps its best
    iterate: after one Arnoldi step that is the one-step GMRES minimiser
    x0 + t r0, which the FP64 oracle's GMRES computes independently (E^{n+theta}
    within the 1e-6 relative field tolerance: both sides assemble the operator
    from the same particles, the GPU from FP32 deposit sums);
  * NaN or infinite values in host arrays passed to gx_fields_set and
    gx_species_add are refused with GX_EINVAL, and the state is left as it was;
  * a right-hand side of zero gives the exact solution 0 with no iteration.
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


def _ctx(gx, wl, **kw):
    cfg = gx.make_config(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, comoving=wl.comoving, lf_on=wl.lf_on,
                         lf_speed_c=wl.lf_speed_c, lf_beta=wl.lf_beta, ns_j=wl.ns_j, nsmooth_u=wl.nsmooth_u, **kw)
    ctx = gx.Context(cfg)
    for s in wl.species:
        ctx.species_add(s["q"], s["m"], np.ascontiguousarray(s["x"]), np.ascontiguousarray(s["y"]),
                        np.ascontiguousarray(s["z"]), np.ascontiguousarray(s["vx"], np.float32),
                        np.ascontiguousarray(s["vy"], np.float32), np.ascontiguousarray(s["vz"], np.float32),
                        np.ascontiguousarray(s["w"], np.float32))
    ctx.fields_set(np.ascontiguousarray(wl.E0), np.ascontiguousarray(wl.B0))
    return ctx


def test_gmres_maxit_returns_noconv_with_the_best_iterate(gx):
    wl = workloads.uniform_drift(n=(24, 16, 1), ppc=16, ns_j=1)
    ctx = _ctx(gx, wl, gmres_maxit=1, gmres_tol=1e-12)
    try:
        rc = gx.lib().gx_field_solve(ctx.h, None, gx.C.byref(st := gx.SolveStats()))
        assert rc == gx.GX_ENOCONV
        assert "best iterate kept" in gx.lib().gx_last_error(ctx.h).decode()
        assert st.converged == 0 and st.iters == 1 and st.relres > 1e-12
        Eth = ctx.get_solution()

        cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
        cfg.gmres_tol, cfg.gmres_maxit = 1e-12, 1
        pl = O.Plasma.from_species(wl.species)
        E, B = wl.E0.copy(), wl.B0.copy()
        r = O.step(cfg, pl, E, B, want=("Eth",))
        assert r["rc"] == 1 and r["iters"] == 1
        assert rel(Eth, r["Eth"]) < 1e-6
        assert st.relres == pytest.approx(r["relres"], rel=1e-4)
        # the one-step correction is real: the iterate moved away from E^n
        assert rel(Eth, wl.E0) > 1e-6

        # the context stays usable: the push follows, and so does the next solve
        ctx.push_and_deposit()
        st2 = ctx.field_solve(allow_noconv=True)
        assert st2.iters == 1 and st2.converged == 0
        ctx.push_and_deposit()
        d = ctx.diagnostics()
        assert np.isfinite(d["total"]) and d["n_particles"] == sum(len(s["x"]) for s in wl.species)
    finally:
        ctx.close()


def test_nonfinite_inputs_are_refused_and_leave_the_state(gx):
    wl = workloads.uniform_drift(n=(16, 8, 1), ppc=8)
    ctx = _ctx(gx, wl)
    try:
        E0, B0 = ctx.get_fields()
        for bad in (np.nan, np.inf, -np.inf):
            E = E0.copy()
            E[1, 0, 3, 5] = bad
            with pytest.raises(gx.GxError) as e:
                ctx.fields_set(E, B0)
            assert e.value.status == gx.GX_EINVAL and "not finite" in str(e.value)
            B = B0.copy()
            B[2, 0, 7, 1] = bad
            with pytest.raises(gx.GxError) as e:
                ctx.fields_set(None, B)
            assert e.value.status == gx.GX_EINVAL
        E1, B1 = ctx.get_fields()
        assert np.array_equal(E1, E0) and np.array_equal(B1, B0)

        s = wl.species[0]
        n = len(s["x"])
        arrays = [np.ascontiguousarray(s[k], np.float64 if k in "xyz" else np.float32)
                  for k in ("x", "y", "z", "vx", "vy", "vz", "w")]
        for k, bad in [(0, np.nan), (1, np.inf), (3, np.nan), (5, -np.inf), (6, np.nan)]:
            a = [v.copy() for v in arrays]
            a[k][n // 2] = bad
            with pytest.raises(gx.GxError) as e:
                ctx.species_add(s["q"], s["m"], *a)
            assert e.value.status == gx.GX_EINVAL and "not finite" in str(e.value)
        # nothing was added; a clean species is still accepted
        assert ctx.species_count(2) == -1
        sid = ctx.species_add(s["q"], s["m"], *arrays)
        assert sid == 2 and ctx.species_count(2) == n
        st = ctx.step(1)
        assert st.converged == 1
    finally:
        ctx.close()


def test_zero_right_hand_side_gives_exactly_zero(gx):
    # vacuum, zero fields: b = 0, and the solve returns E^{n+theta} = 0 at once
    cfg = gx.make_config((32, 16, 1), (0.1, 0.1, 1.0), comoving=0, lf_on=1, lf_speed_c=1)
    ctx = gx.Context(cfg)
    try:
        z = np.zeros((3, 1, 16, 32))
        ctx.fields_set(z, z)
        st = ctx.field_solve()
        assert st.converged == 1 and st.iters == 0 and st.relres == 0.0
        assert not np.any(ctx.get_solution())
    finally:
        ctx.close()
