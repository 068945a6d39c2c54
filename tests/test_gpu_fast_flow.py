"""The paper's remaining 1D tests on the GPU path, against the oracle.

* Uniform fast flow (Sec. 3.2): a solar-wind plasma (400 km/s, 5 nT, m_i/m_e =
  100) in 20 periodic cells, converted to the package's normalised units
  (c dt / dx ~ 142).  Parity: E and B after two steps within 2e-6 relative of
  the oracle (the 1e-6 per-step field tolerance, once per step).  Behaviour, as
  the paper reports it: with the comoving current and one current filter pass
  the total particle momentum stays within 2e-3 of its start over 400 steps;
  with the standard current it drifts by more than 1 % (one filter pass) or
  decays at least ten times faster than with the comoving current (no filter;
  that run heats the electrons until the push reports a particle crossing
  more than one cell).  The oracle (FP64, same reading) shows 2.5e-4, 4 % and
  a 92 % loss on the same inputs.
* Top-hat light wave with the digital filter on E in place of the LF term on E
  (Sec. 3.1): 100 steps (t = 0.4) with one and with three filter passes,
  GPU within 1e-5 of the oracle (the filter sweeps are FP32 on the GPU: about
  1e-7 per step).
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


def test_fast_flow_two_steps_match_oracle(gx):
    wl = workloads.fast_flow_1d(comoving=1, ns_j=1)
    ctx = gx.from_workload(wl, gmres_tol=1e-12)
    for _ in range(2):
        st = ctx.step(1)
        assert st.converged == 1
    E1, B1 = ctx.get_fields()
    ctx.close()
    cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
    cfg.gmres_tol = 1e-12
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    for _ in range(2):
        assert O.step(cfg, pl, E, B)["rc"] == 0
    errs = {"E": rel(E1, E), "B": rel(B1, B)}
    assert all(v <= 2e-6 for v in errs.values()), errs


def _momentum_history(gx, comoving, ns_j, steps=400):
    """Relative change of the total particle x momentum every 10 steps, up to
    `steps` or until the push reports a particle moving more than one cell."""
    wl = workloads.fast_flow_1d(comoving=comoving, ns_j=ns_j)
    ctx = gx.from_workload(wl)
    p0 = ctx.diagnostics()["momentum"][0]
    hist, cfl_stop = [], False
    for _ in range(steps // 10):
        try:
            ctx.step(10)
        except gx.GxError as e:
            assert e.status == gx.GX_ECFL
            cfl_stop = True
            break
        hist.append(ctx.diagnostics()["momentum"][0] / p0 - 1.0)
    ctx.close()
    return np.array(hist), cfl_stop


def test_fast_flow_comoving_current_keeps_particle_momentum(gx):
    cm, stop = _momentum_history(gx, comoving=1, ns_j=1)
    assert not stop and len(cm) == 40
    assert np.abs(cm).max() < 2e-3, cm
    # standard current with one filter pass: a steady loss of the flow
    std1, stop1 = _momentum_history(gx, comoving=0, ns_j=1)
    assert np.abs(std1).max() > 1e-2, std1
    # standard current, no filter: the flow decays fast and heats the electrons
    # until one crosses more than a cell in a step (the binned push stops the
    # run with GX_ECFL; the FP64 oracle runs on and loses ~90 % of the momentum)
    std0, stop0 = _momentum_history(gx, comoving=0, ns_j=0)
    assert stop0 or std0[-1] < -0.3, std0
    assert abs(std0[3]) > 10 * np.abs(cm[:4]).max(), (std0, cm)


@pytest.mark.parametrize("npass", [1, 3])
def test_tophat_with_E_filter_matches_oracle(gx, npass):
    wl = workloads.tophat_1d(lf_on=1, lf_beta=1.0)
    steps = 100
    cfg = gx.make_config(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, comoving=0, lf_on=1, lf_speed_c=1,
                         lf_beta=1.0, gmres_tol=1e-13, nsmooth_e=npass)
    ctx = gx.Context(cfg)
    e, f = np.zeros(0), np.zeros(0, np.float32)
    ctx.species_add(-1.0, 0.04, e, e, e, f, f, f, f)
    ctx.fields_set(wl.E0, wl.B0)
    for _ in range(steps):
        ctx.step(1)
    E, B = ctx.get_fields()
    ctx.close()
    ocfg = O.make_cfg(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, lf_on=1, lf_speed_c=1, lf_beta=1.0,
                      gmres_tol=1e-13, nsmooth_u=0, nsmooth_e=npass)
    z = np.zeros(0)
    empty = O.Plasma([-1.0], [0.04], np.zeros(0, np.int32), z, z, z, z, z, z, z)
    Eo, Bo = wl.E0.copy(), wl.B0.copy()
    for _ in range(steps):
        assert O.step(ocfg, empty, Eo, Bo)["rc"] == 0
    assert rel(E, Eo) < 1e-5 and rel(B, Bo) < 1e-5, (rel(E, Eo), rel(B, Bo))
    # three passes smear the top-hat far more than one (Sec. 3.1): the range of
    # E_y stays ~1 with one pass and drops to ~0.8 with three (oracle: 1.0003, 0.795)
    if npass == 1:
        assert np.ptp(E[1]) > 0.99
    else:
        assert np.ptp(E[1]) < 0.85


def test_E_filter_with_plasma_matches_oracle(gx):
    """The E-field filter with particles: the 32 x 32 drifting plasma with
    nsmooth_e = 2 (and so no LF term on E), two steps against the oracle (fields
    within 2e-6, the per-step field tolerance once per step)."""
    wl = workloads.uniform_drift(n=(32, 32, 1), ppc=32, ns_j=1)
    cfg = gx.make_config(wl.n, wl.dx, c=wl.c, theta=wl.theta, dt=wl.dt, comoving=wl.comoving, lf_on=1,
                         lf_beta=wl.lf_beta, ns_j=wl.ns_j, nsmooth_u=wl.nsmooth_u, gmres_tol=1e-12, nsmooth_e=2)
    ctx = gx.Context(cfg)
    for sp in wl.species:
        ctx.species_add(sp["q"], sp["m"], sp["x"], sp["y"], sp["z"], sp["vx"], sp["vy"], sp["vz"], sp["w"])
    ctx.fields_set(wl.E0, wl.B0)
    for _ in range(2):
        assert ctx.step(1).converged == 1
    E1, B1 = ctx.get_fields()
    ctx.close()
    ocfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
    ocfg.gmres_tol, ocfg.nsmooth_e = 1e-12, 2
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    for _ in range(2):
        assert O.step(ocfg, pl, E, B)["rc"] == 0
    errs = {"E": rel(E1, E), "B": rel(B1, B)}
    assert all(v <= 2e-6 for v in errs.values()), errs
