"""Whole-step pins of the oracle (Sec. 1.1 and 2.1):

* plain ECSIM (theta = 0.5, no comoving current, no LF, no smoothing) conserves
  particle + field energy to the solver tolerance;
* with the comoving current the energy changes by exactly the work of the
  dropped current (a ledger that closes to the solver tolerance);
* Gauss consistency: with the E diffusion off, div(E^{n+1} - E^n) equals
  -4 pi dt div(Jbar) for the current the particles actually carry;
* a cold neutral beam in its own motional field is an exact equilibrium.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads


def small(**kw):
    base = dict(n=(10, 8, 1), ppc=6, gmres_tol=1e-13)
    base.update(kw)
    return workloads.uniform_drift(**base)


def _setup(wl):
    cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
    cfg.gmres_tol = 1e-13
    pl = O.Plasma.from_species(wl.species)
    return cfg, pl, wl.E0.copy(), wl.B0.copy()


@pytest.mark.parametrize("dim3", [False, True])
def test_plain_ecsim_conserves_energy(dim3):
    kw = dict(n=(5, 4, 3), dx=(0.1, 0.1, 0.1)) if dim3 else {}
    wl = small(comoving=0, lf_on=0, ns_j=0, theta=0.5, vth_e=0.2, vth_i=0.05, dt=0.05, **kw)
    cfg, pl, E, B = _setup(wl)
    W0 = O.energy(cfg, pl, E, B)["total"]
    for _ in range(4):
        r = O.step(cfg, pl, E, B)
        assert r["rc"] == 0
        W = O.energy(cfg, pl, E, B)["total"]
        assert abs(W - W0) / W0 < 1e-10
        W0 = W


def test_comoving_energy_ledger():
    # Energy change = dt dV sum_g (Jbar_particles - Jbar_solve) . E^{n+theta},
    # where Jbar_solve = J_C + M (E^{n+theta} - E_M) / dV is what the field saw
    # and Jbar_particles what the particles carry (Sec. 2.1, Eq. 33-35).
    wl = small(comoving=1, lf_on=0, ns_j=0, theta=0.5, vth_e=0.1, vth_i=0.02, dt=0.05)
    cfg, pl, E, B = _setup(wl)
    N = cfg.nn
    dV = cfg.dx[0] * cfg.dx[1] * cfg.dx[2]
    before = O.energy(cfg, pl, E, B)["total"]
    x0 = pl.copy()
    Bn = O.node_avg(cfg, B)
    r = O.step(cfg, pl, E, B, want=("Eth", "J", "M", "u", "vbar"))
    after = O.energy(cfg, pl, E, B)["total"]
    Eth, JC, M, u, vbar = r["Eth"], r["J"], r["M"], r["u"], r["vbar"]
    probe = O.Plasma(x0.q, x0.q, x0.sp, x0.x, x0.y, x0.z, vbar[:, 0], vbar[:, 1], vbar[:, 2], x0.w)
    _, Jp = O.bulk_moments(cfg, probe)
    Jp = Jp / dV
    EM = -np.cross(np.moveaxis(u, 0, -1), np.moveaxis(Bn, 0, -1)) / cfg.c
    EM = np.moveaxis(EM, -1, 0)
    from test_oracle_deposit import _neighbour_gather
    Mr = M.reshape(N, 27, 3, 3)
    MEc = np.einsum("goij,goj->gi", Mr, _neighbour_gather(cfg, Eth - EM)).T.reshape(3, *cfg.shape)
    Jsolve = JC + MEc / dV
    ledger = cfg.dt * dV * ((Jp - Jsolve) * Eth).sum()
    scale = abs(cfg.dt * dV * (Jp * Eth).sum()) + 1e-300
    assert abs((after - before) - ledger) < 1e-9 * max(scale, abs(after - before))
    assert abs(after - before) > 1e3 * abs((after - before) - ledger)   # the ledger is not trivially zero


def test_gauss_consistency_without_e_diffusion():
    wl = small(comoving=1, lf_on=0, ns_j=0, theta=0.6, vth_e=0.1, dt=0.05)
    cfg, pl, E, B = _setup(wl)
    dV = cfg.dx[0] * cfg.dx[1] * cfg.dx[2]
    # a non-trivial field so the plasma responds
    E = E + 0.01 * np.random.default_rng(2).standard_normal(E.shape)
    x0 = pl.copy()
    E0 = E.copy()
    r = O.step(cfg, pl, E, B, want=("vbar",))
    # comoving mode drops the net-charge current, so compare with what the
    # field equation used: Jbar_solve differs from the particle current by
    # a divergence we can compute -- use the standard mode instead for the
    # clean statement, below.
    wl2 = small(comoving=0, lf_on=0, ns_j=0, theta=0.6, vth_e=0.1, dt=0.05)
    cfg2, pl2, E2, B2 = _setup(wl2)
    E2 = E2 + 0.01 * np.random.default_rng(2).standard_normal(E2.shape)
    x2 = pl2.copy()
    E20 = E2.copy()
    r2 = O.step(cfg2, pl2, E2, B2, want=("vbar",))
    vb = r2["vbar"]
    probe = O.Plasma(x2.q, x2.q, x2.sp, x2.x, x2.y, x2.z, vb[:, 0], vb[:, 1], vb[:, 2], x2.w)
    _, Jp = O.bulk_moments(cfg2, probe)
    Jp /= dV
    lhs = O.div_C(cfg2, E2 - E20)
    rhs = -4 * math.pi * cfg2.dt * O.div_C(cfg2, Jp)
    assert np.abs(lhs - rhs).max() < 1e-9 * np.abs(rhs).max()


def test_cold_beam_is_exact_equilibrium_only_in_comoving_frame():
    # v = u for every particle and E = -u x B / c.  With random particle
    # positions the charge density is noisy, so the standard current carries the
    # net-charge transport rho_g u (Eq. 28, second term) and disturbs the field;
    # the comoving current drops exactly that term (Sec. 2.1), which makes the
    # beam an exact equilibrium.
    def run(cm):
        wl = small(comoving=cm, lf_on=1, ns_j=1, vth_e=0.0, vth_i=0.0, u=(0.3, 0.1, 0.0), B=(0.0, 0.05, 0.1))
        cfg, pl, E, B = _setup(wl)
        E0, B0, v0 = E.copy(), B.copy(), pl.vx.copy()
        O.step(cfg, pl, E, B)
        return np.abs(E - E0).max(), np.abs(B - B0).max(), np.abs(pl.vx - v0).max()

    dE, dB, dv = run(1)
    assert dE < 1e-13 and dB < 1e-14 and dv < 1e-13
    dE0, _, _ = run(0)
    assert dE0 > 1e-4 and dE0 > 1e5 * dE
