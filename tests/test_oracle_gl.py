"""Pins of the oracle's Gauss's-law position correction (the GL of GL-ECSIM; the
paper cites the method without an equation, so the oracle follows a stated
reading: one steepest-descent step on F = (dV / 2) sum_c R_c^2, R_c the Gauss
residual (div_C E) / (4 pi) - rhobar of cell c):

* the displacement is exactly -gamma eps dF/dx_p, checked against central
  differences of F (F is quadratic in a particle's position inside its cell),
  with eps = 1 / (Q2 sum_d 4 / dx_d^2), Q2 = sum_p q_p^2 / V;
* no displacement where Gauss's law holds (a neutral plasma of coincident
  pairs in E = 0);
* one particle in a 1D box: the hand-computed displacement;
* repeated steps decrease F monotonically for gamma <= 1, and a step keeps the
  total charge.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads


def plasma(n, dx, ppc, seed=4):
    wl = workloads.uniform_drift(n=n, dx=dx, ppc=ppc, seed=seed)
    rng = np.random.default_rng(seed)
    for s in wl.species:      # a non-uniform density so that the residual has structure
        L = np.array([n[d] * dx[d] for d in range(3)])
        s["x"] = (s["x"] + 0.3 * L[0] * rng.random(len(s["x"])) ** 3) % L[0]
    return wl


def eps_of(cfg, pl):
    V = cfg.n[0] * cfg.n[1] * cfg.n[2] * cfg.dx[0] * cfg.dx[1] * cfg.dx[2]
    Q2 = float(np.sum((pl.q[pl.sp] * pl.w) ** 2)) / V
    lap = sum(4.0 / cfg.dx[d] ** 2 for d in range(3) if cfg.n[d] > 1)
    return 1.0 / (Q2 * lap)


@pytest.mark.parametrize("dims", [((10, 8, 1), (0.1, 0.1, 1.0)), ((6, 5, 4), (0.1, 0.12, 0.08))])
def test_displacement_is_steepest_descent(dims):
    n, dx = dims
    wl = plasma(n, dx, ppc=6)
    cfg = O.make_cfg(n, dx)
    pl = O.Plasma.from_species(wl.species)
    E = 0.02 * np.random.default_rng(9).standard_normal((3,) + cfg.shape)
    gamma = 0.7
    gx_, gy_, gz_, F0 = O.gl_displacement(cfg, pl, E, gamma)
    ge = gamma * eps_of(cfg, pl)
    keys = ("x", "y", "z")
    disp = (gx_, gy_, gz_)
    rng = np.random.default_rng(1)
    checked = 0
    for p in rng.choice(pl.np, 12, replace=False):
        for d in range(3):
            if cfg.n[d] == 1:
                assert disp[d][p] == 0.0
                continue
            arr = getattr(pl, keys[d])
            f = arr[p] / cfg.dx[d] - math.floor(arr[p] / cfg.dx[d])
            if f < 1e-3 or f > 1 - 1e-3:
                continue
            h = 1e-5 * cfg.dx[d]
            Fs = []
            for sgn in (1, -1):
                q = pl.copy()
                getattr(q, keys[d])[p] += sgn * h
                Fs.append(O.gl_displacement(cfg, q, E, gamma)[3])
            dF = (Fs[0] - Fs[1]) / (2 * h)
            assert disp[d][p] == pytest.approx(-ge * dF, rel=1e-6, abs=1e-12 * cfg.dx[d]), (p, d)
            checked += 1
    assert checked >= 12


def test_no_displacement_where_gauss_holds():
    cfg = O.make_cfg((8, 6, 1), (0.1, 0.1, 1.0))
    rng = np.random.default_rng(3)
    m = 40
    x, y = rng.random(m) * 0.8, rng.random(m) * 0.6
    w = rng.random(m) + 0.5
    # electron and ion of each pair consecutive: every node's running charge returns to exactly 0
    sp = np.tile([0, 1], m).astype(np.int32)
    rep = lambda a: np.repeat(a, 2)
    z = np.zeros(2 * m)
    pl = O.Plasma([-1.0, 1.0], [0.04, 1.0], sp, rep(x), rep(y), z, z, z, z, rep(w))
    d = O.gl_displacement(cfg, pl, np.zeros((3,) + cfg.shape), 1.0)
    assert d[3] == 0.0
    assert all(np.all(v == 0.0) for v in d[:3])


def test_single_particle_hand_value():
    # 1D, 6 cells of width h, one unit charge at 0.25 h, E = 0.  rho = (0.75, 0.25)/h on
    # nodes 0, 1; cell means rhobar_5 = 0.375/h, rhobar_0 = 0.5/h, rhobar_1 = 0.125/h; R = -rhobar;
    # phi_0 = (R_5 + R_0)/2 = -0.4375/h, phi_1 = (R_0 + R_1)/2 = -0.3125/h, grad phi = 0.125/h^2;
    # Q2 = 1/(6 h), eps = 1/(Q2 4/h^2) = 1.5 h^3, so dx = gamma 1.5 h^3 0.125/h^2 = 0.1875 gamma h
    # (toward the middle of the cell, where the charge's footprint is most even).
    h = 0.05
    cfg = O.make_cfg((6, 1, 1), (h, 1.0, 1.0))
    pl = O.Plasma([1.0], [1.0], [0], [0.25 * h], [0.0], [0.0], [0.0], [0.0], [0.0], [1.0])
    for gamma in (1.0, 0.4):
        dx, dy, dz, F = O.gl_displacement(cfg, pl, np.zeros((3,) + cfg.shape), gamma)
        assert dx[0] == pytest.approx(0.1875 * gamma * h, rel=1e-13)
        assert dy[0] == 0.0 and dz[0] == 0.0
    # F = (h/2) sum_c R_c^2 = (h/2) (0.375^2 + 0.5^2 + 0.125^2) / h^2
    assert F == pytest.approx(0.5 * (0.375 ** 2 + 0.5 ** 2 + 0.125 ** 2) / h, rel=1e-13)


@pytest.mark.parametrize("gamma", [0.25, 0.5, 1.0])
def test_repeated_steps_decrease_the_residual(gamma):
    n, dx = (12, 10, 1), (0.1, 0.1, 1.0)
    wl = plasma(n, dx, ppc=8, seed=6)
    cfg = O.make_cfg(n, dx)
    pl = O.Plasma.from_species(wl.species)
    E = 0.05 * np.random.default_rng(2).standard_normal((3,) + cfg.shape)
    L = [n[d] * dx[d] for d in range(3)]
    Fs = []
    for _ in range(6):
        d = O.gl_displacement(cfg, pl, E, gamma)
        Fs.append(d[3])
        pl.x = (pl.x + d[0]) % L[0]
        pl.y = (pl.y + d[1]) % L[1]
    assert all(b < a for a, b in zip(Fs[:-1], Fs[1:])), Fs
    assert Fs[-1] < 0.9 * Fs[0]


def test_step_with_correction_adds_the_displacement_and_keeps_charge():
    wl = plasma((10, 8, 1), (0.1, 0.1, 1.0), ppc=6)
    cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
    cfg_gl = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs(), gl_gamma=0.5)
    pl0 = O.Plasma.from_species(wl.species)
    d = O.gl_displacement(cfg, pl0, wl.E0, 0.5)
    res = {}
    for key, c in (("plain", cfg), ("gl", cfg_gl)):
        pl = pl0.copy()
        E, B = wl.E0.copy(), wl.B0.copy()
        assert O.step(c, pl, E, B)["rc"] == 0
        res[key] = pl
    L = [wl.n[k] * wl.dx[k] for k in range(3)]
    for key, k in (("x", 0), ("y", 1)):
        diff = (getattr(res["gl"], key) - getattr(res["plain"], key) - d[k] + 0.5 * L[k]) % L[k] - 0.5 * L[k]
        assert np.abs(diff).max() < 1e-12
    Bn = O.node_avg(cfg, wl.B0)
    q = [O.deposit(cfg, res[k], Bn)[0].sum() for k in ("plain", "gl")]
    assert q[1] == pytest.approx(q[0], rel=1e-12, abs=1e-12)
