"""Pins of the oracle's open x boundaries (the shock runs of Sec. 3.3; the paper
prints the two plasma states, not the boundary treatment, so the treatment is
a reading: boundary cells held at a fixed state and refilled after every push).

  * the counter-based generator is Philox4x64-10 exactly as numpy implements it
    (numpy advances its counter before the first block, so numpy's stream from
    counter c - 1 is the oracle's block at c), including the carry across words;
  * the refill draws are uniform inside their cell and Maxwellian with the
    source's bulk velocity and thermal speed (moments within sampling error);
  * E at boundary nodes and B in boundary cells do not change over steps, while
    the interior evolves;
  * the Dirichlet rows act locally: a vacuum pulse far from the boundaries
    evolves as in the periodic box to 1e-12 in the middle of the domain;
  * after a refill every boundary cell holds exactly ppc particles of each
    species, and interior particles are untouched.
"""
import numpy as np
import pytest

import oracle as O
import workloads


@pytest.mark.parametrize("key,ctr", [
    ((0, 0), (1, 0, 0, 0)),
    ((0x1234567890ABCDEF, 0x0FEDCBA987654321), (7, 3, 2**63 + 5, 11)),
    ((2**64 - 1, 42), (0, 1, 0, 0)),                 # numpy's c - 1 wraps word 0: a carry into word 1
    ((99, 1), (123456789, 2**40 + 17, 5, 2**64 - 1)),
])
def test_philox_matches_numpy(key, ctr):
    prev = list(ctr)
    i = 0
    while prev[i] == 0:                               # prev = ctr - 1 with borrow
        prev[i] = 2**64 - 1
        i += 1
    prev[i] -= 1
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    assert O.philox4x64(key, ctr) == [int(v) for v in g.random_raw(4)]


def test_refill_draws_are_uniform_and_maxwellian():
    cfg = O.make_cfg((40, 1, 1), (0.4, 1.0, 1.0), bc_cells=8)
    u, vth = (0.1, -0.05, 0.02), 0.07
    xs, vs = [], []
    for step in range(1, 6):
        for i in (0, 3, 39):
            x, y, vx, vy, vz = O.bc_sample(cfg, 2024, 1, step, i, 0, 500, u, vth)
            off = x / 0.4 - i
            assert np.all((off >= 0) & (off < 1)) and np.all(y == 0)
            xs.append(off)
            vs.append(np.stack([vx, vy, vz]))
    off = np.concatenate(xs)
    v = np.concatenate(vs, axis=1)
    n = off.size
    assert abs(off.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    for d in range(3):
        assert abs(v[d].mean() - u[d]) < 4 * vth / np.sqrt(n)
        assert abs(v[d].std() / vth - 1) < 4 / np.sqrt(2 * n)
    # different species or steps draw different particles
    a = O.bc_sample(cfg, 2024, 0, 1, 0, 0, 8, u, vth)[2]
    b = O.bc_sample(cfg, 2024, 1, 1, 0, 0, 8, u, vth)[2]
    c = O.bc_sample(cfg, 2024, 0, 2, 0, 0, 8, u, vth)[2]
    assert not np.allclose(a, b) and not np.allclose(a, c)


def _small_shock(**kw):
    return workloads.shock_1d(dx=0.4, length=48.0, ppc=16, **kw)


def test_boundary_fields_stay_and_refill_counts():
    wl = _small_shock()
    bc = wl.notes["bc"]
    G, nx = bc["cells"], wl.n[0]
    cfg = O.make_cfg(wl.n, wl.dx, bc_cells=G, **wl.grid_kwargs())
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    bn = np.r_[0:G, nx - G + 1:nx]
    bcl = np.r_[0:G, nx - G:nx]
    for step in range(1, 4):
        r = O.step(cfg, pl, E, B)
        assert r["rc"] == 0
        ci = np.floor(pl.x / wl.dx[0]).astype(int) % nx
        inner = (ci >= G) & (ci < nx - G)
        kept = {k: getattr(pl, k)[inner].copy() for k in ("x", "vx", "w")}
        pl = O.refill_boundaries(cfg, pl, bc["sources"], step, bc["seed"])
        ci = np.floor(pl.x / wl.dx[0]).astype(int) % nx
        for s in range(2):
            counts = np.bincount(ci[pl.sp == s], minlength=nx)
            assert np.all(counts[bcl] == bc["sources"][0][s]["ppc"])
        inner = (ci >= G) & (ci < nx - G)
        for k, v in kept.items():
            assert np.array_equal(getattr(pl, k)[inner], v)
    E0, B0 = wl.E0.reshape(3, -1), wl.B0.reshape(3, -1)
    assert np.array_equal(E.reshape(3, -1)[:, bn], E0[:, bn])
    assert np.array_equal(B.reshape(3, -1)[:, bcl], B0[:, bcl])
    mid = slice(G + 2, nx - G - 2)
    assert np.abs(B.reshape(3, -1)[:, mid] - B0[:, mid]).max() > 1e-6     # the interior evolves


def test_dirichlet_rows_act_locally():
    n, dx, c = 120, 0.02, 1.0
    dt = 0.4 * dx / c
    B = np.zeros((3, 1, 1, n))
    E = np.zeros((3, 1, 1, n))
    B[2, 0, 0, 55:65] = 1.0
    E[1, 0, 0, 55:66] = 1.0
    e = np.zeros(0)
    empty = O.Plasma([-1.0], [1.0], np.zeros(0, np.int32), e, e, e, e, e, e, e)
    res = {}
    for G in (0, 8):
        cfg = O.make_cfg((n, 1, 1), (dx, 1.0, 1.0), c=c, dt=dt, lf_on=1, lf_speed_c=1, lf_beta=1.0,
                         gmres_tol=1e-14, nsmooth_u=0, bc_cells=G)
        Ek, Bk = E.copy(), B.copy()
        for _ in range(5):
            assert O.step(cfg, empty, Ek, Bk)["rc"] == 0
        res[G] = (Ek, Bk)
    mid = slice(40, 80)
    assert np.abs(res[8][0][..., mid] - res[0][0][..., mid]).max() <= 1e-12
    assert np.abs(res[8][1][..., mid] - res[0][1][..., mid]).max() <= 1e-12


def test_wall_reflects_specularly():
    """With no fields the mover moves a particle in a straight line (alpha = I);
    one crossing the wall face x_w = (nx - G) dx comes back at 2 x_w - x with
    v_x reversed, exactly, and the others are untouched."""
    nx, G, dx, dt = 40, 8, 0.1, 0.05
    cfg = O.make_cfg((nx, 1, 1), (dx, 1.0, 1.0), dt=dt, bc_cells=G, bc_wall=1)
    xw = (nx - G) * dx
    x0 = np.array([xw - 0.01, xw - 0.05, 1.0, xw - 0.002])
    vx0 = np.array([0.8, -0.3, 0.5, 0.05])
    z = np.zeros(4)
    pl = O.Plasma([1.0], [1.0], np.zeros(4, np.int32), x0.copy(), z.copy(), z.copy(), vx0.copy(),
                  np.full(4, 0.1), z.copy(), np.ones(4))
    O.mover(cfg, pl, np.zeros((3, 1, 1, nx)), np.zeros((3, 1, 1, nx)))
    moved = x0 + dt * vx0
    refl = moved >= xw
    assert refl.tolist() == [True, False, False, True]
    assert np.array_equal(pl.x, np.where(refl, 2 * xw - moved, moved))
    assert np.array_equal(pl.vx, np.where(refl, -vx0, vx0))
    assert np.array_equal(pl.vy, np.full(4, 0.1))


def test_wall_region_stays_empty_and_field_free():
    wl = workloads.shock_wall(nx=96, ny=1, ppc=16, steps=4)
    bc = wl.notes["bc"]
    G, nx = bc["cells"], wl.n[0]
    cfg = O.make_cfg(wl.n, wl.dx, bc_cells=G, bc_wall=1, **wl.grid_kwargs())
    pl = O.Plasma.from_species(wl.species)
    E, B = wl.E0.copy(), wl.B0.copy()
    n_in = pl.np
    for step in range(1, 5):
        assert O.step(cfg, pl, E, B)["rc"] == 0
        ci = np.floor(pl.x / wl.dx[0]).astype(int) % nx
        assert not np.any(ci >= nx - G)                        # nothing crosses the wall
        assert pl.np == n_in                                   # nor leaves through it
        pl = O.refill_boundaries(cfg, pl, bc["sources"], step, bc["seed"])
        n_in = pl.np
    Ew = E.reshape(3, -1)[:, nx - G:]
    assert np.all(Ew == 0.0)                                   # the conductor holds E = 0 from its face on
    assert np.array_equal(B.reshape(3, -1)[:, nx - G:], wl.B0.reshape(3, -1)[:, nx - G:])
