"""Pins of the oracle's particle-to-grid moments (Sec. 2.1, Eq. 27-35):
hand-computed one- and two-particle mass matrices, symmetry, partition of unity,
the predicted-current identity against the mover's own vbar (through a
different oracle routine), the motional-field identity inside the deposit, the
cold-beam comoving current, and charge conservation of the deposit."""
import math

import numpy as np
import pytest

import oracle as O
import workloads


def offset(ox, oy, oz=0):
    return (ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)


def test_single_particle_on_node_hand_values():
    # A particle exactly on node (2,3): W = 1 there and 0 elsewhere, so
    # M_gg = beta q alpha and no other block; rho = q / dV.
    q, m, dt, c = -1.0, 0.04, 0.02, 1.0
    cfg = O.make_cfg((6, 5, 1), (0.125, 0.25, 1.0), dt=dt, c=c)
    pl = O.Plasma([q], [m], [0], [0.25], [0.75], [0.0], [0.01], [0.02], [0.0], [2.5])
    Bc = np.zeros((3,) + cfg.shape)
    Bc[2] = 0.3
    Bc[0] = -0.1
    Bn = O.node_avg(cfg, Bc)
    rho, J, M = O.deposit(cfg, pl, Bn)
    beta = q * dt / (2 * m)
    al = O.alpha(beta * np.array([-0.1, 0.0, 0.3]) / c)
    dV = 0.125 * 0.25 * 1.0
    assert rho[0, 3, 2] == pytest.approx(q * 2.5 / dV, rel=1e-14)
    assert np.count_nonzero(rho) == 1
    assert np.allclose(M[0, 3, 2, offset(0, 0)], beta * q * 2.5 * al, rtol=1e-14, atol=0)
    Mz = M.copy()
    Mz[0, 3, 2, offset(0, 0)] = 0
    assert np.abs(Mz).max() == 0.0
    assert np.allclose(J[:, 0, 3, 2], q * 2.5 * al @ np.array([0.01, 0.02, 0.0]) / dV, rtol=1e-14)


def test_particle_at_cell_centre_quarter_weights():
    # At the centre of cell (1,1) every corner weight is 1/4, so each of the 16
    # ordered corner pairs gets beta q alpha / 16 and rho = q/(4 dV) on 4 nodes.
    q, m, dt = 1.0, 1.0, 0.1
    cfg = O.make_cfg((4, 4, 1), (1.0, 1.0, 1.0), dt=dt)
    pl = O.Plasma([q], [m], [0], [1.5], [1.5], [0.0], [0.0], [0.0], [0.0], [1.0])
    Bn = np.zeros((3,) + cfg.shape)
    Bn[2] = 2.0
    rho, J, M = O.deposit(cfg, pl, Bn)
    beta = q * dt / (2 * m)
    al = O.alpha(np.array([0, 0, beta * 2.0]))
    corners = [(1, 1), (2, 1), (1, 2), (2, 2)]
    for (i, j) in corners:
        assert rho[0, j, i] == pytest.approx(0.25, rel=1e-15)
        for (k, l) in corners:
            blk = M[0, j, i, offset(k - i, l - j)]
            assert np.allclose(blk, beta * q * al / 16, rtol=1e-14, atol=0)
    assert np.abs(M).sum() == pytest.approx(16 * np.abs(beta * q * al / 16).sum(), rel=1e-14)


def test_two_particles_hand_values():
    # Particle A at offsets (0.25, 0) in cell (0,0): weights 3/4 on node (0,0),
    # 1/4 on node (1,0).  Particle B (other species) at node (1,0) exactly.
    dt = 0.2
    cfg = O.make_cfg((4, 4, 1), (1.0, 1.0, 1.0), dt=dt)
    qs, ms = [1.0, -1.0], [1.0, 0.5]
    pl = O.Plasma(qs, ms, [0, 1], [0.25, 1.0], [0.0, 0.0], [0.0, 0.0], [0, 0], [0, 0], [0, 0], [1.0, 3.0])
    Bn = np.zeros((3,) + cfg.shape)            # B = 0: alpha = I
    rho, J, M = O.deposit(cfg, pl, Bn)
    bA = 1.0 * dt / 2
    bB = -1.0 * dt / (2 * 0.5)
    I = np.eye(3)
    assert np.allclose(M[0, 0, 0, offset(0, 0)], bA * 1.0 * (9 / 16) * I)
    assert np.allclose(M[0, 0, 0, offset(1, 0)], bA * 1.0 * (3 / 16) * I)
    assert np.allclose(M[0, 0, 1, offset(-1, 0)], bA * 1.0 * (3 / 16) * I)
    assert np.allclose(M[0, 0, 1, offset(0, 0)], bA * (1 / 16) * I + bB * (-1.0) * 3.0 * I)
    assert rho[0, 0, 0] == pytest.approx(0.75) and rho[0, 0, 1] == pytest.approx(0.25 - 3.0)


def _random_plasma(cfg, n=200, seed=1, species=((1.0, 1.0), (-1.0, 0.04))):
    rng = np.random.default_rng(seed)
    L = [cfg.n[d] * cfg.dx[d] for d in range(3)]
    sp = rng.integers(0, len(species), n)
    x = rng.random(n) * L[0]
    y = rng.random(n) * L[1]
    z = rng.random(n) * L[2] if cfg.n[2] > 1 else np.zeros(n)
    v = rng.standard_normal((3, n)) * 0.1
    w = 0.5 + rng.random(n)
    return O.Plasma([s[0] for s in species], [s[1] for s in species], sp, x, y, z, v[0], v[1], v[2], w)


@pytest.fixture(params=[(6, 5, 1), (4, 5, 3)])
def grid(request):
    n = request.param
    return O.make_cfg(n, (0.1, 0.13, 0.07), dt=0.05, c=1.7)


def _random_B(cfg, seed=3):
    return np.random.default_rng(seed).standard_normal((3,) + cfg.shape) * 0.5


def test_mass_matrix_block_symmetry(grid):
    # M_{g g'} = M_{g' g} as 3x3 blocks (the W_pg W_pg' weight is symmetric).
    pl = _random_plasma(grid)
    Bn = O.node_avg(grid, _random_B(grid))
    _, _, M = O.deposit(grid, pl, Bn)
    nz, ny, nx = grid.shape
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for o in range(27):
                    ox, oy, oz = o % 3 - 1, (o // 3) % 3 - 1, o // 9 - 1
                    back = offset(-ox, -oy, -oz)
                    nb = ((k + oz) % nz, (j + oy) % ny, (i + ox) % nx)
                    assert np.allclose(M[k, j, i, o], M[nb][back], rtol=1e-13, atol=1e-15)


def test_mass_matrix_partition_of_unity_no_field(grid):
    # B = 0: alpha = I and sum over all blocks = sum_p beta_s q_p I.
    pl = _random_plasma(grid)
    _, _, M = O.deposit(grid, pl, np.zeros((3,) + grid.shape))
    beta = pl.q[pl.sp] * grid.dt / (2 * pl.m[pl.sp])
    tot = M.reshape(-1, 3, 3).sum(axis=0)
    assert np.allclose(tot, (beta * pl.q[pl.sp] * pl.w).sum() * np.eye(3), rtol=1e-12, atol=1e-15)


def test_charge_conservation_of_deposit(grid):
    # sum_g rho_g dV = sum_p q_p (the weights of a particle sum to 1).
    pl = _random_plasma(grid)
    rho, _, _ = O.deposit(grid, pl, np.zeros((3,) + grid.shape))
    dV = grid.dx[0] * grid.dx[1] * grid.dx[2]
    assert rho.sum() * dV == pytest.approx((pl.q[pl.sp] * pl.w).sum(), rel=1e-12, abs=1e-13)


def test_predicted_current_matches_mover_vbar(grid):
    # Eq. 29 and Eq. 33: J_hat + (1/dV) M E^{n+theta} equals
    # (1/dV) sum_p q_p vbar_p W_pg with vbar from the mover.  The right side is
    # computed with the mass/momentum routine (m := q, v := vbar), a different
    # code path from the deposit.
    pl = _random_plasma(grid, n=150)
    Bn = O.node_avg(grid, _random_B(grid))
    Eth = np.random.default_rng(5).standard_normal((3,) + grid.shape) * 0.2
    rho, J, M = O.deposit(grid, pl, Bn)
    N = grid.nn
    ME = np.einsum("goij,goj->gi", M.reshape(N, 27, 3, 3), _neighbour_gather(grid, Eth))
    dV = grid.dx[0] * grid.dx[1] * grid.dx[2]
    Jbar = J.reshape(3, N).T + ME / dV
    moved = pl.copy()
    _, vbar = O.mover(grid, moved, Eth, Bn, want_vbar=True)
    probe = O.Plasma(pl.q, pl.q, pl.sp, pl.x, pl.y, pl.z, vbar[:, 0], vbar[:, 1], vbar[:, 2], pl.w)
    _, P = O.bulk_moments(grid, probe)
    assert np.allclose(Jbar, P.reshape(3, N).T / dV, rtol=1e-11, atol=1e-12)


def _neighbour_gather(cfg, F):
    """F at g + o for each node g and offset o: shape (N, 27, 3)."""
    nz, ny, nx = cfg.shape
    out = np.zeros((nz, ny, nx, 27, 3))
    for o in range(27):
        ox, oy, oz = o % 3 - 1, (o // 3) % 3 - 1, o // 9 - 1
        out[:, :, :, o, :] = np.moveaxis(np.roll(F, shift=(-oz, -oy, -ox), axis=(1, 2, 3)), 0, -1)
    return out.reshape(-1, 27, 3)


def test_motional_identity_inside_deposit(grid):
    # Sec. 2.1: with a uniform comoving velocity U and uniform B, the standard
    # and comoving predicted currents differ by exactly rho U:
    #   (J - J_C) + (1/dV) M E_M = rho U,  E_M = -U x B / c.
    pl = _random_plasma(grid)
    Bv = np.array([0.2, -0.4, 0.7])
    Bn = np.zeros((3,) + grid.shape)
    for d in range(3):
        Bn[d] = Bv[d]
    U = np.array([0.3, -0.1, 0.05])
    Uf = np.zeros((3,) + grid.shape)
    for d in range(3):
        Uf[d] = U[d]
    rho, J, M = O.deposit(grid, pl, Bn)
    _, JC, _ = O.deposit(grid, pl, Bn, u=Uf)
    EM = -np.cross(U, Bv) / grid.c
    N = grid.nn
    dV = grid.dx[0] * grid.dx[1] * grid.dx[2]
    ME = M.reshape(N, 27, 3, 3).sum(axis=1) @ EM
    lhs = (J - JC).reshape(3, N).T + ME / dV
    assert np.allclose(lhs, rho.reshape(N, 1) * U[None, :], rtol=1e-11, atol=1e-12)


def test_single_pass_comoving_identity_one_species(grid):
    # J_C = J - (1/dV) sum_g' M0_gg' u_g'  with M0 the mass matrix without beta;
    # for one species M0 = M / beta.  Holds for any (non-uniform) u field.
    pl = _random_plasma(grid, species=((-1.0, 0.04),))
    beta = -1.0 * grid.dt / (2 * 0.04)
    Bn = O.node_avg(grid, _random_B(grid))
    u = np.random.default_rng(9).standard_normal((3,) + grid.shape) * 0.3
    _, J, M = O.deposit(grid, pl, Bn)
    _, JC, _ = O.deposit(grid, pl, Bn, u=u)
    N = grid.nn
    dV = grid.dx[0] * grid.dx[1] * grid.dx[2]
    Mu = np.einsum("goij,goj->gi", M.reshape(N, 27, 3, 3), _neighbour_gather(grid, u)) / beta
    assert np.allclose(JC.reshape(3, N).T, J.reshape(3, N).T - Mu / dV, rtol=1e-10, atol=1e-12)


def test_cold_beam_comoving_current_vanishes():
    # Sec. 2.1: a cold uniform neutral beam (every particle moving with u) has
    # plasma velocity u everywhere and zero comoving-frame current.
    wl = workloads.uniform_drift(n=(8, 6, 1), ppc=9, vth_e=0.0, vth_i=0.0, u=(0.3, -0.05, 0.02))
    cfg = O.make_cfg(wl.n, wl.dx, **wl.grid_kwargs())
    pl = O.Plasma.from_species(wl.species)
    rm, P = O.bulk_moments(cfg, pl)
    u = O.bulk_velocity(cfg, rm, P)
    U = np.array([0.3, -0.05, 0.02], dtype=np.float32).astype(np.float64)
    for d in range(3):
        assert np.allclose(u[d], U[d], rtol=1e-13, atol=1e-15)
    Bn = O.node_avg(cfg, wl.B0)
    _, JC, _ = O.deposit(cfg, pl, Bn, u=u)
    _, J, _ = O.deposit(cfg, pl, Bn)
    assert np.abs(JC).max() < 1e-12 * np.abs(J).max() + 1e-14
