"""Pins of the oracle's divergence cleaning of B (Sec. 1.3, "div B correction").

The paper fixes the continuous system (d phi/dt + c_h^2 div B = -(c_h^2/c_p^2)
phi, dB/dt = ... - grad phi) and its parameters (c_h = 0.8 dx/dt, dt c_h^2/c_p^2
= 0.1), not the discretisation; the oracle's reading is central differences at
cell centres, B updated with grad phi^n, then phi with div B^{n+1} and an exact
decay factor exp(-0.1).  These tests pin that reading to facts that do not come
from the oracle's code:
  * a field whose central divergence vanishes identically (B_x depending on y
    only, B_y on x only) with phi = 0 is left exactly as it is;
  * on the periodic grid the central divergence sums to zero, so the sum of
    phi decays by exactly exp(-0.1) per step whatever B is;
  * a single Fourier mode B_x = b sin(kx), phi = p cos(kx) stays a mode, and its
    amplitudes follow the 2 x 2 recurrence b' = b + dt kappa p,
    p' = exp(-0.1) (p - dt c_h^2 kappa b') with kappa = sin(k dx)/dx, evaluated
    here by matrix powers; the recurrence is stable (spectral radius < 1).
"""
import numpy as np

import oracle as O


def cfg2(nx, ny, dx=0.1, dy=0.07, dt=0.02):
    return O.make_cfg((nx, ny, 1), (dx, dy, 1.0), dt=dt, divb_clean=1)


def test_divergence_free_field_is_untouched():
    nx, ny = 12, 10
    cfg = cfg2(nx, ny)
    rng = np.random.default_rng(1)
    B = np.zeros((3, 1, ny, nx))
    B[0] = rng.standard_normal(ny)[None, :, None]        # B_x(y)
    B[1] = rng.standard_normal(nx)[None, None, :]        # B_y(x)
    B[2] = rng.standard_normal((1, ny, nx))              # B_z: no derivative along z in 2D
    B = np.ascontiguousarray(B.reshape(-1))
    B0 = B.copy()
    phi = np.zeros(nx * ny)
    for _ in range(3):
        O.divb_clean(cfg, B, phi)
    assert np.array_equal(B, B0)
    assert np.all(phi == 0.0)


def test_phi_sum_decays_by_exactly_the_damping_factor():
    nx, ny = 9, 14
    cfg = cfg2(nx, ny)
    rng = np.random.default_rng(2)
    B = rng.standard_normal(3 * nx * ny)
    phi = rng.standard_normal(nx * ny)
    for _ in range(4):
        s0 = phi.sum()
        O.divb_clean(cfg, B, phi)
        assert abs(phi.sum() - np.exp(-0.1) * s0) <= 1e-12 * (abs(s0) + np.abs(phi).sum())


def test_fourier_mode_follows_its_recurrence():
    nx, dx, dt = 16, 0.1, 0.02
    cfg = O.make_cfg((nx, 1, 1), (dx, 1.0, 1.0), dt=dt, divb_clean=1)
    k = 2 * np.pi * 3 / (nx * dx)
    x = (np.arange(nx) + 0.5) * dx
    b0, p0 = 0.7, -0.3
    B = np.zeros(3 * nx)
    B[:nx] = b0 * np.sin(k * x)
    phi = p0 * np.cos(k * x)
    ch = 0.8 * dx / dt
    kappa = np.sin(k * dx) / dx
    # one step as a matrix on (b, p): b' = b + dt kappa p, p' = e (p - dt ch^2 kappa b')
    e = np.exp(-0.1)
    Mb = np.array([[1.0, dt * kappa], [0.0, 1.0]])
    Mp = np.array([[1.0, 0.0], [-e * dt * ch ** 2 * kappa, e]])
    M = Mp @ Mb
    assert max(abs(np.linalg.eigvals(M))) < 1.0
    steps = 7
    for _ in range(steps):
        O.divb_clean(cfg, B, phi)
    b, p = np.linalg.matrix_power(M, steps) @ np.array([b0, p0])
    assert np.allclose(B[:nx], b * np.sin(k * x), rtol=0, atol=1e-12)
    assert np.allclose(phi, p * np.cos(k * x), rtol=0, atol=1e-12)
    assert np.all(B[nx:] == 0.0)                          # y, z components untouched in 1D
