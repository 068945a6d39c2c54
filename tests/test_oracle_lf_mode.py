"""Pin of the oracle's vacuum step with the Lax-Friedrichs terms on E and B
(Sec. 1.2, Eq. 17-20) by a closed form derived here from the discrete operators.

With beta = 0 the limiter is off (phi = 0) and a = c, so both LF terms are
linear and a single 1D Fourier mode, E_y = Re(e exp(i k x_i)) at the nodes and
B_z = Re(b exp(i k x_{i+1/2})) at the cell centres, stays a mode.  With
K = 2 sin(k dx / 2) / dx, s = c theta dt K, nu = c dt / dx and
sigma = 2 sin^2(k dx / 2):
  * LF on B adds D = (nu / 2) delta^2 B to B^{n+1}, i.e. -mu b with mu = nu sigma;
  * LF on E (read as diffusion, the sign of reading A3) adds theta nu sigma e_theta
    to the left-hand side;
  * the right-hand side curls B^n + theta D (B^{n+theta} with the LF increment);
so
    e_theta = (e - i s (1 - theta mu) b) / (1 + s^2 + theta nu sigma),
    b'      = (1 - mu) b - i (s / theta) e_theta,
    e'      = (e_theta - (1 - theta) e) / theta.
A wrong LF sign, a dropped theta D, or the B increment taken at another time
level moves the amplitudes well above the 1e-10 checked.  The same recurrence
shows why theta D belongs in the solve: at theta = 1/2 and c dt / dx >> 1 the
modes stay bounded with it, and grow by about 1 + mu per step without it.
"""
import numpy as np
import pytest

import oracle as O


def empty_plasma():
    e = np.zeros(0)
    return O.Plasma([-1.0], [1.0], np.zeros(0, np.int32), e, e, e, e, e, e, e)


def mode_fields(n, dx, k, e, b):
    xn = np.arange(n) * dx
    xc = xn + 0.5 * dx
    E = np.zeros((3, 1, 1, n))
    B = np.zeros((3, 1, 1, n))
    E[1, 0, 0] = (e * np.exp(1j * k * xn)).real
    B[2, 0, 0] = (b * np.exp(1j * k * xc)).real
    return E, B


def mode_matrix(s, theta, nu, sigma, with_theta_d=True):
    mu = nu * sigma
    M = np.zeros((2, 2), complex)
    for j, (e, b) in enumerate(((1.0, 0.0), (0.0, 1.0))):
        bt = (1 - theta * mu) * b if with_theta_d else b
        et = (e - 1j * s * bt) / (1 + s * s + theta * nu * sigma)
        M[:, j] = ((et - (1 - theta) * e) / theta, (1 - mu) * b - 1j * (s / theta) * et)
    return M


@pytest.mark.parametrize("m,theta,cfl", [(3, 0.5, 0.4), (7, 0.5, 0.9), (11, 0.6, 3.0), (19, 0.5, 2.0)])
def test_lf_fourier_mode_follows_closed_form(m, theta, cfl):
    n, dx, c = 40, 0.02, 1.0
    dt = cfl * dx / c
    k = 2 * np.pi * m / (n * dx)
    e, b = 0.4 - 0.2j, 0.6 + 0.3j
    E, B = mode_fields(n, dx, k, e, b)
    cfg = O.make_cfg((n, 1, 1), (dx, 1.0, 1.0), c=c, theta=theta, dt=dt, lf_on=1, lf_speed_c=1, lf_beta=0.0,
                     gmres_tol=1e-14, nsmooth_u=0)
    K = 2 * np.sin(k * dx / 2) / dx
    M = mode_matrix(c * theta * dt * K, theta, c * dt / dx, 2 * np.sin(k * dx / 2) ** 2)
    steps = 5
    for _ in range(steps):
        assert O.step(cfg, empty_plasma(), E, B)["rc"] == 0
    e, b = np.linalg.matrix_power(M, steps) @ np.array([e, b])
    Ee, Be = mode_fields(n, dx, k, e, b)
    assert np.abs(E - Ee).max() <= 1e-10
    assert np.abs(B - Be).max() <= 1e-10


def test_lf_increment_in_the_solve_keeps_fast_light_modes_bounded():
    """At theta = 1/2 and c dt / dx = 50 the recurrence with theta D has spectral
    radius <= 1 for every mode, without it the shortest modes grow (radius
    1 + mu - O(1/s))."""
    theta, nu = 0.5, 0.38
    radii_with, radii_without = [], []
    for kdx in np.linspace(0.1, np.pi, 40):
        s = theta * 50.0 * 2 * np.sin(kdx / 2)
        sigma = 2 * np.sin(kdx / 2) ** 2
        radii_with.append(max(abs(np.linalg.eigvals(mode_matrix(s, theta, nu, sigma)))))
        radii_without.append(max(abs(np.linalg.eigvals(mode_matrix(s, theta, nu, sigma, False)))))
    assert max(radii_with) <= 1.0 + 1e-12
    assert max(radii_without) > 1.5


@pytest.mark.parametrize("m,cfl", [(5, 0.4), (13, 2.0)])
def test_printed_form_follows_its_own_closed_form(m, cfl):
    """With lf_rhs_printed the solve curls B^n alone, as Eq. 7 prints it: the
    same mode then follows the recurrence without the theta D term, and leaves
    the one with it (so the switch selects exactly that term)."""
    n, dx, c, theta = 40, 0.02, 1.0, 0.5
    dt = cfl * dx / c
    k = 2 * np.pi * m / (n * dx)
    e0, b0 = 0.3 + 0.1j, -0.5 + 0.4j
    E, B = mode_fields(n, dx, k, e0, b0)
    cfg = O.make_cfg((n, 1, 1), (dx, 1.0, 1.0), c=c, theta=theta, dt=dt, lf_on=1, lf_speed_c=1, lf_beta=0.0,
                     gmres_tol=1e-14, nsmooth_u=0, lf_rhs_printed=1)
    args = (c * theta * dt * 2 * np.sin(k * dx / 2) / dx, theta, c * dt / dx, 2 * np.sin(k * dx / 2) ** 2)
    steps = 4
    for _ in range(steps):
        assert O.step(cfg, empty_plasma(), E, B)["rc"] == 0
    e, b = np.linalg.matrix_power(mode_matrix(*args, with_theta_d=False), steps) @ np.array([e0, b0])
    Ee, Be = mode_fields(n, dx, k, e, b)
    assert np.abs(E - Ee).max() <= 1e-10 and np.abs(B - Be).max() <= 1e-10
    e, b = np.linalg.matrix_power(mode_matrix(*args), steps) @ np.array([e0, b0])
    Ee, _ = mode_fields(n, dx, k, e, b)
    assert np.abs(E - Ee).max() > 1e-6
