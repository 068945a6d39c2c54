"""Pins of the oracle's vacuum field step with the digital filter on E (Sec. 3.1:
the top-hat light wave smoothed by a filter on E instead of the LF term on E).

The pin is a closed form derived here from the discrete operators, not from the
oracle's code.  In 1D vacuum a single Fourier mode E_y = Re(e exp(i k x_i)) at
the nodes and B_z = Re(b exp(i k x_{i+1/2})) at the cell centres stays a mode:
with K = 2 sin(k dx / 2) / dx the node curl of B_z is -i K b and the cell curl of
E_y is i K e, so the theta scheme (E^{n+theta} from the implicit equation,
B^{n+1} = B^n - c dt curl E^{n+theta}, E^{n+1} = (E^{n+theta} - (1 - theta) E^n)
/ theta) becomes, with s = c theta dt K,
    e_theta = (e - i s b) / (1 + s^2),
    b'      = b - i (s / theta) e_theta,
    e'      = (e_theta - (1 - theta) e) / theta,
and each filter pass of stride d multiplies e' by 0.5 + 0.5 cos(k d dx)
(Eq. 26 with phi = 0.5).  A dropped curl term, a wrong sign or a wrong stride
order changes the amplitudes at the 1e-3 level or more.
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


@pytest.mark.parametrize("npass,theta,cfl", [(0, 0.5, 0.4), (1, 0.5, 0.4), (3, 0.5, 0.4), (2, 0.6, 2.0)])
def test_fourier_mode_follows_closed_form(npass, theta, cfl):
    n, dx, c = 40, 0.02, 1.0
    dt = cfl * dx / c
    m = 3
    k = 2 * np.pi * m / (n * dx)
    e, b = 0.8 + 0.1j, -0.3 + 0.5j
    E, B = mode_fields(n, dx, k, e, b)
    cfg = O.make_cfg((n, 1, 1), (dx, 1.0, 1.0), c=c, theta=theta, dt=dt, lf_on=0, gmres_tol=1e-14,
                     nsmooth_u=0, nsmooth_e=npass)
    K = 2 * np.sin(k * dx / 2) / dx
    s = c * theta * dt * K
    filt = np.prod([0.5 + 0.5 * np.cos(k * (1 if p % 2 == 0 else 2) * dx) for p in range(npass)])
    steps = 6
    for _ in range(steps):
        assert O.step(cfg, empty_plasma(), E, B)["rc"] == 0
        et = (e - 1j * s * b) / (1 + s * s)
        b = b - 1j * (s / theta) * et
        e = filt * (et - (1 - theta) * e) / theta
    Ee, Be = mode_fields(n, dx, k, e, b)
    assert np.abs(E - Ee).max() <= 1e-10
    assert np.abs(B - Be).max() <= 1e-10


def test_filter_replaces_lf_on_E_only():
    """With nsmooth_e > 0 and lf_on the E solve has no LF term (its solution is
    the solve without kappa, not the one with it), and E^{n+1} is one d = 1
    filter pass, 0.5 E_i + 0.25 (E_{i-1} + E_{i+1}), of (E^{n+theta} - (1 -
    theta) E^n) / theta."""
    n, dx, c = 40, 0.02, 1.0
    dt = 0.4 * dx / c
    B = np.zeros((3, 1, 1, n))
    B[2, 0, 0, 10:20] = 1.0
    E = np.zeros_like(B)
    E[1, 0, 0, 5:25] = 0.3
    cfg = O.make_cfg((n, 1, 1), (dx, 1.0, 1.0), c=c, dt=dt, lf_on=1, lf_speed_c=1, lf_beta=1.0,
                     gmres_tol=1e-14, nsmooth_u=0, nsmooth_e=1)
    E1, B1 = E.copy(), B.copy()
    Eth = O.step(cfg, empty_plasma(), E1, B1, want=("Eth",))["Eth"]
    b = O.rhs(cfg, E, B, np.zeros_like(E))
    x_plain = O.gmres(cfg, b, E)[0]
    x_lf = O.gmres(cfg, b, E, kappa=O.lf_kappa_E(cfg, E))[0]
    assert np.abs(Eth - x_plain).max() <= 1e-12
    assert np.abs(Eth - x_lf).max() > 1e-4
    Ey = ((Eth - 0.5 * E) / 0.5)[1].reshape(-1)
    ref = 0.5 * Ey + 0.25 * (np.roll(Ey, 1) + np.roll(Ey, -1))
    assert np.abs(E1[1].reshape(-1) - ref).max() <= 1e-12
