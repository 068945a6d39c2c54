"""Checks of the synthetic workloads against physics the paper states, so that
a mistyped printed number or a wrong unit conversion fails here.

* The two shocks (Sec. 3.3-3.4): the printed upstream and downstream states
  satisfy the MHD jump conditions across a shock at rest, i.e. continuity of
  the mass flux rho u_x, of the normal field B_x and of the tangential electric
  field (u x B)_t, to the rounding of the printed digits (0.5 %).  The code-unit
  states built from them keep those invariants, and the upstream Alfven Mach
  numbers are the printed 7 and 4.
* The fast flow (Sec. 3.2): the conversion reproduces the printed ion inertial
  length (102 km) and Alfven speed (49 km/s), and the printed time step is a
  flow CFL of about 0.2 on the printed 8 km cells.
"""
import math

import numpy as np
import pytest

import workloads


def _jumps(up, dn):
    ru, uu, bu = up[0], np.array(up[1]), np.array(up[2])
    rd, ud, bd = dn[0], np.array(dn[1]), np.array(dn[2])
    mass = (ru * uu[0], rd * ud[0])
    bx = (bu[0], bd[0])
    e_t_up, e_t_dn = np.cross(uu, bu)[1:], np.cross(ud, bd)[1:]     # (u x B)_y, (u x B)_z
    return mass, bx, (e_t_up, e_t_dn)


@pytest.mark.parametrize("kind", ["parallel", "perpendicular"])
def test_printed_shock_states_satisfy_jump_conditions(kind):
    P = workloads.SHOCKS[kind]
    mass, bx, (eu, ed) = _jumps(P["up"], P["down"])
    assert abs(mass[0] - mass[1]) <= 5e-3 * abs(mass[0])
    assert bx[0] == bx[1]
    assert np.all(np.abs(eu - ed) <= 5e-3 * np.abs(eu).max())


@pytest.mark.parametrize("kind,mach", [("parallel", 7.0), ("perpendicular", 4.0)])
def test_code_unit_shock_states(kind, mach):
    wl = workloads.shock_1d(kind, length=48.0, ppc=4)
    up, dn = wl.notes["up"], wl.notes["down"]
    # the code-unit states keep the jump invariants (densities in units of the upstream one)
    assert abs(up["n"] * up["u"][0] - dn["n"] * dn["u"][0]) <= 5e-3 * abs(up["n"] * up["u"][0])
    assert abs(up["B"][0] - dn["B"][0]) <= 1e-12
    eu, ed = np.cross(up["u"], up["B"])[1:], np.cross(dn["u"], dn["B"])[1:]
    assert np.all(np.abs(eu - ed) <= 5e-3 * np.abs(eu).max())
    # upstream Alfven Mach number |u_x| / v_A, v_A = |B| in these units (n = 1/(4 pi), m_i = 1)
    assert abs(abs(up["u"][0]) / math.sqrt(sum(b * b for b in up["B"])) - mach) <= 0.02 * mach
    # the initial E is the motional field -u x B (u rounded to FP32 like the particles): downstream
    # at the first node, upstream at the last
    E = wl.E0[:, 0, 0]
    for st, node in ((dn, 0), (up, -1)):
        u32 = np.asarray(st["u"], np.float32).astype(np.float64)
        assert np.allclose(E[:, node], -np.cross(u32, st["B"]), rtol=0, atol=1e-15)


def test_fast_flow_conversion_reproduces_printed_scales():
    wl = workloads.fast_flow_1d(ppc=4)
    n = wl.notes
    assert abs(n["d_i_km"] - 102.0) <= 1.0
    assert abs(n["v_A"] * 299792.458 - 49.0) <= 0.5
    cfl = n["u"][0] * wl.dt / wl.dx[0]
    assert abs(cfl - 0.2) <= 0.02
    assert wl.n[0] * n["d_i_km"] * wl.dx[0] == pytest.approx(160.0, rel=1e-9)   # the printed 160 km domain
