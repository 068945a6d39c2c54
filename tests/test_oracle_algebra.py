"""Pins of the oracle's particle algebra against what the paper and mathematics
fix (Sec. 2.1, Eq. 29-30): properties of the rotation tensor alpha, the motional-
field identity, the exact gyration of the implicit mover, and the E x B drift
as a fixed point.  None of these re-types the oracle's formula: each checks a
consequence that a dropped term, a wrong sign or a transposed operand breaks."""
import math

import numpy as np
import pytest

import oracle as O


@pytest.fixture(params=range(6))
def bvec(request):
    rng = np.random.default_rng(100 + request.param)
    return rng.standard_normal(3) * (0.2 + request.param)


def test_alpha_leaves_b_invariant(bvec):
    # alpha b = b: the field-aligned velocity is not rotated.
    assert np.allclose(O.alpha(bvec) @ bvec, bvec, rtol=1e-14, atol=1e-14)


def test_alpha_inverse_is_identity_minus_cross(bvec):
    # alpha solves vbar = a + vbar x b, so alpha^{-1} a = a - a x b.
    al = O.alpha(bvec)
    rng = np.random.default_rng(7)
    for _ in range(5):
        a = rng.standard_normal(3)
        inv = a - np.cross(a, bvec)
        assert np.allclose(al @ inv, a, rtol=1e-13, atol=1e-13)


def test_motional_field_identity(bvec):
    # Sec. 2.1: alpha [u + beta E_M] = u with E_M = -u x B / c (b = beta B / c).
    rng = np.random.default_rng(11)
    for _ in range(5):
        u = rng.standard_normal(3)
        beta_EM = -np.cross(u, bvec)
        assert np.allclose(O.alpha(bvec) @ (u + beta_EM), u, rtol=1e-14, atol=1e-14)


def test_alpha_closed_form_rotation_angle(bvec):
    # With E = 0 the mover's map v -> 2 alpha v - v is the rotation about b by
    # phi with tan(phi/2) = |b| (the implicit-midpoint gyration).
    al = O.alpha(bvec)
    R = 2 * al - np.eye(3)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-13)           # orthogonal
    assert abs(np.linalg.det(R) - 1.0) < 1e-13                   # proper
    bn = np.linalg.norm(bvec)
    phi = 2 * math.atan(bn)
    # the trace of a rotation by phi is 1 + 2 cos phi
    assert abs(np.trace(R) - (1 + 2 * math.cos(phi))) < 1e-13
    # sense of rotation: for b along +z, a velocity along x turns toward -y when
    # q B > 0 (v x B force on a positive charge) -- R e_x . e_y = -sin(phi)
    bz = np.array([0.0, 0.0, bn])
    Rz = 2 * O.alpha(bz) - np.eye(3)
    assert abs(Rz[1, 0] - (-math.sin(phi))) < 1e-13


def test_mc_limiter_special_cases():
    L = O.mc_limiter
    for r in np.linspace(-3, 5, 33):
        assert L(r, 0.0) == 0.0                                   # beta = 0: first order
        assert abs(L(r, 1.0) - max(0.0, min(r, 1.0))) < 1e-15     # beta = 1: minmod
        for beta in (1.0, 1.5, 2.0):
            assert 0.0 <= L(r, beta) <= beta + 1e-15
    for beta in (1.0, 1.5, 2.0):
        assert abs(L(1.0, beta) - 1.0) < 1e-15                    # smooth data: second order
        assert L(-1.0, beta) == 0.0                               # extremum: first order
    # beta = 2 is van Leer's monotonized-central limiter
    assert abs(L(0.5, 2.0) - 0.75) < 1e-15 and abs(L(3.0, 2.0) - 2.0) < 1e-15 and abs(L(0.2, 2.0) - 0.4) < 1e-15


def _one_particle_grid(q=1.0, m=1.0, v=(0.1, 0.0, 0.0), pos=(0.3, 0.4, 0.0), E=(0, 0, 0), B=(0, 0, 0.5),
                       dt=0.1, c=1.0):
    cfg = O.make_cfg((8, 8, 1), (1.0, 1.0, 1.0), c=c, dt=dt)
    pl = O.Plasma([q], [m], [0], [pos[0]], [pos[1]], [pos[2]], [v[0]], [v[1]], [v[2]], [1.0])
    Eth = np.zeros((3,) + cfg.shape)
    Bn = np.zeros((3,) + cfg.shape)
    for d in range(3):
        Eth[d] = E[d]
        Bn[d] = B[d]
    return cfg, pl, Eth, Bn


def test_mover_gyration_preserves_speed_and_angle():
    q, m, dt, B = -1.0, 0.04, 0.05, 0.7
    cfg, pl, Eth, Bn = _one_particle_grid(q=q, m=m, v=(0.2, 0.1, 0.05), dt=dt, B=(0, 0, B))
    v0 = np.array([pl.vx[0], pl.vy[0], pl.vz[0]])
    O.mover(cfg, pl, Eth, Bn)
    v1 = np.array([pl.vx[0], pl.vy[0], pl.vz[0]])
    assert abs(np.linalg.norm(v1) - np.linalg.norm(v0)) < 1e-15
    beta = q * dt / (2 * m)
    phi = 2 * math.atan(abs(beta * B))
    ang = math.atan2(v1[1], v1[0]) - math.atan2(v0[1], v0[0])
    ang = (ang + math.pi) % (2 * math.pi) - math.pi
    # a negative charge in +z field gyrates counter-clockwise seen from +z
    assert abs(ang - phi) < 1e-13
    assert v1[2] == v0[2]


def test_mover_exb_drift_is_fixed_point():
    # v = c E x B / B^2 with E perpendicular to B is an exact fixed point.
    E = np.array([0.0, 0.03, 0.0])
    B = np.array([0.0, 0.0, 0.4])
    c = 2.0
    vd = c * np.cross(E, B) / B.dot(B)
    cfg, pl, Eth, Bn = _one_particle_grid(q=1.0, m=1.0, v=tuple(vd), E=tuple(E), B=tuple(B), dt=0.3, c=c)
    x0 = pl.x[0]
    O.mover(cfg, pl, Eth, Bn)
    assert np.allclose([pl.vx[0], pl.vy[0], pl.vz[0]], vd, rtol=0, atol=1e-15)
    assert abs((pl.x[0] - x0) - 0.3 * vd[0]) < 1e-15


def test_mover_free_streaming_and_wrap():
    cfg, pl, Eth, Bn = _one_particle_grid(v=(3.0, -2.5, 0.0), pos=(7.9, 0.2, 0.0), B=(0, 0, 0), dt=0.1)
    O.mover(cfg, pl, Eth, Bn)
    assert abs(pl.x[0] - ((7.9 + 0.3) - 8.0)) < 1e-14
    assert abs(pl.y[0] - ((0.2 - 0.25) + 8.0)) < 1e-14
