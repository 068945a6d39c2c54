"""Pins of the oracle against values the paper prints (fixtures under
tests/golden/, each with its citation in its header).

* velocity_filter_sec2_1.txt: the comoving-frame velocity is the plasma
  velocity smoothed by five passes of the Eq. 26 filter with phi = 0.5 and
  strides 1, 2, 1, 2, 1 (Sec. 2.1); the current smoothing is one pass, d = 1
  (Sec. 2.2, Sec. 3).  The oracle's bulk velocity and current smoothing must
  equal those passes applied one by one, and one pass must be the printed
  three-point formula.
"""
import os

import numpy as np

import oracle as O


def golden(name):
    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    for line in open(path):
        line = line.split("#", 1)[0].strip()
        if "=" in line:
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = v
    return out


VF = golden("velocity_filter_sec2_1.txt")


def test_filter_pass_is_the_printed_three_point_formula():
    # Eq. 26: v*_i = phi v_i + (1 - phi)/2 (v_{i-d} + v_{i+d}), here along x on a 1D grid
    phi = float(VF["phi"])
    cfg = O.make_cfg((11, 1, 1), (0.1, 1.0, 1.0))
    v = np.random.default_rng(3).standard_normal((1, 1, 11))
    for d in (1, 2):
        out = O.filter_pass(cfg, v, d, phi)
        ref = phi * v + 0.5 * (1 - phi) * (np.roll(v, d, axis=2) + np.roll(v, -d, axis=2))
        assert np.allclose(out, ref, atol=1e-15)


def test_bulk_velocity_uses_the_printed_smoothing_schedule():
    passes, phi = int(VF["passes"]), float(VF["phi"])
    strides = [int(x) for x in VF["strides"].split()]
    assert len(strides) == passes
    cfg = O.make_cfg((9, 7, 1), (0.1, 0.12, 1.0), nsmooth_u=passes)
    rng = np.random.default_rng(5)
    rho_m = 1.0 + rng.random(cfg.shape)
    P = rng.standard_normal((3,) + cfg.shape)
    u = O.bulk_velocity(cfg, rho_m, P)
    ref = P / rho_m
    for d in strides:
        ref = O.filter_pass(cfg, ref, d, phi)
    assert np.allclose(u, ref, atol=1e-14)


def test_current_smoothing_is_one_pass_of_stride_one():
    cfg = O.make_cfg((8, 6, 1), (0.1, 0.1, 1.0))
    J = np.random.default_rng(9).standard_normal((3,) + cfg.shape)
    out = O.smooth_current(cfg, J, int(VF["current_passes"]))
    ref = J
    for _ in range(int(VF["current_passes"])):
        ref = O.filter_pass(cfg, ref, int(VF["current_stride"]), float(VF["phi"]))
    assert np.allclose(out, ref, atol=1e-14)
