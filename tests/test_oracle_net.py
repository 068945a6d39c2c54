"""Pins of the oracle's preconditioner network (a project addition, not in the
paper): the forward pass against an independent scipy.ndimage correlation, and
the backward pass against central finite differences of the loss."""
import numpy as np
import pytest
from scipy import ndimage

import oracle as O


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(O.net_param_count()) * scale


def _scipy_forward(params, x, periodic):
    mode = "wrap" if periodic else "constant"
    h = x
    layers = O.net_split(params)
    for l, (w, b) in enumerate(layers):
        cout, cin = w.shape[:2]
        y = np.zeros((cout,) + h.shape[1:])
        for co in range(cout):
            acc = np.full(h.shape[1:], b[co])
            for ci in range(cin):
                acc = acc + ndimage.correlate(h[ci], w[co, ci], mode=mode, cval=0.0)
            y[co] = acc
        h = np.maximum(y, 0.0) if l < 3 else y
    return h


@pytest.mark.parametrize("periodic", [True, False])
def test_forward_matches_scipy_correlation(periodic):
    p = _params(1)
    x = np.random.default_rng(2).standard_normal((3, 7, 9))
    y = O.net_forward(p, x, periodic=periodic)
    ref = _scipy_forward(p, x, periodic)
    assert np.allclose(y, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("periodic", [True, False])
def test_backward_matches_finite_differences(periodic):
    p = _params(3, 0.25)
    rng = np.random.default_rng(4)
    x = rng.standard_normal((3, 5, 6))
    t = rng.standard_normal((3, 5, 6))
    L, gp, gx = O.net_loss_backward(p, x, t, periodic=periodic)
    y = O.net_forward(p, x, periodic=periodic)
    assert L == pytest.approx(0.5 * np.mean((y - t) ** 2), rel=1e-13)
    # within one ReLU region the loss is exactly quadratic in any single
    # parameter or input, so a central difference has no truncation error
    h = 1e-4
    idx = rng.choice(p.size, 60, replace=False)
    # include every bias of the last layer and some first-layer weights
    idx = np.unique(np.concatenate([idx, np.arange(p.size - 3, p.size), np.arange(0, 5)]))
    pattern = O.net_forward(p, x, periodic, want_acts=True)[1] > 0

    def same_pattern(pa, xa):
        # a central difference across a ReLU kink is not a derivative: skip it
        return np.array_equal(O.net_forward(pa, xa, periodic, want_acts=True)[1] > 0, pattern)

    checked = 0
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        if not (same_pattern(pp, x) and same_pattern(pm, x)):
            continue
        fd = (O.net_loss_backward(pp, x, t, periodic)[0] - O.net_loss_backward(pm, x, t, periodic)[0]) / (2 * h)
        assert gp[i] == pytest.approx(fd, rel=1e-7, abs=1e-11), i
        checked += 1
    assert checked >= 0.9 * len(idx)
    for flat in rng.choice(x.size, 12, replace=False):
        xp, xm = x.copy(), x.copy()
        xp.flat[flat] += h
        xm.flat[flat] -= h
        if not (same_pattern(p, xp) and same_pattern(p, xm)):
            continue
        fd = (O.net_loss_backward(p, xp, t, periodic)[0] - O.net_loss_backward(p, xm, t, periodic)[0]) / (2 * h)
        assert gx.flat[flat] == pytest.approx(fd, rel=1e-7, abs=1e-11)
