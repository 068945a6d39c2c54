"""Pins of the oracle's grid averages that every other pin sees only with
uniform data: B carried from cell centres to nodes (the mesh of Sec. 1.1, B at
cell centres and E at nodes, averaged to nodes before the particles gather it),
and the diffusion speed a of the limited Lax-Friedrichs terms (Sec. 1.2,
Eq. 17-20), |u| averaged over the two nodes of an edge for E and over the
nodes of a face for B.

Each test puts a single nonzero value in one cell or at one node, so the
expected result is a handful of hand-computed entries and zeros elsewhere.  A
stencil shifted by one cell, a wrong face or edge, or a wrong divisor puts the
values somewhere else or scales them, and fails here."""
import numpy as np
import pytest

import oracle as O


def _nonzero(a):
    return {tuple(int(v) for v in k): a[tuple(k)] for k in np.argwhere(a != 0)}


@pytest.mark.parametrize("dims", [(6, 5, 1), (5, 4, 6)])
def test_node_average_of_one_cell(dims):
    # B only in cell (i0, j0, k0): each of the cell's 2^d corner nodes (i0..i0+1,
    # j0..j0+1, k0..k0+1) holds B / 2^d, every other node 0.  The cell spans
    # [i0, i0+1] x [j0, j0+1] x [k0, k0+1] node spacings (Sec. 1.1 mesh).
    cfg = O.make_cfg(dims, (0.1, 0.2, 0.3))
    nz, ny, nx = cfg.shape
    i0, j0, k0 = nx - 1, 2, (nz - 1 if nz > 1 else 0)    # at the periodic seam in x and z
    b = np.array([0.7, -1.3, 2.9])
    Bc = np.zeros((3,) + cfg.shape)
    Bc[:, k0, j0, i0] = b
    Bn = O.node_avg(cfg, Bc)
    dim = 3 if nz > 1 else 2
    want = {}
    for dk in (range(2) if dim == 3 else [0]):
        for dj in range(2):
            for di in range(2):
                want[((k0 + dk) % nz, (j0 + dj) % ny, (i0 + di) % nx)] = 1
    for comp in range(3):
        got = _nonzero(Bn[comp])
        assert set(got) == set(want), comp
        for key in want:
            assert got[key] == pytest.approx(b[comp] / 2 ** dim, rel=1e-15)


def test_node_average_two_cells_superpose_with_distinct_values():
    # Two cells with different values: the node they share holds the sum of
    # both quarters; the others hold one quarter each (2D).
    cfg = O.make_cfg((7, 6, 1), (0.1, 0.1, 1.0))
    Bc = np.zeros((3,) + cfg.shape)
    Bc[0, 0, 2, 3] = 4.0           # cell (3, 2)
    Bc[0, 0, 3, 4] = 8.0           # cell (4, 3): shares node (4, 3) with it
    Bn = O.node_avg(cfg, Bc)[0, 0]
    assert Bn[3, 4] == pytest.approx(1.0 + 2.0, rel=1e-15)
    for (j, i) in [(2, 3), (2, 4), (3, 3)]:
        assert Bn[j, i] == pytest.approx(1.0, rel=1e-15)
    for (j, i) in [(3, 5), (4, 4), (4, 5)]:
        assert Bn[j, i] == pytest.approx(2.0, rel=1e-15)
    assert np.count_nonzero(Bn) == 7


@pytest.mark.parametrize("dims", [(6, 5, 1), (5, 4, 6)])
def test_lf_kappa_edges_of_one_node(dims):
    # E^n = 0 makes every smoothness ratio 0/0 -> r = 0 and phi_E = MC(0) = 0, so
    # kappa = (1 - phi) a / 2 = a / 2 with a the mean of |u| over the edge's two
    # nodes (Eq. 19-20 with the diffusion speed |u|).  |u| = U only at node n0:
    # the two edges of each resolved axis that touch n0 get U/4, the rest 0, for
    # every field component.
    cfg = O.make_cfg(dims, (0.1, 0.2, 0.3), lf_on=1, lf_speed_c=0, lf_beta=1.0)
    nz, ny, nx = cfg.shape
    n0 = (nz // 2, 1, 0)                   # (k, j, i), i = 0 at the periodic seam
    u = np.zeros((3,) + cfg.shape)
    uvec = np.array([0.3, -0.4, 1.2])      # |u| = 1.3
    u[(slice(None),) + n0] = uvec
    U = float(np.linalg.norm(uvec))
    kappa = O.lf_kappa_E(cfg, np.zeros((3,) + cfg.shape), u)
    axes = [d for d in range(3) if cfg.n[d] > 1]
    for d in range(3):
        for comp in range(3):
            got = _nonzero(kappa[d, comp])
            if d not in axes:
                assert not got
                continue
            k, j, i = n0
            m = [i, j, k]
            m[d] -= 1
            lower = (m[2] % nz, m[1] % ny, m[0] % nx)
            assert set(got) == {n0, lower}, (d, comp)
            for key in got:
                assert got[key] == pytest.approx(U / 4, rel=1e-15)


def test_lf_kappa_uses_the_limiter_of_its_own_edge():
    # A ramp E_x = i (interior, away from the seam) has r = 1 on the edges
    # between i = 2..5: phi = MC(1, beta) = min(beta, 1, beta).  With beta = 0.5
    # kappa = (1 - 0.5) a / 2 = a / 4; with beta = 1, kappa = 0.  Uniform
    # |u| = U there, so a = U.
    for beta, fac in [(0.5, 0.25), (1.0, 0.0), (0.0, 0.5)]:
        cfg = O.make_cfg((9, 4, 1), (0.1, 0.1, 1.0), lf_on=1, lf_speed_c=0, lf_beta=beta)
        E = np.zeros((3,) + cfg.shape)
        E[0] = np.arange(9)[None, None, :]
        u = np.zeros((3,) + cfg.shape)
        u[2] = 0.8
        kappa = O.lf_kappa_E(cfg, E, u)
        for i in range(2, 6):
            assert kappa[0, 0, 0, :, i] == pytest.approx(np.full(4, 0.8 * fac), rel=1e-15, abs=0), (beta, i)


@pytest.mark.parametrize("dims", [(6, 5, 1), (5, 4, 6)])
def test_lf_b_increment_faces_of_one_node(dims):
    # |u| = U only at node n0 = (i0, j0, k0); B_z = b only in cell c0 = (i0, j0, k0).
    # A face between cell c and c + e_d has its nodes at index c_d + 1 along d;
    # a is |u| averaged over the face's nodes (4 in 3D; in 2D the collapsed z
    # pairs them, so each node counts twice): U/4 in 3D, U/2 in 2D on the faces
    # that contain n0.  Of the faces next to c0, only its low face along each
    # axis d (between c0 - e_d and c0, nodes at index i0 along d) contains n0.
    # The ratio there is (B[c0-e_d] - B[c0-2e_d]) / (B[c0] - B[c0-e_d]) = 0/b, so
    # phi_B = 0 and F = a/2 (b - 0); every other face has a = 0 or no jump.
    # Hence, with f_d = dt/dx_d (Eq. 17-18):
    #   D(c0) = -sum_d f_d a b / 2,   D(c0 - e_d) = +f_d a b / 2.
    cfg = O.make_cfg(dims, (0.1, 0.2, 0.3), lf_on=1, lf_speed_c=0, lf_beta=1.0, dt=0.05)
    nz, ny, nx = cfg.shape
    dim = 3 if nz > 1 else 2
    i0, j0, k0 = 0, 2, (1 if nz > 1 else 0)
    U, b = 1.7, 0.9
    u = np.zeros((3,) + cfg.shape)
    u[1, k0, j0, i0] = -U
    Bc = np.zeros((3,) + cfg.shape)
    Bc[2, k0, j0, i0] = b
    D = O.lf_b_increment(cfg, Bc, u)
    a = U / 4 if dim == 3 else U / 2
    want = {(k0, j0, i0): 0.0}
    for d in range(dim):
        f = cfg.dt / cfg.dx[d]
        m = [i0, j0, k0]
        m[d] -= 1
        want[(k0, j0, i0)] -= f * a * b / 2
        want[(m[2] % nz, m[1] % ny, m[0] % nx)] = f * a * b / 2
    assert not _nonzero(D[0]) and not _nonzero(D[1])
    got = _nonzero(D[2])
    assert set(got) == set(want)
    for key, v in want.items():
        assert got[key] == pytest.approx(v, rel=1e-14), key
