"""Device-side species initialisation (gx_species_maxwellian) against the oracle.

The device draws every particle from the counter-based generator (Philox4x64-10,
key (seed, species), counter (0, cell, k, 0)); the oracle evaluates the same
draws (or_bc_sample at step 0).  Positions are exact (24-bit offsets, identical
in FP32 and FP64), velocities agree to FP32 rounding of the Box-Muller
transform (<= 1e-6 of the largest speed), weights to FP32 rounding; the charge,
current and mass-matrix moments of the two particle sets agree to 1e-5.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    g.lib()
    return g


SPECIES = [(-1.0, 0.04, 32, 1.0 / (4 * np.pi), (0.2, -0.05, 0.0), 0.08),
           (1.0, 1.0, 32, 1.0 / (4 * np.pi), (0.2, -0.05, 0.0), 0.015)]


@pytest.mark.parametrize("n,dx", [((24, 16, 1), (0.1, 0.08, 1.0)), ((40, 1, 1), (0.1, 1.0, 1.0))])
def test_device_maxwellian_matches_oracle_draws(gx, n, dx):
    seed = 77
    cfg = gx.make_config(n, dx, dt=0.02, comoving=1, lf_on=1, seed=seed, track_ids=1)
    ctx = gx.Context(cfg)
    ocfg = O.make_cfg(n, dx, dt=0.02, comoving=1, lf_on=1)
    ref = []
    for s, (q, m, ppc, n0, u, vth) in enumerate(SPECIES):
        assert ctx.species_maxwellian(q, m, ppc, n0, u, vth) == s
        ref.append(O.maxwellian_species(ocfg, seed, s, ppc, n0, u, vth))
    B = np.zeros((3, 1, n[1], n[0]))
    B[2] = 0.1
    E = np.zeros_like(B)
    ctx.fields_set(E, B)
    for s, r in enumerate(ref):
        p = ctx.get_particles(s, ids=True)
        assert len(p["x"]) == len(r["x"]) == n[0] * n[1] * SPECIES[s][2]
        order = np.argsort(p["id"])                 # ids are cell * ppc + k: the oracle's order
        assert np.array_equal(p["x"][order], r["x"]) and np.array_equal(p["y"][order], r["y"])
        vmax = max(np.abs(r[k]).max() for k in ("vx", "vy", "vz"))
        for k in ("vx", "vy", "vz"):
            assert np.abs(p[k][order] - r[k]).max() <= 1e-6 * vmax, k
        assert np.allclose(p["w"][order], r["w"], rtol=1e-7, atol=0)
    ctx.deposit()
    rho, J, M, u = ctx.get_moments()
    ctx.close()
    pl = O.Plasma([s[0] for s in SPECIES], [s[1] for s in SPECIES],
                  np.concatenate([np.full(len(r["x"]), s, np.int32) for s, r in enumerate(ref)]),
                  *[np.concatenate([r[k] for r in ref]) for k in ("x", "y", "z", "vx", "vy", "vz", "w")])
    Bn = O.node_avg(ocfg, B)
    rm, P = O.bulk_moments(ocfg, pl)
    uo = O.bulk_velocity(ocfg, rm, P)
    orho, oJ, oM = O.deposit(ocfg, pl, Bn, u=uo)

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(rho, orho) <= 1e-5 and rel(J, oJ) <= 1e-5 and rel(M, oM) <= 1e-5, (rel(rho, orho), rel(J, oJ))


def test_device_maxwellian_rejects_bad_arguments(gx):
    ctx = gx.Context(gx.make_config((8, 8, 1), (0.1, 0.1, 1.0)))
    for args in ((-1.0, 0.04, 0, 1.0, (0, 0, 0), 0.1), (-1.0, 0.0, 8, 1.0, (0, 0, 0), 0.1),
                 (-1.0, 0.04, 8, 1.0, (0, 0, 0), -0.1)):
        with pytest.raises(gx.GxError) as e:
            ctx.species_maxwellian(*args)
        assert e.value.status == gx.GX_EINVAL
    ctx.close()


def test_dense_cells_one_step_matches_oracle(gx):
    """Dense cells: 2048 particles per cell and species on 8 x 8 cells (a bin of
    3,328 slots streamed through 32 chunks per cell and push): one whole step
    against the oracle on the same drawn particles, fields within 1e-6 and the
    particle count unchanged."""
    n, dx, seed, ppc = (8, 8, 1), (0.1, 0.1, 1.0), 5, 2048
    cfg = gx.make_config(n, dx, dt=0.02, comoving=1, lf_on=1, seed=seed, gmres_tol=1e-12)
    ctx = gx.Context(cfg)
    ocfg = O.make_cfg(n, dx, dt=0.02, comoving=1, lf_on=1, gmres_tol=1e-12)
    ref = []
    for s, (q, m, _, n0, u, vth) in enumerate(SPECIES):
        ctx.species_maxwellian(q, m, ppc, n0, u, vth)
        ref.append(O.maxwellian_species(ocfg, seed, s, ppc, n0, u, vth))
    B = np.zeros((3, 1, n[1], n[0]))
    B[2] = 0.1
    E = np.zeros_like(B)
    E[1] = -0.2 * 0.1            # -u x B for u = 0.2 x, B = 0.1 z
    ctx.fields_set(E, B)
    assert ctx.step(1).converged == 1
    E1, B1 = ctx.get_fields()
    counts = [ctx.species_count(s) for s in range(2)]
    ctx.close()
    pl = O.Plasma([s[0] for s in SPECIES], [s[1] for s in SPECIES],
                  np.concatenate([np.full(len(r["x"]), s, np.int32) for s, r in enumerate(ref)]),
                  *[np.concatenate([r[k] for r in ref]) for k in ("x", "y", "z", "vx", "vy", "vz", "w")])
    Eo, Bo = E.copy(), B.copy()
    assert O.step(ocfg, pl, Eo, Bo)["rc"] == 0

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(E1, Eo) <= 1e-6 and rel(B1, Bo) <= 1e-6, (rel(E1, Eo), rel(B1, Bo))
    assert counts == [n[0] * n[1] * ppc] * 2


def test_four_species_step_matches_oracle(gx):
    """The largest species count (4: electrons, protons, alpha particles and a
    heavy ion): one whole step against the oracle on the same drawn particles
    (fields within 1e-6), and a fifth species is refused."""
    n, dx, seed = (16, 12, 1), (0.1, 0.1, 1.0), 9
    sp4 = [(-1.0, 0.04, 24, 1.4 / (4 * np.pi), (0.2, 0.0, 0.0), 0.08),
           (1.0, 1.0, 24, 1.0 / (4 * np.pi), (0.2, 0.0, 0.0), 0.015),
           (2.0, 4.0, 16, 0.15 / (4 * np.pi), (0.2, 0.0, 0.0), 0.01),
           (1.0, 16.0, 8, 0.1 / (4 * np.pi), (0.1, 0.05, 0.0), 0.005)]
    cfg = gx.make_config(n, dx, dt=0.02, comoving=1, lf_on=1, seed=seed, gmres_tol=1e-12)
    ctx = gx.Context(cfg)
    ocfg = O.make_cfg(n, dx, dt=0.02, comoving=1, lf_on=1, gmres_tol=1e-12)
    ref = []
    for s, (q, m, ppc, n0, u, vth) in enumerate(sp4):
        assert ctx.species_maxwellian(q, m, ppc, n0, u, vth) == s
        ref.append(O.maxwellian_species(ocfg, seed, s, ppc, n0, u, vth))
    with pytest.raises(gx.GxError) as e:
        ctx.species_maxwellian(1.0, 1.0, 4, 0.01, (0, 0, 0), 0.01)
    assert e.value.status == gx.GX_EINVAL
    B = np.zeros((3, 1, n[1], n[0]))
    B[2] = 0.1
    E = np.zeros_like(B)
    ctx.fields_set(E, B)
    assert ctx.step(1).converged == 1
    E1, B1 = ctx.get_fields()
    ctx.close()
    pl = O.Plasma([s[0] for s in sp4], [s[1] for s in sp4],
                  np.concatenate([np.full(len(r["x"]), s, np.int32) for s, r in enumerate(ref)]),
                  *[np.concatenate([r[k] for r in ref]) for k in ("x", "y", "z", "vx", "vy", "vz", "w")])
    Eo, Bo = E.copy(), B.copy()
    assert O.step(ocfg, pl, Eo, Bo)["rc"] == 0

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(E1, Eo) <= 1e-6 and rel(B1, Bo) <= 1e-6, (rel(E1, Eo), rel(B1, Bo))
