"""The allocation-free particle gather against the allocating one, through the
C ABI.  Both copy the same FP32/FP64 values in the same bin order, so the
comparison is exact (tolerance 0).  The gather exists for callers that cannot
allocate, so the tests also check that calls leave the device's free memory
unchanged, including the first call in a fresh process (its scratch lookup
and module load happen when the context is created).  Collected last so that
it also runs after every other test has used the device; it passes alone in a
fresh process too.
"""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "vx", "vy", "vz", "w", "id")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    g.lib()
    return g, torch


def device_out(torch, n):
    f64 = dict(dtype=torch.float64, device="cuda")
    f32 = dict(dtype=torch.float32, device="cuda")
    out = {k: torch.full((n,), -7.0, **f64) for k in ("x", "y", "z")}
    out.update({k: torch.full((n,), -7.0, **f32) for k in ("vx", "vy", "vz", "w")})
    out["id"] = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    return out


def check_same(torch, ctx, s):
    ref = ctx.get_particles(s, ids=True)
    n = ctx.species_count(s)
    assert n == ref["x"].size and n > 0
    for _ in range(2):      # two calls in a row on the same scratch
        out = ctx.get_particles_noalloc(s, device_out(torch, n))
        torch.cuda.synchronize()
        for k in FIELDS:
            assert np.array_equal(out[k].cpu().numpy(), ref[k]), k


def test_noalloc_gather_matches_allocating_gather(env):
    g, torch = env
    wl = workloads.uniform_drift(n=(40, 24, 1), ppc=16, ns_j=1)
    ctx = g.from_workload(wl, track_ids=1)
    try:
        for s in range(len(wl.species)):
            check_same(torch, ctx, s)
        # after a push the bins hold stayers (front) and arrivals (back)
        ctx.step(2)
        for s in range(len(wl.species)):
            check_same(torch, ctx, s)
        # repeated calls allocate nothing: the device's free memory stays put
        outs = [device_out(torch, ctx.species_count(s)) for s in range(len(wl.species))]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            for s in range(len(wl.species)):
                ctx.get_particles_noalloc(s, outs[s])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        ctx.close()


def test_first_call_in_a_fresh_process_allocates_nothing(env):
    # A new process: the context's creation looks the scratch up and loads the
    # gather's code, so even the very first gather leaves free memory unchanged.
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import torch
        import paper_2506_11320_gb300 as g
        import workloads
        torch.cuda.init()
        wl = workloads.uniform_drift(n=(24, 16, 1), ppc=8)
        ctx = g.from_workload(wl)
        n = ctx.species_count(0)
        out = {k: torch.zeros(n, dtype=torch.float64, device="cuda") for k in ("x", "y", "z")}
        out.update({k: torch.zeros(n, dtype=torch.float32, device="cuda") for k in ("vx", "vy", "vz", "w")})
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        ctx.get_particles_noalloc(0, out)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        ref = ctx.get_particles(0)
        assert all((out[k].cpu().numpy() == ref[k]).all() for k in out)
        print("FREE", free0, free1)
        ctx.close()
    """) % root
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("FREE")][-1]
    free0, free1 = (int(v) for v in line.split()[1:])
    assert free0 == free1, (free0, free1)


def test_noalloc_gather_rejects_large_grids_and_bad_arguments(env):
    g, torch = env
    L = g.lib()
    maxc = int(L.gx_noalloc_max_cells())
    assert maxc == 1 << 18
    nx = 1024
    ny = maxc // nx + 1                      # one row more than the scratch holds
    ctx = g.Context(g.make_config((nx, ny, 1), (0.1, 0.1, 1.0)))
    try:
        n = 64
        rng = np.random.default_rng(1)
        ctx.species_add(-1.0, 1.0, rng.random(n) * nx * 0.1, rng.random(n) * ny * 0.1, np.zeros(n),
                        np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros(n, np.float32),
                        np.ones(n, np.float32))
        out = device_out(torch, n)
        out["id"] = None                     # this context carries no ids
        with pytest.raises(g.GxError) as e:
            ctx.get_particles_noalloc(0, out)
        assert e.value.status == g.GX_EINVAL
        assert "fixed scratch" in str(e.value)
        assert L.gx_get_particles_noalloc(ctx.h, 5, None, None, None, None, None, None, None, None, None) \
            == g.GX_EINVAL
    finally:
        ctx.close()
    assert L.gx_get_particles_noalloc(None, 0, None, None, None, None, None, None, None, None, None) \
        == g.GX_EINVAL
