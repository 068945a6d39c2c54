"""GPU parity of the learned preconditioner's kernels (BF16 tensor-core 3x3
convolutions with FP32 accumulation: forward, data gradient, weight gradient)
against the FP64 oracle network, and the gain of the trained network inside
FGMRES.

Tolerances.  The oracle runs on the same BF16-rounded weights and inputs, so
what remains is the BF16 rounding (relative 2^-9) of the three hidden
activations and, backwards, of the propagated gradients, plus FP32
accumulation.  Against the FP64 oracle: relative L2 <= 1e-2 for the network
output and the loss; <= 5e-2 for every layer's weight and bias gradient (the
first layer's weight gradient sums products of three times re-rounded
back-propagated values over all pixels with cancellation; a BF16 emulation in
plain PyTorch shows the same 2-4 % on these inputs).  Against that emulation,
which rounds at the same points as the kernels, the kernels agree to 2e-3 in
the output and 1e-2 in the gradients (FP32 against FP64 accumulation moves a
few values across a BF16 rounding boundary, and the first layer's weight
gradient amplifies that by the same cancellation).
"""
import numpy as np
import pytest

import oracle as O
import workloads

pytestmark = pytest.mark.gpu

TOL_FWD = 1e-2
TOL_GRAD = 5e-2
TOL_EMU = 2e-3
TOL_EMU_GRAD = 1e-2


def rel(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_11320_gb300 as g
    g.lib()
    ctx = g.Context(g.make_config((16, 8, 1), (0.1, 0.1, 1.0)))
    yield g, torch, ctx
    ctx.close()


def bf16(torch, a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def random_params(seed, bias_scale=0.1):
    """He-scaled weights and small biases, in the oracle's layout."""
    rng = np.random.default_rng(seed)
    chans = [3, 32, 32, 32, 3]
    out = []
    for l in range(4):
        cin, cout = chans[l], chans[l + 1]
        out.append(rng.standard_normal(cout * cin * 9) * np.sqrt(2.0 / (9 * cin)))
        out.append(rng.standard_normal(cout) * bias_scale)
    p = np.concatenate(out)
    assert p.size == O.net_param_count()
    return p


def weights_bf16(torch, p):
    """Round every weight (not the biases, which stay FP32) to BF16."""
    q = p.copy()
    chans = [3, 32, 32, 32, 3]
    off = 0
    for l in range(4):
        nw = chans[l + 1] * chans[l] * 9
        q[off:off + nw] = bf16(torch, p[off:off + nw])
        off += nw + chans[l + 1]
    return q


def layer_slices():
    chans = [3, 32, 32, 32, 3]
    off, out = 0, []
    for l in range(4):
        nw = chans[l + 1] * chans[l] * 9
        out.append((f"W{l + 1}", slice(off, off + nw)))
        out.append((f"b{l + 1}", slice(off + nw, off + nw + chans[l + 1])))
        off += nw + chans[l + 1]
    return out


def emulate_bf16(torch, p, x, t=None, periodic=True):
    """The network in plain PyTorch (CPU, FP64 arithmetic) rounding to BF16 at
    the points where the kernels store BF16: the input, the hidden
    activations, and backwards the output gradient and the propagated
    gradients.  Returns y, or (y, grads by layer name) when t is given."""
    F = torch.nn.functional
    chans = [3, 32, 32, 32, 3]
    off, Ws, bs = 0, [], []
    for l in range(4):
        nw = chans[l + 1] * chans[l] * 9
        Ws.append(torch.tensor(p[off:off + nw], dtype=torch.float64).reshape(chans[l + 1], chans[l], 3, 3))
        bs.append(torch.tensor(p[off + nw:off + nw + chans[l + 1]], dtype=torch.float64))
        off += nw + chans[l + 1]

    def rb(a):
        return a.to(torch.bfloat16).to(torch.float64)

    def pad(a):
        return F.pad(a, (1, 1, 1, 1), mode="circular") if periodic else F.pad(a, (1, 1, 1, 1))

    h = [rb(torch.tensor(x, dtype=torch.float64)[None])]
    for l in range(4):
        a = F.conv2d(pad(h[-1]), Ws[l]) + bs[l][None, :, None, None]
        h.append(rb(torch.relu(a)) if l < 3 else a)
    y = h[-1]
    if t is None:
        return y[0].numpy()
    assert not periodic
    H, W = x.shape[1:]
    d = rb((y - torch.tensor(t, dtype=torch.float64)[None]) / y.numel())
    grads = {}
    for l in range(3, -1, -1):
        hl = pad(h[l])
        gw = torch.zeros_like(Ws[l])
        for ky in range(3):
            for kx in range(3):
                gw[:, :, ky, kx] = torch.einsum("bohw,bihw->oi", d, hl[:, :, ky:ky + H, kx:kx + W])
        grads[f"W{l + 1}"] = gw.reshape(-1).numpy()
        grads[f"b{l + 1}"] = d.sum((0, 2, 3)).numpy()
        if l > 0:
            d = rb(F.conv_transpose2d(d, Ws[l], padding=1) * (h[l] > 0))
    return y[0].numpy(), grads


# (H, W): the convolution works on units of 4 rows x 128 columns.  Narrow
# images (one partial unit per row pair, odd heights), one exact unit, and
# rows of several units with a ragged last one (the periodic halo crossing
# unit and image edges).
SHAPES = [(24, 40), (8, 16), (5, 7), (33, 50), (2, 128), (7, 300), (4, 256)]


@pytest.mark.parametrize("H,W", SHAPES)
def test_forward_matches_oracle(env, H, W):
    g, torch, ctx = env
    p = random_params(11)
    ctx.precond_set_weights(p.astype(np.float32))
    x = np.random.default_rng(H * 1000 + W).standard_normal((3, H, W))
    xb = bf16(torch, x)
    y_ref = O.net_forward(weights_bf16(torch, p.astype(np.float32)), xb, periodic=True)
    xd = torch.from_numpy(xb.astype(np.float32)).cuda()
    yd = torch.zeros((3, H, W), dtype=torch.float32, device="cuda")
    ctx.precond_forward(xd, yd)
    y = yd.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(y))
    assert rel(y, y_ref) <= TOL_FWD, rel(y, y_ref)
    y_emu = emulate_bf16(torch, weights_bf16(torch, p.astype(np.float32)), xb)
    assert rel(y, y_emu) <= TOL_EMU, rel(y, y_emu)


@pytest.mark.parametrize("H,W", [(16, 24), (9, 13), (24, 40)])
def test_loss_and_gradients_match_oracle(env, H, W):
    g, torch, ctx = env
    p = random_params(23)
    ctx.precond_set_weights(p.astype(np.float32))
    rng = np.random.default_rng(7 + H)
    xb = bf16(torch, rng.standard_normal((3, H, W)))
    t = rng.standard_normal((3, H, W)).astype(np.float32).astype(np.float64)
    pb = weights_bf16(torch, p.astype(np.float32))
    L_ref, g_ref, _ = O.net_loss_backward(pb, xb, t, periodic=False)
    _, g_emu = emulate_bf16(torch, pb, xb, t, periodic=False)
    xd = torch.from_numpy(xb.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    gd = torch.zeros(O.net_param_count(), dtype=torch.float32, device="cuda")
    L = ctx.precond_loss_grad(xd, td, gd)
    grad = gd.cpu().numpy().astype(np.float64)
    assert abs(L - L_ref) <= TOL_FWD * abs(L_ref), (L, L_ref)
    for name, sl in layer_slices():
        e = rel(grad[sl], g_ref[sl])
        assert e <= TOL_GRAD, (name, e)
        e = rel(grad[sl], g_emu[name])
        assert e <= TOL_EMU_GRAD, (name, "vs BF16 emulation", e)


def test_solver_application_matches_oracle(env):
    """The network as FGMRES applies it to a Krylov column v (unit norm): the
    input is v / s (s = 1/sqrt(3N)) rounded to BF16, the last layer writes
    z = D^-1 v + s N(v/s) itself.  With zero weights N = 0, so that call gives
    D^-1 v, which must equal the block-Jacobi preconditioner's output; the
    difference of the two calls, divided by s, is N(v/s), compared with the
    oracle's forward pass.  The grid (160 x 13) has rows of two units (the
    second ragged) and an odd number of rows."""
    g, torch, _ = env
    wl = workloads.harris(nx=160, ny=13, ppc=4, steps=1)
    net = g.from_workload(wl, precond=g.GX_PRECOND_NET)
    jac = g.from_workload(wl, precond=g.GX_PRECOND_JACOBI)
    try:
        for c in (net, jac):
            assert c.step(1).converged
        H, W = 13, 160
        N = H * W
        v = np.random.default_rng(5).standard_normal(3 * N)
        v /= np.linalg.norm(v)
        s = 1.0 / np.sqrt(3 * N)
        vd = torch.from_numpy(v).cuda()
        z1 = torch.zeros_like(vd)
        z0 = torch.zeros_like(vd)
        zj = torch.zeros_like(vd)
        p = random_params(11)
        net.precond_set_weights(p.astype(np.float32))
        net.precond_apply(vd, z1)
        net.precond_set_weights(np.zeros(O.net_param_count(), np.float32))
        net.precond_apply(vd, z0)
        jac.precond_apply(vd, zj)
        z0h, zjh = z0.cpu().numpy(), zj.cpu().numpy()
        assert np.all(np.isfinite(z0h)) and rel(z0h, zjh) <= 1e-6, rel(z0h, zjh)
        y = ((z1.cpu().numpy() - z0h) / s).reshape(3, H, W)
        xb = bf16(torch, (v / s).reshape(3, H, W))
        pb = weights_bf16(torch, p.astype(np.float32))
        y_ref = O.net_forward(pb, xb, periodic=True)
        assert rel(y, y_ref) <= TOL_FWD, rel(y, y_ref)
        y_emu = emulate_bf16(torch, pb, xb)
        assert rel(y, y_emu) <= TOL_EMU, rel(y, y_emu)
    finally:
        net.close()
        jac.close()


def test_set_get_weights_roundtrip_and_errors(env):
    g, torch, ctx = env
    p = random_params(5).astype(np.float32)
    ctx.precond_set_weights(p)
    assert np.array_equal(ctx.precond_get_weights(), p)
    L = g.lib()
    assert L.gx_precond_set_weights(ctx.h, p.ctypes.data, p.size - 1, 0) == g.GX_EINVAL
    # training without collected pairs is a state error, not a crash
    assert L.gx_precond_train(ctx.h, 4, 8, 2, 1, 1e-3, 0, None, None) == g.GX_ESTATE


def test_trained_network_reduces_gmres_iterations(env):
    """Collect training pairs from the run's own solves, train on the GPU,
    then compare FGMRES with the trained network against plain GMRES (and
    block Jacobi, reported) on the same plasma: fewer matrix-vector products
    per solve, the same true relative residual, the same fields."""
    g, torch, _ = env
    wl = workloads.harris(nx=64, ny=32, ppc=16, steps=40)
    ctxs = {k: g.from_workload(wl, precond=p) for k, p in
            (("plain", g.GX_PRECOND_NONE), ("jacobi", g.GX_PRECOND_JACOBI), ("net", g.GX_PRECOND_NET))}
    try:
        net = ctxs["net"]
        net.precond_collect(256)
        its = {k: [] for k in ctxs}
        for _ in range(24):
            for k, c in ctxs.items():
                its[k].append(c.step(1).iters)
        assert net.precond_pairs() >= 24
        losses = net.precond_train(npairs=256, crop=16, batch=32, epochs=300, lr=3e-3, seed=3)
        assert np.all(np.isfinite(losses))
        assert losses[-1] < 0.5 * losses[0], losses
        net.precond_collect(0)
        after = {k: [] for k in ctxs}
        for _ in range(8):
            for k, c in ctxs.items():
                st = c.step(1)
                assert st.converged and st.relres <= wl.gmres_tol, (k, st.relres)
                after[k].append(st.iters)
        Ep, Bp = ctxs["plain"].get_fields()
        En, Bn = net.get_fields()
        assert rel(En, Ep) <= 1e-5 and rel(Bn, Bp) <= 1e-5
        info = (after, its, losses)
        assert np.mean(after["net"]) < np.mean(after["plain"]), info
    finally:
        for c in ctxs.values():
            c.close()


def _splitmix64(x):
    m = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & m
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & m
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & m
    return x ^ (x >> 31)


def test_crop_store_geometry_and_training(env):
    """The crop store (gx_precond_collect_crops): every collected pair is cut into
    per_pair windows at the documented hash positions; windows of one pair agree
    wherever they overlap on the periodic grid (same field values, same scale),
    the scale is the pair's s > 0, the count is the ring's, and a network trained
    on the crops alone still cuts the Krylov steps of the solve."""
    g, torch, _ = env
    wl = workloads.harris(nx=64, ny=32, ppc=16, steps=40)
    C, per, seed = 16, 48, 11
    S = C + 8
    ctxs = {k: g.from_workload(wl, precond=p) for k, p in
            (("plain", g.GX_PRECOND_NONE), ("net", g.GX_PRECOND_NET))}
    try:
        net = ctxs["net"]
        net.precond_collect_crops(4096, C, per, seed)
        its = {k: [] for k in ctxs}
        for _ in range(12):
            for k, c in ctxs.items():
                its[k].append(c.step(1).iters)
        n = net.precond_pairs()
        assert n == min(4096, 12 * 7 * per), n           # (r0, e) and 6 Krylov pairs per solve
        # the first pair's windows: positions from the hash, overlaps consistent
        nx, ny = wl.n[0], wl.n[1]
        full = np.full((6, ny, nx), np.nan)
        scales = set()
        for b in range(per):
            crop, s = net.precond_crop(b, C)
            assert np.all(np.isfinite(crop)) and s > 0
            scales.add(s)
            h = _splitmix64(seed ^ _splitmix64(b))
            x0, y0 = (h & 0xFFFFFFFF) % nx, (h >> 32) % ny
            vals = crop.reshape(6, S, S)
            ys = (y0 + np.arange(S)) % ny
            xs = (x0 + np.arange(S)) % nx
            prev = full[:, ys[:, None], xs[None, :]]
            seen = np.isfinite(prev)
            assert np.array_equal(prev[seen], vals[seen]), b
            full[:, ys[:, None], xs[None, :]] = vals
        assert len(scales) == 1                          # one pair, one scale
        assert np.isfinite(full).mean() > 0.9            # the windows cover most of the grid
        losses = net.precond_train(npairs=256, crop=C, batch=32, epochs=300, lr=3e-3, seed=3)
        assert np.all(np.isfinite(losses)) and losses[-1] < 0.5 * losses[0], losses
        net.precond_collect(0)
        after = {k: [] for k in ctxs}
        for _ in range(8):
            for k, c in ctxs.items():
                st = c.step(1)
                assert st.converged and st.relres <= wl.gmres_tol, (k, st.relres)
                after[k].append(st.iters)
        assert np.mean(after["net"]) < np.mean(after["plain"]), (after, its)
    finally:
        for c in ctxs.values():
            c.close()
