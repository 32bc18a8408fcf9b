"""The BF16 surrogate network against the FP64 CPU oracle (forward and
gradients), its training, checkpointing, and the surrogate weights path
(projection, residual check, FP64 fallback)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

N_IN, N_OUT, H, L = 50, 25, 256, 3


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1912_13282_gb300 import _build
    _build.build()
    import paper_1912_13282_gb300 as pkg
    return pkg


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


def blocks(n_in, n_out):
    """(name, size) of the plain parameter layout."""
    out, ins, outs = [], [n_in, H, H, H], [H, H, H, n_out]
    for l in range(4):
        out += [(f"W{l + 1}", ins[l] * outs[l]), (f"b{l + 1}", outs[l])]
    return out


def split(v, n_in, n_out):
    res, o = {}, 0
    for name, sz in blocks(n_in, n_out):
        res[name] = v[o:o + sz]
        o += sz
    return res


def test_forward_and_gradients_match_oracle(P, ctx, oracle):
    net = P.MLP(ctx, N_IN, N_OUT, seed=3)
    npar = net.num_params
    assert npar == oracle.mlp_nparams(N_IN, H, L, N_OUT)
    rng = np.random.default_rng(0)
    params = net.get_params().astype(np.float64)
    # nonzero biases so every parameter block is exercised
    sp = split(params, N_IN, N_OUT)
    for name in ("b1", "b2", "b3", "b4"):
        sp[name][:] = rng.normal(scale=0.1, size=sp[name].shape)
    net.set_params(params.astype(np.float32))
    params = net.get_params().astype(np.float64)
    Bn = 512
    x = rng.uniform(-1, 1, size=(Bn, N_IN))
    t = rng.normal(size=(Bn, N_OUT))
    xd = torch.from_numpy(x.astype(np.float32)).cuda()
    td = torch.from_numpy(t.astype(np.float32)).cuda()
    y = torch.empty((Bn, N_OUT), dtype=torch.float32, device="cuda")
    net.forward(xd, y)
    torch.cuda.synchronize()
    yref, _ = oracle.mlp_forward(N_IN, H, L, N_OUT, params, x.astype(np.float32).astype(np.float64))
    rel = np.linalg.norm(y.cpu().numpy() - yref) / np.linalg.norm(yref)
    assert rel <= 2e-2, rel
    loss, g = net.grad(xd, td)
    lref, gref = oracle.mlp_grad(N_IN, H, L, N_OUT, params, x.astype(np.float32).astype(np.float64), t.astype(np.float32).astype(np.float64))
    assert abs(loss - lref) <= 2e-2 * lref
    gs, gr = split(g.astype(np.float64), N_IN, N_OUT), split(gref, N_IN, N_OUT)
    errs = {name: float(np.linalg.norm(gs[name] - gr[name]) / max(np.linalg.norm(gr[name]), 1e-30))
            for name, _ in blocks(N_IN, N_OUT)}
    # BF16 operands (u = 2^-8) in the forward and backward GEMMs, FP32 sums:
    # about 1e-2 relative in norm per parameter block
    assert max(errs.values()) <= 1e-2, errs
    net.close()


def _bf16_forward_sigma(params, x, mean_std=None):
    """Per-element scale of |y_bf16 - y| for the network evaluated with BF16
    weights and activations and FP32 accumulation, from the layer widths, by
    probabilistic rounding-error analysis (Higham & Mary, SIAM J. Sci.
    Comput. 2019: independent rounding errors of unit roundoff u add up like
    sqrt(n) u instead of n u).  Each rounding is modelled as a relative error
    uniform in [-u, u] (variance u^2/3), u = 2^-8 for BF16: the input, every
    weight and every stored activation; the hardware tanh of GELU adds an
    absolute error below 2^-11 |z|.  Variances propagate through layer l as
        V_l = W_l^2 v_{l-1} + (u^2/3) W_l^2 h_{l-1}^2,
        v_l = 1.13^2 V_l + (u^2/3) h_l^2 + (2^-22/3) z_l^2,  v_0 = (u^2/3) x^2,
    sums over the layer's input width, 1.13 the largest slope of GELU.  The
    FP64 activations h_l, z_l are recomputed here only to evaluate the scale;
    returns sqrt(V_4) times the output scaling."""
    u2 = 2.0 ** -16 / 3
    sp = split(params, N_IN, N_OUT)
    c = np.sqrt(2 / np.pi)
    h = x
    v = u2 * x * x
    for l in range(1, 5):
        W, b = sp[f"W{l}"].reshape(-1, h.shape[1]), sp[f"b{l}"]
        W2 = W * W
        z = h @ W.T + b
        V = v @ W2.T + u2 * ((h * h) @ W2.T)
        if l == 4:
            out = np.sqrt(V)
            break
        h = 0.5 * z * (1 + np.tanh(c * (z + 0.044715 * z ** 3)))
        v = 1.13 ** 2 * V + u2 * h * h + 2.0 ** -22 / 3 * z * z
    if mean_std is not None:
        out = out * np.abs(mean_std[1])[None, :]
    return out


@pytest.mark.parametrize("B", [1, 127, 129, 65536 + 129])
def test_fused_inference_matches_oracle_elementwise(P, ctx, oracle, B):
    """The fused tensor-core forward (tcgen05) against the FP64 oracle forward
    of the same FP32 parameters, element by element: every output within
    lambda = 4 of the rounding-error scale of _bf16_forward_sigma (a sum of
    independent roundings exceeds 4 sigma with probability below 2 exp(-8)
    per element; the scale's GELU slope 1.13 already overstates the typical
    one, and a BF16 emulation of the network stays below 0.7 sigma), for a
    single row, a partial tile, one row past a tile and more tiles than SMs
    with a ragged tail.  Also: the model is not loose (the 99th percentile
    of |error| / sigma is at least 0.1)."""
    net = P.MLP(ctx, N_IN, N_OUT, seed=17)
    rng = np.random.default_rng(B)
    p = net.get_params()
    p += rng.normal(scale=0.02, size=p.shape).astype(np.float32)   # nonzero biases too
    net.set_params(p)
    mean, std = rng.normal(size=N_OUT), rng.uniform(0.5, 2.0, size=N_OUT)
    net.set_output_scaling(mean, std)
    mean, std = mean.astype(np.float32).astype(np.float64), std.astype(np.float32).astype(np.float64)
    x = rng.uniform(-1, 1, size=(B, N_IN)).astype(np.float32)
    y = torch.full((B, N_OUT), float("nan"), device="cuda")
    net.forward(torch.from_numpy(x).cuda(), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    params = net.get_params().astype(np.float64)
    # the oracle in chunks (its forward holds B x 256 activations per layer)
    ref = np.empty_like(got)
    bound = np.empty_like(got)
    for a in range(0, B, 8192):
        xb = x[a:a + 8192].astype(np.float64)
        yo, _ = oracle.mlp_forward(N_IN, H, L, N_OUT, params, xb)
        ref[a:a + 8192] = yo * std + mean
        bound[a:a + 8192] = _bf16_forward_sigma(params, xb, (mean, std))
    assert np.isfinite(got).all()
    ratio = np.abs(got - ref) / bound
    worst = np.unravel_index(np.argmax(ratio), ratio.shape)
    assert ratio.max() <= 4.0, (float(ratio.max()), worst, float(got[worst]), float(ref[worst]),
                                float(bound[worst]))
    if B >= 127:
        assert np.quantile(ratio, 0.99) >= 0.1, float(np.quantile(ratio, 0.99))
    net.close()


@pytest.mark.parametrize("B", [1, 127, 128, 300, 5000, 65536 + 129])
def test_fused_inference_matches_layered(P, ctx, B):
    """The fused tensor-core forward (tcgen05, one launch for all rows) equals
    the layer-by-layer forward of the same BF16 network to BF16 rounding, for
    ragged row counts (partial last tile, more tiles than SMs, more rows than
    one layered batch)."""
    net = P.MLP(ctx, N_IN, N_OUT, seed=11)
    rng = np.random.default_rng(2)
    p = net.get_params()
    p += rng.normal(scale=0.02, size=p.shape).astype(np.float32)   # nonzero biases too
    net.set_params(p)
    net.set_output_scaling(rng.normal(size=N_OUT), rng.uniform(0.5, 2.0, size=N_OUT))
    x = torch.from_numpy(rng.uniform(-1, 1, size=(B, N_IN)).astype(np.float32)).cuda()
    y_f = torch.full((B, N_OUT), float("nan"), device="cuda")
    y_l = torch.full((B, N_OUT), float("nan"), device="cuda")
    net.forward(x, y_f)
    ctx.set_option(P.binding.OPT_MLP_INFER, P.binding.MLP_LAYERED)
    try:
        net.forward(x, y_l)
    finally:
        ctx.set_option(P.binding.OPT_MLP_INFER, P.binding.MLP_FUSED)
    torch.cuda.synchronize()
    assert torch.isfinite(y_f).all()
    err = (y_f - y_l).abs().max().item()
    scale = y_l.abs().max().item()
    assert err <= 2e-2 * scale, (err, scale)
    net.close()


def test_targets_and_output_scaling_on_gpu(P, ctx):
    """mm_surrogate_targets (w s^2 per row, FP32) and mm_mlp_fit_output_scaling
    (column mean and standard deviation, n - 1 denominator) against numpy."""
    rng = np.random.default_rng(7)
    rows, n = 3000, N_OUT
    rp = torch.arange(rows + 1, dtype=torch.int64, device="cuda") * n
    vals = torch.from_numpy(rng.normal(size=rows * n)).cuda()
    scale = torch.from_numpy(rng.uniform(0.01, 0.1, size=rows - 100)).cuda()
    out = torch.full((rows - 100, n), float("nan"), dtype=torch.float32, device="cuda")
    P.binding.surrogate_targets(ctx, rp, 50, rows - 50, n, vals, scale, 2, out)
    torch.cuda.synchronize()
    v = vals.cpu().numpy().reshape(rows, n)[50:rows - 50]
    ref = (v * scale.cpu().numpy()[:, None] ** 2).astype(np.float32)
    assert np.array_equal(out.cpu().numpy(), ref)
    net = P.MLP(ctx, N_IN, N_OUT, seed=1)
    t = torch.from_numpy((rng.normal(size=(5000, N_OUT)) * 3 + 1).astype(np.float32)).cuda()
    net.fit_output_scaling(t)
    th = t.cpu().numpy().astype(np.float64)
    mean, std = th.mean(0), th.std(0, ddof=1)
    y = torch.empty((1, N_OUT), device="cuda")
    # the scaling is what the network undoes: zero weights and biases but an
    # output bias of 1 give y = 1 * std + mean
    p = np.zeros(net.num_params, dtype=np.float32)
    p[-N_OUT:] = 1.0
    net.set_params(p)
    net.forward(torch.zeros((1, N_IN), device="cuda"), y)
    torch.cuda.synchronize()
    assert np.allclose(y.cpu().numpy()[0], mean + std, rtol=1e-5, atol=1e-5), (y, mean + std)
    net.close()


def test_params_and_checkpoint_roundtrip(P, ctx, tmp_path):
    net = P.MLP(ctx, N_IN, N_OUT, seed=5)
    rng = np.random.default_rng(1)
    p = rng.normal(scale=0.05, size=net.num_params).astype(np.float32)
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    x = torch.rand((300, N_IN), device="cuda") * 2 - 1
    t = torch.randn((300, N_OUT), device="cuda")
    net.set_output_scaling(np.full(N_OUT, 0.5), np.full(N_OUT, 2.0))
    for _ in range(3):
        net.train_step(x, t, 1e-3)
    net.save(tmp_path / "ck.bin")
    y1 = torch.empty((300, N_OUT), device="cuda")
    net.forward(x, y1)
    net2 = P.MLP(ctx, N_IN, N_OUT, seed=9)
    net2.load(tmp_path / "ck.bin")
    y2 = torch.empty_like(y1)
    net2.forward(x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    # the Adam state came along: one more step on both stays identical
    net.train_step(x, t, 1e-3)
    net2.train_step(x, t, 1e-3)
    assert np.array_equal(net.get_params(), net2.get_params())
    net.close()
    net2.close()


@pytest.fixture(scope="module")
def trained(P, ctx):
    from paper_1912_13282_gb300 import surrogate as S
    data = S.make_dataset(ctx, 1 << 16, seed=1)
    net = P.MLP(ctx, N_IN, N_OUT, seed=0)
    losses = S.train(net, data["x"], data["t"], epochs=40, batch=2048, lr=3e-3, lr_final=1e-4)
    return net, losses


def test_training_reduces_loss(trained):
    net, losses = trained
    assert np.isfinite(losses).all()
    # normalised MSE starts near 1 (predicting the mean); the configured MLP on
    # rank-ordered offsets levels off well above 0 (its inputs permute under jitter)
    first, last = losses[:20].mean(), losses[-50:].mean()
    assert last < 0.8 * first, (first, last)


@pytest.mark.parametrize("wide", ["ff", "fp64"])
def test_surrogate_weights_path(P, ctx, oracle, trained, wide):
    """Held-out stencils: accepted rows reproduce the monomials to 1e-12 and
    equal the oracle's FP64 projection of the same prediction; rejected rows
    equal the FP64 solve; the residual check's rho agrees with the oracle's.
    The projection runs in double-FP32 (ff) or native FP64."""
    from paper_1912_13282_gb300 import surrogate as S
    net, _ = trained
    ctx.set_option(P.binding.OPT_WIDE, P.binding.WIDE_FP64 if wide == "fp64" else P.binding.WIDE_FF)
    try:
        _surrogate_path_checks(P, ctx, oracle, net, S)
    finally:
        ctx.set_option(P.binding.OPT_WIDE, P.binding.WIDE_FF)


def _surrogate_path_checks(P, ctx, oracle, net, S):
    count = 4096
    pts, rp, col = S.make_stencils(ctx, count, seed=10 ** 6)
    n, k, m = 25, 5, 4
    x = torch.empty((count, 2 * n), dtype=torch.float32, device="cuda")
    scale = torch.empty(count, dtype=torch.float64, device="cuda")
    P.stencil_features(ctx, pts, rp, col, 0, count, n, x, scale)
    pred = torch.empty((count, n), dtype=torch.float32, device="cuda")
    net.forward(x, pred)
    vals = torch.zeros(count * n, dtype=torch.float64, device="cuda")
    status = torch.empty(count, dtype=torch.int32, device="cuda")
    rho = torch.empty(count, dtype=torch.float32, device="cuda")
    tau = 1e-3
    P.rbffd_weights_surrogate(ctx, net, k, m, pts, rp, col, 0, count, n, tau, vals, status, rho)
    ref = torch.zeros_like(vals)
    ctx.rbffd_weights(P.LAP, k, m, pts, rp, col, [ref], row_end=count, n_max=n, precision=P.FP64)
    refir = torch.zeros_like(vals)
    ctx.rbffd_weights(P.LAP, k, m, pts, rp, col, [refir], row_end=count, n_max=n, precision=P.FP32_IR)
    vir = torch.zeros_like(vals)
    stir = torch.empty_like(status)
    P.rbffd_weights_surrogate(ctx, net, k, m, pts, rp, col, 0, count, n, tau, vir, stir,
                              fallback=P.FP32_IR)
    torch.cuda.synchronize()
    st, w, w64 = status.cpu().numpy(), vals.cpu().numpy(), ref.cpu().numpy()
    r = rho.cpu().numpy()
    acc = st == P.binding.ST_ACCEPTED
    fb = st == P.binding.ST_FALLBACK
    assert (acc | fb).all()
    assert acc.mean() > 0.2, acc.mean()
    assert np.array_equal(w.reshape(count, n)[fb], w64.reshape(count, n)[fb])
    assert (r[acc] <= tau).all()
    # FP32+IR fallback: same accepted rows and weights; the rejected rows
    # equal the FP32+IR solve (or the FP64 one for its own stragglers)
    st2, w2, wir = stir.cpu().numpy(), vir.cpu().numpy(), refir.cpu().numpy()
    assert np.array_equal(st2 == P.binding.ST_ACCEPTED, acc)
    assert np.array_equal(w2.reshape(count, n)[acc], w.reshape(count, n)[acc])
    rej_ok = (st2 == P.binding.ST_OK)
    rej_fb = (st2 == P.binding.ST_FALLBACK)
    assert (acc | rej_ok | rej_fb).all()
    assert np.array_equal(w2.reshape(count, n)[rej_ok], wir.reshape(count, n)[rej_ok])
    assert np.array_equal(w2.reshape(count, n)[rej_fb], w64.reshape(count, n)[rej_fb])
    pts_h, rp_h, col_h = pts.cpu().numpy(), rp.cpu().numpy(), col.cpu().numpy()
    pred_h, s_h = pred.cpu().numpy().astype(np.float64), scale.cpu().numpy()
    from _helpers import monomial_residual
    rows = np.nonzero(acc)[0][:300]
    assert monomial_residual(pts_h, None, rp_h, col_h, w, "lap", m, rows) <= 1e-12
    for i in rows[:120]:
        stn = col_h[rp_h[i]:rp_h[i + 1]]
        proj = oracle.project_lap(pts_h, stn, k, m, pred_h[i])
        got = w[rp_h[i]:rp_h[i + 1]] * s_h[i] ** 2
        assert np.abs(got - proj).max() <= 1e-9 * np.abs(proj).max()
    # rho against the oracle's, relatively, on accepted and rejected rows; the
    # accept/reject decision equals the oracle's wherever rho is clear of tau
    # by more than that tolerance (the GPU check runs in FP32: about u32 times
    # sum |A_ij w_j| ~ 1e-5 of ||l_phi|| absolute)
    sample = np.concatenate([np.nonzero(acc)[0][:200], np.nonzero(~acc)[0][:200]])
    rho_o = np.empty(len(sample))
    for t, i in enumerate(sample):
        stn = col_h[rp_h[i]:rp_h[i + 1]]
        proj = oracle.project_lap(pts_h, stn, k, m, pred_h[i])
        rho_o[t] = oracle.phi_residual_lap(pts_h, stn, k, m, proj)
    rho_g = r[sample].astype(np.float64)
    tol = 0.02 * rho_o + 2e-5
    assert (np.abs(rho_g - rho_o) <= tol).all(), float((np.abs(rho_g - rho_o) / (rho_o + 1e-30)).max())
    clear = np.abs(rho_o - tau) > 0.02 * tau + 2e-5
    assert clear.sum() >= 0.8 * len(sample)
    assert np.array_equal(acc[sample][clear], rho_o[clear] <= tau)
