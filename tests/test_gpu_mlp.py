"""GPU parity of the surrogate network's kernels with the FP64 oracle
(oracle/mlp.py): forward, MSE loss, back-propagated gradient, one Adam step,
and that native training reduces the loss."""
import numpy as np
import pytest

import workloads
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

SIZES = omlp.layer_sizes(5, 256, 4)


@pytest.fixture(scope="module")
def gb():
    import torch
    assert torch.cuda.is_available()
    import paper_1906_02818_gb300 as gb
    return gb


def _data(n, seed=1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n, 5)).astype(np.float32)
    t = (np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2] - 0.5 * x[:, 3] ** 2 + 0.1 * x[:, 4]).astype(np.float32)
    return x, t


def test_forward_fp32_matches_oracle(gb):
    import torch
    init = workloads.mlp_init()
    net = gb.Mlp(5, 256, 4, init)
    x, _ = _data(1000)
    y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = omlp.forward(omlp.unpack(init.astype(np.float64), SIZES), x.astype(np.float64))
    assert np.max(np.abs(y - want)) <= 1e-5 * np.max(np.abs(want)) + 1e-6
    net.close()


def test_loss_and_gradient_match_oracle(gb):
    import torch
    init = workloads.mlp_init(seed=7)
    net = gb.Mlp(5, 256, 4, init)
    x, t = _data(777, seed=2)
    loss, g = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    P = omlp.unpack(init.astype(np.float64), SIZES)
    l_ref, G = omlp.loss_and_grads(P, x.astype(np.float64), t.astype(np.float64))
    g_ref = omlp.pack(G)
    assert abs(loss - l_ref) <= 1e-5 * l_ref
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * scale, np.max(np.abs(g - g_ref)) / scale
    net.close()


def test_one_adam_step_matches_oracle(gb):
    import torch
    init = workloads.mlp_init(seed=8)
    net = gb.Mlp(5, 256, 4, init)
    x, t = _data(512, seed=3)
    net.train(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), epochs=1, batch=512, lr=1e-3)
    P = omlp.unpack(init.astype(np.float64), SIZES)
    _, G = omlp.loss_and_grads(P, x.astype(np.float64), t.astype(np.float64))
    Z = [(np.zeros_like(W), np.zeros_like(b)) for W, b in P]
    P1, _, _ = omlp.adam_step(P, G, Z, Z, 1, 1e-3)
    got, want, g = net.params(), omlp.pack(P1), np.abs(omlp.pack(G))
    big = g > 1e-4 * g.max()  # Adam's first step is lr * sign(g): compare where the sign is resolved
    assert np.max(np.abs(got[big] - want[big])) <= 1e-6 + 1e-6 * np.max(np.abs(want))
    net.close()


def test_training_reduces_loss(gb):
    import torch
    net = gb.Mlp(5, 256, 4, workloads.mlp_init(seed=9))
    x, t = _data(1 << 15, seed=4)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l0, _ = net.loss_grad(xd, td)
    l1 = net.train(xd, td, epochs=20, batch=1024, lr=1e-3)
    assert l1 < 0.05 * l0, (l0, l1)
    net.close()


# ----------------------------- BF16 inference ------------------------------

def _bf16_emulation(P, x):
    """The bf16 kernel's arithmetic in FP64: layer 0 as x_hi W_hi + x_lo W_hi
    + x_hi W_lo (hi = bf16 rounding, lo = bf16 of the FP32 remainder), every
    hidden operand rounded to bf16 after the SiLU, the last hidden layer's
    SiLU and the output layer unrounded."""
    from quant import to_bf16
    (W0, b0), hid, (Wo, bo) = P[0], P[1:-1], P[-1]
    x32 = np.asarray(x, dtype=np.float32)
    xh = to_bf16(x32)
    xl = to_bf16((x32 - xh.astype(np.float32)).astype(np.float32))
    w32 = W0.astype(np.float32)
    wh = to_bf16(w32)
    wl = to_bf16((w32 - wh.astype(np.float32)).astype(np.float32))
    z = xh @ wh + xl @ wh + xh @ wl + b0
    for W, b in hid:
        z = to_bf16(omlp.silu(z)) @ to_bf16(W) + b
    return (omlp.silu(z) @ Wo + bo)[:, 0]


def _bf16_case(gb, n_in, width, hidden, n, seed):
    import torch
    sizes = omlp.layer_sizes(n_in, width, hidden)
    rng = np.random.default_rng(seed)
    P = [(rng.normal(0, np.sqrt(2.0 / i), size=(i, o)), rng.normal(0, 0.1, size=o)) for i, o in zip(sizes, sizes[1:])]
    flat = omlp.pack(P).astype(np.float32)
    P = omlp.unpack(flat.astype(np.float64), sizes)
    net = gb.Mlp(n_in, width, hidden, flat)
    x = rng.uniform(-1.5, 1.5, size=(n, n_in)).astype(np.float32)
    y = net.forward(torch.from_numpy(x).cuda(), precision="bf16").cpu().numpy()
    net.close()
    return y, _bf16_emulation(P, x.astype(np.float64)), omlp.forward(P, x.astype(np.float64))[0]


@pytest.mark.parametrize("n", [1, 100, 128, 129, 384, 1000, 100003])
def test_forward_bf16_matches_emulation(gb, n):
    """Surrogate shape (5 -> 256 x 4 -> 1): ragged tile counts, one or two
    tiles per CTA pair, many pairs per CTA."""
    y, emu, exact = _bf16_case(gb, 5, 256, 4, n, seed=n)
    assert np.all(np.isfinite(y))
    scale = np.max(np.abs(exact)) + 1e-3
    e_emu = np.max(np.abs(y - emu)) / scale
    r_emu = np.sqrt(np.mean((y - emu) ** 2)) / scale
    e_ex = np.max(np.abs(y - exact)) / scale
    print(f"n={n}: |bf16 - emulation| max {e_emu:.2e} rms {r_emu:.2e}, |bf16 - fp64| max {e_ex:.2e} of max|y|")
    # The emulation differs from the kernel by tanh.approx in the SiLU (relative
    # 2^-11) and FP32 accumulation; each moves some activations across a bf16
    # rounding boundary (one bf16 ulp, 2^-8 relative, each), which the next
    # layers carry to the output: a few 1e-3 of max|y| at worst, far less on
    # average.  Against unrounded FP64, bf16 operands in three 256-wide layers.
    assert e_emu <= 6e-3 and r_emu <= 1e-3
    assert e_ex <= 3e-2


@pytest.mark.parametrize("n_in,width,hidden", [(1, 32, 1), (10, 64, 2), (3, 96, 3), (5, 128, 5), (8, 256, 2)])
def test_forward_bf16_shapes(gb, n_in, width, hidden):
    y, emu, exact = _bf16_case(gb, n_in, width, hidden, 777, seed=width + hidden)
    scale = np.max(np.abs(exact)) + 1e-3
    print(f"{n_in}->{width}x{hidden}: {np.max(np.abs(y - emu)) / scale:.2e} vs emulation, "
          f"{np.max(np.abs(y - exact)) / scale:.2e} vs fp64")
    assert np.max(np.abs(y - emu)) <= 6e-3 * scale
    assert np.max(np.abs(y - exact)) <= 3e-2 * scale


def test_forward_bf16_tracks_parameter_updates(gb):
    """The bf16 operand image is rebuilt after set_params and training."""
    import torch
    init = workloads.mlp_init(seed=3)
    net = gb.Mlp(5, 256, 4, init)
    x, t = _data(4096, seed=5)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y0 = net.forward(xd, precision="bf16").cpu().numpy()
    net.train(xd, td, epochs=2, batch=1024, lr=1e-3)
    y1 = net.forward(xd, precision="bf16").cpu().numpy()
    f1 = net.forward(xd).cpu().numpy()
    assert np.max(np.abs(y1 - y0)) > 1e-3
    assert np.max(np.abs(y1 - f1)) <= 3e-2 * np.max(np.abs(f1))
    net.set_params(init)
    assert np.array_equal(net.forward(xd, precision="bf16").cpu().numpy(), y0)
    net.close()


def test_forward_bf16_rejects_unsupported_shapes(gb):
    import torch
    from paper_1906_02818_gb300.native import MCError
    for n_in, width, hidden in [(5, 48, 2), (11, 64, 2), (5, 320, 2)]:
        sizes = omlp.layer_sizes(n_in, width, hidden)
        flat = np.zeros(sum(i * o + o for i, o in zip(sizes, sizes[1:])), dtype=np.float32)
        net = gb.Mlp(n_in, width, hidden, flat)
        with pytest.raises(MCError, match="bf16"):
            net.forward(torch.zeros((4, n_in), device="cuda"), precision="bf16")
        net.close()


def test_apply_grad_is_one_training_step(gb):
    """An Adam step with the batch gradient from loss_grad (the data-parallel
    path's update) equals one step of native training on that batch."""
    import torch
    init = workloads.mlp_init(seed=12)
    a, b = gb.Mlp(5, 256, 4, init), gb.Mlp(5, 256, 4, init)
    x, t = _data(1024, seed=6)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    _, g = a.loss_grad(xd, td)
    a.apply_grad(g, 1e-3)
    b.train(xd, td, epochs=1, batch=1024, lr=1e-3)
    assert np.max(np.abs(a.params() - b.params())) <= 1e-7
    a.close()
    b.close()


@pytest.mark.parametrize("mode", ["fp32", "tf32x3"])
def test_device_sums_equal_the_host_path(gb, mode):
    """The data-parallel building blocks on the device: two part-batch
    gradient sums (mc_mlp_loss_grad_sums) add up to n times the full batch's
    mean gradient and MSE (mc_mlp_loss_grad), and a summed gradient applied
    with scale 1/n (mc_mlp_apply_grad_sums) is the host path's Adam step
    (mc_mlp_apply_grad), three steps in a row."""
    import torch
    init = workloads.mlp_init(seed=13)
    a, b = gb.Mlp(5, 256, 4, init), gb.Mlp(5, 256, 4, init)
    a.set_train_mode(mode)
    b.set_train_mode(mode)
    x, t = _data(2048, seed=8)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    for step in range(3):
        loss, g = a.loss_grad(xd, td)
        # split batch: the summed halves reproduce the full batch's mean
        tot = b.loss_grad_sums(xd[:1000], td[:1000]) + b.loss_grad_sums(xd[1000:], td[1000:])
        assert abs(float(tot[-1]) / 2048 - loss) <= 1e-5 * loss, (step, float(tot[-1]) / 2048, loss)
        gd = tot[:-1].cpu().numpy() / 2048
        assert np.max(np.abs(gd - g)) <= 2e-5 * np.max(np.abs(g)), step
        # the update: the full batch's sums scaled by 1 / n, as the host step
        a.apply_grad(g, 1e-3)
        b.apply_grad_sums(b.loss_grad_sums(xd, td), 1.0 / 2048, 1e-3)
    pa, pb = a.params(), b.params()
    assert np.max(np.abs(pa - pb)) <= 1e-6 * max(1.0, np.max(np.abs(pa)))
    a.close()
    b.close()


@pytest.mark.parametrize("n", [130, 777, 4096])
def test_tf32x3_loss_and_gradient_match_oracle(gb, n):
    """Tensor-core training products (three-pass TF32, FP32 accumulation)
    against the FP64 oracle at the FP32 path's tolerances, and against the
    FP32 SIMT path; n = 130 (two row tiles, ragged), 777 (ragged K of the
    weight-gradient products), 4096 (the training batch, split K)."""
    import torch
    init = workloads.mlp_init(seed=7)
    net = gb.Mlp(5, 256, 4, init)
    x, t = _data(n, seed=2)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    l32, g32 = net.loss_grad(xd, td)
    net.set_train_mode("tf32x3")
    loss, g = net.loss_grad(xd, td)
    P = omlp.unpack(init.astype(np.float64), SIZES)
    l_ref, G = omlp.loss_and_grads(P, x.astype(np.float64), t.astype(np.float64))
    g_ref = omlp.pack(G)
    assert abs(loss - l_ref) <= 1e-5 * l_ref
    scale = np.max(np.abs(g_ref))
    err = np.max(np.abs(g - g_ref)) / scale
    print(f"n={n}: tf32x3 gradient max err {err:.2e} of max|g| (fp32 SIMT {np.max(np.abs(g32 - g_ref)) / scale:.2e})")
    assert err <= 1e-4
    # every layer's weights and biases, against its own scale
    off = 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        for cnt in (a * b, b):
            seg = slice(off, off + cnt)
            ls = np.max(np.abs(g_ref[seg]))
            assert np.max(np.abs(g[seg] - g_ref[seg])) <= 2e-4 * ls + 1e-12, (a, b, cnt)
            off += cnt
    net.close()


def test_tf32x3_training_tracks_fp32_training(gb):
    """Three epochs of Adam from the same initialisation in both arithmetics:
    both reduce the loss, and the final losses agree to 1 %."""
    import torch
    init = workloads.mlp_init(seed=5)
    x, t = _data(1 << 14, seed=4)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    out = {}
    for mode in ("fp32", "tf32x3"):
        net = gb.Mlp(5, 256, 4, init)
        net.set_train_mode(mode)
        l0, _ = net.loss_grad(xd, td)
        out[mode] = (l0, net.train(xd, td, epochs=3, batch=1024, lr=1e-3))
        net.close()
    print("training losses", out)
    for l0, l1 in out.values():
        assert l1 < 0.5 * l0
    assert abs(out["tf32x3"][1] - out["fp32"][1]) <= 0.01 * out["fp32"][1]


def test_train_mode_checks(gb):
    """Tensor-core training needs a width that is a multiple of 64; unknown
    modes are rejected."""
    from paper_1906_02818_gb300 import native
    sizes = omlp.layer_sizes(5, 100, 3)
    count = sum(a * b + b for a, b in zip(sizes[:-1], sizes[1:]))
    net = gb.Mlp(5, 100, 3, np.zeros(count, dtype=np.float32))
    with pytest.raises(native.MCError):
        net.set_train_mode("tf32x3")
    assert native.lib().mc_mlp_set_train_mode(net.handle, 7) == native.MC_EINVAL
    net.close()


S_SCALE, V_SCALE = 1.0 / 0.55, 1.0 / 0.15  # d input / d(S/K) and d input / d sigma of the surrogate's input map


@pytest.mark.parametrize("mode", ["fp32", "tf32x3"])
@pytest.mark.parametrize("n", [131, 777])
def test_derivative_loss_gradient_matches_oracle(gb, n, mode):
    """The derivative-label loss (mc_mlp_loss_grad_d: prices plus two input
    gradients, some labels missing) and its gradient against the FP64 oracle
    (oracle/mlp.py dloss_and_grads, pinned by finite differences), in both
    training arithmetics (FP32 SIMT products; the width -> width products on
    the tensor cores in three-pass TF32, stacked rows 393 and 2331: ragged
    tiles and transposes).  The library compares scale_k dy/dx with g_k; the
    oracle's form is the same loss with weight scale^2 and label g / scale."""
    import torch
    init = workloads.mlp_init(seed=9)
    net = gb.Mlp(5, 256, 4, init)
    if mode == "tf32x3":
        net.set_train_mode("tf32x3")
    tol_parts = 1e-5 if mode == "fp32" else 5e-5
    x, t = _data(n, seed=4)
    rng = np.random.default_rng(5)
    g = rng.uniform(-1, 1, (n, 2)).astype(np.float32)
    g[::7, 0] = np.nan
    g[3::11, 1] = np.nan
    dirs, scales, weights = [0, 1], [S_SCALE, V_SCALE], [0.5, 2.0]
    parts, grad = net.loss_grad_d(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(g).cuda(),
                                  dirs, scales, weights)
    P = omlp.unpack(init.astype(np.float64), SIZES)
    sc = np.array(scales)
    loss, p_ref, G = omlp.dloss_and_grads(P, x.astype(np.float64), t.astype(np.float64), g.astype(np.float64) / sc,
                                          dirs, list(np.array(weights) * sc * sc))
    g_ref = omlp.pack(G)
    for a, b in zip(parts, p_ref):
        assert abs(a - b) <= tol_parts * b + 1e-9, (mode, parts, p_ref)
    scale = np.max(np.abs(g_ref))
    print("derivative loss (%s): parts" % mode, parts,
          "max grad err / max |grad| %.2e" % (np.max(np.abs(grad - g_ref)) / scale))
    assert np.max(np.abs(grad - g_ref)) <= 1e-4 * scale
    # no directions: the plain loss and gradient
    parts0, grad0 = net.loss_grad_d(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), None, [], [], [])
    l_plain, g_plain = net.loss_grad(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    assert abs(parts0[0] - l_plain) <= (1e-6 if mode == "fp32" else 1e-5) * l_plain
    assert np.max(np.abs(grad0 - g_plain)) <= (1e-5 if mode == "fp32" else 1e-4) * np.max(np.abs(g_plain))
    net.close()


def test_training_on_greeks_gains_over_prices_alone(gb):
    """What the derivative labels buy (Sec. I.A.3's sensitivities as training
    signal): two networks from the same initial weights train on the same
    2^14 European points of the surrogate's box, each labelled by 2^10 Monte
    Carlo paths, one on the prices alone and one on the prices plus the
    pathwise delta and vega labels of the same paths.  On 4096 fresh points
    both are scored against the Black-Scholes closed forms: the Greek-trained network's
    delta error and its price error must be the smaller."""
    import math
    import torch
    from closed_forms import bs_call
    n_tr, n_te = 1 << 14, 4096
    pts = workloads.surrogate_points(n_tr + n_te, seed=21)
    pts[:, 4] = 0.0  # European
    P = torch.from_numpy(pts).cuda()
    lab, dl, x = gb.surrogate_label_greeks(P[:n_tr], 1 << 10, with_inputs=True)
    _, _, xt = gb.surrogate_label_greeks(P[n_tr:], 1, with_inputs=True)
    te = pts[n_tr:].astype(np.float64)
    M = np.maximum(1, np.rint(te[:, 2] * 252))
    T = M * (te[:, 2] / M)
    price = np.array([bs_call(s, 1.0, r, v, tt) for s, v, r, tt in zip(te[:, 0], te[:, 1], te[:, 3], T)])
    d1 = (np.log(te[:, 0]) + (te[:, 3] + 0.5 * te[:, 1] ** 2) * T) / (te[:, 1] * np.sqrt(T))
    delta = 0.5 * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in d1]))
    init = workloads.mlp_init(seed=17)
    res = {}
    for name, dirs in (("prices", []), ("prices+greeks", [0, 1])):
        net = gb.Mlp(5, 256, 4, init)
        sc, wt = [S_SCALE, V_SCALE][:len(dirs)], [0.2, 0.05][:len(dirs)]
        for lr, ep in ((1e-3, 30), (3e-4, 15), (1e-4, 15)):
            net.train_d(x, lab, dl, dirs, sc, wt, epochs=ep, batch=512, lr=lr)
        xq = xt.clone().requires_grad_(False)
        y = net.forward(xq).double().cpu().numpy()
        h = 1e-3  # central difference of the network in S/K: input 0 moves by h / 0.55
        xp, xm = xt.clone(), xt.clone()
        xp[:, 0] += h * S_SCALE
        xm[:, 0] -= h * S_SCALE
        dnet = (net.forward(xp).double() - net.forward(xm).double()).cpu().numpy() / (2 * h)
        res[name] = (float(np.sqrt(np.mean((y - price) ** 2))), float(np.sqrt(np.mean((dnet - delta) ** 2))))
        net.close()
    print("test RMSE vs Black-Scholes (price, delta):", res)
    (p0, d0), (p1, d1_) = res["prices"], res["prices+greeks"]
    assert d1_ < 0.7 * d0, res
    assert p1 < 0.8 * p0, res
