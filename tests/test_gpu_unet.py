"""Warm-start network kernels against the FP64 oracle (gpu).

Convolution forward against oracle.unet.conv3d; weight and data gradients
against central differences of the oracle (the convolution is linear, so the
differences are exact up to rounding); the full network's forward and
gradients against the oracle network and its finite differences.  BF16
activations bound the agreement: 1e-2 relative per convolution, and a
gradient cosine above 0.99 for the whole network.
"""
import numpy as np
import pytest

import oracle.unet as OU

pytestmark = pytest.mark.gpu


def _bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda().contiguous()


@pytest.mark.parametrize("ci,co,shape,periodic", [
    (16, 16, (2, 4, 6, 10), 1), (16, 32, (2, 4, 6, 10), 1), (48, 16, (2, 4, 6, 10), 1),
    (96, 32, (2, 4, 6, 10), 1), (192, 64, (2, 4, 6, 10), 1), (64, 128, (2, 4, 6, 10), 1),
    (64, 192, (2, 4, 6, 10), 1), (16, 8, (2, 4, 6, 10), 1),
    # several 8 x 16 output blocks with ragged edges, and zero padding in y, z
    (32, 64, (1, 5, 37, 19), 1), (32, 64, (1, 5, 37, 19), 0), (16, 16, (3, 3, 17, 9), 0)])
def test_conv_forward(cuda_lib, ci, co, shape, periodic):
    import torch

    from paper_1410_1914_gb300 import warmstart as W
    rng = np.random.default_rng(ci * 1000 + co + periodic)
    N, D, H, Wd = shape
    x = _bf16(rng.standard_normal((N, D, H, Wd, ci)))
    w = _bf16(rng.standard_normal((27, co, ci)) / np.sqrt(27 * ci))
    b = rng.standard_normal(co)
    ref = OU.conv3d(x, w, b, periodic_yz=bool(periodic))
    out = torch.empty(N, D, H, Wd, co, dtype=torch.bfloat16, device="cuda")
    # keep the device copies alive until the kernel has run
    xd, wd, bd = _dev(x, torch.bfloat16), _dev(w, torch.bfloat16), _dev(b, torch.float32)
    W._call("cl_nn_conv3d", W._p(xd), W._p(wd), W._p(bd), W._p(out), N, D, H, Wd, ci, co, ci, 0, co, 0, 0, periodic,
            None)
    W._call("cl_nn_check", None)
    got = out.float().cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-2, atol=1e-2 * np.abs(ref).max())


@pytest.mark.parametrize("ci,co", [(16, 16), (48, 16), (64, 128)])
def test_conv_gradients_against_differences(cuda_lib, ci, co):
    import torch

    from paper_1410_1914_gb300 import warmstart as W
    rng = np.random.default_rng(ci + co)
    N, D, H, Wd = 1, 4, 4, 6
    x = _bf16(rng.standard_normal((N, D, H, Wd, ci)))
    w = _bf16(rng.standard_normal((27, co, ci)) / np.sqrt(27 * ci))
    gy = _bf16(rng.standard_normal((N, D, H, Wd, co)))
    zero_b = np.zeros(co)
    f = lambda xx, ww: float(np.sum(OU.conv3d(xx, ww, zero_b) * gy))
    # GPU weight gradient
    M = N * D * H * Wd
    ws = torch.empty(W._lib().cl_nn_wgrad_workspace(N, D, H, Wd, ci, co) // 4 + 1, dtype=torch.float32, device="cuda")
    dw = torch.empty(27, co, ci, dtype=torch.float32, device="cuda")
    dx_in = _dev(x, torch.bfloat16)
    dgy = _dev(gy, torch.bfloat16)
    W._call("cl_nn_conv3d_wgrad", W._p(dx_in), W._p(dgy), W._p(ws), W._p(dw), N, D, H, Wd, ci, co, ci, 0, co, 0, 1, None)
    # GPU data gradient: the convolution with flipped, transposed weights
    wd = torch.empty(27, ci, co, dtype=torch.bfloat16, device="cuda")
    w_dev = _dev(w, torch.bfloat16)
    W._call("cl_nn_wt_dgrad", W._p(w_dev), W._p(wd), co, ci, None)
    gx = torch.empty(N, D, H, Wd, ci, dtype=torch.bfloat16, device="cuda")
    W._call("cl_nn_conv3d", W._p(dgy), W._p(wd), None, W._p(gx), N, D, H, Wd, co, ci, co, 0, ci, 0, 0, 1, None)
    torch.cuda.synchronize()
    dw = dw.cpu().numpy()
    gx = gx.float().cpu().numpy()
    h = 0.5
    for _ in range(12):
        t, o, i = rng.integers(27), rng.integers(co), rng.integers(ci)
        wp, wm = w.copy(), w.copy()
        wp[t, o, i] += h
        wm[t, o, i] -= h
        fd = (f(x, wp) - f(x, wm)) / (2 * h)
        assert dw[t, o, i] == pytest.approx(fd, rel=1e-2, abs=1e-2 * (1 + abs(fd)))
    for _ in range(12):
        idx = tuple(rng.integers(s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (f(xp, w) - f(xm, w)) / (2 * h)
        assert gx[idx] == pytest.approx(fd, rel=2e-2, abs=2e-2 * (1 + abs(fd)))


@pytest.mark.parametrize("ci,co,shape,periodic", [
    (16, 16, (1, 3, 5, 7), 1), (48, 16, (2, 4, 4, 6), 1), (96, 32, (1, 4, 6, 6), 1), (192, 64, (1, 3, 4, 8), 1),
    (64, 128, (1, 5, 3, 9), 1), (16, 128, (2, 2, 2, 2), 1), (16, 32, (1, 4, 21, 11), 1), (16, 16, (2, 3, 19, 9), 0),
    (32, 32, (1, 3, 19, 9), 0)])
def test_wgrad_full_tensor(cuda_lib, ci, co, shape, periodic):
    """Every entry of dW[t][o][i] = sum_v gy[v][o] x_t[v][i], where x_t (the
    input shifted by tap t, with the padding rules) comes from the oracle's
    convolution with an identity kernel at that tap.  Products of BF16
    values are exact in FP32, so only the summation order differs."""
    import torch

    from paper_1410_1914_gb300 import warmstart as W
    rng = np.random.default_rng(7 * ci + co)
    N, D, H, Wd = shape
    x = _bf16(rng.standard_normal((N, D, H, Wd, ci)))
    gy = _bf16(rng.standard_normal((N, D, H, Wd, co)))
    exp = np.zeros((27, co, ci))
    for tap in range(27):
        wid = np.zeros((27, ci, ci))
        wid[tap] = np.eye(ci)
        xt = OU.conv3d(x, wid, np.zeros(ci), periodic_yz=bool(periodic)).reshape(-1, ci)
        exp[tap] = gy.reshape(-1, co).T @ xt
    ws = torch.empty(W._lib().cl_nn_wgrad_workspace(N, D, H, Wd, ci, co) // 4 + 1, dtype=torch.float32, device="cuda")
    dw = torch.empty(27, co, ci, dtype=torch.float32, device="cuda")
    xd, gd = _dev(x, torch.bfloat16), _dev(gy, torch.bfloat16)
    W._call("cl_nn_conv3d_wgrad", W._p(xd), W._p(gd), W._p(ws), W._p(dw), N, D, H, Wd, ci, co, ci, 0, co, 0, periodic,
            None)
    W._call("cl_nn_check", None)
    np.testing.assert_allclose(dw.cpu().numpy(), exp, rtol=0, atol=1e-5 * np.abs(exp).max() + 1e-6)


def _oracle_params(net):
    P = {}
    for name, ci, co in OU.CONV_LAYERS:
        w, b = net.params[name]
        P[name] = (_bf16(w.cpu().numpy()), b.cpu().numpy().astype(np.float64))
    hw, hb = net.params["head"]
    P["head"] = (hw.cpu().numpy().astype(np.float64), float(hb.cpu().numpy()[0]))
    return P


def test_network_forward_and_gradients(cuda_lib):
    import torch

    from paper_1410_1914_gb300 import warmstart as W
    rng = np.random.default_rng(5)
    net = W.UNet(seed=3)
    # non-trivial biases so that ReLUs are mixed
    for name, _, co in W.CONV_LAYERS:
        net.params[name][1].copy_(torch.from_numpy(rng.standard_normal(co).astype(np.float32) * 0.1).cuda())
    net.params["head"][0].copy_(torch.from_numpy(rng.standard_normal(16).astype(np.float32) * 0.3).cuda())
    N, D = 1, 8
    x = _bf16(rng.standard_normal((N, D, D, D, 16)))
    target = rng.standard_normal(N * D ** 3)
    mask = (rng.random(N * D ** 3) < 0.7).astype(np.uint8)
    xd = _dev(x, torch.bfloat16)
    out = net.forward(xd, N, D)
    P = _oracle_params(net)
    ref = OU.forward(P, x).reshape(-1)
    got = out.cpu().numpy().astype(np.float64)
    assert np.corrcoef(got, ref)[0, 1] > 0.999
    np.testing.assert_allclose(got, ref, rtol=0, atol=0.05 * np.abs(ref).max())
    tt = _dev(target, torch.float32)
    mm = _dev(mask, torch.uint8)
    net.backward(tt, mm)
    torch.cuda.synchronize()
    assert net.loss_value() == pytest.approx(OU.masked_mse(ref.reshape(-1), target, mask), rel=2e-2)
    # finite differences of the oracle loss for sampled parameters of every layer
    ga, gf = [], []
    h = 1e-3
    for name in [n for n, _, _ in OU.CONV_LAYERS] + ["head"]:
        gw = net.grads[name][0].cpu().numpy()
        for _ in range(3):
            idx = tuple(rng.integers(s) for s in gw.shape)
            Pp = dict(P)
            Pm = dict(P)
            wp, wm = P[name][0].copy(), P[name][0].copy()
            wp[idx] += h
            wm[idx] -= h
            Pp[name] = (wp, P[name][1])
            Pm[name] = (wm, P[name][1])
            lp = OU.masked_mse(OU.forward(Pp, x).reshape(-1), target, mask)
            lm = OU.masked_mse(OU.forward(Pm, x).reshape(-1), target, mask)
            gf.append((lp - lm) / (2 * h))
            ga.append(float(gw[idx]))
    ga, gf = np.array(ga), np.array(gf)
    cos = float(np.dot(ga, gf) / (np.linalg.norm(ga) * np.linalg.norm(gf)))
    assert cos > 0.99, (cos, ga, gf)
    assert np.linalg.norm(ga) == pytest.approx(np.linalg.norm(gf), rel=0.05)


def test_features_target_and_warm_field(cuda_lib):
    """Solver glue: the 16 input channels against the oracle's set-up
    (active set, D/D_max of Eq. 7-9, the series-resistor profile written out
    here in numpy), the training target against the solver's own field, and
    the warm-started field against ramp + prediction."""
    import torch

    import oracle
    from paper_1410_1914_gb300 import Solver, inputs
    from paper_1410_1914_gb300 import warmstart as W
    ph, _, params = inputs.batch_workloads(2, seed0=7, edge_range=(24, 24))[1]
    nz, ny, nx = ph.shape
    o = oracle.OracleLBM(ph, **params)
    act = o.active().astype(bool)
    rel = np.where(act, o.D() / o.D_max, 0.0)
    x = np.arange(nx)
    ramp = 1.0 - (x + 0.5) / nx
    # series resistors: inlet half cell, harmonic links between planes, outlet half cell
    a, b = rel[:, :, :-1], rel[:, :, 1:]
    both = act[:, :, :-1] & act[:, :, 1:]
    g_link = np.where(both, 2 * a * b / np.where(both, a + b, 1.0), 0.0).sum(axis=(0, 1)) / (ny * nz)
    R = np.concatenate([[1 / (2 * rel[:, :, 0].sum() / (ny * nz))], 1 / g_link,
                        [1 / (2 * rel[:, :, -1].sum() / (ny * nz))]])
    series = 1.0 - np.cumsum(R)[:-1] / R.sum()
    exp = np.zeros(ph.shape + (16,))
    exp[..., 0] = act
    exp[..., 1] = ph == 1
    exp[..., 2] = ph == 2
    exp[..., 3] = ph == 3
    exp[..., 4] = np.where(act, np.maximum(0.0, 1.0 + np.log(np.maximum(rel, 1e-6)) / 6.0), 0.0)
    exp[..., 5] = ramp
    exp[..., 6] = series
    exp[..., 7] = (series - ramp) * nx / 4.0
    with Solver(ph.shape, storage="fp32", **params) as s:
        s.set_structure(ph)
        f = W.features(s)[0].float().cpu().numpy()
        np.testing.assert_allclose(f, exp, rtol=2 ** -7, atol=1e-5)
        # target: (C - ramp) * nx / (c_in - c_out) on active cells
        s.step(300)
        C = s.field()
        t = W.target(s).cpu().numpy().reshape(ph.shape)
        np.testing.assert_allclose(t, np.where(act, (C - ramp) * nx, 0.0), rtol=1e-6, atol=1e-5)
        # warm field: ramp + prediction (target units: times (c_in - c_out) / nx) on active cells, 0 elsewhere
        pred = np.random.default_rng(0).standard_normal(ph.size).astype(np.float32)
        pd = torch.from_numpy(pred).cuda()
        W._call("cl_lbm_init_warm", __import__("ctypes").c_void_p(s.h), W._p(pd))
        torch.cuda.synchronize()
        C0 = s.field()
        np.testing.assert_allclose(C0, np.where(act, ramp + pred.reshape(ph.shape) / nx, 0.0), rtol=0, atol=1e-6)
