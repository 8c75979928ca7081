"""GPU parity of the neural-operator kernels (BF16 tensor-core convolutions
with FP32 accumulation) against the FP64 oracle.

Tolerances: single layers get BF16-exact inputs and weights, so only the
FP32 accumulation order differs: relative L-infinity 1e-5 (K <= 9 x 320
terms of size ~1, eps32 * sqrt(K) ~ 1e-5 relative to the largest output).
The whole 23-layer network stores activations and gradients in BF16
(eps = 2^-8 = 3.9e-3 per rounding); forward relative L2 error <= 3e-2 and
gradients relative L2 <= 8e-2 with cosine similarity >= 0.99.
"""
import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()
    return lbib


def bf16(shape, seed, scale=1.0):
    import torch
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(*shape, generator=g) * scale).to(torch.bfloat16)


def f64(t):
    return t.float().numpy().astype(np.float64)


def rel_inf(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_conv_forward_and_concat_upsample(lb, orc):
    import torch
    from oracle import nn as onn
    N, H, W, C1, C2, Co = 2, 16, 24, 16, 32, 48
    x1 = bf16((N, H, W, C1), 1)
    x2 = bf16((N, H // 2, W // 2, C2), 2)
    w = bf16((3, 3, C1 + C2, Co), 3, 0.1)
    b = torch.randn(Co, generator=torch.Generator().manual_seed(4)).float()
    st = torch.cuda.current_stream().cuda_stream
    dw = w.float().cuda()
    wf = torch.empty((9, Co, C1 + C2), dtype=torch.bfloat16, device="cuda")
    wd = torch.empty((9, C1 + C2, Co), dtype=torch.bfloat16, device="cuda")
    lb.load().lbib_nn_weight_copies(C1 + C2, Co, C1 + C2, Co, dw.data_ptr(), wf.data_ptr(),
                                    wd.data_ptr(), st)
    torch.cuda.synchronize()
    out = torch.empty((N, H, W, Co), dtype=torch.float32, device="cuda")
    dx1, dx2, dbias = x1.cuda(), x2.cuda(), b.cuda()   # kept alive across the calls
    rc = lb.load().lbib_nn_conv3x3(N, H, W, C1, C2, Co, dx1.data_ptr(), dx2.data_ptr(),
                                   wf.data_ptr(), dbias.data_ptr(), out.data_ptr(), 0, 1, st)
    assert rc == 0
    xin = np.concatenate([f64(x1), onn.upsample2(f64(x2))], axis=3)
    ref = orc.conv3x3(xin, f64(w), b.double().numpy())
    assert rel_inf(out.cpu().numpy(), ref) < 1e-5
    # ReLU and BF16 output
    outb = torch.empty((N, H, W, Co), dtype=torch.bfloat16, device="cuda")
    lb.load().lbib_nn_conv3x3(N, H, W, C1, C2, Co, dx1.data_ptr(), dx2.data_ptr(),
                              wf.data_ptr(), dbias.data_ptr(), outb.data_ptr(), 1, 0, st)
    assert rel_inf(f64(outb.cpu()), np.maximum(ref, 0)) < 8e-3


def test_conv_data_gradient_with_flipped_weights(lb, orc):
    import torch
    N, H, W, Ci, Co = 2, 12, 20, 48, 32
    g = bf16((N, H, W, Co), 5)
    w = bf16((3, 3, Ci, Co), 6, 0.1)
    st = torch.cuda.current_stream().cuda_stream
    wf = torch.empty((9, Co, Ci), dtype=torch.bfloat16, device="cuda")
    wd = torch.empty((9, Ci, Co), dtype=torch.bfloat16, device="cuda")
    dwf32, dg = w.float().cuda(), g.cuda()
    lb.load().lbib_nn_weight_copies(Ci, Co, Ci, Co, dwf32.data_ptr(), wf.data_ptr(),
                                    wd.data_ptr(), st)
    out = torch.empty((N, H, W, Ci), dtype=torch.float32, device="cuda")
    # the data gradient is a forward convolution of g with the flipped copy
    rc = lb.load().lbib_nn_conv3x3(N, H, W, Co, 0, Ci, dg.data_ptr(), None,
                                   wd.data_ptr(), None, out.data_ptr(), 0, 1, st)
    assert rc == 0
    ref = orc.conv3x3_dgrad(f64(g), f64(w))
    assert rel_inf(out.cpu().numpy(), ref) < 1e-5


@pytest.mark.parametrize("C1,C2,Co", [(32, 0, 48), (16, 32, 16)])
def test_conv_weight_gradient(lb, orc, C1, C2, Co):
    import torch
    from oracle import nn as onn
    N, H, W = 2, 16, 32
    x1 = bf16((N, H, W, C1), 7)
    x2 = bf16((N, H // 2, W // 2, C2), 8) if C2 else None
    g = bf16((N, H, W, Co), 9)
    st = torch.cuda.current_stream().cuda_stream
    dw = torch.zeros((9, C1 + C2, Co), dtype=torch.float32, device="cuda")
    db = torch.zeros(Co, dtype=torch.float32, device="cuda")
    dx1, dg = x1.cuda(), g.cuda()
    dx2 = x2.cuda() if C2 else None
    rc = lb.load().lbib_nn_conv3x3_wgrad(N, H, W, C1, C2, Co, dx1.data_ptr(),
                                         dx2.data_ptr() if C2 else None,
                                         dg.data_ptr(), dw.data_ptr(), db.data_ptr(), st)
    assert rc == 0
    xin = f64(x1) if not C2 else np.concatenate([f64(x1), onn.upsample2(f64(x2))], axis=3)
    rw, rb = orc.conv3x3_wgrad(xin, f64(g))
    assert rel_inf(dw.cpu().numpy().reshape(3, 3, C1 + C2, Co), rw) < 1e-5
    assert rel_inf(db.cpu().numpy(), rb) < 1e-5


def _net_inputs(seed, n, H):
    rng = np.random.default_rng(seed)
    mask = (rng.uniform(size=(n, H, H)) < 0.5).astype(np.uint8)
    src = (mask * (rng.uniform(size=(n, H, H)) < 0.3)).astype(np.uint8)
    D = rng.uniform(0.05, 0.2, n)
    k = rng.uniform(1e-4, 1e-2, n)
    s = np.full(n, 1e-3)
    phi = rng.uniform(0, 1, (n, H, H)) * (s / k)[:, None, None]
    return mask, src, D, k, s, phi


def _bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy() \
        .astype(np.float64)


@pytest.mark.parametrize("H,n", [
    (32, 2),    # every level on the warp-level convolution
    (256, 1),   # 256^2 and 128^2 on the tcgen05 convolution (forward and data
                # gradient with the fused ReLU backward), the weights re-tiled
                # by the fused refresh
])
def test_network_forward_and_gradient_match_oracle(lb, orc, H, n):
    import torch
    from oracle import nn as onn
    net = lb.NeuralOperator(n, H, H)
    shapes = onn.nop_shapes()
    assert net.layers() == [(ci, co) for _, ci, co in shapes]
    assert net.n_params == onn.nop_num_params()
    p = li.nop_init_params(21, shapes)
    p = p + 0.01 * np.random.default_rng(3).normal(size=p.size)   # non-zero biases
    p = p.astype(np.float32).astype(np.float64)
    net.set_params(p)
    mask, src, D, k, s, phi = _net_inputs(5, n, H)
    dm = torch.from_numpy(mask).cuda()
    ds = torch.from_numpy(src).cuda()
    out = net.forward(dm, ds, D, k, s).cpu().numpy()
    # oracle on the same (BF16-rounded) features and BF16-rounded weights
    x = onn.features(mask, src, D, k)
    x[..., 2:] = _bf16_round(x[..., 2:])
    pb = _bf16_round(p)
    y, cache = onn.forward(pb, x)
    ref = y[..., 0] * (s / k)[:, None, None]
    assert rel_l2(out, ref) < 3e-2
    # gradient of the loss (no update)
    loss = net.train_step(dm, ds, D, k, s, torch.from_numpy(phi.astype(np.float32)).cuda(),
                          update=False)
    tgt = (phi * (k / s)[:, None, None])[..., None]
    rloss, dy = onn.loss(y, tgt)
    assert loss == pytest.approx(rloss, rel=5e-2)
    g_ref = onn.backward(dy, cache)
    g = net.get_grads().astype(np.float64)
    assert rel_l2(g, g_ref) < 8e-2
    assert float(g @ g_ref / (np.linalg.norm(g) * np.linalg.norm(g_ref))) > 0.99
    net.close()


def test_adam_step_matches_oracle(lb):
    import torch
    from oracle import nn as onn
    H, n = 32, 2
    net = lb.NeuralOperator(n, H, H)
    p = li.nop_init_params(22, onn.nop_shapes())
    net.set_params(p)
    mask, src, D, k, s, phi = _net_inputs(6, n, H)
    args = (torch.from_numpy(mask).cuda(), torch.from_numpy(src).cuda(), D, k, s,
            torch.from_numpy(phi.astype(np.float32)).cuda())
    net.train_step(*args, update=False)
    g = net.get_grads().astype(np.float64)
    net.train_step(*args, lr=1e-3, update=True)
    q = net.get_params().astype(np.float64)
    qr, _, _ = onn.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    # the first step is lr * g / (|g| + eps): exact where |g| >> eps, and at
    # most lr in size everywhere (recomputed gradients differ in atomic order)
    big = np.abs(g) > 1e-5
    assert big.sum() > 1000
    assert np.abs(q - qr)[big].max() < 2e-6
    # (plus the FP32 rounding of parameters of size ~0.3: ulp 3e-8)
    assert np.abs(q - p).max() <= 1e-3 + 1e-7
    net.close()


def test_training_reduces_loss(lb):
    import torch
    H, n = 64, 4
    net = lb.NeuralOperator(n, H, H)
    from oracle import nn as onn
    net.set_params(li.nop_init_params(23, onn.nop_shapes()))
    mask, src, D, k, s, phi = _net_inputs(7, n, H)
    args = (torch.from_numpy(mask).cuda(), torch.from_numpy(src).cuda(), D, k, s,
            torch.from_numpy(phi.astype(np.float32)).cuda())
    first = net.train_step(*args, lr=1e-3)
    for _ in range(40):
        last = net.train_step(*args, lr=1e-3)
    assert last < 0.5 * first, (first, last)
    net.close()
