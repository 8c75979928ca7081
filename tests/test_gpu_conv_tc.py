"""GPU parity of the tcgen05 convolution (lbib_nn_conv3x3_tc: tensor-memory
accumulator, TMA-staged operands) against the FP64 oracle and against the
warp-level mma.sync kernel of lbib_nn_conv3x3.

Tolerances as for the other layer tests: BF16-exact inputs and weights, so
only the FP32 accumulation order differs: relative L-infinity 1e-5 in FP32
output; BF16 output within 8e-3 (one rounding of 2^-8 relative).  The
kernel's error word stays zero.  Shapes cover tiles of rows of 128 (one
accumulator per row; W = 128, 256, 640, 1280) and of whole narrower rows
(accumulators over the row-major halo positions; W = 8 .. 64, and 48, not a
power of two), one and several accumulators per CTA, tiles that overhang
the image's last row, 16- and 32-channel chunks (32- and 64-byte
swizzles), the decoder's upsampled second input in both, an output wider
than one CTA (two N tiles), the one-channel final layer and the data
gradient through flipped weights.
"""
import numpy as np
import pytest

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


def _weights(lb, w, Ci, Co, st):
    """Forward (9, Co, Ci) and flipped (9, Ci, Co) BF16 copies and the tiled
    forward copy of FP32 weights w (3, 3, Ci, Co)."""
    import ctypes
    import torch
    dw = w.float().cuda()
    wf = torch.empty((9, Co, Ci), dtype=torch.bfloat16, device="cuda")
    wd = torch.empty((9, Ci, Co), dtype=torch.bfloat16, device="cuda")
    assert lb.load().lbib_nn_weight_copies(Ci, Co, Ci, Co, dw.data_ptr(), wf.data_ptr(),
                                           wd.data_ptr(), st) == 0
    n = ctypes.c_uint64(0)
    assert lb.load().lbib_nn_tile_weights_tc(Ci, Co, None, None, ctypes.byref(n), st) == 0
    wt = torch.empty(int(n.value), dtype=torch.bfloat16, device="cuda")
    assert lb.load().lbib_nn_tile_weights_tc(Ci, Co, wf.data_ptr(), wt.data_ptr(), None, st) == 0
    return dw, wf, wd, wt


@pytest.mark.parametrize("N,H,W,C1,C2,Co", [
    (2, 16, 32, 16, 32, 48),    # 16-channel chunks, upsampled input, overhanging tile
    (1, 32, 16, 32, 0, 64),     # 32-channel chunk, narrow rows
    (2, 8, 64, 16, 32, 32),     # upsampled
    (1, 3, 128, 64, 0, 96),     # rows of 128, two chunks
    (2, 2, 256, 32, 0, 192),    # two N tiles of 96, two tiles per row
    (1, 16, 16, 48, 0, 320),    # two N tiles of 160
    (1, 16, 64, 32, 0, 1),      # the one-channel final layer
    (4, 8, 8, 32, 0, 64),       # the 8 x 8 level: one tile per image
    (3, 50, 48, 32, 0, 32),     # W = 48, 50 rows
    (2, 32, 256, 32, 32, 32),   # upsampled input in a 32-channel chunk
    (2, 128, 640, 16, 32, 48),  # rows of 128, 4 accumulators, upsampled input
    (1, 64, 1280, 16, 0, 192),  # rows of 128, 192 channels in one CTA
    (40, 64, 64, 16, 32, 32),   # 7 rows x 66 halo positions in 4 accumulators
])
def test_tc_conv_matches_oracle_and_mma_sync(lb, orc, N, H, W, C1, C2, Co):
    import torch
    from oracle import nn as onn
    assert lb.load().lbib_nn_conv3x3_tc_supported(H, W, C1, C2, Co) == 1
    Ci = C1 + C2
    x1 = bf16((N, H, W, C1), 11)
    x2 = bf16((N, H // 2, W // 2, C2), 12) if C2 else None
    w = bf16((3, 3, Ci, Co), 13, 0.1)
    b = torch.randn(Co, generator=torch.Generator().manual_seed(14)).float()
    st = torch.cuda.current_stream().cuda_stream
    dw, wf, wd, wt = _weights(lb, w, Ci, Co, st)
    dx1, dbias = x1.cuda(), b.cuda()
    dx2 = x2.cuda() if C2 else None
    p2 = dx2.data_ptr() if C2 else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((N, H, W, Co), float("nan"), dtype=torch.float32, device="cuda")
    rc = lb.load().lbib_nn_conv3x3_tc(N, H, W, C1, C2, Co, dx1.data_ptr(), p2, wt.data_ptr(),
                                      dbias.data_ptr(), out.data_ptr(), 0, 1, err.data_ptr(), st)
    assert rc == 0, lb.lbib_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    xin = f64(x1) if not C2 else np.concatenate([f64(x1), onn.upsample2(f64(x2))], axis=3)
    ref = orc.conv3x3(xin, f64(w), b.double().numpy())
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel_inf(got, ref) < 1e-5
    # the warp-level kernel on the same inputs (its path takes Co even)
    if Co % 2 == 0:
        out2 = torch.empty((N, H, W, Co), dtype=torch.float32, device="cuda")
        assert lb.load().lbib_nn_conv3x3(N, H, W, C1, C2, Co, dx1.data_ptr(), p2, wf.data_ptr(),
                                         dbias.data_ptr(), out2.data_ptr(), 0, 1, st) == 0
        assert rel_inf(got, out2.cpu().numpy()) < 1e-5
    # ReLU and BF16 output
    outb = torch.empty((N, H, W, Co), dtype=torch.bfloat16, device="cuda")
    assert lb.load().lbib_nn_conv3x3_tc(N, H, W, C1, C2, Co, dx1.data_ptr(), p2, wt.data_ptr(),
                                        dbias.data_ptr(), outb.data_ptr(), 1, 0, err.data_ptr(),
                                        st) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert rel_inf(f64(outb.cpu()), np.maximum(ref, 0)) < 8e-3


def test_tc_conv_data_gradient(lb, orc):
    """The data gradient: a forward convolution of the output gradient with
    the tap-flipped, transposed weights."""
    import ctypes
    import torch
    N, H, W, Ci, Co = 2, 16, 32, 48, 32
    g = bf16((N, H, W, Co), 15)
    w = bf16((3, 3, Ci, Co), 16, 0.1)
    st = torch.cuda.current_stream().cuda_stream
    dw, wf, wd, _ = _weights(lb, w, Ci, Co, st)
    n = ctypes.c_uint64(0)
    lb.load().lbib_nn_tile_weights_tc(Co, Ci, None, None, ctypes.byref(n), st)
    wdt = torch.empty(int(n.value), dtype=torch.bfloat16, device="cuda")
    assert lb.load().lbib_nn_tile_weights_tc(Co, Ci, wd.data_ptr(), wdt.data_ptr(), None, st) == 0
    dg = g.cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((N, H, W, Ci), dtype=torch.float32, device="cuda")
    assert lb.load().lbib_nn_conv3x3_tc(N, H, W, Co, 0, Ci, dg.data_ptr(), None, wdt.data_ptr(),
                                        None, out.data_ptr(), 0, 1, err.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = orc.conv3x3_dgrad(f64(g), f64(w))
    assert rel_inf(out.cpu().numpy(), ref) < 1e-5


def test_tc_conv_shape_support(lb):
    L = lb.load()
    assert L.lbib_nn_conv3x3_tc_supported(16, 192, 32, 0, 32) == 0   # W > 128, not rows of 128
    assert L.lbib_nn_conv3x3_tc_supported(16, 16, 8, 0, 32) == 0     # C1 not a multiple of 16
    assert L.lbib_nn_conv3x3_tc_supported(16, 16, 16, 16, 32) == 0   # 32-channel chunks, C1 = 16
    assert L.lbib_nn_conv3x3_tc_supported(15, 16, 32, 16, 32) == 0   # upsampled input, odd H
    assert L.lbib_nn_conv3x3_tc_supported(8, 8, 32, 0, 32) == 1
    assert L.lbib_nn_conv3x3_tc_supported(2, 32, 16, 0, 32) == 1
    assert L.lbib_nn_conv3x3_tc_supported(256, 256, 16, 0, 32) == 1


@pytest.mark.parametrize("N,H,W,C1,C2,Co", [
    (2, 16, 32, 32, 0, 32),     # whole narrow rows, one 32-channel chunk (64-byte swizzle)
    (2, 8, 16, 16, 32, 48),     # 16-channel chunks (eight shifts per M), upsampled input
    (1, 5, 128, 64, 0, 64),     # rows of 128, two chunks, a row tile overhanging the image
    (1, 4, 256, 32, 32, 192),   # two tiles per row, two N tiles of 96, upsampled 32-channel chunk
    (4, 64, 64, 48, 0, 16),     # the smallest N tile (four accumulator sets), 32 + 16 channels
    (1, 4, 256, 32, 48, 32),    # upsampled 48 channels: a 32- and a 16-channel chunk
    (2, 8, 32, 16, 16, 32),     # 16-channel chunks of both inputs
])
def test_tc_wgrad_matches_oracle_and_mma_sync(lb, orc, N, H, W, C1, C2, Co):
    """The weight gradient on tcgen05 (MN-major operands, the input channels of
    three tap shifts as M; 32-channel chunks where an input has them, 16 for a
    remainder) against the FP64 oracle and the warp-level kernel: BF16-exact
    inputs, FP32 accumulation in a different order."""
    import torch
    from oracle import nn as onn
    L = lb.load()
    assert L.lbib_nn_conv3x3_wgrad_tc_supported(H, W, C1, C2, Co) == 1
    Ci = C1 + C2
    x1 = bf16((N, H, W, C1), 21)
    x2 = bf16((N, H // 2, W // 2, C2), 22) if C2 else None
    g = bf16((N, H, W, Co), 23)
    st = torch.cuda.current_stream().cuda_stream
    dx1, dg = x1.cuda(), g.cuda()
    dx2 = x2.cuda() if C2 else None
    p2 = dx2.data_ptr() if C2 else None
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    dw = torch.zeros((9, Ci, Co), dtype=torch.float32, device="cuda")
    db = torch.zeros(Co, dtype=torch.float32, device="cuda")
    assert L.lbib_nn_conv3x3_wgrad_tc(N, H, W, C1, C2, Co, dx1.data_ptr(), p2, dg.data_ptr(),
                                      dw.data_ptr(), db.data_ptr(), err.data_ptr(), st) == 0, \
        lb.lbib_last_error(None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    xin = f64(x1) if not C2 else np.concatenate([f64(x1), onn.upsample2(f64(x2))], axis=3)
    rw, rb = orc.conv3x3_wgrad(xin, f64(g))
    got = dw.cpu().numpy().reshape(3, 3, Ci, Co)
    assert np.isfinite(got).all()
    assert rel_inf(got, rw) < 1e-5
    assert rel_inf(db.cpu().numpy(), rb) < 1e-5
    dw2 = torch.zeros((9, Ci, Co), dtype=torch.float32, device="cuda")
    db2 = torch.zeros(Co, dtype=torch.float32, device="cuda")
    assert L.lbib_nn_conv3x3_wgrad(N, H, W, C1, C2, Co, dx1.data_ptr(), p2, dg.data_ptr(),
                                   dw2.data_ptr(), db2.data_ptr(), st) == 0
    torch.cuda.synchronize()
    assert rel_inf(got, dw2.cpu().numpy().reshape(3, 3, Ci, Co)) < 1e-5


def test_tc_wgrad_shape_support(lb):
    L = lb.load()
    assert L.lbib_nn_conv3x3_wgrad_tc_supported(8, 8, 32, 0, 32) == 0     # W below 16
    assert L.lbib_nn_conv3x3_wgrad_tc_supported(8, 40, 32, 0, 32) == 0    # W not a multiple of 16
    assert L.lbib_nn_conv3x3_wgrad_tc_supported(8, 32, 32, 0, 40) == 0    # Co not a multiple of 16
    assert L.lbib_nn_conv3x3_wgrad_tc_supported(8, 32, 16, 0, 32) == 1    # one 16-channel chunk
    assert L.lbib_nn_conv3x3_wgrad_tc_supported(8, 32, 16, 16, 32) == 1   # a 16-channel chunk of each input
    assert L.lbib_nn_conv3x3_wgrad_tc_supported(256, 256, 16, 0, 32) == 1
