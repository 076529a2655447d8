"""f3, layer by layer: each tensor-core convolution of the learned-guess network
(forward, weight gradient, bias gradient, data gradient) against the FP64 oracle
(``oracle/convnet.py`` ``conv3x3`` / ``conv3x3_backward``) element by element, on
the GPU's own BF16 operands.

Bounds. The operands are BF16, so every product w*x is exact in FP32 (8 x 8
significant bits); the only errors are the FP32 accumulation and, for BF16 outputs,
the final rounding. For an output that sums K products with magnitude sum
S = sum |w||x| (+ |bias| + |res|):

    FP32 accumulation      |acc - exact| <= (K + 2) * 2^-22 * S
                           (2^-24 per addition for round-to-nearest; 4x that for the
                           tensor cores' internal alignment and the split partials)
    BF16 output rounding   |bf16(y) - y| <= 2^-8 * |y|

so |y_gpu - y_oracle| <= 2^-8 |y_oracle| + (K + 2) 2^-22 S (+ 2^-8 of that). A wrong
tap, a transposed chunk or a dropped channel block moves an output by O(|w x|), far
above this bound on a random tensor, so every such mistake fails element-wise.
K: forward 9 Cin, data gradient 9 Cout, weight gradient the pixel count (plus the
number of pixel splits), bias gradient the pixel count (plus its partial blocks).
"""
import numpy as np
import pytest

from oracle import convnet as CN
from paper_2406_00878_gb300 import pit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (Cin, Cout): the network's lift (2 channels padded to 16 -> C), block (C -> C), head
# (C -> M)
# at the benchmark's C = 64, M = 128, tile-splitting shapes, and 64- and 128-channel inputs
# with narrow and wide outputs (the TMA kernels' accumulator rings of 4 and 8 blocks)
LAYERS = [(16, 64), (64, 64), (64, 128), (80, 144), (16, 32), (32, 16), (64, 16), (64, 96), (128, 64), (128, 32)]
# (B, H, W): image rows longer than one 128-pixel segment with a ragged tail, row
# counts that are not multiples of the 4-row CTA tile, and a tiny image
IMAGES = [(2, 6, 130), (1, 5, 9), (3, 1, 17)]


def _bf16(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).cuda().contiguous()


def _f64(t):
    return t.float().cpu().numpy().astype(np.float64)


def _operands(seed, Cin, Cout, B, H, Wd):
    rng = np.random.default_rng(seed)
    X = _bf16(rng.standard_normal((B, H, Wd, Cin)))
    Wt = _bf16(rng.standard_normal((Cout, 3, 3, Cin)) * np.sqrt(2.0 / (9 * Cin)))
    return rng, X, Wt


@pytest.mark.parametrize("B,H,Wd", IMAGES)
@pytest.mark.parametrize("Cin,Cout", LAYERS)
@pytest.mark.parametrize("mode", ["plain", "relu", "residual"])
def test_conv_forward_layer_matches_oracle_elementwise(Cin, Cout, B, H, Wd, mode):
    rng, X, Wt = _operands(Cin * 7 + Cout + H, Cin, Cout, B, H, Wd)
    bias = torch.as_tensor(0.1 * rng.standard_normal(Cout), dtype=torch.float32).cuda()
    res = _bf16(rng.standard_normal((B, H, Wd, Cout))) if mode == "residual" else None
    Y = torch.empty((B, H, Wd, Cout), dtype=torch.bfloat16, device="cuda")
    pit.pit_conv3x3_forward(X, Wt, bias, res, Y, B, H, Wd, Cin, Cout, relu=(mode == "relu"))
    x, w, b = _f64(X), _f64(Wt), bias.double().cpu().numpy()
    ref = CN.conv3x3(x, w, b)
    S = CN.conv3x3(np.abs(x), np.abs(w), np.abs(b))
    if res is not None:
        ref = ref + _f64(res)
        S = S + np.abs(_f64(res))
    if mode == "relu":
        ref = np.maximum(ref, 0.0)
    tol = 2.0 ** -8 * np.abs(ref) + (9 * Cin + 2) * 2.0 ** -22 * S * (1 + 2.0 ** -8)
    err = np.abs(_f64(Y) - ref)
    assert np.all(err <= tol), (float(err.max()), float((err / np.maximum(tol, 1e-300)).max()))


@pytest.mark.parametrize("B,H,Wd", IMAGES)
@pytest.mark.parametrize("Cin,Cout", LAYERS)
def test_conv_backward_layer_matches_oracle_elementwise(Cin, Cout, B, H, Wd):
    rng, X, Wt = _operands(Cin * 11 + Cout + Wd, Cin, Cout, B, H, Wd)
    dY = _bf16(rng.standard_normal((B, H, Wd, Cout)))
    dX = torch.empty((B, H, Wd, Cin), dtype=torch.bfloat16, device="cuda")
    dW = torch.empty((Cout, 3, 3, Cin), dtype=torch.float32, device="cuda")
    db = torch.empty(Cout, dtype=torch.float32, device="cuda")
    pit.pit_conv3x3_backward(X, Wt, dY, dX, dW, db, B, H, Wd, Cin, Cout)
    x, w, dy = _f64(X), _f64(Wt), _f64(dY)
    rdx, rdW, rdb = CN.conv3x3_backward(x, w, dy)
    Sdx, SdW, Sdb = CN.conv3x3_backward(np.abs(x), np.abs(w), np.abs(dy))
    P = B * H * Wd
    # weight gradient: FP32 over P pixels (tensor cores) plus up to 160 split partials
    err = np.abs(dW.double().cpu().numpy() - rdW)
    tol = (P + 160 + 2) * 2.0 ** -22 * SdW
    assert np.all(err <= tol), ("dW", float(err.max()), float((err / np.maximum(tol, 1e-300)).max()))
    # bias gradient: FP32 sum over P pixels in up to 2048 partial blocks
    err = np.abs(db.double().cpu().numpy() - rdb)
    tol = (P + 2048 + 2) * 2.0 ** -22 * Sdb
    assert np.all(err <= tol), ("db", float(err.max()))
    # data gradient: the forward kernel on flipped, transposed weights, BF16 output
    err = np.abs(_f64(dX) - rdx)
    tol = 2.0 ** -8 * np.abs(rdx) + (9 * Cout + 2) * 2.0 ** -22 * Sdx * (1 + 2.0 ** -8)
    assert np.all(err <= tol), ("dX", float(err.max()), float((err / np.maximum(tol, 1e-300)).max()))


def test_conv_layer_bound_catches_a_wrong_tap():
    # the bound of this file is tight enough to see one mistaken tap: the oracle with the
    # weights of tap (0, 1) moved to tap (1, 0) must fail it on the GPU's output
    Cin, Cout, B, H, Wd = 64, 64, 1, 5, 40
    rng, X, Wt = _operands(5, Cin, Cout, B, H, Wd)
    bias = torch.zeros(Cout, dtype=torch.float32, device="cuda")
    Y = torch.empty((B, H, Wd, Cout), dtype=torch.bfloat16, device="cuda")
    pit.pit_conv3x3_forward(X, Wt, bias, None, Y, B, H, Wd, Cin, Cout, relu=False)
    x, w = _f64(X), _f64(Wt)
    wrong = w.copy()
    wrong[:, 1, 0, :], wrong[:, 0, 1, :] = w[:, 0, 1, :], w[:, 1, 0, :]
    ref = CN.conv3x3(x, wrong, np.zeros(Cout))
    S = CN.conv3x3(np.abs(x), np.abs(w), np.zeros(Cout))
    tol = 2.0 ** -8 * np.abs(ref) + (9 * Cin + 2) * 2.0 ** -22 * S * (1 + 2.0 ** -8)
    assert np.mean(np.abs(_f64(Y) - ref) > tol) > 0.5
