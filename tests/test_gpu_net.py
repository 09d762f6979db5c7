"""The CUDA warm-start network against the FP64 reference (oracle/nn.py):
forward outputs and every parameter gradient, in the FP32 mode (tight) and
the BF16 mode (BF16 storage, FP32 accumulation)."""
import numpy as np
import pytest

from oracle import nn
from paper_2012_14707_gb300 import build as lbm_build
from paper_2012_14707_gb300 import lbm

pytestmark = pytest.mark.gpu


def _flat(p, levels, base):
    parts = []
    for name, kind, ci, co in nn.layer_shapes(3, 3, base, levels):
        parts.append(p[name + ".w"].reshape(-1))
        parts.append(p[name + ".b"].reshape(-1))
    return np.concatenate(parts)


@pytest.mark.parametrize("precision,rtol,grad_rtol", [("fp32", 2e-5, 2e-5), ("bf16", 3e-2, 8e-2)])
def test_forward_and_gradients_match_reference(precision, rtol, grad_rtol):
    """FP32 mode: forward and every gradient within 2e-5 (rel. L2 per
    tensor).  BF16 mode: forward within 3 %; gradients within 8 % -- the
    activation gradients are stored in BF16 at every one of the 14 layers
    they pass through, so the first layer's error compounds (measured
    4.7 %)."""
    import torch

    lbm_build.build()
    torch.cuda.set_device(0)
    levels, base, H, W, N = 3, 8, 16, 24, 2
    rng = np.random.default_rng(11)
    p = nn.init_params(5, base=base, levels=levels)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.05
    x = rng.standard_normal((N, H, W, 3))
    t = rng.standard_normal((N, H, W, 3))
    y_ref, cache = nn.forward(p, x, levels)
    g_ref = nn.backward(p, cache, y_ref, t, levels)
    net = lbm.Net(H, W, base=base, levels=levels, precision=precision, max_batch=N)
    flat = _flat(p, levels, base)
    assert net.n_params == flat.size
    net.set_params(flat)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    yd = torch.empty((N, H, W, 3), dtype=torch.float32, device="cuda")
    net.forward(xd.data_ptr(), N, yd.data_ptr())
    y = yd.cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= rtol * np.linalg.norm(y_ref)
    g, loss = net.gradients(xd.data_ptr(), td.data_ptr(), N)
    assert loss == pytest.approx(nn.mse(y_ref, t), rel=rtol)
    g_ref_flat = _flat(g_ref, levels, base)
    # per layer tensor, relative L2 of the gradient
    off = 0
    for name, kind, ci, co in nn.layer_shapes(3, 3, base, levels):
        for suffix in (".w", ".b"):
            size = g_ref[name + suffix].size
            a, b = g[off:off + size], g_ref_flat[off:off + size]
            off += size
            assert np.linalg.norm(a - b) <= grad_rtol * np.linalg.norm(b) + 1e-12, (name + suffix)


def test_training_lowers_the_loss():
    import torch

    lbm_build.build()
    torch.cuda.set_device(0)
    H = W = 32
    net = lbm.Net(H, W, base=8, levels=3, precision="bf16", max_batch=4, seed=3)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, H, W, 3)).astype(np.float32)
    t = np.stack([np.tanh(x[..., 0]), x[..., 1] * 0.5, x[..., 2] ** 2 * 0.2], axis=-1).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    td = torch.tensor(t, device="cuda")
    first = net.train_step(xd.data_ptr(), td.data_ptr(), 4, 3e-3)
    for _ in range(200):
        last = net.train_step(xd.data_ptr(), td.data_ptr(), 4, 3e-3)
    assert last < 0.3 * first


def test_bf16_tensor_core_path_matches_fp32_at_full_width():
    """The full-width network (base 32, 4 levels: up to 384 input and 256
    output channels, two 128-channel output tiles, 64-channel K chunks) in
    BF16 mode -- the tensor-core convolutions -- against the FP32 mode
    (CUDA cores) with the same parameters: forward within 3 % (rel. L2),
    gradients of every layer within 10 %."""
    import torch

    lbm_build.build()
    torch.cuda.set_device(0)
    H = W = 64
    N = 2
    n32 = lbm.Net(H, W, base=32, levels=4, precision="fp32", max_batch=N, seed=7)
    n16 = lbm.Net(H, W, base=32, levels=4, precision="bf16", max_batch=N, seed=7)
    p = n32.get_params()
    rng = np.random.default_rng(4)
    p = p + 0.0  # He-normal weights, zero biases; give the biases some size
    n32.set_params(p)
    n16.set_params(p)
    x = rng.standard_normal((N, H, W, 3)).astype(np.float32)
    t = rng.standard_normal((N, H, W, 3)).astype(np.float32)
    xd = torch.tensor(x, device="cuda")
    td = torch.tensor(t, device="cuda")
    y32 = torch.empty((N, H, W, 3), device="cuda")
    y16 = torch.empty((N, H, W, 3), device="cuda")
    n32.forward(xd.data_ptr(), N, y32.data_ptr())
    n16.forward(xd.data_ptr(), N, y16.data_ptr())
    a, b = y16.cpu().numpy(), y32.cpu().numpy()
    assert np.isfinite(a).all()
    assert np.linalg.norm(a - b) <= 3e-2 * np.linalg.norm(b)
    g32, _ = n32.gradients(xd.data_ptr(), td.data_ptr(), N)
    g16, _ = n16.gradients(xd.data_ptr(), td.data_ptr(), N)
    off = 0
    for name, kind, ci, co in nn.layer_shapes(3, 3, 32, 4):
        size = (9 if kind == "c3" else 1) * ci * co
        ga, gb = g16[off:off + size], g32[off:off + size]
        assert np.linalg.norm(ga - gb) <= 0.1 * np.linalg.norm(gb) + 1e-12, name
        off += size + co


@pytest.mark.parametrize("precision,rtol,grad_rtol", [("fp32", 2e-5, 2e-5), ("bf16", 3e-2, 0.1)])
def test_full_width_network_matches_reference(precision, rtol, grad_rtol):
    """The full-width network of the warm start (base 32, 4 levels: 32 to
    256 channels, 384 input channels in the decoder, two 128-channel output
    tiles of the tensor-core convolutions) on a 32 x 32 lattice, against the
    FP64 reference (oracle/nn.py): forward and the gradient of every tensor.
    BF16 tolerances as in the full-width BF16-against-FP32 test: every
    activation and activation gradient is stored with 8 significant bits,
    and the deepest level (4 x 4 pixels here) sums its weight gradients over
    few pixels, so little of that rounding averages out."""
    import torch

    lbm_build.build()
    torch.cuda.set_device(0)
    levels, base, H, W, N = 4, 32, 32, 32, 2
    rng = np.random.default_rng(21)
    p = nn.init_params(9, base=base, levels=levels)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.05
    x = rng.standard_normal((N, H, W, 3))
    t = rng.standard_normal((N, H, W, 3))
    y_ref, cache = nn.forward(p, x, levels)
    g_ref = nn.backward(p, cache, y_ref, t, levels)
    net = lbm.Net(H, W, base=base, levels=levels, precision=precision, max_batch=N)
    net.set_params(_flat(p, levels, base))
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    td = torch.tensor(t, dtype=torch.float32, device="cuda")
    yd = torch.empty((N, H, W, 3), dtype=torch.float32, device="cuda")
    net.forward(xd.data_ptr(), N, yd.data_ptr())
    y = yd.cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= rtol * np.linalg.norm(y_ref)
    g, loss = net.gradients(xd.data_ptr(), td.data_ptr(), N)
    g_ref_flat = _flat(g_ref, levels, base)
    off = 0
    for name, kind, ci, co in nn.layer_shapes(3, 3, base, levels):
        for suffix in (".w", ".b"):
            size = g_ref[name + suffix].size
            a, b = g[off:off + size], g_ref_flat[off:off + size]
            off += size
            assert np.linalg.norm(a - b) <= grad_rtol * np.linalg.norm(b) + 1e-12, (name + suffix)
