"""The learned near-contact correction's tensor-core kernels against the FP64
oracle (oracle/mlp.py), through the C ABI.

Bars: forward outputs and the loss within 2e-2 relative, the gradient within
3e-2 relative to its largest component: weights and activations are rounded
to BF16 (8 significant bits, relative step 2^-8 = 3.9e-3) before every
product, and a product of 64 terms accumulated in FP32 keeps that order of
error.  Training: Adam on the GPU cuts the loss of a teacher-student fit by
more than 20 times.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    import torch

    torch.cuda.init()
    yield


def _data(seed, B):
    from oracle import mlp

    rng = np.random.default_rng(seed)
    theta = mlp.init_params(seed) + rng.normal(0, 0.05, mlp.N_PARAMS)
    mx, sx = rng.normal(0, 1, 14), rng.uniform(0.5, 2.0, 14)
    my, sy = rng.normal(0, 1, 6), rng.uniform(0.5, 2.0, 6)
    x = mx + sx * rng.normal(0, 1, (B, 14))
    y = my + sy * rng.normal(0, 1, (B, 6))
    norm = np.concatenate([mx, sx, my, sy])
    return theta, norm, x, y


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


def test_forward_loss_and_gradient_match_oracle():
    import torch

    from oracle import mlp
    from paper_1005_2594_gb300 import bloodlb as bl

    theta, norm, x, y = _data(21, 333)  # a ragged last tile
    m = bl.bl_mlp_create()
    bl.bl_mlp_params_set(m, theta, norm)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    out = torch.zeros((x.shape[0], 6), dtype=torch.float32, device="cuda")
    bl.bl_mlp_forward(m, xd, out)
    torch.cuda.synchronize()
    xs = (x - norm[:14]) / norm[14:28]
    ys = (y - norm[28:34]) / norm[34:40]
    yo, _ = mlp.forward(theta, xs)
    y_raw = yo * norm[34:40] + norm[28:34]
    assert rel(out.cpu().numpy(), y_raw) < 2e-2
    loss_o, g_o = mlp.loss_and_grad(theta, xs, ys)
    loss_g, g_g = bl.bl_mlp_grad(m, xd, yd, want_grad=True)
    print("loss gpu %.6f oracle %.6f, grad rel err %.3e" % (loss_g, loss_o, rel(g_g, g_o)))
    assert abs(loss_g - loss_o) < 2e-2 * loss_o
    assert rel(g_g, g_o) < 3e-2
    # the same data give the same gradient (fixed reduction order)
    _, g_again = bl.bl_mlp_grad(m, xd, yd, want_grad=True)
    assert rel(g_again, g_g) < 1e-5
    bl.bl_mlp_destroy(m)


def test_adam_training_fits_a_teacher():
    import torch

    from oracle import mlp
    from paper_1005_2594_gb300 import bloodlb as bl

    rng = np.random.default_rng(5)
    teacher = mlp.init_params(99) * 2.0
    x = rng.normal(0, 1, (4096, 14))
    y, _ = mlp.forward(teacher, x)
    norm = np.concatenate([np.zeros(14), np.ones(14), np.zeros(6), np.ones(6)])
    m = bl.bl_mlp_create()
    bl.bl_mlp_params_set(m, mlp.init_params(7), norm)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    first = None
    for it in range(600):
        loss, _ = bl.bl_mlp_grad(m, xd, yd)
        if it == 0:
            first = loss
        bl.bl_mlp_adam(m, lr=3e-3)
    last, _ = bl.bl_mlp_grad(m, xd, yd)
    print("teacher fit: loss %.4e -> %.4e" % (first, last))
    assert last < first / 20
    bl.bl_mlp_destroy(m)
