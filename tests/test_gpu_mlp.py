"""The learned operator's network on the tensor cores (tcgen05) against the
FP64 oracle: forward values, the loss and its gradient (BF16 operands and
activations, FP32 accumulation: agreement to the BF16 rounding level), and a
training run that must reduce the loss."""
import math

import numpy as np
import pytest

import oracle as O
from tests.gpu_util import bf16_round, random_params
import paper_1503_00707_gb300 as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1503_00707_gb300 import _build
    _build.build()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_forward_matches_oracle():
    s = D.Solver(D.F32, D.COLL_NONE, 1.0)
    params = random_params(1, gain=1.5)
    s.set_weights(params)
    rng = np.random.default_rng(2)
    x = bf16_round(rng.normal(size=(300, 64)))  # 2 full 128-row tiles and a ragged one
    y = s.mlp_forward(x)
    ref = O.mlp_forward(params.astype(np.float64), x.astype(np.float64))
    assert rel(y, ref) < 2e-2
    assert np.max(np.abs(y - ref)) < 5e-2 * np.max(np.abs(ref))


def test_loss_and_gradient_match_oracle():
    s = D.Solver(D.F32, D.COLL_NONE, 1.0)
    params = random_params(3, gain=1.5)
    s.set_weights(params)
    rng = np.random.default_rng(4)
    x = bf16_round(rng.normal(size=(200, 64)))
    t = rng.normal(size=(200, 64)).astype(np.float32)
    loss, g = s.mlp_loss_grad(x, t)
    gref, lref = O.mlp_backward(params.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lref) < 1e-2 * lref
    off = 0
    for (r, c), nb in O.MLP_SHAPES:
        for n in (r * c, nb):
            assert rel(g[off:off + n], gref[off:off + n]) < 5e-2, (r, c, n)
            off += n


def test_training_reduces_loss():
    """Fit a fixed teacher network's outputs with Adam on the GPU."""
    teacher = random_params(5, gain=1.0)
    rng = np.random.default_rng(6)
    x = bf16_round(rng.normal(size=(4096, 64)))
    t = O.mlp_forward(teacher.astype(np.float64), x.astype(np.float64)).astype(np.float32)
    s = D.Solver(D.F32, D.COLL_NONE, 1.0)
    s.set_weights(random_params(7, gain=1.0))
    l0, _ = s.mlp_loss_grad(x, t, want_grad=False)
    l1 = s.train(x, t, epochs=40, batch=512, lr=1e-3, seed=1)
    l2, _ = s.mlp_loss_grad(x, t, want_grad=False)
    assert l2 < 0.2 * l0, (l0, l1, l2)
    # the weights moved and can be read back
    w = s.get_weights()
    assert w.shape == (D.MLP_NPARAM,) and np.isfinite(w).all()
