"""What the trained near-contact correction gains over the coarse method.

Training data are approach runs the library generates itself (prescribed
motion, coarse and 2x resolution under diffusive scaling); the network is
trained by the library's BF16 tensor-core kernels with the symmetry
augmentation and early stopping on held-back runs.  Bar: on approach runs
of other seeds that took no part in training, the mean squared error of the
coarse hydrodynamic force and torque against the 2x run (each of the six
body-frame outputs divided by its spread in the training data) is below 0.9
of its value without the correction.
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


def test_trained_correction_reduces_the_error_on_held_out_runs():
    from paper_1005_2594_gb300 import bloodlb as bl
    from paper_1005_2594_gb300 import learned

    X, Y, _, runs = learned.approach_samples(64, seed=11)
    Xh, Yh, _, _ = learned.approach_samples(20, seed=12)
    m, info = learned.fit(X, Y, runs, seed=0)
    e0, e1 = learned.errors(m, Xh, Yh, Y.std(axis=0))
    print("training samples %d (augmented), validation %d, held-out %d; held-out error %.4f -> %.4f (ratio %.3f)"
          % (info["train_samples"], info["val_samples"], Xh.shape[0], e0, e1, e1 / e0))
    assert info["loss_last"] < info["loss_first"]
    assert e1 < 0.9 * e0
    bl.bl_mlp_destroy(m)
