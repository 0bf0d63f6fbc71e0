"""Training with the library's Adam step (fv_inverse_step): the loss and the
solution error fall, and in the inverse problem eps moves towards its true
value (paper Sec. 4.7.1: eps starts at 2, the data come from eps = 0.3)."""
import numpy as np
import pytest

import fv_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_12063_b300 import build
    build.build()
    from paper_2404_12063_b300 import api
    return api.Context(0)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_training_lowers_loss_and_error(ctx, precision):
    from paper_2404_12063_b300 import train
    prob = fi.config1_tiny()
    h = train.train(ctx, prob, precision, epochs=600, lr=3e-3, every=200)
    assert h[-1][2] < 0.2 * h[1][2]          # loss
    assert h[-1][3] < h[0][3]                # relative L2 error of u


def test_inverse_problem_eps_moves_to_truth(ctx):
    from paper_2404_12063_b300 import train
    prob = fi.config4_inverse(8)
    h = train.train(ctx, prob, "fp32", epochs=1500, lr=1e-2, every=500, train_eps=True)
    eps_path = [r[4] for r in h]
    assert abs(eps_path[-1] - 0.3) < 0.5 * abs(eps_path[0] - 0.3)
