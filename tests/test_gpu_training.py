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
    prob = fi.tiny_square()
    h = train.train(ctx, prob, precision, epochs=600, lr=3e-3, every=200)
    assert h[-1][2] < 0.2 * h[1][2]          # loss
    assert h[-1][3] < h[0][3]                # relative L2 error of u


def test_inverse_problem_eps_moves_to_truth(ctx):
    from paper_2404_12063_b300 import train
    prob = fi.inverse_cd2d(8)
    h = train.train(ctx, prob, "fp32", epochs=1500, lr=1e-2, every=500, train_eps=True)
    eps_path = [r[4] for r in h]
    assert abs(eps_path[-1] - 0.3) < 0.5 * abs(eps_path[0] - 0.3)


@pytest.mark.parametrize("k,precision", [("inverse", "fp32"), ("disc", "fp16"), ("tiny", "fp64")])
def test_step_graph_equals_individual_steps(ctx, k, precision):
    """A captured graph of n training steps (loss + grad + Adam) gives bitwise
    the parameters, eps, gradient and loss of n fv_inverse_step calls."""
    from paper_2404_12063_b300 import api
    prob = fi.WORKLOADS[k]()
    pb = api.problem_from_inputs(ctx, prob, precision)
    n = 4
    res = []
    for graph in (False, True):
        params = torch.tensor(prob.params, dtype=pb.dtype, device="cuda")
        eps = torch.tensor([prob.eps], dtype=torch.float64, device="cuda")
        adam = api.Adam(ctx, pb.net.n_params, precision, with_eps=(k == "inverse"))
        grad = torch.empty_like(params)
        out = torch.zeros(5, dtype=torch.float64, device="cuda")
        if graph:
            g = api.StepGraph(pb, params, eps, adam, 1e-3, n_steps=n, grad=grad, out=out)
            g.launch()
            g.launch()
        else:
            for _ in range(2 * n):
                pb.inverse_step(params, eps, adam, 1e-3, grad, out)
        torch.cuda.synchronize()
        res.append((params.clone(), eps.clone(), grad.clone(), out.clone()))
        if graph:
            g.close()
    for a, b in zip(*res):
        assert torch.equal(a, b)
