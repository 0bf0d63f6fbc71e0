"""Element-sharded evaluation over world-size-2 gloo ranks on the CPU: the sum
over ranks of the per-shard (loss parts, gradient) equals the unsharded
result.  The per-shard evaluator here is the CPU oracle (the library's CUDA
evaluator plugs into the same host logic on GPU ranks)."""
import os
import socket

import numpy as np
import pytest

import fv_inputs as fi

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle_evaluator(sub):
    import oracle
    b = oracle.Bound(sub)

    def ev(params):
        r = b.loss_grad(params)
        return np.array([r["loss"], r["Lv"], r["Lb"], r["Ls"], r["dL_deps"]]), r["grad"]
    return ev


def _worker(rank, world, port, cfg, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2404_12063_b300.parallel import ShardedLoss
    prob = fi.inverse_cd2d(24) if cfg == "inverse" else fi.skewed_disc()
    sl = ShardedLoss(prob, rank, world, _oracle_evaluator)
    out, grad = sl.loss_grad(prob.params)
    if rank == 0:
        np.save(result_path, np.concatenate([out, grad]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("cfg", ["disc", "inverse"])
def test_two_rank_shards_sum_to_the_whole(tmp_path, cfg):
    import torch.multiprocessing as mp
    import oracle
    world = 2
    res = str(tmp_path / "r.npy")
    mp.start_processes(_worker, args=(world, _free_port(), cfg, res), nprocs=world, join=True, start_method="spawn")
    got = np.load(res)
    prob = fi.inverse_cd2d(24) if cfg == "inverse" else fi.skewed_disc()
    ref = oracle.Bound(prob).loss_grad(prob.params)
    want = np.concatenate([[ref["loss"], ref["Lv"], ref["Lb"], ref["Ls"], ref["dL_deps"]], ref["grad"]])
    np.testing.assert_allclose(got[:5], want[:5], rtol=1e-12)
    assert np.linalg.norm(got[5:] - want[5:]) < 1e-12 * np.linalg.norm(want[5:])


def test_shard_ranges_cover_and_balance():
    from paper_2404_12063_b300.parallel import shard_ranges
    for n, w in ((1024, 2), (8192, 8), (10, 3), (5, 8)):
        r = shard_ranges(n, w)
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [hi - lo for lo, hi in r]
        assert max(sizes) - min(sizes) <= 1
