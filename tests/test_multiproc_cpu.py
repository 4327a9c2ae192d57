"""The multi-rank path on CPU: two gloo ranks, each decoding its own batch with the oracle,
must together reproduce the single-process result, and the timing reduction must take
the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2507_10424_gb300 import inputs, shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, F, out_dir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    code = inputs.cfg_regular_576()
    llr = inputs.all_zero_awgn_llr(F, code.N, 2.0, code.design_rate, shard.rank_seed(40, rank))
    g = oracle.Graph.from_code(code)
    bits, iters, ok, _ = oracle.decode_f32(g, llr, 20, threads=1, soft=False)
    t = shard.max_over_ranks(1.0 + rank)  # stands in for this rank's step time
    np.savez(os.path.join(out_dir, f"r{rank}.npz"), bits=bits, iters=iters, ok=ok, t=t)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_decode(tmp_path):
    import oracle
    world, F = 2, 64
    mp.start_processes(_worker, args=(world, _free_port(), F, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    code = inputs.cfg_regular_576()
    g = oracle.Graph.from_code(code)
    for rank in range(world):
        res = np.load(tmp_path / f"r{rank}.npz")
        llr = inputs.all_zero_awgn_llr(F, code.N, 2.0, code.design_rate, shard.rank_seed(40, rank))
        bits, iters, ok, _ = oracle.decode_f32(g, llr, 20, soft=False)
        assert (res["bits"] == bits).all() and (res["iters"] == iters).all()
        assert float(res["t"]) == 2.0  # the maximum over ranks


@pytest.mark.parametrize("total,world", [(10, 3), (65536, 8), (5, 8), (0, 2)])
def test_frame_range_partitions_exactly(total, world):
    spans = [shard.frame_range(total, r, world) for r in range(world)]
    assert spans[0][0] == 0 and spans[-1][1] == total
    for (a, b), (c, d) in zip(spans, spans[1:]):
        assert b == c and b - a >= d - c >= b - a - 1
