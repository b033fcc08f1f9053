"""The multi-rank path on CPU: world size 2 over gloo (no GPU). Each rank takes its shard of
a score vector, forms its local log normaliser with the oracle, and the combined log Z must
equal the oracle's over the whole vector; timings combine by their maximum."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2312_08715_gb300 import multigpu, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ll = synth.random_ll(np.random.default_rng(99), n).astype(np.float64)
    b, e = multigpu.shard_range(n, rank, world)
    local = oracle.lse(ll[b:e])[0] if e > b else -np.inf
    z = multigpu.combine_logz(torch.tensor([local], dtype=torch.float64))
    t = multigpu.max_over_ranks(10.0 + rank)
    out[rank] = (float(z), t, b, e)
    dist.destroy_process_group()


@pytest.mark.parametrize("n", [1, 145800])
def test_sharded_log_normaliser_matches_oracle(orc, n):
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), n, out), nprocs=world, join=True)
    ll = synth.random_ll(np.random.default_rng(99), n).astype(np.float64)
    z_ref, _ = orc.lse(ll)
    for r in range(world):
        z, t, b, e = out[r]
        assert z == pytest.approx(z_ref, abs=1e-9)
        assert t == 11.0
    assert out[0][2] == 0 and out[0][3] == out[1][2] and out[1][3] == n


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 7, 145800):
        for world in (1, 2, 3, 8):
            spans = [multigpu.shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in spans]
            assert max(sizes) - min(sizes) <= 1
