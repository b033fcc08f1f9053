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


def _local_draws(ll_shard, base, m, seed, stage, before, mass, logz, oracle):
    """A rank's part of the draw, restated in FP64 (what b3d_lse_resample_shard computes on a
    GPU rank): draw k, with u_k the oracle's 24-bit Philox uniform, is this rank's when it
    falls in [before, before + mass); its index is the shard's inverse CDF at
    (u_k - before) / mass. Other ranks' draws are -1 / -inf."""
    idx = np.full(m, -1, np.int64)
    logq = np.full(m, -np.inf)
    if ll_shard.size == 0 or mass <= 0:
        return idx, logq
    w = np.exp(ll_shard - ll_shard.max())
    cdf = np.cumsum(w)
    for k in range(m):
        u = oracle.uniform24(int(oracle.philox([k, stage, 0, 0], [seed, 0])[0]))
        if before <= u < before + mass:
            h = int(np.searchsorted(cdf, (u - before) / mass * cdf[-1], side="right"))
            h = min(h, ll_shard.size - 1)
            idx[k] = base + h
            logq[k] = ll_shard[h] - logz
    return idx, logq


def _draw_worker(rank, world, port, n, m, seed, stage, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from oracle import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ll = synth.random_ll(np.random.default_rng(7), n).astype(np.float64)
    b, e = multigpu.shard_range(n, rank, world)
    local = oracle.lse(ll[b:e])[0] if e > b else -np.inf
    logz, before, mass = multigpu.shard_masses(multigpu.gather_logz(local), rank)
    idx, logq = _local_draws(ll[b:e], b, m, seed, stage, before, mass, logz, oracle)
    i, q = multigpu.gather_draws(torch.as_tensor(idx), torch.as_tensor(logq))
    out[rank] = (logz, before, mass, i.numpy().copy(), q.numpy().copy())
    dist.destroy_process_group()


@pytest.mark.parametrize("n,world", [(145800, 2), (5, 2), (1, 2)])
def test_sharded_draws_match_unsharded_oracle(orc, n, world):
    """One categorical split over two gloo ranks: after the all-gather of the shards' log
    normalisers and the all-reduce of the draws, every rank holds the draws orc.resample
    makes on the whole vector (except a draw whose CDF margin is below 1e-5, where the split
    sums may round the other way), with logq = ll - log Z."""
    m, seed, stage = 100, 21, 1
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_draw_worker, args=(world, _free_port(), n, m, seed, stage, out), nprocs=world, join=True)
    ll = synth.random_ll(np.random.default_rng(7), n).astype(np.float64)
    idx, logq, margin = orc.resample(ll, m, seed, stage)
    z_ref, _ = orc.lse(ll)
    firm = margin >= 1e-5
    assert firm.mean() > 0.9
    masses = [out[r][2] for r in range(world)]
    assert sum(masses) == pytest.approx(1.0, abs=1e-12) and out[0][1] == 0.0
    for r in range(world):
        logz, _, _, i, q = out[r]
        assert logz == pytest.approx(z_ref, abs=1e-9)
        assert (i >= 0).all()  # every draw has an owner
        np.testing.assert_array_equal(i[firm], idx[firm])
        np.testing.assert_allclose(q[firm], logq[firm], rtol=0, atol=1e-9)
        np.testing.assert_array_equal(i, out[0][3])  # the same on every rank


def test_shard_masses_cover_the_unit_interval():
    z = [-3.0, 0.5, -np.inf, 2.0]
    parts = [multigpu.shard_masses(z, r) for r in range(len(z))]
    logz = parts[0][0]
    assert logz == pytest.approx(np.logaddexp.reduce([-3.0, 0.5, 2.0]))
    assert all(p[0] == logz for p in parts)
    # intervals [before, before + mass) tile [0, 1) in rank order; the empty shard owns nothing
    assert parts[0][1] == 0.0
    for a, b in zip(parts, parts[1:]):
        assert b[1] == pytest.approx(a[1] + a[2], abs=1e-15)
    assert parts[2][2] == 0.0
    assert parts[-1][1] + parts[-1][2] == 1.0
    assert multigpu.shard_masses([-np.inf, -np.inf], 1) == (-np.inf, 0.0, 0.0)
