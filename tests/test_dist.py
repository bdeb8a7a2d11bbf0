"""Multi-rank path on CPU ranks (torch.distributed, gloo, world size 2): the
chain sharding plus the integer all-reduce of the histograms reproduces the
single-process run exactly; a rank that leaves before the exchange makes
the other rank's collective fail with an error instead of hanging."""
import datetime
import os
import socket

import numpy as np
import pytest

from paper_2007_07379_gb300 import dist as D
from paper_2007_07379_gb300 import workloads as W


def test_shard_covers_all_chains():
    for chains in (1, 31, 32, 33, 4096, 4100, 65536):
        for world in (1, 2, 3, 8):
            parts = [D.shard(chains, r, world) for r in range(world)]
            assert sum(c for c, _ in parts) == chains
            g0s = [g for _, g in parts]
            assert g0s == sorted(g0s)
            # consecutive ranks own consecutive group ranges
            for (c, g0), (_, g1) in zip(parts, parts[1:]):
                assert g0 + (c + 31) // 32 == g1 or c == 0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, mode):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    try:
        import oracle
        n, d = 4, 6
        g = W.random_circuit(n, d, 19)
        chains = 100
        c, g0 = D.shard(chains, rank, world)
        if mode == "leave" and rank == 1:
            q.put((rank, "left"))
            return  # leaves before the exchange
        if mode == "phase":  # a general-gate model: FP64 phase sums + exact counters
            gu, mu = W.random_general_circuit(n, d, 19, frac_u=0.6)
            r = oracle.u_gibbs(n, d, gu, mu, J=3.0, seed=7, chains=c, chain0=g0 * 32, sweeps=15)
            sums, cnt, valid, samples = D.allreduce_phase_sums(r["sum"], r["cnt"], r["valid"],
                                                               r["samples"])
            q.put((rank, (sums.tolist(), cnt.tolist(), valid, samples)))
            return
        r = oracle.gibbs(n, d, g, J=3.0, seed=7, chains=c, chain0=g0 * 32, sweeps=15)
        try:
            cnt, valid, samples = D.allreduce_histogram(r["cnt"], r["valid"], r["samples"])
            q.put((rank, (cnt.tolist(), valid, samples)))
        except Exception as e:  # noqa: BLE001
            q.put((rank, "error: " + type(e).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _spawn(mode):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, mode)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        rank, val = q.get(timeout=120)
        out[rank] = val
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return out


def test_two_rank_reduction_equals_single_run():
    import oracle
    out = _spawn("ok")
    n, d = 4, 6
    g = W.random_circuit(n, d, 19)
    ref = oracle.gibbs(n, d, g, J=3.0, seed=7, chains=100, sweeps=15)
    for rank in (0, 1):
        cnt, valid, samples = out[rank]
        assert np.array_equal(np.array(cnt, dtype=np.uint64), ref["cnt"])
        assert valid == ref["valid"] and samples == ref["samples"]


def test_rank_leaving_before_the_exchange_is_detected():
    out = _spawn("leave")
    assert out[1] == "left"
    assert isinstance(out[0], str) and out[0].startswith("error"), out[0]



def test_two_rank_phase_sums_equal_single_run():
    """General one-qubit gates: the counters reduce exactly and the FP64 phase
    sums to rounding."""
    import oracle
    out = _spawn("phase")
    n, d = 4, 6
    gu, mu = W.random_general_circuit(n, d, 19, frac_u=0.6)
    ref = oracle.u_gibbs(n, d, gu, mu, J=3.0, seed=7, chains=100, sweeps=15)
    for rank in (0, 1):
        sums, cnt, valid, samples = out[rank]
        assert np.array_equal(np.array(cnt, dtype=np.uint64), ref["cnt"])
        assert valid == ref["valid"] and samples == ref["samples"]
        assert np.allclose(np.array(sums), ref["sum"], rtol=0, atol=1e-9)
