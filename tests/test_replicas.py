"""The multi-GPU path of bench.py is replicas only (independent evaluations,
no collective on the data path): the timed region is the slowest rank's and
the value counts the units of all ranks.  Exercised here with two gloo ranks
on the CPU."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = bench.max_over_ranks(2.0 + rank, torch.device("cpu"))          # rank 1 is the slowest
        gathered = bench.gather_over_ranks({"rank": rank, "lat": [0.1 * (rank + 1)] * (rank + 2)})
        value = bench.replica_value(3, seconds, world)
        q.put((rank, seconds, gathered, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, seconds, gathered, value in out:
        assert seconds == 3.0                                     # max over the ranks
        assert [g["rank"] for g in gathered] == [0, 1]            # rank order
        assert sum(len(g["lat"]) for g in gathered) == 5
        assert value == pytest.approx(2 * 3 / 3.0)                # units of both ranks / slowest time


def test_single_process_is_the_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import torch

    import bench
    assert bench.max_over_ranks(1.5, torch.device("cpu")) == 1.5
    assert bench.gather_over_ranks({"a": 1}) == [{"a": 1}]
    assert bench.replica_value(4, 2.0, 1) == 2.0


def test_mle_checkpoint_round_trip(tmp_path):
    """The MLE bench saves the Nelder-Mead state (a plain host struct) and its
    step records after every step; a later run resumes from them."""
    sys.path.insert(0, ROOT)
    import bench
    import paper_2008_07437_gb300 as geo
    st = geo.geo_mle_init(geo.Theta((1.0, 1.2), 0.1, (0.5, 1.0), 0.4))
    st.iter, st.evals = 3, 17
    path = str(tmp_path / "mle.ckpt")
    assert bench._mle_load(path, geo) == (None, [])
    recs = [{"step": 1, "seconds": 2.5, "evals": 11, "best_loglik": -1.0},
            {"step": 2, "seconds": 1.5, "evals": 2, "best_loglik": -0.5}]
    bench._mle_save(path, st, recs)
    st2, recs2 = bench._mle_load(path, geo)
    assert bytes(st2) == bytes(st) and recs2 == recs
    assert st2.evals == 17 and st2.iter == 3


def test_workload_overrides_for_the_emulated_form():
    """--oz-cut switches the level cut of the emulated workloads (and names the variant);
    the configuration the bench prints says which form ran."""
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    base = dict(workload="bivariate-n20000", n=0, n_pred=-1, nb=0, tlr_tol=0.0, dst=0, oz_cut=-1,
                tlr_z="model")
    w = bench.workload(argparse.Namespace(**base))
    assert w.extra.get("oz_cut") == 1 and w.extra.get("oz_slices") == 8
    assert "level cut" in bench.config_json(w, argparse.Namespace(**base))["form"]
    w0 = bench.workload(argparse.Namespace(**dict(base, oz_cut=0)))
    assert w0.name.endswith("-nocut") and w0.extra["oz_cut"] == 0
    assert "level cut" not in bench.config_json(w0, argparse.Namespace(**base))["form"]
    # the native form has no cut to switch
    wn = bench.workload(argparse.Namespace(**dict(base, workload="bivariate-n20000-native", oz_cut=1)))
    assert "oz_cut" not in wn.extra and "fp64_gemm" not in wn.extra
