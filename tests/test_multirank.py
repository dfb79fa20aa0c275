"""The multi-rank host logic of bench.py, on CPU with two gloo ranks.

bench.py runs one process per GPU under torchrun.  What the ranks share is
the aggregation (the max over ranks of the timed region, the sums over ranks
of the units processed) and, for the batch workload, the split of a larger
batch into per-rank blocks of independent systems.
"""
import multiprocessing
import os
import socket

import numpy as np

import bench
import snp_synth


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: a timed region of 10 + 5 r ms, 100 (r + 1) units and 7 launches
        ms, counts = bench.aggregate_ranks(10.0 + 5.0 * rank, [100 * (rank + 1), 7], dist, "cpu")
        out.put((rank, ms, counts, bench.rank_info()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_sum_the_units():
    ctx = multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[0] for g in got] == [0, 1]
    for rank, ms, counts, info in got:
        assert ms == 15.0
        assert counts == [300.0, 14.0]
        assert info == (rank, 2, rank)


def test_one_rank_passes_its_numbers_through():
    assert bench.aggregate_ranks(3.5, [4, 5]) == (3.5, [4.0, 5.0])


def _same_system(a, b) -> bool:
    return all(np.array_equal(np.asarray(getattr(a, f)), np.asarray(getattr(b, f)))
               for f in ("rule_neuron", "rule_i", "rule_j", "M", "c0"))


def test_batch_ranks_take_consecutive_blocks_of_one_larger_batch():
    w = dict(bench.WORKLOADS["batch4096"], n=5)
    assert bench.batch_seed_base(w, 0) == w["base_seed"]
    whole = snp_synth.batch_systems(3 * w["n"], w["base_seed"])
    for r in range(3):
        block = snp_synth.batch_systems(w["n"], bench.batch_seed_base(w, r))
        assert all(_same_system(a, b) for a, b in zip(block, whole[r * w["n"]:(r + 1) * w["n"]]))
    # rank 0's block is the single-GPU batch
    assert all(_same_system(a, b) for a, b in zip(snp_synth.batch_systems(w["n"], w["base_seed"]), whole))
