"""Parity of the batch engine (snp_explore_batch): every system of a batch must
give exactly what the oracle gives for it alone (discovery order, per-depth
counts), whatever the pass size, tile and warps per CTA."""
import numpy as np
import pytest

import bruteforce as bf
import oracle
import snp_synth

pytestmark = pytest.mark.gpu


def assert_matches_oracle(s, system, depth, cap, budget, max_expand=-1):
    e = oracle.Oracle(system).explore(depth, cap=cap, budget=budget, max_expand=max_expand)
    got = s.reachable()
    assert got.shape == e.configs.shape
    assert (got == e.configs).all()
    st = s.depth_stats()
    assert len(st) == len(e.depths)
    for d, (a, b) in enumerate(zip(st, e.depths)):
        assert a.new == b.new, d
        if d > 0:
            assert (a.examined, a.candidates, a.truncated) == (b.examined, b.candidates, b.truncated), d


def test_batch_systems_match_oracle(gpu):
    systems = snp_synth.batch_systems(24)
    handles = [gpu.System(x) for x in systems]
    st = gpu.explore_batch(handles, 4, cap=512, budget=8192)
    assert (st == 0).all()
    for h, x in zip(handles, systems):
        assert_matches_oracle(h, x, 4, 512, 8192)


@pytest.mark.parametrize("cap,budget", [(1, 0), (3, 7), (50, 0), (7, 40)])
def test_batch_tiny_systems(gpu, cap, budget):
    rng = np.random.default_rng(3000 + cap * 17 + budget)
    systems = [bf.tiny_system(rng, m_max=4, r_max=9) for _ in range(40)]
    handles = [gpu.System(x) for x in systems]
    st = gpu.explore_batch(handles, 5, cap=cap, budget=budget)
    assert (st == 0).all()
    for h, x in zip(handles, systems):
        assert_matches_oracle(h, x, 5, cap, budget)


@pytest.mark.parametrize("chunk,tile,warps", [(32, 2, 4), (1024, 8, 8), (4096, 32, 4), (100, 5, 8)])
def test_batch_plan_does_not_change_results(gpu, chunk, tile, warps):
    systems = snp_synth.batch_systems(10)
    handles = [gpu.System(x) for x in systems]
    gpu.explore_batch(handles, 3, cap=300, budget=5000, chunk=chunk, tile=tile, warps=warps)
    for h, x in zip(handles, systems):
        assert_matches_oracle(h, x, 3, 300, 5000)


def test_batch_equals_single_explores_at_batch_settings(gpu):
    """cap 2^12, budget 2^16, depth 6: the batch configuration's settings."""
    systems = snp_synth.batch_systems(64)
    handles = [gpu.System(x) for x in systems]
    st = gpu.explore_batch(handles, 6, cap=1 << 12, budget=1 << 16)
    assert (st == 0).all()
    for k in range(0, 64, 9):
        single = gpu.System(systems[k])
        single.explore(6, cap=1 << 12, budget=1 << 16)
        assert (single.reachable() == handles[k].reachable()).all()
        assert [(a.new, a.examined) for a in single.depth_stats()] == \
               [(a.new, a.examined) for a in handles[k].depth_stats()]
    for k in (0, 31):
        assert_matches_oracle(handles[k], systems[k], 6, 1 << 12, 1 << 16)


def test_batch_replay_and_reuse(gpu):
    paper = snp_synth.paper_example()
    handles = [gpu.System(paper), gpu.System(snp_synth.random_64(1))]
    gpu.explore_batch(handles, 40, cap=1 << 10, budget=1 << 14, max_expand=9)
    assert_matches_oracle(handles[0], paper, 40, 1 << 10, 1 << 14, max_expand=9)
    # a handle can explore alone afterwards, and batch again
    handles[1].explore(2, cap=100, budget=1000)
    assert_matches_oracle(handles[1], snp_synth.random_64(1), 2, 100, 1000)
    gpu.explore_batch(handles, 2, cap=100, budget=1000)
    assert_matches_oracle(handles[1], snp_synth.random_64(1), 2, 100, 1000)


def test_batch_autotune(gpu):
    systems = snp_synth.batch_systems(32)
    handles = [gpu.System(x) for x in systems]
    o = gpu.snp_explore_opts_init()
    o.depth, o.frontier_cap, o.candidate_budget = 3, 256, 4096
    chunk, tile, warps = gpu.snp_batch_autotune([h.h for h in handles], o)
    assert chunk in (1024, 2048, 4096) and tile in (8, 16, 32) and warps in (4, 8)
    gpu.explore_batch(handles, 3, cap=256, budget=4096, chunk=chunk, tile=tile, warps=warps)
    assert_matches_oracle(handles[5], systems[5], 3, 256, 4096)


def test_batch_rejects_bad_options(gpu):
    h = [gpu.System(snp_synth.paper_example())]
    o = gpu.snp_explore_opts_init()
    o.depth = 3
    o.frontier_cap = 0
    with pytest.raises(gpu.SnpError) as ei:
        gpu.snp_explore_batch([x.h for x in h], o)
    assert ei.value.code == gpu.SNP_E_INVALID


# --- the fp8 tensor-core form in the batch engine ---

def test_batch_tc_systems_match_oracle(gpu):
    systems = snp_synth.batch_systems(24)
    handles = [gpu.System(x) for x in systems]
    st = gpu.explore_batch(handles, 4, cap=512, budget=8192, transition=gpu.SNP_T_TC_F8)
    assert (st == 0).all()
    for h, x in zip(handles, systems):
        assert_matches_oracle(h, x, 4, 512, 8192)


@pytest.mark.parametrize("cap,budget,chunk", [(1, 0, 0), (3, 7, 32), (50, 0, 100), (7, 40, 0)])
def test_batch_tc_tiny_systems(gpu, cap, budget, chunk):
    rng = np.random.default_rng(4000 + cap * 17 + budget)
    systems = [bf.tiny_system(rng, m_max=4, r_max=9) for _ in range(40)]
    handles = [gpu.System(x) for x in systems]
    st = gpu.explore_batch(handles, 5, cap=cap, budget=budget, chunk=chunk, transition=gpu.SNP_T_TC_F8)
    assert (st == 0).all()
    for h, x in zip(handles, systems):
        assert_matches_oracle(h, x, 5, cap, budget)


def test_batch_tc_wide_and_many_rule_systems(gpu):
    """Rows of 129 to 700 neurons (several 128-column chunks) and a system of
    16 rules per neuron (more rule blocks than the operand holds at once)."""
    systems = [snp_synth.random_system(60 + k, m, (1, 3), (2, 6), (0, 5), "sparse")
               for k, m in enumerate((129, 300, 700))]
    systems.append(snp_synth.random_system(77, 128, (16, 16), (2, 4), (0, 6), "sparse"))
    handles = [gpu.System(x) for x in systems]
    st = gpu.explore_batch(handles, 3, cap=400, budget=4000, transition=gpu.SNP_T_TC_F8)
    assert (st == 0).all()
    for h, x in zip(handles, systems):
        assert_matches_oracle(h, x, 3, 400, 4000)


def test_batch_tc_equals_sparse_at_batch_settings(gpu):
    systems = snp_synth.batch_systems(64)
    a = [gpu.System(x) for x in systems]
    b = [gpu.System(x) for x in systems]
    assert (gpu.explore_batch(a, 6, cap=1 << 12, budget=1 << 16) == 0).all()
    assert (gpu.explore_batch(b, 6, cap=1 << 12, budget=1 << 16, transition=gpu.SNP_T_TC_F8) == 0).all()
    for x, y in zip(a, b):
        assert (x.reachable() == y.reachable()).all()
        assert [(p.new, p.examined) for p in x.depth_stats()] == [(p.new, p.examined) for p in y.depth_stats()]


def test_batch_tc_refusals(gpu):
    systems = snp_synth.batch_systems(2)
    handles = [gpu.System(x) for x in systems]
    with pytest.raises(gpu.SnpError) as ei:
        gpu.explore_batch(handles, 2, cap=16, transition=gpu.SNP_T_TC_I8)
    assert ei.value.code == gpu.SNP_E_INVALID
    big = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [17, 1], [[1], [0]], [3, 3])
    with pytest.raises(gpu.SnpError) as ei:
        gpu.explore_batch([gpu.System(big)], 2, cap=16, transition=gpu.SNP_T_TC_F8)
    assert ei.value.code == gpu.SNP_E_RANGE
