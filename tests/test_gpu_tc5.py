"""Parity of the fp8 tensor-core transition (SNP_T_TC_F8: tcgen05, TMEM
accumulators) with the CPU oracle and the sparse int32 path, through the C ABI.

The product is exact (integer operands of at most 16 in magnitude, partial
sums below 2^24), so every comparison is bit for bit: discovery-ordered
configurations, per-depth counts, sums of Psi and truncation flags.  Cases
cover both operand forms (the difference from a reference spiking vector for
tiles inside one parent of a wide system; the full 0/1 spiking vector for rows
of at most 128 neurons and for tiles that cross parents), tiles cut by the
pass size, several column chunks, groups of more rule blocks than shared memory
holds at once, and the refusal of entries beyond 16.
"""
import numpy as np
import pytest

import bruteforce as bf
import oracle
import snp_synth
from conftest import read_golden
from test_gpu_parity import (assert_same, broadcast_system, digest, few_choice_system, golden_digests,
                             many_duplicates_system, saturating_system)

pytestmark = pytest.mark.gpu


def explore_f8(gpu, system, depth, **kw):
    s = gpu.System(system)
    s.explore(depth, transition=gpu.SNP_T_TC_F8, **kw)
    return s


def test_f8_paper_example_and_replay(gpu):
    g = read_golden("paper_run.txt")
    paper = snp_synth.paper_example()
    s = explore_f8(gpu, paper, 10)
    assert_same(s, oracle.Oracle(paper).explore(10))
    s = explore_f8(gpu, paper, 1000, max_expand=9)
    assert ["-".join(str(int(x)) for x in r) for r in s.reachable()] == g["allGenCk"].split()
    exact = snp_synth.paper_example(exact=True)
    assert_same(explore_f8(gpu, exact, 6), oracle.Oracle(exact).explore(6))


@pytest.mark.parametrize("cap,budget,chunk", [(0, 0, 0), (1, 0, 0), (3, 0, 1), (0, 7, 0), (5, 11, 3), (2, 1, 0)])
def test_f8_tiny_systems(gpu, cap, budget, chunk):
    rng = np.random.default_rng(3000 + 7 * cap + 13 * budget + chunk)
    for _ in range(25):
        system = bf.tiny_system(rng, m_max=4, r_max=9)
        s = explore_f8(gpu, system, 5, cap=cap, budget=budget, chunk=chunk)
        assert_same(s, oracle.Oracle(system).explore(5, cap=cap, budget=budget))


@pytest.mark.parametrize("m", [1, 5, 31, 64, 100, 127, 128, 129, 200, 255, 256, 257, 300, 513, 1024])
def test_f8_neuron_counts(gpu, m):
    """Rows of 1 to 1024 neurons: one to four column chunks of up to 256,
    chunks of 16 to 256 columns, rows that are and are not a multiple of 4."""
    system = snp_synth.random_system(800 + m, m, (1, 4), (1, min(8, max(1, m - 1))), (0, 6), "sparse")
    s = explore_f8(gpu, system, 3, cap=300, budget=3000)
    assert_same(s, oracle.Oracle(system).explore(3, cap=300, budget=3000))


@pytest.mark.parametrize("m,chunk", [(64, 1), (64, 127), (64, 129), (200, 128), (200, 200), (300, 1000)])
def test_f8_pass_sizes(gpu, m, chunk):
    """Passes that cut tiles (chunk not a multiple of 128) and tiles that
    start inside a parent."""
    system = snp_synth.random_system(850 + m + chunk, m, (2, 3), (2, 4), (0, 6), "sparse")
    s = explore_f8(gpu, system, 3, cap=1500, budget=15000, chunk=chunk)
    assert_same(s, oracle.Oracle(system).explore(3, cap=1500, budget=15000))


@pytest.mark.parametrize("m,k,chunk,depth", [(160, 2, 0, 6), (301, 3, 17, 6), (1024, 4, 0, 5)])
def test_f8_tiles_across_parents(gpu, m, k, chunk, depth):
    """Wide rows whose parents have at most 2^k spiking vectors: every tile
    crosses parents (the full product with the parent row as base)."""
    system = few_choice_system(m + k, m, k)
    s = explore_f8(gpu, system, depth, cap=3000, budget=30000, chunk=chunk)
    assert_same(s, oracle.Oracle(system).explore(depth, cap=3000, budget=30000))


@pytest.mark.parametrize("m,k,chunk", [(800, 6, 0), (801, 7, 50)])
def test_f8_large_supports(gpu, m, k, chunk):
    system = broadcast_system(m, k, m)
    s = explore_f8(gpu, system, 3, cap=800, budget=6000, chunk=chunk)
    assert_same(s, oracle.Oracle(system).explore(3, cap=800, budget=6000))


@pytest.mark.parametrize("m,k,chunk", [(64, 6, 0), (200, 7, 9), (1024, 5, 0)])
def test_f8_duplicates(gpu, m, k, chunk):
    system = many_duplicates_system(m, k)
    s = explore_f8(gpu, system, 4, chunk=chunk)
    assert_same(s, oracle.Oracle(system).explore(4))


@pytest.mark.parametrize("kind", ["steady", "drain"])
def test_f8_saturated_psi(gpu, kind):
    system = saturating_system(kind)
    s = explore_f8(gpu, system, 3, cap=20000, budget=1 << 16)
    assert_same(s, oracle.Oracle(system).explore(3, cap=20000, budget=1 << 16))


def test_f8_many_rule_blocks(gpu):
    """A 128-neuron system with 16 rules per neuron (2048 rules, 64 blocks):
    a tile's full spiking vectors touch more rule blocks than shared memory
    holds at once, so the product runs in several groups per column chunk."""
    system = snp_synth.random_system(77, 128, (16, 16), (2, 4), (0, 6), "sparse")
    s = explore_f8(gpu, system, 3, cap=1000, budget=8000)
    assert_same(s, oracle.Oracle(system).explore(3, cap=1000, budget=8000))


def test_f8_random64_small(gpu):
    g = golden_digests()["random64_seed1_small"]
    p = g["params"]
    s = explore_f8(gpu, snp_synth.random_64(1), p["depth"], cap=p["cap"], budget=p["budget"])
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()] == g["per_depth"]
    assert digest(s.reachable()) == g["sha256"]


def test_f8_dense1024_small_matches_sparse_and_oracle(gpu):
    g = golden_digests()["dense1024_seed3_small"]
    p = g["params"]
    system = snp_synth.dense_1024(3)
    s = explore_f8(gpu, system, p["depth"], cap=p["cap"], budget=p["budget"])
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()] == g["per_depth"]
    assert digest(s.reachable()) == g["sha256"]
    sp = gpu.System(system)
    sp.explore(p["depth"], cap=p["cap"], budget=p["budget"])
    assert (sp.reachable() == s.reachable()).all()


def test_f8_union_rules(gpu):
    rng = np.random.default_rng(91)
    for _ in range(20):
        system = bf.tiny_union_system(rng, m_max=4, r_max=8)
        s = explore_f8(gpu, system, 5, cap=40, budget=400)
        assert_same(s, oracle.Oracle(system).explore(5, cap=40, budget=400))


def test_f8_large_spike_counts(gpu):
    """Applicability tables that fold, a period too long for a table and a
    threshold of 400 spikes, reached from C0 = (13, 400, 401)."""
    rules = [  # (neuron, terms, c, p)
        (0, [(3, 4), (1, 6)], 1, 1), (0, [(2, 0), (9, 4)], 2, 1),
        (1, [(1, 7), (2, 9), (3, 11)], 1, 2), (1, [(1, 1)], 1, 1),
        (2, [(400, 0), (1, 2)], 1, 1), (2, [(401, 1)], 3, 1),
    ]
    terms = [t for _, t, _, _ in rules]
    system = snp_synth.make_system(3, [r[0] for r in rules], [t[0][0] for t in terms], [t[0][1] for t in terms],
                                   [r[2] for r in rules], [r[3] for r in rules], [[1, 2], [2, 0], [0, 1]],
                                   [13, 400, 401], terms=terms)
    s = explore_f8(gpu, system, 6, cap=2000)
    assert_same(s, oracle.Oracle(system).explore(6, cap=2000))


def test_f8_parent_records(gpu):
    system = snp_synth.random_system(61, 150, (1, 3), (2, 4), (0, 5), "sparse")
    s = gpu.System(system)
    s.explore(3, cap=500, budget=5000, transition=gpu.SNP_T_TC_F8, record_parents=True)
    rows = s.reachable()
    parent, index = s.parents()
    o = oracle.Oracle(system)
    for k in range(1, rows.shape[0], 7):
        assert (o.child(rows[parent[k]], int(index[k])) == rows[k]).all()


def test_f8_resume_equals_one_run(gpu):
    system = snp_synth.random_64(1)
    one = gpu.System(system)
    one.explore(5, cap=2048, budget=1 << 15, transition=gpu.SNP_T_TC_F8)
    part = gpu.System(system)
    part.explore(2, cap=2048, budget=1 << 15, transition=gpu.SNP_T_TC_F8)
    ck = part.checkpoint()
    later = gpu.System(system)
    later.resume(ck, 5, cap=2048, budget=1 << 15, transition=gpu.SNP_T_TC_F8)
    assert (later.reachable() == one.reachable()).all()


def test_f8_refuses_entries_beyond_16(gpu):
    system = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [17, 1], [[1], [0]], [3, 3])
    s = gpu.System(system)
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(2, transition=gpu.SNP_T_TC_F8)
    assert ei.value.code == gpu.SNP_E_RANGE
    s.explore(2, transition=gpu.SNP_T_TC_I8)  # within int8: the other forms take it
    ok = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [16, 1], [[1], [0]], [3, 3])
    assert_same(explore_f8(gpu, ok, 4), oracle.Oracle(ok).explore(4))
