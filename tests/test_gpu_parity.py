"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work: everything must match bit for bit -- the discovery-ordered
configurations, the per-depth counts of new configurations and examined
candidates, the sums of Psi and the truncation flags.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import bruteforce as bf
import oracle
import snp_synth
from conftest import GOLDEN, read_golden

pytestmark = pytest.mark.gpu


def digest(configs: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(configs, dtype="<i4").tobytes()).hexdigest()


def golden_digests():
    with open(os.path.join(GOLDEN, "oracle_digests.json")) as f:
        return json.load(f)


def explore_both(gpu, system, depth, cap=0, budget=0, max_expand=-1, chunk=0, **kw):
    s = gpu.System(system)
    s.explore(depth, cap=cap, budget=budget, max_expand=max_expand, chunk=chunk, **kw)
    e = oracle.Oracle(system).explore(depth, cap=cap, budget=budget, max_expand=max_expand)
    return s, e


def assert_same(s, e):
    got = s.reachable()
    assert got.shape == e.configs.shape
    assert (got == e.configs).all()
    stats = s.depth_stats()
    assert len(stats) == len(e.depths)
    for d, (a, b) in enumerate(zip(stats, e.depths)):
        assert a.new == b.new, d
        if d > 0:
            assert a.examined == b.examined, d
            assert a.candidates == b.candidates, d
            assert a.truncated == b.truncated, d
    assert s.depth_reached == e.depth_reached
    assert s.per_depth_new() == [d.new for d in e.depths[: e.depth_reached + 1]]


# --- the paper's example ---

def test_paper_example_depth10(gpu):
    s, e = explore_both(gpu, snp_synth.paper_example(), 10)
    assert_same(s, e)
    assert s.per_depth_new() == [1, 2, 4, 6, 6, 6, 5, 5, 5, 5, 5]


def test_paper_replay_reproduces_allgenck(gpu):
    g = read_golden("paper_run.txt")
    s, e = explore_both(gpu, snp_synth.paper_example(), 1000, max_expand=9)
    assert_same(s, e)
    assert ["-".join(str(int(x)) for x in r) for r in s.reachable()] == g["allGenCk"].split()


def test_paper_exact_reading(gpu):
    s, e = explore_both(gpu, snp_synth.paper_example(exact=True), 100)
    assert_same(s, e)
    assert s.count() == 8


def test_step_matches_oracle_and_paper(gpu):
    paper = snp_synth.paper_example()
    s = gpu.System(paper)
    kids, psi = s.step([2, 1, 1])
    assert psi == 2
    assert ["-".join(str(int(x)) for x in r) for r in kids] == read_golden("paper_run.txt")["after_C0"].split()[1:]
    rng = np.random.default_rng(3)
    o = oracle.Oracle(paper)
    for _ in range(50):
        C = rng.integers(0, 12, size=3).astype(np.int32)
        kids, psi = s.step(C)
        assert psi == o.psi(C)
        assert (kids == o.step(C)).all()


def test_step_with_device_buffers(gpu):
    import torch
    system = snp_synth.random_64(1)
    s = gpu.System(system)
    o = oracle.Oracle(system)
    C = torch.tensor(system.c0, dtype=torch.int32, device="cuda")
    out = torch.zeros((5000, system.m), dtype=torch.int32, device="cuda")
    psi = gpu.snp_step(s.h, C, 5000, out)
    assert psi == o.psi(system.c0) == 147456
    assert (out.cpu().numpy() == o.step(system.c0, cap=5000)).all()


# --- small random systems, every truncation mode, several chunk sizes ---

@pytest.mark.parametrize("cap,budget,chunk", [(0, 0, 0), (1, 0, 0), (3, 0, 1), (0, 7, 0), (5, 11, 3), (2, 1, 0),
                                              (4, 0, 2)])
def test_tiny_systems(gpu, cap, budget, chunk):
    rng = np.random.default_rng(1000 + 7 * cap + 13 * budget + chunk)
    for _ in range(30):
        system = bf.tiny_system(rng, m_max=4, r_max=9)
        s, e = explore_both(gpu, system, 5, cap=cap, budget=budget, chunk=chunk)
        assert_same(s, e)


@pytest.mark.parametrize("m", [1, 2, 31, 32, 33, 63, 64, 65, 100, 255, 256, 257, 511, 1024])
def test_neuron_counts(gpu, m):
    system = snp_synth.random_system(500 + m, m, (1, 4), (1, min(8, max(1, m - 1))), (0, 6), "sparse")
    s, e = explore_both(gpu, system, 3, cap=300, budget=3000)
    assert_same(s, e)


# --- rows of more than 128 neurons: built on demand by the whole warp ---

@pytest.mark.parametrize("m,rules,chunk", [(129, (1, 2), 0), (130, (1, 3), 5), (150, (1, 4), 0),
                                           (200, (2, 3), 1000), (257, (1, 2), 37), (1023, (1, 2), 0)])
def test_wide_rows(gpu, m, rules, chunk):
    """Block mode and crossing batches, rows with and without a multiple of
    four neurons, one to four rules per neuron, several pass sizes."""
    system = snp_synth.random_system(900 + m, m, rules, (1, 4), (0, 4), "sparse")
    s, e = explore_both(gpu, system, 4, cap=2000, budget=20000, chunk=chunk)
    assert_same(s, e)


def few_choice_system(seed, m, k):
    """Neurons 0 .. k-1 with two rules each (one or two spikes sent for one
    consumed), the others with one rule (fire while holding a spike): at most
    2^k spiking vectors per parent, so with k < 5 every candidate goes through
    a crossing batch."""
    rng = np.random.default_rng(seed)
    rn, ri, rj, rc, rp = [], [], [], [], []
    for n in range(m):
        for p in ((1, 2) if n < k else (1,)):
            rn.append(n)
            ri.append(1)
            rj.append(1)
            rc.append(1)
            rp.append(p)
    targets = [sorted(rng.choice([t for t in range(m) if t != n], size=2, replace=False).tolist()) for n in range(m)]
    c0 = [5] * k + rng.integers(0, 2, size=m - k).tolist()
    return snp_synth.make_system(m, rn, ri, rj, rc, rp, targets, c0, name="few-choice")


@pytest.mark.parametrize("m,k,chunk,depth", [(160, 2, 0, 6), (301, 3, 17, 6), (1024, 4, 0, 5)])
def test_wide_rows_in_crossing_batches(gpu, m, k, chunk, depth):
    s, e = explore_both(gpu, few_choice_system(m + k, m, k), depth, cap=3000, budget=30000, chunk=chunk)
    assert_same(s, e)


def broadcast_system(m, k, seed):
    """Neurons 0 .. k-1 with two rules each and a synapse to every other
    neuron, the others with one rule and two synapses: the supports of the
    multi-choice neurons are too large for the low neurons' swap table, so
    rows are built with swaps read from global memory."""
    rng = np.random.default_rng(seed)
    rn, ri, rj, rc, rp = [], [], [], [], []
    for n in range(m):
        for p in ((1, 2) if n < k else (1,)):
            rn.append(n)
            ri.append(1)
            rj.append(1)
            rc.append(1)
            rp.append(p)
    targets = [[t for t in range(m) if t != n] if n < k else
               sorted(rng.choice([t for t in range(m) if t != n], size=2, replace=False).tolist()) for n in range(m)]
    c0 = [3] * k + rng.integers(0, 2, size=m - k).tolist()
    return snp_synth.make_system(m, rn, ri, rj, rc, rp, targets, c0, name="broadcast")


@pytest.mark.parametrize("m,k,chunk", [(800, 6, 0), (801, 7, 50)])
def test_wide_rows_with_large_supports(gpu, m, k, chunk):
    s, e = explore_both(gpu, broadcast_system(m, k, m), 3, cap=800, budget=6000, chunk=chunk)
    assert_same(s, e)


def many_duplicates_system(m, k):
    """k neurons with two rules each, both consuming one spike, one sending a
    spike to the last neuron and one forgetting: a parent's 2^k spiking vectors
    give only k + 1 children, so most candidates meet a row that another lane
    of the same warp has just claimed."""
    rn, ri, rj, rc, rp = [], [], [], [], []
    for n in range(k):
        for p in (1, 0):
            rn.append(n)
            ri.append(1)
            rj.append(1)
            rc.append(1)
            rp.append(p)
    targets = [[m - 1] for _ in range(k)] + [[] for _ in range(m - k)]
    return snp_synth.make_system(m, rn, ri, rj, rc, rp, targets, [3] * k + [0] * (m - k), name="duplicates")


@pytest.mark.parametrize("m,k,chunk", [(64, 6, 0), (200, 6, 0), (200, 7, 9), (1024, 5, 0), (1022, 8, 100)])
def test_duplicates_within_a_warp(gpu, m, k, chunk):
    s, e = explore_both(gpu, many_duplicates_system(m, k), 4, chunk=chunk)
    assert_same(s, e)


def saturating_system(kind):
    """'steady': 100 neurons with two rules each (a+ / a -> a or a^2) that stay
    applicable, so every configuration has 2^100 spiking vectors.  'drain': 70
    neurons with one spike and two rules (a -> lambda, a -> a into a private
    sink): the root has 2^70 spiking vectors, its children have one each."""
    rn, ri, rj, rc, rp = [], [], [], [], []
    if kind == "steady":
        m = 100
        for n in range(m):
            for p in (1, 2):
                rn += [n]
                ri += [1]
                rj += [1]
                rc += [1]
                rp += [p]
        targets = [[(n + 1) % m, (n + 7) % m] for n in range(m)]
        return snp_synth.make_system(m, rn, ri, rj, rc, rp, targets, [6] * m, name="steady")
    k = 70
    for n in range(k):
        for p in (0, 1):
            rn += [n]
            ri += [1]
            rj += [0]
            rc += [1]
            rp += [p]
    targets = [[k + n] for n in range(k)] + [[] for _ in range(k)]
    return snp_synth.make_system(2 * k, rn, ri, rj, rc, rp, targets, [1] * k + [0] * k, name="drain")


@pytest.mark.parametrize("kind", ["steady", "drain"])
def test_saturated_psi_sums(gpu, kind):
    """Frontiers of 20000 rows after a depth whose Psi sum saturated: the
    first 8192 rows go first, and the rest are read only when those do not
    already give 2^64 - 1 candidates ('steady': they do; 'drain': they
    do not)."""
    s, e = explore_both(gpu, saturating_system(kind), 3, cap=20000, budget=1 << 16)
    assert_same(s, e)
    assert e.depths[1].candidates == 2**64 - 1
    assert (e.depths[2].candidates == 2**64 - 1) == (kind == "steady")


def test_batch_style_systems(gpu):
    for system in snp_synth.batch_systems(6):
        s, e = explore_both(gpu, system, 4, cap=1 << 9, budget=1 << 13)
        assert_same(s, e)


# --- the 64-neuron workload ---

@pytest.mark.parametrize("chunk", [0, 1000, 4097, 65536])
def test_random64_small_all_chunkings(gpu, chunk):
    g = golden_digests()["random64_seed1_small"]
    system = snp_synth.random_64(1)
    s = gpu.System(system)
    p = g["params"]
    s.explore(p["depth"], cap=p["cap"], budget=p["budget"], chunk=chunk)
    got = s.reachable()
    assert digest(got) == g["sha256"]
    st = s.depth_stats()
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in st] == g["per_depth"]


def test_random64_small_against_oracle_directly(gpu):
    s, e = explore_both(gpu, snp_synth.random_64(1), 3, cap=1 << 12, budget=1 << 16)
    assert_same(s, e)


@pytest.mark.slow
def test_random64_full_size(gpu):
    """Depth 8, cap 2^20, budget 2^24 (the benchmark's launch configuration)."""
    g = golden_digests()["random64_seed1_full"]
    system = snp_synth.random_64(1)
    s = gpu.System(system)
    p = g["params"]
    s.explore(p["depth"], cap=p["cap"], budget=p["budget"], record_parents=True)
    got = s.reachable()
    assert got.shape[0] == g["count"]
    st = s.depth_stats()
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in st] == g["per_depth"]
    assert digest(got) == g["sha256"]
    # sampled: each configuration is its recorded parent's child at the recorded index
    par, idx = s.parents()
    o = oracle.Oracle(system)
    rng = np.random.default_rng(0)
    for k in rng.choice(got.shape[0] - 1, size=200, replace=False) + 1:
        ch = o.child(got[par[k]], int(idx[k]))
        assert ch is not None and (ch == got[k]).all()


def test_dense1024_small(gpu):
    g = golden_digests()["dense1024_seed3_small"]
    system = snp_synth.dense_1024(3)
    s = gpu.System(system)
    p = g["params"]
    s.explore(p["depth"], cap=p["cap"], budget=p["budget"])
    st = s.depth_stats()
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in st] == g["per_depth"]
    assert digest(s.reachable()) == g["sha256"]


# --- parent records, streams, device outputs ---

def test_parent_records(gpu):
    system = snp_synth.random_64(2)
    s = gpu.System(system)
    s.explore(3, cap=5000, budget=80000, record_parents=True)
    rows = s.reachable()
    par, idx = s.parents()
    assert par[0] == -1 and idx[0] == 0
    o = oracle.Oracle(system)
    for k in range(1, rows.shape[0], 97):
        assert (o.child(rows[par[k]], int(idx[k])) == rows[k]).all()
    # the parent of a depth-d configuration lies in depth d - 1
    per = s.per_depth_new()
    start = np.cumsum([0] + per)
    for d in range(1, len(per)):
        sl = slice(start[d], start[d + 1])
        assert (par[sl] >= start[d - 1]).all() and (par[sl] < start[d]).all()


def test_explore_on_a_side_stream_into_device_memory(gpu):
    import torch
    system = snp_synth.random_64(1)
    s = gpu.System(system)
    stream = torch.cuda.Stream()
    s.explore(3, cap=1 << 12, budget=1 << 16, stream=stream)
    n = s.count()
    out = torch.empty((n, system.m), dtype=torch.int32, device="cuda")
    gpu.snp_reachable(s.h, out, n)
    e = oracle.Oracle(system).explore(3, cap=1 << 12, budget=1 << 16)
    assert (out.cpu().numpy() == e.configs).all()


def test_repeated_explores_reuse_the_handle(gpu):
    system = snp_synth.random_64(1)
    s = gpu.System(system)
    e = oracle.Oracle(system).explore(2, cap=1 << 10, budget=1 << 14)
    for cap in (1 << 10, 1 << 12, 1 << 10):
        s.explore(2, cap=cap, budget=1 << 14)
    assert (s.reachable() == e.configs).all()


# --- edge cases and errors ---

def test_depth_zero_and_quiet_system(gpu):
    system = snp_synth.random_64(1)
    s = gpu.System(system)
    s.explore(0)
    assert s.count() == 1 and (s.reachable()[0] == system.c0).all()
    quiet = snp_synth.make_system(3, [0, 1], [5, 5], [0, 0], [1, 1], [1, 1], [[1], [2], []], [0, 0, 0])
    s, e = explore_both(gpu, quiet, 5)
    assert_same(s, e)
    assert s.count() == 1 and s.depth_reached == 0


def test_cap_one_and_budget_one(gpu):
    system = snp_synth.random_64(3)
    for cap, budget in [(1, 0), (0, 1), (1, 1)]:
        s, e = explore_both(gpu, system, 4, cap=cap, budget=budget)
        assert_same(s, e)


def test_overflow_is_reported(gpu):
    big = 2 ** 31 - 3
    system = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [5, 5], [[1], [0]], [big, big])
    s = gpu.System(system)
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(3)
    assert ei.value.code == gpu.SNP_E_OVERFLOW
    with pytest.raises(gpu.SnpError) as ei:
        s.step(system.c0)
    assert ei.value.code == gpu.SNP_E_OVERFLOW
    # Counts grow by 4 a step (gain 5): the frontier of depth 3 holds 2^31 - 5,
    # whose children could pass 2^31 - 1; depth 2 is still fine.
    m = 2 ** 31 - 1
    system = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [5, 5], [[1], [0]], [m - 12, 1])
    s = gpu.System(system)
    s.explore(2)
    assert s.reachable().tolist() == [[m - 12, 1], [m - 8, 5], [m - 4, 9]]
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(3)
    assert ei.value.code == gpu.SNP_E_OVERFLOW
    s.explore(2, cap=1)
    assert s.count() == 3


@pytest.mark.parametrize("m,cap", [(64, 2000), (128, 3000), (256, 1500)])
def test_psi_rows_with_large_counts(gpu, m, cap):
    """Frontier rows that hold spike counts of 64 or more in some neurons (the
    direct applicability table stops at 63): such rows leave the fast Psi loop
    for the general one; with small caps the parent records are built too."""
    system = snp_synth.random_system(4400 + m, m, (2, 3), (2, 4), (0, 6), "sparse")
    rng = np.random.default_rng(m)
    system.c0[:] = np.where(rng.random(m) < 0.2, rng.integers(60, 300, size=m), rng.integers(0, 7, size=m))
    s, e = explore_both(gpu, system, 3, cap=cap, budget=20 * cap)
    assert_same(s, e)


def test_overflow_bound_against_the_oracle(gpu):
    """The device refuses to expand a configuration from which some column
    could leave int32 in one step (the per-column bound: the sum over neurons
    of their largest entry in that column, whatever fires); the oracle, in
    int64, flags only a child that does leave it.  They agree on an actual
    overflow and differ, by design, where the bound fires and no child
    overflows (the oracle pins use the same two systems)."""
    big = 2 ** 31 - 3
    actual = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [5, 0], [[1], [0]], [1, big])
    assert oracle.Oracle(actual).explore(3).error == 1
    s = gpu.System(actual)
    for t in (gpu.SNP_T_SPARSE_I32, gpu.SNP_T_TC_I8, gpu.SNP_T_TC_F8):
        with pytest.raises(gpu.SnpError) as ei:
            s.explore(3, transition=t)
        assert ei.value.code == gpu.SNP_E_OVERFLOW
    bound_only = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [5, 0], [[1], [0]], [0, big])
    e = oracle.Oracle(bound_only).explore(3)
    assert e.error == 0 and e.configs.shape[0] == 4
    s = gpu.System(bound_only)
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(3)
    assert ei.value.code == gpu.SNP_E_OVERFLOW


def test_state_and_buffer_errors(gpu):
    s = gpu.System(snp_synth.paper_example())
    with pytest.raises(gpu.SnpError) as ei:
        gpu.snp_reachable(s.h, None, 0)
    assert ei.value.code == gpu.SNP_E_STATE
    s.explore(3)
    out = np.zeros((2, 3), dtype=np.int32)
    with pytest.raises(gpu.SnpError) as ei:
        gpu.snp_reachable(s.h, out, 2)
    assert ei.value.code == gpu.SNP_E_BUFFER
    with pytest.raises(gpu.SnpError) as ei:
        gpu.snp_parents(s.h, None, None, 100)
    assert ei.value.code == gpu.SNP_E_STATE


# --- the exact int8 tensor-core transition (SNP_T_TC_I8) ---

def explore_tc(gpu, system, depth, **kw):
    s = gpu.System(system)
    s.explore(depth, transition=gpu.SNP_T_TC_I8, **kw)
    return s


def test_tc_paper_example_and_replay(gpu):
    g = read_golden("paper_run.txt")
    paper = snp_synth.paper_example()
    s = explore_tc(gpu, paper, 10)
    assert_same(s, oracle.Oracle(paper).explore(10))
    s = explore_tc(gpu, paper, 1000, max_expand=9)
    assert ["-".join(str(int(x)) for x in r) for r in s.reachable()] == g["allGenCk"].split()


@pytest.mark.parametrize("cap,budget,chunk", [(0, 0, 0), (3, 0, 1), (5, 11, 3), (2, 1, 0)])
def test_tc_tiny_systems(gpu, cap, budget, chunk):
    rng = np.random.default_rng(2000 + 7 * cap + 13 * budget + chunk)
    for _ in range(25):
        system = bf.tiny_system(rng, m_max=4, r_max=9)
        s = explore_tc(gpu, system, 5, cap=cap, budget=budget, chunk=chunk)
        assert_same(s, oracle.Oracle(system).explore(5, cap=cap, budget=budget))


@pytest.mark.parametrize("m", [1, 5, 31, 64, 100, 129, 257, 1024])
def test_tc_neuron_counts(gpu, m):
    system = snp_synth.random_system(700 + m, m, (1, 4), (1, min(8, max(1, m - 1))), (0, 6), "sparse")
    s = explore_tc(gpu, system, 3, cap=300, budget=3000)
    assert_same(s, oracle.Oracle(system).explore(3, cap=300, budget=3000))


def test_tc_random64_small(gpu):
    g = golden_digests()["random64_seed1_small"]
    p = g["params"]
    s = explore_tc(gpu, snp_synth.random_64(1), p["depth"], cap=p["cap"], budget=p["budget"])
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()] == g["per_depth"]
    assert digest(s.reachable()) == g["sha256"]


def test_tc_dense1024_matches_sparse_and_oracle(gpu):
    g = golden_digests()["dense1024_seed3_small"]
    p = g["params"]
    system = snp_synth.dense_1024(3)
    s = explore_tc(gpu, system, p["depth"], cap=p["cap"], budget=p["budget"])
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()] == g["per_depth"]
    assert digest(s.reachable()) == g["sha256"]
    sp = gpu.System(system)
    sp.explore(p["depth"], cap=p["cap"], budget=p["budget"])
    assert (sp.reachable() == s.reachable()).all()


def test_tc_refuses_entries_beyond_int8(gpu):
    system = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [200, 1], [[1], [0]], [3, 3])
    s = gpu.System(system)
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(2, transition=gpu.SNP_T_TC_I8)
    assert ei.value.code == gpu.SNP_E_RANGE
    s.explore(2)  # the sparse path takes it


def test_tc_peak_probe(gpu):
    tops = gpu.snp_tc_peak_tops(2000)
    assert tops > 1.0


def test_rules_with_identical_rows(gpu):
    """Neurons whose rules share a row of M_Pi but differ in their regexes: the
    candidates that choose a later rule repeat earlier ones, and the result must
    not depend on how the simulator exploits that."""
    rng = np.random.default_rng(77)
    for _ in range(20):
        m = int(rng.integers(2, 7))
        rn, ri, rj, rc, rp = [], [], [], [], []
        for n in range(m):
            k = int(rng.integers(1, 5))
            c, p = int(rng.integers(1, 3)), int(rng.integers(0, 3))
            for _ in range(k):
                rn.append(n)
                ri.append(int(rng.integers(1, 4)))
                rj.append(int(rng.integers(0, 3)))
                same = rng.random() < 0.7
                rc.append(c if same else int(rng.integers(1, 3)))
                rp.append(p if same else int(rng.integers(0, 3)))
        targets = [sorted(rng.choice([t for t in range(m) if t != n], size=min(2, m - 1), replace=False).tolist())
                   for n in range(m)]
        system = snp_synth.make_system(m, rn, ri, rj, rc, rp, targets, rng.integers(0, 6, size=m))
        for transition in (gpu.SNP_T_SPARSE_I32, gpu.SNP_T_TC_I8):
            s = gpu.System(system)
            s.explore(6, cap=40, budget=400, transition=transition)
            assert_same(s, oracle.Oracle(system).explore(6, cap=40, budget=400))


def large_count_system():
    """Neurons whose rule sets give every kind of applicability lookup: period
    L = 6 (folded by multiply and shift), L = 8, L = lcm(5, 7, 3) = 105 and a
    threshold of 300 (both evaluated from the rules), a threshold of 200 with
    L = 3, and two rules with identical rows."""
    rules = [  # (neuron, i, j, c, p)
        (0, 1, 2, 1, 1), (0, 2, 3, 2, 1),
        (1, 3, 4, 1, 2), (1, 1, 0, 1, 1), (1, 5, 8, 3, 1),
        (2, 2, 5, 1, 1), (2, 3, 7, 2, 2), (2, 1, 3, 1, 1),
        (3, 200, 1, 200, 1), (3, 1, 3, 1, 1),
        (4, 300, 2, 1, 1),
        (5, 1, 1, 1, 1), (5, 1, 1, 1, 1),
    ]
    rn, ri, rj, rc, rp = (list(x) for x in zip(*rules))
    targets = [[1, 2], [2, 3], [3, 4], [4, 5], [5, 0], [0, 1]]
    return snp_synth.make_system(6, rn, ri, rj, rc, rp, targets, [0] * 6, name="large-count")


def test_applicability_at_large_spike_counts(gpu):
    system = large_count_system()
    s = gpu.System(system)
    o = oracle.Oracle(system)
    rng = np.random.default_rng(11)
    for k in range(300):
        band = rng.integers(0, 3, size=6)
        C = np.where(band == 0, rng.integers(0, 20, size=6),
                     np.where(band == 1, rng.integers(180, 330, size=6), rng.integers(10**6, 10**7, size=6)))
        C = C.astype(np.int32)
        kids, psi = s.step(C)
        assert psi == o.psi(C), C
        assert (kids == o.step(C)).all(), C


def test_explore_from_large_spike_counts(gpu):
    system = large_count_system()
    rng = np.random.default_rng(12)
    for k in range(4):
        system.c0[:] = rng.integers(10**5, 10**6, size=6).astype(np.int32)
        if k == 1:
            system.c0[3] = 250
            system.c0[4] = 301
        s = gpu.System(system)
        s.explore(4, cap=3000, budget=40000)
        e = oracle.Oracle(system).explore(4, cap=3000, budget=40000)
        assert (s.reachable() == e.configs).all()
        assert [x.examined for x in s.depth_stats()] == [x.examined for x in e.depths]


@pytest.mark.parametrize("chunk", [0, 4096])
def test_uncapped_growth_rebuilds_the_table(gpu, chunk):
    """No cap and no budget: the store, the row map and the hash table all
    grow during the run (the table is rebuilt from the rows found so far,
    through the row map); small passes keep two in flight most of the time."""
    system = snp_synth.random_system(8, 12, (2, 3), (2, 4), (0, 6), "sparse")
    s = gpu.System(system)
    s.explore(3, chunk=chunk, record_parents=True)
    e = oracle.Oracle(system).explore(3)
    got = s.reachable()
    assert got.shape[0] == 159140  # well past the first table (sized for 4096 + 65536 rows)
    assert (got == e.configs).all()
    assert [(x.new, x.examined) for x in s.depth_stats()] == [(x.new, x.examined) for x in e.depths]
    parent, index = s.parents()
    o = oracle.Oracle(system)
    for k in range(1, got.shape[0], 4999):  # each row is the index-th child of its parent
        assert (o.child(got[parent[k]], int(index[k])) == got[k]).all()


# --- general rules: unions of terms a^i (a^j)* ---

@pytest.mark.parametrize("cap,budget", [(0, 0), (3, 0), (0, 40)])
def test_union_rule_systems(gpu, cap, budget):
    rng = np.random.default_rng(5000 + 7 * cap + budget)
    for _ in range(25):
        system = bf.tiny_union_system(rng, m_max=4, r_max=8)
        s, e = explore_both(gpu, system, 5, cap=cap, budget=budget)
        assert_same(s, e)
        o = oracle.Oracle(system)
        for _ in range(3):
            C = rng.integers(0, 14, size=system.m).astype(np.int32)
            kids, psi = s.step(C)
            assert psi == o.psi(C)
            assert (kids == o.step(C)).all()


def test_union_rules_at_large_spike_counts(gpu):
    """Union rules whose tables fold (period lcm(4, 6) = 12), whose period is
    too long for a table (lcm(7, 9, 11) = 693) or whose threshold is (a^400)."""
    rules = [  # (neuron, terms, c, p)
        (0, [(3, 4), (1, 6)], 1, 1), (0, [(2, 0), (9, 4)], 2, 1),
        (1, [(1, 7), (2, 9), (3, 11)], 1, 2), (1, [(1, 1)], 1, 1),
        (2, [(400, 0), (1, 2)], 1, 1), (2, [(401, 1)], 3, 1),
    ]
    terms = [t for _, t, _, _ in rules]
    system = snp_synth.make_system(3, [r[0] for r in rules], [t[0][0] for t in terms], [t[0][1] for t in terms],
                                   [r[2] for r in rules], [r[3] for r in rules], [[1, 2], [2, 0], [0, 1]],
                                   [0, 0, 0], terms=terms)
    s = gpu.System(system)
    o = oracle.Oracle(system)
    rng = np.random.default_rng(17)
    for _ in range(300):
        band = rng.integers(0, 3, size=3)
        C = np.where(band == 0, rng.integers(0, 30, size=3),
                     np.where(band == 1, rng.integers(380, 420, size=3), rng.integers(10**5, 10**7, size=3)))
        C = C.astype(np.int32)
        kids, psi = s.step(C)
        assert psi == o.psi(C), C
        assert (kids == o.step(C)).all(), C
    system.c0[:] = [13, 400, 401]
    s, e = explore_both(gpu, system, 6, cap=2000)
    assert_same(s, e)


def test_union_rules_in_the_batch_engine(gpu):
    rng = np.random.default_rng(77)
    systems = [bf.tiny_union_system(rng, m_max=4, r_max=8) for _ in range(30)]
    handles = [gpu.System(x) for x in systems]
    st = gpu.explore_batch(handles, 5, cap=64, budget=512)
    assert (st == 0).all()
    for h, x in zip(handles, systems):
        e = oracle.Oracle(x).explore(5, cap=64, budget=512)
        assert (h.reachable() == e.configs).all()
        assert [(a.new, a.examined) for a in h.depth_stats()] == [(b.new, b.examined) for b in e.depths]


# --- checkpoint and resume at depth boundaries ---

def same_run(a, b):
    assert (a.reachable() == b.reachable()).all()
    key = lambda x: (x.new, x.examined, x.candidates, x.truncated, x.parents)
    assert [key(x) for x in a.depth_stats()] == [key(x) for x in b.depth_stats()]
    assert a.depth_reached == b.depth_reached


@pytest.mark.parametrize("at", [0, 1, 4])
def test_resume_equals_one_run(gpu, tmp_path, at):
    system = snp_synth.random_64(1)
    opts = dict(cap=4096, budget=1 << 16)
    first = gpu.System(system)
    first.explore(at, **opts)
    rows, stats = first.checkpoint()
    np.save(tmp_path / "rows.npy", rows)
    np.save(tmp_path / "stats.npy", stats)
    later = gpu.System(system)
    later.resume((np.load(tmp_path / "rows.npy"), np.load(tmp_path / "stats.npy")), 8, **opts)
    fresh = gpu.System(system)
    fresh.explore(8, **opts)
    same_run(later, fresh)
    e = oracle.Oracle(system).explore(8, **opts)
    assert (later.reachable() == e.configs).all()


def test_resume_from_device_rows_and_other_transition(gpu):
    import torch
    system = snp_synth.random_64(1)
    first = gpu.System(system)
    first.explore(2, cap=2048, budget=1 << 15)
    rows, stats = first.checkpoint()
    later = gpu.System(system)
    later.resume((torch.from_numpy(rows).cuda(), stats), 5, cap=2048, budget=1 << 15, transition=gpu.SNP_T_TC_I8)
    fresh = gpu.System(system)
    fresh.explore(5, cap=2048, budget=1 << 15)
    assert (later.reachable() == fresh.reachable()).all()


def test_resume_after_the_search_ended(gpu):
    paper = snp_synth.paper_example()
    first = gpu.System(paper)
    first.explore(60, max_expand=9)  # the replay ends by repetition before depth 60
    ckpt = first.checkpoint()
    later = gpu.System(paper)
    later.resume(ckpt, 80, max_expand=9)
    fresh = gpu.System(paper)
    fresh.explore(80, max_expand=9)
    same_run(later, fresh)
    assert later.count() == 48


def test_resume_rejects_inconsistent_checkpoints(gpu):
    system = snp_synth.random_64(1)
    first = gpu.System(system)
    first.explore(2, cap=100, budget=1000)
    rows, stats = first.checkpoint()
    later = gpu.System(system)
    with pytest.raises(gpu.SnpError) as ei:
        later.resume((rows[:-1], stats), 4, cap=100, budget=1000)
    assert ei.value.code == gpu.SNP_E_INVALID
    with pytest.raises(gpu.SnpError) as ei:
        later.resume((rows, stats), 1, cap=100, budget=1000)  # the checkpoint is already at depth 2
    assert ei.value.code == gpu.SNP_E_INVALID
    later.resume((rows, stats), 4, cap=100, budget=1000)  # the handle is still usable
    fresh = gpu.System(system)
    fresh.explore(4, cap=100, budget=1000)
    same_run(later, fresh)


# --- failure detection on the host (no GPU fault involved) ---

def test_allocation_failures_leave_handles_usable(gpu):
    """Each device allocation of a load and an exploration is refused in turn
    (the library's fault-injection hook): the call reports SNP_E_NOMEM, and the
    same handle then explores correctly once allocations succeed again."""
    system = snp_synth.random_64(1)
    want = oracle.Oracle(system).explore(3, cap=2000, budget=20000)
    refused = 0
    try:
        for k in range(1, 200):
            gpu.snp_debug_fail_allocation(k)
            try:
                s = gpu.System(system)
            except gpu.SnpError as e:
                assert e.code == gpu.SNP_E_NOMEM
                refused += 1
                continue
            try:
                s.explore(3, cap=2000, budget=20000)
            except gpu.SnpError as e:
                assert e.code == gpu.SNP_E_NOMEM
                refused += 1
                gpu.snp_debug_fail_allocation(0)
                s.explore(3, cap=2000, budget=20000)
                assert (s.reachable() == want.configs).all()
                continue
            gpu.snp_debug_fail_allocation(0)
            assert (s.reachable() == want.configs).all()  # k is past the last allocation
            break
        else:
            raise AssertionError("the hook never ran out of allocations to refuse")
    finally:
        gpu.snp_debug_fail_allocation(0)
    assert refused > 10
