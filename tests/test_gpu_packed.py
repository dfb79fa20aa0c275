"""Packed configurations: the store keeps each spike count in 1 or 2 bytes
where a bound on every reachable count allows it (snp_explore_opts.packed).

The result must not depend on the store's width: every packed exploration is
compared with the oracle (or with the oracle's stored digests) exactly as the
int32 path is, and the width chosen is checked against the bound (counts
start at C0 and grow by at most gain[j] per step in column j).
"""
import numpy as np
import pytest

import oracle
import snp_synth
from test_gpu_parity import assert_same, digest, explore_both, few_choice_system, golden_digests

pytestmark = pytest.mark.gpu


def column_gain(system) -> np.ndarray:
    """gain[j]: the most one step can add to column j -- per neuron the
    largest entry of column j among its rules (at most one fires), summed."""
    M = np.asarray(system.M, dtype=np.int64).reshape(system.R, system.m)
    rn = np.asarray(system.rule_neuron)
    g = np.zeros(system.m, dtype=np.int64)
    for n in range(system.m):
        rows = M[rn == n]
        if len(rows):
            g += np.maximum(rows.max(axis=0), 0)
    return g


def expected_width(system, depth: int) -> int:
    b = int((np.asarray(system.c0, dtype=np.int64) + depth * column_gain(system)).max())
    if b <= 255 and system.m % 16 == 0:
        return 1
    if b <= 65535 and system.m % 8 == 0:
        return 2
    return 4


@pytest.mark.parametrize("m", [16, 32, 48, 64, 128, 144, 256, 1024])
def test_packed_uint8_against_the_oracle(gpu, m):
    """uint8 rows through the narrow (m <= 128) and wide expand kernels."""
    system = snp_synth.random_system(500 + m, m, (1, 4), (1, min(8, m - 1)), (0, 6), "sparse")
    s, e = explore_both(gpu, system, 3, cap=300, budget=3000, packed=True)
    assert s.row_width() == expected_width(system, 3) == 1
    assert_same(s, e)


@pytest.mark.parametrize("m,lo,hi", [(24, 0, 6), (64, 200, 250), (136, 300, 900)])
def test_packed_uint16_against_the_oracle(gpu, m, lo, hi):
    """uint16 rows: m a multiple of 8 but not of 16, or counts past 255."""
    system = snp_synth.random_system(700 + m, m, (1, 4), (1, 6), (lo, hi), "sparse")
    s, e = explore_both(gpu, system, 3, cap=400, budget=4000, packed=True)
    assert s.row_width() == expected_width(system, 3) == 2
    assert_same(s, e)


def test_packed_falls_back_to_int32(gpu):
    """Rows that are no whole number of 16-byte pieces, counts that could pass
    65535, and the tensor-core forms keep int32 rows."""
    cases = [snp_synth.random_system(41, 20, (1, 3), (1, 4), (0, 6), "sparse"),
             snp_synth.random_system(42, 64, (1, 3), (1, 4), (65000, 65530), "sparse")]
    for system in cases:
        s, e = explore_both(gpu, system, 3, cap=200, budget=2000, packed=True)
        assert s.row_width() == 4
        assert_same(s, e)
    system = snp_synth.random_64(1)
    for t in (gpu.SNP_T_TC_F8, gpu.SNP_T_TC_I8):
        s, e = explore_both(gpu, system, 3, cap=500, budget=5000, packed=True, transition=t)
        assert s.row_width() == 4
        assert_same(s, e)
    s, e = explore_both(gpu, system, 3, cap=500, budget=5000)
    assert s.row_width() == 4
    assert_same(s, e)


@pytest.mark.parametrize("chunk", [0, 1000, 4097])
def test_packed_random64_small_digest(gpu, chunk):
    """The 64-neuron system at depth 4 (uint8 rows) against the oracle's
    stored digest and per-depth records, several pass sizes."""
    g = golden_digests()["random64_seed1_small"]
    p = g["params"]
    s = gpu.System(snp_synth.random_64(1))
    s.explore(p["depth"], cap=p["cap"], budget=p["budget"], chunk=chunk, packed=True)
    assert s.row_width() == 1
    assert digest(s.reachable()) == g["sha256"]
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()] == g["per_depth"]


def test_packed_dense1024_cap_2_16(gpu):
    """The 1024-neuron system with cap 2^16, budget 2^19, depth 3 (uint16
    rows: the bound reaches 1975) against the oracle's digest."""
    g = golden_digests()["dense1024_seed3_mid"]
    p = g["params"]
    system = snp_synth.dense_1024(3)
    s = gpu.System(system)
    s.explore(p["depth"], cap=p["cap"], budget=p["budget"], packed=True)
    assert s.row_width() == expected_width(system, p["depth"]) == 2
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()] == g["per_depth"]
    got = s.reachable()
    assert got.shape[0] == g["count"]
    assert digest(got) == g["sha256"]


@pytest.mark.parametrize("m,k,chunk,depth", [(160, 2, 0, 6), (1024, 4, 0, 5), (64, 3, 7, 6)])
def test_packed_crossing_batches(gpu, m, k, chunk, depth):
    """Few spiking vectors per parent: every candidate goes through a crossing
    batch (parent rows unpacked per lane, parent records from the Psi scan)."""
    system = few_choice_system(m + k, m, k)
    s, e = explore_both(gpu, system, depth, cap=3000, budget=30000, chunk=chunk, packed=True)
    assert s.row_width() == 1
    assert_same(s, e)


def test_packed_parent_records(gpu):
    system = snp_synth.random_64(2)
    s = gpu.System(system)
    s.explore(3, cap=5000, budget=80000, record_parents=True, packed=True)
    assert s.row_width() == 1
    rows = s.reachable()
    par, idx = s.parents()
    o = oracle.Oracle(system)
    for k in range(1, rows.shape[0], 97):
        assert (o.child(rows[par[k]], int(idx[k])) == rows[k]).all()
    e = o.explore(3, cap=5000, budget=80000)
    assert (rows == e.configs).all()


def test_packed_uncapped_growth_rebuilds_the_table(gpu):
    """No cap: the store and the table grow, and the table is rebuilt from
    the packed rows found so far (183734 configurations)."""
    system = snp_synth.random_system(8, 16, (2, 3), (2, 4), (0, 6), "sparse")
    s, e = explore_both(gpu, system, 4, packed=True)
    assert s.row_width() == 1
    assert s.count() == 183734
    assert_same(s, e)


@pytest.mark.parametrize("device_rows", [False, True])
def test_packed_resume(gpu, device_rows):
    """A checkpoint (int32 rows) resumed into a packed store gives the result
    of one exploration; the width then comes from the checkpoint's largest
    count and the depths still to run."""
    import torch
    system = snp_synth.random_64(1)
    one = gpu.System(system)
    one.explore(5, cap=20000, budget=300000)
    a = gpu.System(system)
    a.explore(2, cap=20000, budget=300000)
    rows, raw = a.checkpoint()
    if device_rows:
        rows = torch.from_numpy(rows).cuda()
    b = gpu.System(system)
    b.resume((rows, raw), 5, cap=20000, budget=300000, packed=True)
    assert b.row_width() == 1
    assert (b.reachable() == one.reachable()).all()
    assert [(x.new, x.examined, x.candidates) for x in b.depth_stats()] == \
        [(x.new, x.examined, x.candidates) for x in one.depth_stats()]


def test_packed_store_after_int32_and_back(gpu):
    """One handle alternating widths: the store's capacity is re-read in rows
    of each exploration's width."""
    system = snp_synth.dense_1024(3)
    s = gpu.System(system)
    e = oracle.Oracle(system).explore(3, cap=1024, budget=8192)
    for packed in (True, False, True):
        s.explore(3, cap=1024, budget=8192, packed=packed)
        assert s.row_width() == (2 if packed else 4)
        assert (s.reachable() == e.configs).all()


@pytest.mark.slow
def test_packed_random64_full_size(gpu):
    """Depth 8, cap 2^20, budget 2^24 (the benchmark's launch configuration)
    with uint8 rows: the oracle's digest and per-depth records."""
    g = golden_digests()["random64_seed1_full"]
    p = g["params"]
    s = gpu.System(snp_synth.random_64(1))
    s.explore(p["depth"], cap=p["cap"], budget=p["budget"], packed=True)
    assert s.row_width() == 1
    got = s.reachable()
    assert got.shape[0] == g["count"]
    assert [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()] == g["per_depth"]
    assert digest(got) == g["sha256"]


@pytest.mark.parametrize("chunk,packed", [(0, False), (20000, False), (9000, True)])
def test_wide_passes_over_several_large_parents(gpu, chunk, packed):
    """Rows of 160 neurons whose parents hold 8192 spiking vectors each, with a
    cap of 30000: a pass spans several parents with at least 4096 of its
    candidates, so the block bases of the wide mode come from several cached
    base children (and from a full decode where a parent has fewer)."""
    system = few_choice_system(173, 160, 13)
    s, e = explore_both(gpu, system, 3, cap=30000, chunk=chunk, packed=packed)
    assert_same(s, e)


def pairs(m):
    """m neurons in pairs passing one spike to each other: C0's only child is C0."""
    return snp_synth.make_system(m, list(range(m)), [1] * m, [1] * m, [1] * m, [1] * m,
                                 [[n ^ 1] for n in range(m)], [1] * m, name="pairs")


@pytest.mark.parametrize("m", [32, 144])
def test_packed_wait_runs_out(gpu, m):
    """A held hash slot makes the wait run out with a packed store too (narrow
    and wide kernels); the handle explores normally afterwards."""
    s = gpu.System(pairs(m))
    gpu.snp_debug_hold_root_slot(True)
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(2, timeout_ms=50, packed=True)
    assert ei.value.code == gpu.SNP_E_TIMEOUT
    s.explore(2, packed=True)
    assert s.row_width() == 1 and s.count() == 1


def test_packed_max_expand(gpu):
    """Rows holding more than max_expand spikes somewhere are kept but not
    expanded, read from uint8 rows."""
    s, e = explore_both(gpu, snp_synth.random_64(1), 4, cap=4000, budget=40000, max_expand=3, packed=True)
    assert s.row_width() == 1
    assert_same(s, e)


def test_packed_wide_parent_records(gpu):
    """Parent records with uint8 rows in the wide mode (256 neurons)."""
    system = snp_synth.random_system(88, 256, (1, 3), (2, 4), (0, 5), "sparse")
    s = gpu.System(system)
    s.explore(3, cap=800, budget=8000, record_parents=True, packed=True)
    assert s.row_width() == expected_width(system, 3) == 1
    rows = s.reachable()
    par, idx = s.parents()
    o = oracle.Oracle(system)
    for k in range(1, rows.shape[0], 13):
        assert (o.child(rows[par[k]], int(idx[k])) == rows[k]).all()
    assert (rows == o.explore(3, cap=800, budget=8000).configs).all()


@pytest.mark.parametrize("m,packed_width", [(64, 1), (1024, 2)])
def test_packed_rows_into_device_memory(gpu, m, packed_width):
    """snp_reachable widens packed rows straight into a device buffer, after an
    exploration on a side stream."""
    import torch
    system = snp_synth.random_64(1) if m == 64 else snp_synth.dense_1024(3)
    kw = dict(cap=1 << 12, budget=1 << 16) if m == 64 else dict(cap=1024, budget=8192)
    s = gpu.System(system)
    stream = torch.cuda.Stream()
    s.explore(3, stream=stream, packed=True, **kw)
    assert s.row_width() == packed_width
    n = s.count()
    out = torch.empty((n, system.m), dtype=torch.int32, device="cuda")
    gpu.snp_reachable(s.h, out, n)
    e = oracle.Oracle(system).explore(3, **kw)
    assert (out.cpu().numpy() == e.configs).all()


def test_packed_passes_of_one_candidate(gpu):
    """uint8 rows with passes of a single candidate (every pass a ragged tail)."""
    system = snp_synth.random_system(901, 16, (1, 3), (1, 4), (0, 4), "sparse")
    s, e = explore_both(gpu, system, 3, cap=50, budget=400, chunk=1, packed=True)
    assert s.row_width() == 1
    assert_same(s, e)


def test_packed_uint16_crossing_batches(gpu):
    """uint16 rows (24 neurons) in the narrow kernel's crossing batches."""
    system = few_choice_system(27, 24, 3)
    s, e = explore_both(gpu, system, 6, cap=2000, budget=20000, packed=True)
    assert s.row_width() == 2
    assert_same(s, e)
