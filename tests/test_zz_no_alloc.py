"""snp_explore_static against snp_explore and the oracle.

snp_explore_static is for callers that may not allocate device memory when
they need an exploration (a caching allocator holds the free memory, or a
loop must not block on the allocator).  It keeps its scratch in one fixed
array inside the library and writes into the caller's buffer.  These tests
check that, called twice in a row, it gives exactly the configurations and
per-depth counts that snp_explore gives (integer results: bit for bit), also
with rows of more than 128 neurons and near its 2^20-configuration limit
where its hash table is rebuilt mid-depth, that it agrees with the oracle, and
that it refuses sizes beyond its fixed limit and buffers it cannot use.

The file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import snp_synth

pytestmark = pytest.mark.gpu


def _opts(snp, depth, cap=0, budget=0, max_expand=-1, stream=None):
    o = snp.snp_explore_opts_init()
    o.depth = depth
    o.frontier_cap = cap
    o.candidate_budget = budget
    o.max_expand_value = max_expand
    if stream is not None:
        o.stream = stream.cuda_stream
    return o


@pytest.mark.parametrize("case", ["random64", "paper_replay"])
def test_static_matches_explore_twice(gpu, case):
    import torch
    snp = gpu
    if case == "random64":
        system, depth, cap, budget, mx = snp_synth.random_64(1), 3, 1 << 12, 1 << 16, -1
    else:
        system, depth, cap, budget, mx = snp_synth.paper_example(), 1000, 0, 0, 9
    ref = snp.System(system)
    ref.explore(depth, cap=cap, budget=budget, max_expand=mx)
    want = ref.reachable()
    want_per_depth = ref.per_depth_new()

    h = snp.snp_load_system(system.m, system.rule_neuron, system.rule_i, system.rule_j, system.M, system.c0)
    try:
        capacity = want.shape[0] + 7
        out = torch.full((capacity, system.m), -1, dtype=torch.int32, device="cuda")
        for _ in range(2):
            pdn = np.zeros(depth + 1, dtype=np.int64)
            n, reached = snp.snp_explore_static(h, _opts(snp, depth, cap, budget, mx), out, capacity, pdn)
            torch.cuda.synchronize()
            got = out[:n].cpu().numpy()
            assert n == want.shape[0]
            assert (got == want).all()
            assert reached == ref.depth_reached
            assert pdn[: reached + 1].tolist() == want_per_depth
    finally:
        snp.snp_free(h)


def test_static_on_a_side_stream(gpu):
    import torch
    snp = gpu
    system = snp_synth.random_64(2)
    ref = snp.System(system)
    ref.explore(2, cap=3000, budget=40000)
    want = ref.reachable()
    h = snp.snp_load_system(system.m, system.rule_neuron, system.rule_i, system.rule_j, system.M, system.c0)
    try:
        stream = torch.cuda.Stream()
        out = torch.empty((want.shape[0], system.m), dtype=torch.int32, device="cuda")
        n, _ = snp.snp_explore_static(h, _opts(snp, 2, 3000, 40000, stream=stream), out, want.shape[0])
        stream.synchronize()
        assert n == want.shape[0] and (out.cpu().numpy() == want).all()
    finally:
        snp.snp_free(h)


def test_static_refuses_sizes_beyond_its_limit(gpu):
    import torch
    snp = gpu
    system = snp_synth.paper_example()
    h = snp.snp_load_system(system.m, system.rule_neuron, system.rule_i, system.rule_j, system.M, system.c0)
    try:
        big = torch.empty(((1 << 20) + 1, 3), dtype=torch.int32, device="cuda")
        with pytest.raises(snp.SnpError) as ei:
            snp.snp_explore_static(h, _opts(snp, 3), big, (1 << 20) + 1)
        assert ei.value.code == snp.SNP_E_INVALID and "limit" in str(ei.value)
        del big
        out = torch.empty((16, 3), dtype=torch.int32, device="cuda")
        with pytest.raises(snp.SnpError) as ei:
            snp.snp_explore_static(h, _opts(snp, 1000, max_expand=9), out, 16)
        assert ei.value.code == snp.SNP_E_BUFFER
        host = np.zeros((16, 3), dtype=np.int32)
        with pytest.raises(snp.SnpError) as ei:
            snp.snp_explore_static(h, _opts(snp, 3), host, 16)
        assert ei.value.code == snp.SNP_E_INVALID
    finally:
        snp.snp_free(h)


def _load(snp, system):
    return snp.snp_load_system(system.m, system.rule_neuron, system.rule_i, system.rule_j, system.M, system.c0)


def test_static_matches_the_oracle(gpu):
    import torch
    snp = gpu
    system = snp_synth.random_64(4)
    e = oracle.Oracle(system).explore(3, cap=3000, budget=30000)
    h = _load(snp, system)
    try:
        out = torch.empty((e.configs.shape[0] + 1, system.m), dtype=torch.int32, device="cuda")
        pdn = np.zeros(4, dtype=np.int64)
        n, reached = snp.snp_explore_static(h, _opts(snp, 3, 3000, 30000), out, out.shape[0], pdn)
        torch.cuda.synchronize()
        assert n == e.configs.shape[0] and (out[:n].cpu().numpy() == e.configs).all()
        assert reached == e.depth_reached and pdn[: reached + 1].tolist() == e.per_depth_new
    finally:
        snp.snp_free(h)


def test_static_wide_rows(gpu):
    """200 neurons: the wide mode (rows built by the whole warp, written to
    staging and copied in by the commit), twice in a row, against snp_explore
    and the oracle."""
    import torch
    snp = gpu
    system = snp_synth.random_system(321, 200, (1, 3), (2, 4), (0, 5), "sparse")
    e = oracle.Oracle(system).explore(3, cap=2000, budget=20000)
    ref = snp.System(system)
    ref.explore(3, cap=2000, budget=20000)
    assert (ref.reachable() == e.configs).all()
    h = _load(snp, system)
    try:
        out = torch.empty((e.configs.shape[0], system.m), dtype=torch.int32, device="cuda")
        for _ in range(2):
            out.fill_(-1)
            n, _ = snp.snp_explore_static(h, _opts(snp, 3, 2000, 20000), out, out.shape[0])
            torch.cuda.synchronize()
            assert n == e.configs.shape[0] and (out.cpu().numpy() == e.configs).all()
    finally:
        snp.snp_free(h)


def test_static_table_rebuild_near_the_limit(gpu):
    """100 neurons whose children are nearly all distinct, 24 depths of 40000
    configurations in passes of 65536 candidates: 960001 configurations (near
    the 2^20 limit) and about 25000 claims past the cap per depth, whose
    tombstones fill the fixed table past three quarters, so it is rebuilt
    mid-depth.  Same result as snp_explore with the same options."""
    import torch
    from test_gpu_parity import saturating_system
    snp = gpu
    system = saturating_system("steady")
    ref = snp.System(system)
    ref.explore(24, cap=40000, chunk=1 << 16)
    want = ref.reachable()
    assert want.shape[0] == 1 + 24 * 40000
    h = _load(snp, system)
    try:
        out = torch.empty((1 << 20, system.m), dtype=torch.int32, device="cuda")
        o = _opts(snp, 24, 40000)
        o.chunk = 1 << 16
        n, reached = snp.snp_explore_static(h, o, out, 1 << 20)
        torch.cuda.synchronize()
        assert n == want.shape[0] and reached == 24
        assert (out[:n].cpu().numpy() == want).all()
    finally:
        snp.snp_free(h)


def test_static_refuses_buffers_it_cannot_use(gpu):
    import torch
    snp = gpu
    system = snp_synth.paper_example()
    h = _load(snp, system)
    try:
        good = torch.empty((16, 3), dtype=torch.int32, device="cuda")
        bad = [torch.empty((16, 3), dtype=torch.int64, device="cuda"),          # not int32
               torch.empty((3, 16), dtype=torch.int32, device="cuda").t(),      # not contiguous
               torch.empty((15, 3), dtype=torch.int32, device="cuda")]          # too small for 16 rows
        for out in bad:
            with pytest.raises(snp.SnpError) as ei:
                snp.snp_explore_static(h, _opts(snp, 3), out, 16)
            assert ei.value.code == snp.SNP_E_INVALID
        for pdn in (np.zeros(3, dtype=np.int64), np.zeros(4, dtype=np.int32)):  # depth + 1 = 4 int64 entries
            with pytest.raises(snp.SnpError) as ei:
                snp.snp_explore_static(h, _opts(snp, 3), good, 16, pdn)
            assert ei.value.code == snp.SNP_E_INVALID
        n, _ = snp.snp_explore_static(h, _opts(snp, 3), good, 16, np.zeros(4, dtype=np.int64))
        assert n > 0
    finally:
        snp.snp_free(h)
