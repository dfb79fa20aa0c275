"""snp_explore_static against snp_explore.

snp_explore_static is for callers that may not allocate device memory when
they need an exploration (a caching allocator holds the free memory, host
callbacks, loops that must not block on the allocator).  It keeps its scratch
in one fixed array inside the library and writes into the caller's buffer.
These tests check that, called twice in a row, it gives exactly the
configurations and per-depth counts that snp_explore gives (integer results:
bit for bit), and that it refuses sizes beyond its fixed limit.

The file is named to be collected last, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

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
        out = torch.empty((16, 3), dtype=torch.int32, device="cuda")
        with pytest.raises(snp.SnpError) as ei:
            snp.snp_explore_static(h, _opts(snp, 3), out, (1 << 20) + 1)
        assert ei.value.code == snp.SNP_E_INVALID and "limit" in str(ei.value)
        with pytest.raises(snp.SnpError) as ei:
            snp.snp_explore_static(h, _opts(snp, 1000, max_expand=9), out, 16)
        assert ei.value.code == snp.SNP_E_BUFFER
        host = np.zeros((16, 3), dtype=np.int32)
        with pytest.raises(snp.SnpError) as ei:
            snp.snp_explore_static(h, _opts(snp, 3), host, 16)
        assert ei.value.code == snp.SNP_E_INVALID
    finally:
        snp.snp_free(h)
