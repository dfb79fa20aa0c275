"""Parity at the sizes the benchmark times.

* The 1024-neuron system with cap 2^16, budget 2^19, depth 3 (196609
  configurations): every transition form against the oracle's digest and
  per-depth records (tests/golden/oracle_digests.json), the sparse form with
  its automatic pass size (several tasks per warp, the Psi shortcut).
* The 1024-neuron system at full size (cap 2^22, budget 2^26, depth 4: 16.8 M
  configurations of 4 KB), sparse and fp8 tensor-core forms and the sparse
  form with a packed (uint16) store: all give the
  same configurations in the same order and the same parent records; every
  configuration is distinct; 1000 sampled configurations are each the
  recorded child of their recorded parent (the oracle recomputes it); the
  per-depth records follow the cap and budget rule.
* All 4096 systems of the batch workload (depth 6, cap 2^12, budget 2^16) in
  one snp_explore_batch call, sparse and fp8 tensor-core forms, each against
  its oracle digest (tests/golden/batch4096_digests.json).
* The serving loop on 200 requests of the serving stream's own ranges (m up
  to 512, depth up to 32, cap 2^12, budget 2^16): each result alone equals
  the result in the mix.
"""
import concurrent.futures as cf
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import snp_synth
from conftest import GOLDEN
from test_gpu_parity import digest, golden_digests

pytestmark = pytest.mark.gpu


def records(s):
    return [[a.new, a.examined, str(a.candidates), a.truncated] for a in s.depth_stats()]


@pytest.mark.parametrize("form", ["sparse", "f8", "i8"])
def test_dense1024_cap_2_16(gpu, form):
    g = golden_digests()["dense1024_seed3_mid"]
    p = g["params"]
    t = {"sparse": gpu.SNP_T_SPARSE_I32, "f8": gpu.SNP_T_TC_F8, "i8": gpu.SNP_T_TC_I8}[form]
    s = gpu.System(snp_synth.dense_1024(3))
    s.explore(p["depth"], cap=p["cap"], budget=p["budget"], transition=t)
    assert records(s) == g["per_depth"]
    got = s.reachable()
    assert got.shape[0] == g["count"]
    assert digest(got) == g["sha256"]


def _row_keys(torch, rows_dev, keys):
    """A 64-bit linear fingerprint of every row (wrapping int64), in chunks."""
    out = []
    for a in range(0, rows_dev.shape[0], 1 << 18):
        out.append((rows_dev[a:a + (1 << 18)].to(torch.int64) * keys).sum(dim=1))
    return torch.cat(out)


@pytest.mark.slow
def test_dense1024_full_size(gpu):
    import torch
    system = snp_synth.dense_1024(3)
    cap, budget, depth = 1 << 22, 1 << 26, 4
    o = oracle.Oracle(system)
    gen = torch.Generator(device="cpu").manual_seed(5)
    keys = (torch.randint(1, 2 ** 62, (system.m,), generator=gen, dtype=torch.int64) * 2 + 1).cuda()
    runs = {}
    for name, form, packed in (("sparse", gpu.SNP_T_SPARSE_I32, False), ("f8", gpu.SNP_T_TC_F8, False),
                               ("packed", gpu.SNP_T_SPARSE_I32, True)):
        s = gpu.System(system)
        s.explore(depth, cap=cap, budget=budget, transition=form, record_parents=True, packed=packed)
        assert s.row_width() == (2 if packed else 4)
        n = s.count()
        assert n == 1 + depth * cap
        rows = torch.empty((n, system.m), dtype=torch.int32, device="cuda")
        gpu.snp_reachable(s.h, rows, n)
        fp = _row_keys(torch, rows, keys)
        assert torch.unique(fp).numel() == n  # every configuration is new once
        par, idx = s.parents()
        rng = np.random.default_rng(form + 7 * packed)
        ks = np.sort(rng.choice(n - 1, size=1000, replace=False) + 1)
        sample = rows[torch.from_numpy(ks).cuda()].cpu().numpy()
        parents = rows[torch.from_numpy(par[ks]).cuda()].cpu().numpy()
        for k, child, parent in zip(ks, sample, parents):
            assert par[k] < k
            ch = o.child(parent, int(idx[k]))
            assert ch is not None and (ch == child).all(), k
        runs[name] = (fp.cpu().numpy(), par, idx, records(s))
        del rows, fp
        s.close()
        torch.cuda.empty_cache()
    a = runs["sparse"]
    for b in (runs["f8"], runs["packed"]):
        assert (a[0] == b[0]).all() and (a[1] == b[1]).all() and (a[2] == b[2]).all() and a[3] == b[3]
    # the cap and budget rule: every depth accepts cap new configurations
    # before its budget runs out, out of more than 2^64 - 1 candidates
    for d, (new, examined, candidates, truncated) in enumerate(a[3]):
        if d == 0:
            continue
        assert new == cap and new <= examined <= budget and truncated == 1 and int(candidates) == 2 ** 64 - 1


def _system_digest(rows: np.ndarray, per_depth) -> str:
    # the digest tests/golden/make_golden.py stores for each batch system
    h = hashlib.sha256(np.ascontiguousarray(rows, dtype="<i4").tobytes())
    h.update(np.asarray(per_depth, dtype="<u8").tobytes())
    return h.hexdigest()[:24]


@pytest.mark.slow
@pytest.mark.parametrize("form", ["sparse", "f8"])
def test_batch4096_every_system(gpu, form):
    with open(os.path.join(GOLDEN, "batch4096_digests.json")) as f:
        g = json.load(f)
    systems = snp_synth.batch_systems(g["n"], g["base_seed"])
    handles = [gpu.System(x) for x in systems]
    t = gpu.SNP_T_SPARSE_I32 if form == "sparse" else gpu.SNP_T_TC_F8
    st = gpu.explore_batch(handles, g["depth"], cap=g["cap"], budget=g["budget"], transition=t)
    assert (st == 0).all()

    def check(k):
        h = handles[k]
        per = [[a.new, a.examined, a.candidates, a.truncated] for a in h.depth_stats()]
        rows = h.reachable()
        return k, rows.shape[0], _system_digest(rows, per)

    with cf.ThreadPoolExecutor(8) as ex:
        for k, count, dig in ex.map(check, range(len(handles))):
            assert [count, dig] == g["systems"][k], k


@pytest.mark.slow
def test_serving_at_stream_sizes(gpu):
    """200 requests of the serving stream (m U[8,512], depth U[4,32], cap
    2^12, budget 2^16), all submitted at once with room for 64 on the device:
    every result equals the same exploration run alone."""
    import time
    reqs = snp_synth.serving_requests(200, 100.0, seed=4)
    systems = [r.system() for r in reqs]
    handles = [gpu.System(x) for x in systems]
    srv = gpu.snp_server_create(32 << 30, 64)
    try:
        for h, r in zip(handles, reqs):
            o = gpu.snp_explore_opts_init()
            o.depth, o.frontier_cap, o.candidate_budget = r.depth, 1 << 12, 1 << 16
            gpu.snp_server_submit(srv, h.h, o)
        gpu.snp_server_wait(srv)
        got = 0
        while got < len(reqs):
            ids, lat, sts = gpu.snp_server_poll(srv)
            assert all(int(x) == 0 for x in sts)
            got += len(ids)
            if len(ids) == 0:
                time.sleep(0.001)
        for h, x, r in zip(handles, systems, reqs):
            a = gpu.System(x)
            a.explore(r.depth, cap=1 << 12, budget=1 << 16)
            assert (h.reachable() == a.reachable()).all()
            assert [(p.new, p.examined, p.candidates, p.truncated) for p in h.depth_stats()] == \
                [(p.new, p.examined, p.candidates, p.truncated) for p in a.depth_stats()]
            a.close()
        info = gpu.snp_server_stats(srv)
        assert info.completed == 200
    finally:
        gpu.snp_server_destroy(srv)
