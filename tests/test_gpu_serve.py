"""The serving loop (snp_server_*): every request's result is the same alone
and in the mix -- bit for bit, since the results are integer configurations
-- whatever else runs beside it, however requests arrive and however little
device memory the server has."""
import threading
import time

import numpy as np
import pytest

import oracle
import snp_synth

pytestmark = pytest.mark.gpu


def requests(n, seed, m_range=(8, 96), depth_range=(3, 7)):
    rng = snp_synth.Rng(seed)
    ms = rng.randint(m_range[0], m_range[1], n)
    depths = rng.randint(depth_range[0], depth_range[1], n)
    systems = [snp_synth.random_system(9000 + seed * 1000 + k, int(ms[k]), (2, 3), (4, 4), (0, 6), "sparse")
               for k in range(n)]
    return systems, [int(d) for d in depths]


def opts(gpu, depth, cap=256, budget=4096):
    o = gpu.snp_explore_opts_init()
    o.depth, o.frontier_cap, o.candidate_budget = depth, cap, budget
    return o


def alone(gpu, system, depth, cap=256, budget=4096):
    s = gpu.System(system)
    s.explore(depth, cap=cap, budget=budget)
    return s.reachable(), [(a.new, a.examined, a.candidates, a.truncated) for a in s.depth_stats()]


def result(h):
    return h.reachable(), [(a.new, a.examined, a.candidates, a.truncated) for a in h.depth_stats()]


def drain(gpu, srv, expect):
    got = {}
    while len(got) < expect:
        ids, lat, sts = gpu.snp_server_poll(srv)
        for i, l, s in zip(ids, lat, sts):
            got[int(i)] = (float(l), int(s))
        if len(got) < expect:
            time.sleep(0.001)
    return got


def test_alone_and_in_the_mix(gpu):
    systems, depths = requests(48, 1)
    srv = gpu.snp_server_create(8 << 30, 64)
    try:
        handles = [gpu.System(x) for x in systems]
        ids = [gpu.snp_server_submit(srv, h.h, opts(gpu, d)) for h, d in zip(handles, depths)]
        gpu.snp_server_wait(srv)
        done = drain(gpu, srv, len(ids))
        assert all(s == 0 for _, s in done.values())
        for h, x, d in zip(handles, systems, depths):
            rows, stats = result(h)
            rows_a, stats_a = alone(gpu, x, d)
            assert (rows == rows_a).all() and stats == stats_a
        # and against the oracle, for a few
        for k in (0, 17, 40):
            e = oracle.Oracle(systems[k]).explore(depths[k], cap=256, budget=4096)
            assert (handles[k].reachable() == e.configs).all()
        info = gpu.snp_server_stats(srv)
        assert info.completed == 48 and info.pending == 0 and info.active == 0
        assert info.p99_ms >= info.p50_ms > 0
    finally:
        gpu.snp_server_destroy(srv)


def test_requests_arriving_while_others_run(gpu):
    systems, depths = requests(60, 2, m_range=(8, 200), depth_range=(4, 12))
    srv = gpu.snp_server_create(8 << 30, 16)
    handles = [gpu.System(x) for x in systems]
    try:
        def client(part):
            for k in part:
                gpu.snp_server_submit(srv, handles[k].h, opts(gpu, depths[k]))
                time.sleep(0.002)
        threads = [threading.Thread(target=client, args=(range(t, 60, 3),)) for t in range(3)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        gpu.snp_server_wait(srv)
        drain(gpu, srv, 60)
        info = gpu.snp_server_stats(srv)
        assert info.completed == 60
        assert info.ticks < sum(depths)  # requests shared launches
        for k in range(0, 60, 7):
            rows, stats = result(handles[k])
            rows_a, stats_a = alone(gpu, systems[k], depths[k])
            assert (rows == rows_a).all() and stats == stats_a
    finally:
        gpu.snp_server_destroy(srv)


def test_admission_by_memory(gpu):
    systems, depths = requests(20, 3, m_range=(32, 64), depth_range=(4, 6))
    # room for about three requests at a time
    srv = gpu.snp_server_create(12 << 20, 64)
    handles = [gpu.System(x) for x in systems]
    try:
        for h, d in zip(handles, depths):
            gpu.snp_server_submit(srv, h.h, opts(gpu, d))
        gpu.snp_server_wait(srv)
        done = drain(gpu, srv, 20)
        assert len(done) == 20
        for k in range(20):
            rows, stats = result(handles[k])
            rows_a, stats_a = alone(gpu, systems[k], depths[k])
            assert (rows == rows_a).all() and stats == stats_a
    finally:
        gpu.snp_server_destroy(srv)


def test_server_refuses_bad_requests(gpu):
    srv = gpu.snp_server_create(4 << 20, 4)
    try:
        h = gpu.System(snp_synth.random_64(1))
        with pytest.raises(gpu.SnpError) as ei:
            gpu.snp_server_submit(srv, h.h, opts(gpu, 4, cap=0))
        assert ei.value.code == gpu.SNP_E_INVALID
        with pytest.raises(gpu.SnpError) as ei:
            gpu.snp_server_submit(srv, h.h, opts(gpu, 8, cap=1 << 20))
        assert ei.value.code == gpu.SNP_E_NOMEM
    finally:
        gpu.snp_server_destroy(srv)
