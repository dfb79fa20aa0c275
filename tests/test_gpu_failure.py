"""Failure detection without a GPU fault: a bounded wait that runs out, and a
cancel flag polled between passes.

A testing hook (snp_debug_hold_root_slot) leaves C0's hash-table slot in the
"being claimed" state.  In a system whose only child is C0 itself (two
neurons passing one spike to each other), the first candidate then finds its
key claimed and never published: it waits, the wait runs out after
timeout_ms, the call returns SNP_E_TIMEOUT, and the handle explores normally
afterwards.  Nothing faults, traps or hangs."""
import threading
import time

import numpy as np
import pytest

import oracle
import snp_synth

pytestmark = pytest.mark.gpu


def ping_pong():
    return snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [1, 1], [[1], [0]], [1, 1], name="ping-pong")


@pytest.mark.parametrize("form", ["sparse", "i8", "f8"])
def test_wait_for_a_held_slot_runs_out(gpu, form):
    t = {"sparse": gpu.SNP_T_SPARSE_I32, "i8": gpu.SNP_T_TC_I8, "f8": gpu.SNP_T_TC_F8}[form]
    system = ping_pong()
    s = gpu.System(system)
    gpu.snp_debug_hold_root_slot(True)
    t0 = time.time()
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(3, transition=t, timeout_ms=50)
    assert ei.value.code == gpu.SNP_E_TIMEOUT
    assert time.time() - t0 < 30
    # the hook was one-shot and the handle is usable
    s.explore(3, transition=t, timeout_ms=50)
    e = oracle.Oracle(system).explore(3)
    assert (s.reachable() == e.configs).all() and s.depth_reached == e.depth_reached == 0


def test_wide_rows_wait_runs_out(gpu):
    """The same in the wide mode (rows of more than 128 neurons): 130 neurons
    in pairs that pass one spike to each other."""
    m = 130
    rn = list(range(m))
    system = snp_synth.make_system(m, rn, [1] * m, [1] * m, [1] * m, [1] * m,
                                   [[n ^ 1] for n in range(m)], [1] * m, name="pairs")
    s = gpu.System(system)
    gpu.snp_debug_hold_root_slot(True)
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(2, timeout_ms=50)
    assert ei.value.code == gpu.SNP_E_TIMEOUT
    s.explore(2)
    assert s.count() == 1


def test_cancel_flag_set_before_the_call(gpu):
    system = snp_synth.random_64(1)
    s = gpu.System(system)
    flag = np.ones(1, dtype=np.int32)
    with pytest.raises(gpu.SnpError) as ei:
        s.explore(4, cap=1 << 12, budget=1 << 16, cancel=flag)
    assert ei.value.code == gpu.SNP_E_CANCELLED
    flag[0] = 0
    s.explore(4, cap=1 << 12, budget=1 << 16, cancel=flag)
    e = oracle.Oracle(system).explore(4, cap=1 << 12, budget=1 << 16)
    assert (s.reachable() == e.configs).all()


def test_cancel_flag_set_during_the_call(gpu):
    """The int8 form on the 1024-neuron system takes seconds: a flag set
    0.3 s in stops it between passes."""
    s = gpu.System(snp_synth.dense_1024(3))
    flag = np.zeros(1, dtype=np.int32)
    timer = threading.Timer(0.3, lambda: flag.__setitem__(0, 1))
    timer.start()
    t0 = time.time()
    try:
        with pytest.raises(gpu.SnpError) as ei:
            s.explore(4, cap=1 << 22, budget=1 << 26, transition=gpu.SNP_T_TC_I8, cancel=flag)
        assert ei.value.code == gpu.SNP_E_CANCELLED
        assert time.time() - t0 < 3.0
    finally:
        timer.cancel()
    with pytest.raises(gpu.SnpError) as ei:
        s.reachable()
    assert ei.value.code == gpu.SNP_E_STATE  # the cancelled exploration was discarded
