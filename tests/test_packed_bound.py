"""The bound a packed store relies on, checked on the oracle (CPU).

Counts never go below 0 (a rule applies only to at least the spikes it
consumes), and one step adds at most gain[j] to column j, the sum over
neurons of the largest entry of column j among the neuron's rules (at most
one rule per neuron fires; the consumption sits on the rule's own column as
a negative entry).  So every configuration at depth d has counts in
[0, C0[j] + d * gain[j]].  Brute force over many small random systems, and a
system that meets the bound with equality, so that a bound one too small
would fail.
"""
import numpy as np

import bruteforce as bf
import oracle
import snp_synth


def column_gain(system) -> np.ndarray:
    M = np.asarray(system.M, dtype=np.int64).reshape(system.R, system.m)
    rn = np.asarray(system.rule_neuron)
    g = np.zeros(system.m, dtype=np.int64)
    for n in range(system.m):
        rows = M[rn == n]
        if len(rows):
            g += np.maximum(rows.max(axis=0), 0)
    return g


def depth_of_rows(e) -> np.ndarray:
    return np.repeat(np.arange(len(e.depths)), [d.new for d in e.depths])


def check_bound(system, depth, **kw):
    e = oracle.Oracle(system).explore(depth, **kw)
    d = depth_of_rows(e)[:, None]
    hi = np.asarray(system.c0, dtype=np.int64)[None, :] + d * column_gain(system)[None, :]
    assert (e.configs >= 0).all()
    assert (e.configs <= hi).all()
    return e, hi


def test_bound_holds_on_small_random_systems():
    rng = np.random.default_rng(77)
    for _ in range(150):
        system = bf.tiny_system(rng, m_max=4, r_max=9)
        check_bound(system, 6)
    for _ in range(40):
        system = bf.tiny_union_system(rng, m_max=4, r_max=8)
        check_bound(system, 6)


def test_bound_holds_on_generated_workload_shapes():
    check_bound(snp_synth.random_64(1), 3, cap=1 << 12, budget=1 << 16)
    check_bound(snp_synth.random_system(8, 16, (2, 3), (2, 4), (0, 6), "sparse"), 3)


def test_bound_is_met_with_equality():
    """Neuron 0 fires a -> a^3 (exactly one spike) into neurons 1 and 2 and
    gets one spike back every step from neuron 1, which fires a(a)* -> a;
    neuron 2's rule (exactly a^1000) never applies.  Column 2 then grows by
    exactly gain[2] = 3 every step."""
    system = snp_synth.make_system(3, [0, 1, 2], [1, 1, 1000], [0, 1, 0], [1, 1, 1], [3, 1, 1],
                                   [[1, 2], [0], [0]], [1, 1, 0])
    assert list(column_gain(system)) == [2, 3, 3]
    e, hi = check_bound(system, 5)
    assert e.depth_reached == 5 and e.configs.shape[0] == 6
    assert (e.configs[:, 2] == hi[:, 2]).all()
