"""Pins of the CPU oracle to facts outside itself.

- values the paper prints for its worked example (tests/golden/paper_*.txt);
- Python's regular-expression engine for rule applicability;
- itertools.product for the order of Algorithm 2, II-3;
- brute force over all 0/1 spiking vectors on small systems;
- closed forms (saturation of Psi) and invariants of Eq. next-config.
"""
import itertools

import numpy as np
import pytest

import bruteforce as bf
import oracle
import snp_synth
from conftest import parse_literal, read_golden


@pytest.fixture(scope="module")
def paper():
    return snp_synth.paper_example()


@pytest.fixture(scope="module")
def orc(paper):
    return oracle.Oracle(paper)


def fmt(rows):
    return ["-".join(str(int(x)) for x in r) for r in rows]


# --- the transcription of the example (Section 2, Eq. snp_mat, Eq. row-maj, Eq. rules) ---

def test_transition_matrix_matches_eq_snp_mat(paper):
    g = read_golden("paper_example.txt")
    M = np.array([[int(x) for x in row.split()] for row in g["M_Pi"].split("|")])
    assert (paper.M == M).all()
    assert paper.M.reshape(-1).tolist() == [int(x) for x in g["M_row_major"].split(",")]
    assert paper.c0.tolist() == [int(x) for x in g["C0"].split()]


def test_rules_file_matches_rule_list(paper):
    g = read_golden("paper_example.txt")
    per_neuron = [[int(x) for x in part.split()] for part in g["rules_file"].split("$")]
    assert per_neuron == parse_literal(g["rule_list"])
    got = [[int(paper.rule_i[r]) for r in range(paper.R) if paper.rule_neuron[r] == n] for n in range(paper.m)]
    assert got == per_neuron


def test_synapses_match(paper):
    g = read_golden("paper_example.txt")
    syn = sorted(tuple(int(v) for v in tok.strip("()").split(",")) for tok in g["syn"].split())
    got = sorted((s + 1, int(t) + 1) for s in range(paper.m) for t in paper.targets(s))
    assert got == syn


# --- Algorithm 2 on C0 (Section 4.2 illustration, Section 5 log) ---

def test_ii1_marks_for_c0(orc):
    g = read_golden("paper_example.txt")
    tmp = parse_literal(g["tmp_final"])
    ok = orc.applicable([2, 1, 1]).tolist()
    marks = [1 if v else 0 for neuron in tmp for v in neuron]
    assert ok == marks


def test_psi_of_c0(orc):
    g = read_golden("paper_example.txt")
    assert orc.psi([2, 1, 1]) == int(g["Psi_C0"])


def test_spiking_vectors_of_c0_in_ii3_order(orc):
    g = read_golden("paper_example.txt")
    S = orc.spiking_vectors([2, 1, 1])
    assert ["".join(str(int(x)) for x in row) for row in S] == g["tmp3"].split()


def test_per_neuron_strings_of_ii2(orc, paper):
    g = read_golden("paper_example.txt")
    want = parse_literal(g["tmpList"])
    ok = orc.applicable([2, 1, 1])
    got = []
    for n in range(paper.m):
        rules = [r for r in range(paper.R) if paper.rule_neuron[r] == n]
        app = [k for k, r in enumerate(rules) if ok[r]]
        # one string per applicable rule: a 1 at that rule's place among the neuron's rules
        got.append(["".join("1" if k == a else "0" for k in range(len(rules))) for a in app])
    assert got == want


# --- the printed run (Section 5) ---

def test_children_of_c0(orc):
    g = read_golden("paper_run.txt")
    kids = fmt(orc.step([2, 1, 1]))
    assert ["2-1-1"] + kids == g["after_C0"].split()


def test_replay_first_expansions(orc):
    g = read_golden("paper_run.txt")
    e = orc.explore(1000, max_expand=9)
    lst = fmt(e.configs)
    assert lst[:3] == g["after_C0"].split()
    assert lst[:5] == g["after_212"].split()
    assert lst[:7] == g["after_112"].split()


def test_replay_full_allgenck(orc):
    g = read_golden("paper_run.txt")
    e = orc.explore(1000, max_expand=9)
    assert fmt(e.configs) == g["allGenCk"].split()
    assert fmt(e.configs)[-4:] == g["tail_109"].split()


def test_replay_stops_by_repetition(orc):
    # the run ends because nothing new is produced (second stopping criterion)
    e = orc.explore(1000, max_expand=9)
    assert e.depths[-1].new == 0
    assert e.depth_reached == len(e.depths) - 2


# --- applicability against Python's regex engine ---

@pytest.mark.parametrize("i", range(0, 6))
@pytest.mark.parametrize("j", range(0, 4))
def test_applicability_matches_regex(i, j):
    s = snp_synth.make_system(2, [0], [i], [j], [1], [1], [[1], []], [0, 0])
    o = oracle.Oracle(s)
    for x in range(0, 30):
        want = bf.in_language(x, i, j) and x >= 1
        assert bool(o.applicable([x, 0])[0]) == want, (x, i, j)


def test_consumption_bound_applies():
    # E = a^1(a^1)* matches 2 spikes, but the rule consumes 3: not applicable (x >= c)
    s = snp_synth.make_system(2, [0], [1], [1], [3], [1], [[1], []], [2, 0])
    o = oracle.Oracle(s)
    assert o.applicable([2, 0]).tolist() == [0]
    assert o.applicable([3, 0]).tolist() == [1]


# --- enumeration order against itertools.product ---

def test_order_is_itertools_product():
    rng = np.random.default_rng(5)
    for _ in range(40):
        s = bf.tiny_system(rng, m_max=4, r_max=10)
        o = oracle.Oracle(s)
        C = rng.integers(0, 6, size=s.m)
        ok = bf.applicable(s, C)
        choices = []
        for n in range(s.m):
            rules = [r for r in range(s.R) if s.rule_neuron[r] == n and ok[r]]
            choices.append(rules if rules else [None])
        want = []
        for combo in itertools.product(*choices):
            S = np.zeros(s.R, dtype=np.uint8)
            for r in combo:
                if r is not None:
                    S[r] = 1
            want.append(S)
        got = o.spiking_vectors(C)
        assert len(got) == len(want) == o.psi(C)
        assert all((a == b).all() for a, b in zip(got, want))


def test_child_by_index_matches_enumeration():
    rng = np.random.default_rng(7)
    for _ in range(30):
        s = bf.tiny_system(rng)
        o = oracle.Oracle(s)
        C = rng.integers(0, 6, size=s.m)
        kids = o.step(C)
        for t in range(len(kids)):
            assert (o.child(C, t) == kids[t]).all()
        assert o.child(C, len(kids)) is None


# --- brute force over all 0/1 vectors ---

def test_children_match_brute_force():
    rng = np.random.default_rng(11)
    for _ in range(150):
        s = bf.tiny_system(rng)
        o = oracle.Oracle(s)
        for _ in range(3):
            C = rng.integers(0, 6, size=s.m)
            want = bf.children_canonical(s, C)
            got = o.step(C)
            assert o.psi(C) == len(want)
            assert got.shape == want.shape and (got == want).all()


def test_bfs_levels_match_brute_force():
    rng = np.random.default_rng(13)
    for _ in range(60):
        s = bf.tiny_system(rng, m_max=3, r_max=6)
        o = oracle.Oracle(s)
        levels = bf.bfs_levels(s, 5)
        e = o.explore(5)
        start = 0
        for d, lvl in enumerate(levels):
            n = e.depths[d].new
            got = {tuple(int(x) for x in r) for r in e.configs[start:start + n]}
            assert got == lvl, d
            start += n
        assert start == len(e.configs)


@pytest.mark.parametrize("cap,budget", [(1, 0), (2, 0), (3, 5), (0, 4), (5, 1), (7, 17)])
def test_truncation_matches_brute_force(cap, budget):
    rng = np.random.default_rng(100 + cap * 31 + budget)
    for _ in range(25):
        s = bf.tiny_system(rng, m_max=3, r_max=7)
        o = oracle.Oracle(s)
        order, stats = bf.bfs_canonical(s, 4, cap=cap, budget=budget)
        e = o.explore(4, cap=cap, budget=budget)
        assert [tuple(int(x) for x in r) for r in e.configs] == order
        for d, st in enumerate(stats):
            assert e.depths[d].new == st["new"]
            if d > 0:
                assert e.depths[d].examined == st["examined"]


# --- general rules: unions of terms a^i (a^j)* ---

def test_union_rule_applicability_by_hand():
    """E = a^2 + a^5 (a^3)*, consuming 2: applicable at 2, 5, 8, 11, ... only."""
    s = snp_synth.make_system(2, [0, 1], [2, 1], [0, 1], [2, 1], [1, 1], [[1], [0]], [0, 0],
                              terms=[[(2, 0), (5, 3)], [(1, 1)]])
    o = oracle.Oracle(s)
    got = [x for x in range(20) if o.applicable(np.array([x, 0], dtype=np.int32))[0]]
    assert got == [2, 5, 8, 11, 14, 17]


def test_union_applicability_matches_regex():
    rng = np.random.default_rng(41)
    for _ in range(200):
        s = bf.tiny_union_system(rng)
        o = oracle.Oracle(s)
        for _ in range(5):
            C = rng.integers(0, 14, size=s.m).astype(np.int32)
            assert (o.applicable(C) == bf.applicable(s, C)).all()


def test_union_systems_match_brute_force():
    rng = np.random.default_rng(43)
    for _ in range(30):
        s = bf.tiny_union_system(rng, m_max=3, r_max=6)
        o = oracle.Oracle(s)
        for _ in range(3):
            C = rng.integers(0, 8, size=s.m)
            want = bf.children_canonical(s, C)
            assert o.psi(C) == len(want)
            assert (o.step(C) == want).all()
        order, stats = bf.bfs_canonical(s, 4, cap=5, budget=0)
        e = o.explore(4, cap=5)
        assert [tuple(int(x) for x in r) for r in e.configs] == order


# --- closed forms and invariants ---

def test_psi_saturates():
    m = 70  # 2^70 valid vectors: two applicable rules in every neuron
    rn = np.repeat(np.arange(m), 2)
    s = snp_synth.make_system(m, rn, [1] * (2 * m), [1] * (2 * m), [1] * (2 * m), [0] * (2 * m),
                              [[] for _ in range(m)], [1] * m)
    o = oracle.Oracle(s)
    assert o.psi(np.ones(m, dtype=np.int32)) == 2 ** 64 - 1
    s2 = snp_synth.make_system(63, rn[:126], [1] * 126, [1] * 126, [1] * 126, [0] * 126,
                               [[] for _ in range(63)], [1] * 63)
    assert oracle.Oracle(s2).psi(np.ones(63, dtype=np.int32)) == 2 ** 63


def test_invariants_on_random64():
    s = snp_synth.random_64(1)
    o = oracle.Oracle(s)
    e = o.explore(2, cap=2000, budget=20000)
    rowsum = s.M.sum(axis=1)
    start = 0
    levels = []
    for d in e.depths:
        levels.append(e.configs[start:start + d.new])
        start += d.new
    assert (e.configs >= 0).all()
    # levels pairwise disjoint; rows distinct
    assert len({r.tobytes() for r in e.configs}) == len(e.configs)
    # every configuration of depth 1 is a child of C0 with the spike sum of Eq. next-config
    kids = {r.tobytes() for r in o.step(s.c0, cap=1 << 20)}
    for r in levels[1]:
        assert r.tobytes() in kids
    for C in levels[1][:50]:
        S = o.spiking_vectors(C, cap=64)
        kids2 = o.step(C, cap=64)
        for Srow, ch in zip(S, kids2):
            assert ch.sum() == C.sum() + int(rowsum[Srow.astype(bool)].sum())
        p = o.psi(C)
        if p <= 4096:
            assert len(o.step(C, cap=p + 1)) == p


def test_textbook_exact_reading_gives_eight():
    # E = a^k exactly (j = 0): a derived fact, cross-checked by brute force
    s = snp_synth.paper_example(exact=True)
    e = oracle.Oracle(s).explore(100)
    levels = bf.bfs_levels(s, 100)
    assert len(e.configs) == sum(len(l) for l in levels) == 8


def test_depth10_of_paper_example_matches_brute_force():
    s = snp_synth.paper_example()
    e = oracle.Oracle(s).explore(10)
    levels = bf.bfs_levels(s, 10)
    assert e.per_depth_new == [len(l) for l in levels]
    assert e.per_depth_new == [1, 2, 4, 6, 6, 6, 5, 5, 5, 5, 5]


def test_overflow_flag_on_actual_overflow():
    """Eq. next-config in int64, flagged when an entry leaves int32: neuron 0
    (one spike) sends 5 spikes to neuron 1, which holds 2^31 - 3 and consumes
    one.  Both neurons have one applicable rule, so the only spiking vector is
    S = (1, 1) and the only child is C + S . M = (0, 2^31 + 1) (Python
    integers below); the oracle's step raises and its exploration stops with
    the error set, keeping only C0."""
    big = 2 ** 31 - 3
    system = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [5, 0], [[1], [0]], [1, big])
    child = [1 + int(system.M[0][0]) + int(system.M[1][0]), big + int(system.M[0][1]) + int(system.M[1][1])]
    assert child == [0, 2 ** 31 + 1]
    o = oracle.Oracle(system)
    C = np.array([1, big], dtype=np.int32)
    assert o.psi(C) == 1
    with pytest.raises(OverflowError):
        o.step(C)
    e = o.explore(3)
    assert e.error == 1 and e.configs.shape[0] == 1


def test_no_overflow_flag_when_no_child_overflows():
    """The same system with neuron 0 empty: neuron 1 fires alone and drains
    (its count only falls), so no child leaves int32 and the oracle explores
    normally, although neuron 1's column could still gain 5 in one step if
    neuron 0 fired (the GPU's per-column bound refuses this case; see the
    GPU test of the same system)."""
    big = 2 ** 31 - 3
    system = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [5, 0], [[1], [0]], [0, big])
    e = oracle.Oracle(system).explore(3)
    assert e.error == 0
    assert e.configs.tolist() == [[0, big], [0, big - 1], [0, big - 2], [0, big - 3]]
