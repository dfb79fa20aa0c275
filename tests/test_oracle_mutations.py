"""Plants plausible mistakes in a copy of the oracle and checks that the pins
catch each one (the mutated copies are built in a temporary directory; the
oracle itself is untouched)."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

import bruteforce as bf
import oracle
import snp_synth
from conftest import read_golden

SRC = os.path.join(os.path.dirname(oracle.__file__), "snp_oracle.cpp")

MUTATIONS = {
    "neuron0_least_significant": ("for (int n = (int)lists.size() - 1; n >= 0; --n) {",
                                  "for (int n = 0; n < (int)lists.size(); ++n) {"),
    "exactly_i_only": ("if (j == 0) return x == i;", "if (true) return x == i;"),
    "no_consumption_bound": ("&& x >= consumed(s, r);", ";"),
    "sign_flip": ("acc[j] += (int64_t)S[r] * s.M", "acc[j] -= (int64_t)S[r] * s.M"),
    "mirrored_column": ("acc[j] += (int64_t)S[r] * s.M[(size_t)r * s.m + j];",
                        "acc[j] += (int64_t)S[r] * s.M[(size_t)r * s.m + (s.m - 1 - j)];"),
    "no_dedup": ("if (visited.find(child) == visited.end()) {", "if (true) {"),
    "cap_off_by_one": ("if (cap > 0 && st.new_configs >= cap)", "if (cap > 0 && st.new_configs > cap)"),
    "budget_off_by_one": ("if (budget > 0 && st.examined >= budget)", "if (budget > 0 && st.examined > budget)"),
    "psi_without_max1": ("p = sat_mul(p, l.empty() ? 1 : l.size());", "p = sat_mul(p, l.size());"),
    "parents_lifo": ("std::memcpy(parent.data(), res->configs.data() + p * s.m",
                     "std::memcpy(parent.data(), res->configs.data() + (level_end - 1 - (p - level_begin)) * s.m"),
    "no_overflow_check": ("if (acc[j] < INT32_MIN || acc[j] > INT32_MAX) return false;", "(void)0;"),
    "rule_order_reversed": ("if (applicable(s, C, r)) lists[s.rule_neuron[r]].push_back(r);",
                            "if (applicable(s, C, r)) lists[s.rule_neuron[r]].insert(lists[s.rule_neuron[r]].begin(), r);"),
}


def pins_pass(lib_path: str) -> bool:
    """A fast subset of the oracle pins; True iff all hold."""
    g = read_golden("paper_run.txt")
    ge = read_golden("paper_example.txt")
    paper = snp_synth.paper_example()
    o = oracle.Oracle(paper, lib_path=lib_path)
    if o.psi([2, 1, 1]) != int(ge["Psi_C0"]):
        return False
    S = ["".join(str(int(x)) for x in r) for r in o.spiking_vectors([2, 1, 1])]
    if S != ge["tmp3"].split():
        return False
    if o.explore(10).per_depth_new != [1, 2, 4, 6, 6, 6, 5, 5, 5, 5, 5]:
        return False  # checked first: a broken deduplication would not terminate the replay below
    e = o.explore(1000, max_expand=9)
    if ["-".join(str(int(x)) for x in r) for r in e.configs] != g["allGenCk"].split():
        return False
    # an actual int32 overflow stops the exploration; a possible one does not
    big = 2 ** 31 - 3
    for c0, want_error in (([1, big], 1), ([0, big], 0)):
        x = snp_synth.make_system(2, [0, 1], [1, 1], [1, 1], [1, 1], [5, 0], [[1], [0]], c0)
        if oracle.Oracle(x, lib_path=lib_path).explore(3).error != want_error:
            return False
    # a budget of B examines exactly B candidates when more are available
    e = oracle.Oracle(snp_synth.random_64(1), lib_path=lib_path).explore(1, budget=100)
    if e.depths[1].examined != 100 or e.depths[1].truncated != 1:
        return False
    rng = np.random.default_rng(2024)
    for _ in range(40):
        s = bf.tiny_system(rng)
        os_ = oracle.Oracle(s, lib_path=lib_path)
        C = rng.integers(0, 6, size=s.m)
        want = bf.children_canonical(s, C)
        got = os_.step(C)
        if os_.psi(C) != len(want) or got.shape != want.shape or not (got == want).all():
            return False
    for cap, budget in [(2, 0), (3, 5), (0, 4)]:
        for _ in range(8):
            s = bf.tiny_system(rng, m_max=3, r_max=7)
            order, stats = bf.bfs_canonical(s, 4, cap=cap, budget=budget)
            e = oracle.Oracle(s, lib_path=lib_path).explore(4, cap=cap, budget=budget)
            if [tuple(int(x) for x in r) for r in e.configs] != order:
                return False
            if [d.new for d in e.depths][: len(stats)] != [st["new"] for st in stats]:
                return False
            if [d.examined for d in e.depths][1: len(stats)] != [st["examined"] for st in stats][1:]:
                return False
    return True


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


def build_variant(workdir: str, name: str, old: str, new: str) -> str:
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation {name}: pattern not found exactly once"
    path = os.path.join(workdir, f"{name}.cpp")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = os.path.join(workdir, f"lib{name}.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", lib, path])
    return lib


def test_unmutated_oracle_passes_the_pins():
    assert pins_pass(oracle.build())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(workdir, name):
    old, new = MUTATIONS[name]
    lib = build_variant(workdir, name, old, new)
    assert not pins_pass(lib), f"the pins do not detect mutation {name}"
