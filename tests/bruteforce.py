"""Brute-force references for small systems, independent of the oracle.

Applicability is decided by Python's regular-expression engine on the string
a^x; spiking vectors are found by trying all 2^R vectors of 0s and 1s and
keeping the valid ones (Section 2.2: in every neuron that has an applicable
rule exactly one applicable rule is used, elsewhere none); children are
C + S @ M with numpy.  Nothing here is shared with oracle/ or the CUDA path.
"""
from __future__ import annotations

import itertools
import re
from functools import lru_cache
from typing import Dict, List, Tuple

import numpy as np


@lru_cache(maxsize=None)
def _regex(i: int, j: int):
    return re.compile(f"a{{{i}}}(a{{{j}}})*")


def in_language(x: int, i: int, j: int) -> bool:
    """a^x in L(a^i (a^j)*), decided by the regex engine."""
    return _regex(i, j).fullmatch("a" * x) is not None


def in_union_language(x: int, terms) -> bool:
    """a^x in the union of the terms' languages, decided by one regex."""
    pattern = "|".join(f"(?:a{{{i}}}(?:a{{{j}}})*)" for i, j in terms)
    return re.fullmatch(f"(?:{pattern})", "a" * x) is not None


def applicable(system, C) -> np.ndarray:
    ok = np.zeros(system.R, dtype=np.uint8)
    for r in range(system.R):
        n = int(system.rule_neuron[r])
        c = -int(system.M[r, n])
        x = int(C[n])
        if getattr(system, "terms", None) is not None:
            member = in_union_language(x, system.terms[r])
        else:
            member = in_language(x, int(system.rule_i[r]), int(system.rule_j[r]))
        ok[r] = 1 if (member and x >= c) else 0
    return ok


def valid_vectors(system, C) -> List[np.ndarray]:
    """All valid spiking vectors of C, by trying every 0/1 vector of length R."""
    ok = applicable(system, C)
    has = np.zeros(system.m, dtype=bool)
    for r in range(system.R):
        if ok[r]:
            has[system.rule_neuron[r]] = True
    out = []
    for bits in itertools.product((0, 1), repeat=system.R):
        S = np.array(bits, dtype=np.int64)
        if np.any(S & (1 - ok)):
            continue  # uses a rule that is not applicable
        per = np.zeros(system.m, dtype=np.int64)
        np.add.at(per, system.rule_neuron, S)
        if np.all(per == has.astype(np.int64)):
            out.append(S)
    return out


def mixed_radix_key(system, C, S) -> Tuple[int, ...]:
    """Per neuron (neuron 0 first): the position of the used rule among the
    neuron's applicable rules, 0 if the neuron does not fire."""
    ok = applicable(system, C)
    key = []
    for n in range(system.m):
        rules = [r for r in range(system.R) if system.rule_neuron[r] == n and ok[r]]
        used = [k for k, r in enumerate(rules) if S[r]]
        key.append(used[0] if used else 0)
    return tuple(key)


def children(system, C) -> np.ndarray:
    vecs = valid_vectors(system, C)
    if not vecs:
        return np.zeros((0, system.m), dtype=np.int64)
    return np.asarray(C, dtype=np.int64)[None, :] + np.stack(vecs) @ system.M.astype(np.int64)


def children_canonical(system, C) -> np.ndarray:
    """Children ordered by the mixed-radix key, neuron 0 most significant."""
    vecs = valid_vectors(system, C)
    vecs.sort(key=lambda S: mixed_radix_key(system, C, S))
    if not vecs:
        return np.zeros((0, system.m), dtype=np.int64)
    return np.asarray(C, dtype=np.int64)[None, :] + np.stack(vecs) @ system.M.astype(np.int64)


def bfs_levels(system, depth: int) -> List[set]:
    """Set of configurations first reached at each depth (no cap)."""
    c0 = tuple(int(x) for x in system.c0)
    seen = {c0}
    levels = [{c0}]
    for _ in range(depth):
        nxt = set()
        for C in levels[-1]:
            for ch in children(system, np.array(C)):
                t = tuple(int(x) for x in ch)
                if t not in seen:
                    seen.add(t)
                    nxt.add(t)
        if not nxt:
            break
        levels.append(nxt)
    return levels


def bfs_canonical(system, depth: int, cap: int = 0, budget: int = 0) -> Tuple[List[Tuple[int, ...]], List[Dict]]:
    """Discovery-ordered BFS with a per-depth cap and candidate budget, the
    candidates of each parent in mixed-radix order (brute-force enumeration)."""
    c0 = tuple(int(x) for x in system.c0)
    seen = {c0}
    order = [c0]
    stats = [dict(new=1, examined=0)]
    frontier = [c0]
    for _ in range(depth):
        nxt, examined, stop = [], 0, False
        for C in frontier:
            if stop:
                break
            for ch in children_canonical(system, np.array(C)):
                if budget > 0 and examined >= budget:
                    stop = True
                    break
                examined += 1
                t = tuple(int(x) for x in ch)
                if t not in seen:
                    seen.add(t)
                    nxt.append(t)
                    order.append(t)
                    if cap > 0 and len(nxt) >= cap:
                        stop = True
                        break
        stats.append(dict(new=len(nxt), examined=examined))
        if not nxt:
            break
        frontier = nxt
    return order, stats


def tiny_union_system(rng: np.random.Generator, m_max: int = 4, r_max: int = 9, t_max: int = 3):
    """tiny_system whose rules have 1..t_max terms a^i (a^j)* each (general rules)."""
    import snp_synth
    base = tiny_system(rng, m_max, r_max)
    terms = [[(int(rng.integers(0, 6)), int(rng.integers(0, 5))) for _ in range(int(rng.integers(1, t_max + 1)))]
             for _ in range(base.R)]
    c = -base.M[np.arange(base.R), base.rule_neuron]
    p = np.array([int(base.M[r].max()) if base.M[r].max() > 0 else 0 for r in range(base.R)])
    targets = [base.targets(s).tolist() for s in range(base.m)]
    return snp_synth.make_system(base.m, base.rule_neuron, [t[0][0] for t in terms], [t[0][1] for t in terms], c, p,
                                 targets, base.c0, name="tiny-union", terms=terms)


def tiny_system(rng: np.random.Generator, m_max: int = 4, r_max: int = 9):
    """A random small system for brute-force checks (uses snp_synth.make_system)."""
    import snp_synth
    m = int(rng.integers(1, m_max + 1))
    while True:
        per = rng.integers(0, 4, size=m)
        if 1 <= per.sum() <= r_max:
            break
    rule_neuron = np.repeat(np.arange(m), per)
    R = len(rule_neuron)
    i = rng.integers(0, 4, size=R)
    c = np.array([int(rng.integers(1, max(1, ii) + 1)) if rng.random() < 0.8 else int(rng.integers(1, 4))
                  for ii in i])
    j = rng.integers(0, 3, size=R)
    p = rng.integers(0, 3, size=R)
    targets = []
    for s in range(m):
        others = [t for t in range(m) if t != s]
        k = int(rng.integers(0, len(others) + 1))
        targets.append(sorted(rng.choice(others, size=k, replace=False).tolist()) if k else [])
    c0 = rng.integers(0, 5, size=m)
    return snp_synth.make_system(m, rule_neuron, i, j, c, p, targets, c0, name="tiny")
