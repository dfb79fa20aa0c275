"""Seeded synthetic SNP systems without delays: the inputs, and nothing else.

This module is shared by the CPU oracle and the GPU path, so it holds none of
the simulation method's arithmetic (no applicability test, no spiking-vector
enumeration, no transition, no deduplication).  It only draws the parameters
of a system (rules, synapses, initial spikes) and lays the spiking transition
matrix M_Pi out as an input array, entry by entry as Definition 2 of the paper
defines it: row r (a rule of neuron s) holds -c at column s, +p at every
column t with (s, t) a synapse, and 0 elsewhere.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw k (k = 1, 2, ...) of a stream with seed s is
mix64(s + k * 0x9E3779B97F4A7C15).  Integers in [lo, hi] are
lo + ((u >> 32) * (hi - lo + 1) >> 32); the draw order of every recipe is fixed
below, so a seed names exactly one system.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

__all__ = [
    "SnpSystem",
    "Rng",
    "paper_example",
    "random_system",
    "random_64",
    "dense_1024",
    "batch_systems",
    "serving_requests",
    "make_system",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


class Rng:
    """Counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = np.uint64(int(seed) & _MASK64)
        self.ctr = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.ctr + 1, self.ctr + n + 1, dtype=np.uint64)
        self.ctr += n
        with np.errstate(over="ignore"):
            return _mix64(self.seed + k * _GAMMA)

    def randint(self, lo, hi, n: int) -> np.ndarray:
        """n integers, element e uniform in [lo_e, hi_e] (inclusive); lo/hi may be arrays."""
        u = self.u64(n) >> np.uint64(32)
        span = (np.asarray(hi, dtype=np.int64) - np.asarray(lo, dtype=np.int64) + 1).astype(np.uint64)
        with np.errstate(over="ignore"):
            off = (u * span) >> np.uint64(32)
        return (np.asarray(lo, dtype=np.int64) + off.astype(np.int64)).astype(np.int64)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1)."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class SnpSystem:
    """An SNP system without delays in the matrix representation of the paper.

    Rules are in the paper's total order, grouped by neuron (rule_neuron is
    non-decreasing).  Rule r of neuron s has regular expression a^i(a^j)*
    (j = 0: exactly a^i), consumes c spikes and sends p spikes along each
    synapse (s, t); p = 0 is a forgetting rule.
    """

    m: int
    rule_neuron: np.ndarray  # int32 [R]
    rule_i: np.ndarray       # int32 [R]
    rule_j: np.ndarray       # int32 [R]
    rule_c: np.ndarray       # int32 [R]
    rule_p: np.ndarray       # int32 [R]
    syn_ptr: np.ndarray      # int32 [m+1]  targets of neuron s: syn_dst[syn_ptr[s]:syn_ptr[s+1]]
    syn_dst: np.ndarray      # int32 [nsyn]
    c0: np.ndarray           # int32 [m]
    M: np.ndarray            # int32 [R, m]  spiking transition matrix (Definition 2)
    name: str = ""
    meta: dict = field(default_factory=dict)
    # General regular expressions (the paper's future work), read as unions of
    # terms: rule r's expression is the union of a^i (a^j)* over terms[r]'s
    # (i, j) pairs.  None: each rule is its single term (rule_i[r], rule_j[r]).
    terms: Optional[List[List[Tuple[int, int]]]] = None

    @property
    def R(self) -> int:
        return int(self.rule_neuron.shape[0])

    def term_arrays(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """(rule_terms [R+1], term_i, term_j): rule r's terms are
        [rule_terms[r], rule_terms[r+1])."""
        terms = self.terms if self.terms is not None else [[(int(i), int(j))] for i, j in zip(self.rule_i, self.rule_j)]
        ptr = np.zeros(self.R + 1, dtype=np.int32)
        ptr[1:] = np.cumsum([len(t) for t in terms])
        ti = np.array([i for t in terms for i, _ in t], dtype=np.int32)
        tj = np.array([j for t in terms for _, j in t], dtype=np.int32)
        return ptr, ti, tj

    def targets(self, s: int) -> np.ndarray:
        return self.syn_dst[self.syn_ptr[s]:self.syn_ptr[s + 1]]


def make_system(m, rule_neuron, rule_i, rule_j, rule_c, rule_p, targets, c0,
                name: str = "", meta: Optional[dict] = None, terms=None) -> SnpSystem:
    """Assemble a system and lay out M_Pi entry by entry (Definition 2).

    targets: per-neuron lists of synapse targets, or a CSR pair (syn_ptr, syn_dst).
    """
    rule_neuron = np.asarray(rule_neuron, dtype=np.int32)
    R = rule_neuron.shape[0]
    if isinstance(targets, tuple):            # already (syn_ptr, syn_dst), rows sorted
        syn_ptr = np.asarray(targets[0], dtype=np.int32)
        syn_dst = np.asarray(targets[1], dtype=np.int32)
    else:
        syn_ptr = np.zeros(m + 1, dtype=np.int32)
        for s in range(m):
            syn_ptr[s + 1] = syn_ptr[s] + len(targets[s])
        syn_dst = np.zeros(int(syn_ptr[-1]), dtype=np.int32)
        for s in range(m):
            syn_dst[syn_ptr[s]:syn_ptr[s + 1]] = np.sort(np.asarray(targets[s], dtype=np.int32))
    rule_c = np.asarray(rule_c, dtype=np.int32)
    rule_p = np.asarray(rule_p, dtype=np.int32)
    M = np.zeros((R, m), dtype=np.int32)
    rows = np.arange(R)
    M[rows, rule_neuron] = -rule_c                      # -c on the rule's own neuron
    outdeg = (syn_ptr[1:] - syn_ptr[:-1])[rule_neuron]  # +p on each synapse target
    rr = np.repeat(rows, outdeg)
    starts = syn_ptr[rule_neuron]
    within = np.arange(rr.shape[0]) - np.repeat(np.cumsum(outdeg) - outdeg, outdeg)
    M[rr, syn_dst[np.repeat(starts, outdeg) + within]] = np.repeat(rule_p, outdeg)
    return SnpSystem(m=m, rule_neuron=rule_neuron, rule_i=np.asarray(rule_i, dtype=np.int32),
                     rule_j=np.asarray(rule_j, dtype=np.int32), rule_c=rule_c, rule_p=rule_p,
                     syn_ptr=syn_ptr, syn_dst=syn_dst, c0=np.asarray(c0, dtype=np.int32), M=M,
                     name=name, meta=dict(meta or {}),
                     terms=None if terms is None else [[(int(i), int(j)) for i, j in t] for t in terms])


def paper_example(exact: bool = False) -> SnpSystem:
    """The paper's 3-neuron, 5-rule system that generates N - {1} (Section 2, Fig. 1).

    Transcription: C0 = <2,1,1>; synapses (1,2),(1,3),(2,1),(2,3); sigma_3 is
    the output neuron and its spikes leave the system, so its rules have no
    positive entries in M.  The rules file "2 2 $ 1 $ 1 2" gives each rule's
    spike threshold k; the printed run is reproduced when a rule of form (b-3)
    applies whenever the neuron holds at least k spikes, i.e. E = a^k(a)*
    (i = k, j = 1).  exact=True gives the other reading, E = a^k (j = 0).
    Consumed spikes c are read off the diagonal of Eq. (snp_mat).
    """
    j = 0 if exact else 1
    return make_system(
        m=3,
        rule_neuron=[0, 0, 1, 2, 2],
        rule_i=[2, 2, 1, 1, 2],
        rule_j=[j] * 5,
        rule_c=[1, 2, 1, 1, 2],
        rule_p=[1, 1, 1, 1, 0],
        targets=[[1, 2], [0, 2], []],
        c0=[2, 1, 1],
        name="paper_example_exact" if exact else "paper_example",
    )


def _floyd_targets(rng: Rng, m: int, deg: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Distinct targets per neuron, no self-loops (Floyd's subset sampling,
    vectorised over neurons; draws one u64 per neuron per step)."""
    n = m - 1
    dmax = int(deg.max()) if m > 0 else 0
    chosen = np.full((m, max(dmax, 1)), -1, dtype=np.int64)
    for k in range(dmax):
        active = k < deg
        jj = n - deg + k                      # Floyd's j for neuron s at this step
        jj_safe = np.where(active, jj, 0)
        t = rng.randint(0, jj_safe, m)
        seen = (chosen[:, :k] == t[:, None]).any(axis=1) if k > 0 else np.zeros(m, dtype=bool)
        pick = np.where(seen, jj_safe, t)
        chosen[:, k] = np.where(active, pick, -1)
    self_idx = np.arange(m)[:, None]
    mapped = np.where(chosen >= self_idx, chosen + 1, chosen)  # map [0, m-1) onto the other neurons
    mapped = np.where(chosen < 0, m, mapped)                   # padding sorts last
    mapped = np.sort(mapped, axis=1)
    syn_ptr = np.zeros(m + 1, dtype=np.int32)
    syn_ptr[1:] = np.cumsum(deg)
    keep = np.arange(mapped.shape[1])[None, :] < deg[:, None]
    return syn_ptr, mapped[keep].astype(np.int32)


def random_system(seed: int, m, rules_per_neuron: Tuple[int, int], outdeg: Tuple[int, int],
                  c0_range: Tuple[int, int], mode: str, name: str = "") -> SnpSystem:
    """A random system.  Draw order: m (if a range), rules per neuron [m],
    then per rule the arrays a, b, j, p, forget [R], out-degree [m], synapse
    targets, initial spikes [m].

    mode "sparse" (configs with 2-3 or 1-4 rules per neuron):
        i = U[1,4], c = U[1,i], j = U{0,1,2}, p = U{1,2}, and with probability
        0.15 the rule forgets (p = 0).
    mode "dense" (1024-neuron tensor-core config):
        c = U[1,8], i = U[c,8], j = U{0,1,2}, p = U[1,8], no forgetting rules.
    """
    rng = Rng(seed)
    if isinstance(m, tuple):
        m = int(rng.randint(m[0], m[1], 1)[0])
    m = int(m)
    nrules = rng.randint(rules_per_neuron[0], rules_per_neuron[1], m)
    R = int(nrules.sum())
    rule_neuron = np.repeat(np.arange(m, dtype=np.int32), nrules)
    if mode == "sparse":
        i = rng.randint(1, 4, R)
        c = rng.randint(1, i, R)
        j = rng.randint(0, 2, R)
        p = rng.randint(1, 2, R)
        forget = rng.uniform(R) < 0.15
        p = np.where(forget, 0, p)
    elif mode == "dense":
        c = rng.randint(1, 8, R)
        i = rng.randint(c, 8, R)
        j = rng.randint(0, 2, R)
        p = rng.randint(1, 8, R)
        rng.uniform(R)  # keeps the draw layout of the sparse mode
    else:
        raise ValueError(mode)
    deg = rng.randint(outdeg[0], outdeg[1], m)
    deg = np.minimum(deg, m - 1)
    targets = _floyd_targets(rng, m, deg)
    c0 = rng.randint(c0_range[0], c0_range[1], m)
    return make_system(m, rule_neuron, i, j, c, p, targets, c0, name=name or f"random_{mode}_seed{seed}",
                       meta={"seed": seed, "mode": mode})


def random_64(seed: int = 1) -> SnpSystem:
    """64 neurons, 2-3 rules each, out-degree 4, initial spikes U[0,6]."""
    return random_system(seed, 64, (2, 3), (4, 4), (0, 6), "sparse", name=f"random64_seed{seed}")


def dense_1024(seed: int = 3) -> SnpSystem:
    """1024 neurons, 4 rules each (4096 rules), out-degree 64, M_Pi in [-8, 8],
    initial spikes U[0,16]."""
    return random_system(seed, 1024, (4, 4), (64, 64), (0, 16), "dense", name=f"dense1024_seed{seed}")


def batch_systems(n: int = 4096, base_seed: int = 1000) -> List[SnpSystem]:
    """n independent systems; system s has seed base_seed + s, neurons U[16,256],
    1-4 rules per neuron, out-degree U[2,8] per neuron, otherwise as random_64."""
    return [random_system(base_seed + s, (16, 256), (1, 4), (2, 8), (0, 6), "sparse", name=f"batch_s{s}")
            for s in range(n)]


@dataclass
class Request:
    idx: int
    arrival_s: float
    seed: int
    depth: int

    def system(self) -> SnpSystem:
        """Neurons U[8,512], 2-3 rules each, out-degree 4, otherwise as random_64."""
        return random_system(self.seed, (8, 512), (2, 3), (4, 4), (0, 6), "sparse", name=f"req{self.idx}")


def serving_requests(n: int, rate_per_s: float, seed: int = 4,
                     depth_range: Tuple[int, int] = (4, 32)) -> List[Request]:
    """A Poisson stream: exponential inter-arrival gaps of mean 1/rate, depth
    U[depth_range]; request k's system has seed 10**7 + k."""
    rng = Rng(seed)
    gaps = -np.log1p(-rng.uniform(n)) / float(rate_per_s)
    arrivals = np.cumsum(gaps)
    depths = rng.randint(depth_range[0], depth_range[1], n)
    return [Request(k, float(arrivals[k]), 10 ** 7 + k, int(depths[k])) for k in range(n)]
