"""Writes the oracle-derived expected values under tests/golden/.

Calls only the CPU oracle (oracle/) and the seeded input generator
(snp_synth); nothing here touches the CUDA simulator.  Each case stores the
exploration's per-depth statistics and a SHA-256 digest of the
discovery-ordered configurations (int32, little endian, row-major), so the
GPU tests can check full-size runs bit for bit without re-running the oracle.

    python tests/golden/make_golden.py [case ...]
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import snp_synth  # noqa: E402

OUT = os.path.join(HERE, "oracle_digests.json")

# name -> (system factory, exploration parameters)
CASES = {
    # the 64-neuron workload at full size (depth 8, cap 2^20, budget 2^24)
    "random64_seed1_full": (lambda: snp_synth.random_64(1), dict(depth=8, cap=1 << 20, budget=1 << 24)),
    # the same system, smaller: several chunks and a ragged tail at every depth
    "random64_seed1_small": (lambda: snp_synth.random_64(1), dict(depth=4, cap=1 << 14, budget=1 << 18)),
    # the 1024-neuron system, reduced cap and budget
    "dense1024_seed3_small": (lambda: snp_synth.dense_1024(3), dict(depth=3, cap=1 << 10, budget=1 << 13)),
}


def digest(configs: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(configs, dtype="<i4").tobytes()).hexdigest()


def run_case(name: str) -> dict:
    make, params = CASES[name]
    system = make()
    t = time.time()
    e = oracle.Oracle(system).explore(params["depth"], cap=params["cap"], budget=params["budget"])
    dt = time.time() - t
    assert e.error == 0
    return {
        "system": system.name,
        "params": params,
        "count": int(e.configs.shape[0]),
        "depth_reached": e.depth_reached,
        "per_depth": [[d.new, d.examined, str(d.candidates), d.truncated] for d in e.depths],
        "sha256": digest(e.configs),
        "oracle_seconds": round(dt, 2),
    }


def main(names):
    data = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            data = json.load(f)
    for name in names or list(CASES):
        print(f"{name} ...", flush=True)
        data[name] = run_case(name)
        print(json.dumps(data[name]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
