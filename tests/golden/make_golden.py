"""Writes the oracle-derived expected values under tests/golden/.

Calls only the CPU oracle (oracle/) and the seeded input generator
(snp_synth); nothing here touches the CUDA simulator.  Each case stores the
exploration's per-depth statistics and a SHA-256 digest of the
discovery-ordered configurations (int32, little endian, row-major), so the
GPU tests can check full-size runs bit for bit without re-running the oracle.

    python tests/golden/make_golden.py [case ...]

The batch case ("batch4096_seed1000") explores every one of the 4096 systems
of the batch workload and stores one short digest per system in
tests/golden/batch4096_digests.json (run in parallel over the host's cores).
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
    # the 1024-neuron system at a cap that spans many passes of wide rows and
    # several tasks per warp (the full-size run is checked by sampled children)
    "dense1024_seed3_mid": (lambda: snp_synth.dense_1024(3), dict(depth=3, cap=1 << 16, budget=1 << 19)),
}

# The batch workload: 4096 systems (seed 1000 + s), depth 6, cap 2^12, budget 2^16.
BATCH = dict(n=4096, base_seed=1000, depth=6, cap=1 << 12, budget=1 << 16)
BATCH_OUT = os.path.join(HERE, "batch4096_digests.json")


def system_digest(configs: np.ndarray, per_depth) -> str:
    """First 24 hex digits of SHA-256 over the discovery-ordered configurations
    (int32, little endian) followed by the per-depth records (new, examined,
    candidates, truncated) as little-endian uint64."""
    h = hashlib.sha256(np.ascontiguousarray(configs, dtype="<i4").tobytes())
    h.update(np.asarray([[int(v) for v in d] for d in per_depth], dtype="<u8").tobytes())
    return h.hexdigest()[:24]


def _batch_one(s: int):
    system = snp_synth.batch_systems(1, BATCH["base_seed"] + s)[0]
    e = oracle.Oracle(system).explore(BATCH["depth"], cap=BATCH["cap"], budget=BATCH["budget"])
    assert e.error == 0
    per = [[d.new, d.examined, d.candidates, d.truncated] for d in e.depths]
    return s, int(e.configs.shape[0]), system_digest(e.configs, per)


def run_batch() -> None:
    import multiprocessing as mp
    t = time.time()
    out = [None] * BATCH["n"]
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for s, count, dig in pool.imap_unordered(_batch_one, range(BATCH["n"]), chunksize=8):
            out[s] = [count, dig]
    data = dict(BATCH, digest="system_digest in make_golden.py", systems=out,
                oracle_seconds=round(time.time() - t, 1), processes=os.cpu_count())
    with open(BATCH_OUT, "w") as f:
        json.dump(data, f, separators=(",", ":"))
    print(f"batch4096: {len(out)} systems in {data['oracle_seconds']} s", flush=True)


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
    names = names or list(CASES) + ["batch4096_seed1000"]
    if "batch4096_seed1000" in names:
        run_batch()
        names = [n for n in names if n != "batch4096_seed1000"]
    for name in names:
        print(f"{name} ...", flush=True)
        data[name] = run_case(name)
        print(json.dumps(data[name]), flush=True)
        with open(OUT, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main(sys.argv[1:])
