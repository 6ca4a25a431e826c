"""Write paper_2106_13281_gb300/data/alg_flops.json: the algorithmic flop count
per environment step of each scene (forward, and the reverse pass as the
tape's reverse-op count: 2 flops per tape edge plus the flops that formed
the local partials), from the oracle's flop-counting scalar
(add/sub/mul/div/sqrt/atan2/min/max = 1 flop; every listed collision pair is
detected every substep; contact response counted for active contacts only).

The sample follows the benchmark recipe of each scene (seeded initial
conditions and uniform[-1,1] actions) over a full-length horizon, so the
mean number of active contacts matches the measured workload.

Usage: python oracle/count_flops.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

from oracle import oracle as orc  # noqa: E402
from paper_2106_13281_gb300 import scenes as S  # noqa: E402

SAMPLES = {  # scene: (envs, steps, seed, height jitter)
    "quadruped": (64, 1000, 1, 0.05),
    "biped": (16, 1000, 2, 0.0),
    "pendulum": (64, 200, 4, 0.0),
    "arm_box": (32, 200, 4, 0.0),
}


def main():
    out = {}
    for name, (N, T, seed, jit) in SAMPLES.items():
        d = S.SCENES[name]()
        rp, rr, ang = S.initial_conditions(d, N, seed, height_jitter=jit)
        st = orc.default_qp(d, N, rp, rr, ang)
        a = S.actions(d, N, T, seed).astype(np.float64)
        counts, n_active = orc.flops(d, st, a)
        es = N * T
        # reverse pass: the tape's reverse-op count on a shorter slice of the
        # same sample (the tape of a long rollout is large)
        Nr, Tr = min(N, 8), min(T, 50)
        rev, nodes = orc.reverse_flops(d, st[:Nr], a[:Tr, :Nr])
        total = sum(counts.values())
        resp = counts["response"]
        out[name] = {
            "flops_per_env_step": total / es,
            "by_category_per_env_step": {k: v / es for k, v in counts.items()},
            "active_contacts_per_substep": n_active / es / d["substeps"],
            "response_flops_per_active_contact": resp / n_active if n_active else 0.0,
            "sample": f"{N} envs x {T} steps, seed {seed}",
            "reverse_flops_per_env_step": rev / (Nr * Tr),
            "reverse_sample": f"{Nr} envs x {Tr} steps (tape: {nodes / (Nr * Tr):.0f} nodes per env-step)",
        }
        print(name, round(total / es), "flops/env-step forward,", round(rev / (Nr * Tr)), "reverse", flush=True)
    path = os.path.join(ROOT, "paper_2106_13281_gb300", "data", "alg_flops.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
