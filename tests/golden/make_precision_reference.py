"""Write tests/golden/precision_rotor256_q27.json: the FP64 oracle's per-step
force and torque on the D3Q27 128x128x256 rotor sub-run (R = 32, TSR 7,
1000 steps) -- the reference of the 16-bit population-storage study.

Calls only ``oracle`` and ``workloads`` (seeded inputs); run from the repo root:

    python tests/golden/make_precision_reference.py [--steps 1000]
"""

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--out", default=os.path.join(ROOT, "tests", "golden", "precision_rotor256_q27.json"))
    args = ap.parse_args()
    wl = W.workload("rotor256_q27")
    o = O.from_workload(wl)
    F, M = [], []
    t0 = time.time()
    for k in range(args.steps):
        o.step(1)
        f, m, _, _ = o.forces()
        F.append([float(v) for v in f[0]])
        M.append([float(v) for v in m[0]])
        if (k + 1) % 100 == 0:
            print(f"step {k + 1}: thrust {f[0][wl.flow_axis]:.6f} torque {m[0][wl.flow_axis]:.6f} "
                  f"({time.time() - t0:.0f} s)", flush=True)
    a = wl.flow_axis
    half = args.steps // 2
    out = {
        "_source": "FP64 oracle (oracle/hlbm_oracle.c) written by tests/golden/make_precision_reference.py",
        "workload": "rotor256_q27", "note": wl.note, "q": wl.q, "shape": [wl.nx, wl.ny, wl.nz],
        "steps": args.steps, "flow_axis": a, "average_from_step": half,
        "thrust_mean": sum(f[a] for f in F[half:]) / (args.steps - half),
        "torque_mean": sum(m[a] for m in M[half:]) / (args.steps - half),
        "force": F, "torque_vector": M,
    }
    with open(args.out, "w") as fh:
        json.dump(out, fh)
    print("wrote", args.out, "thrust_mean", out["thrust_mean"], "torque_mean", out["torque_mean"])


if __name__ == "__main__":
    main()
