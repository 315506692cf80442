"""Writes the stored oracle results used by the GPU parity tests.

Calls only the oracle (oracle/) and the input generators; run from the repo
root:  python tests/golden/make_golden.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2203_11733_gb300 import workloads as W  # noqa: E402


def crossing_bus_2x2():
    boxes, params = W.crossing_bus_2x2()
    a, g, c = O.mesh_boxes(boxes, **params)
    t = time.time()
    A = O.assemble(a, g)
    C = O.capacitance_from_matrix(A, c, W.EPS_R_SIO2)
    out = {
        "what": "Maxwell capacitance matrix (F) of the 2x2 crossing bus, eps_r 3.9, computed by the FP64 oracle",
        "workload": "crossing_bus_2x2", "params": params, "n_panels": int(len(a)), "eps_r": W.EPS_R_SIO2,
        "oracle_seconds": round(time.time() - t, 1), "threads": O.max_threads(),
        "C": C.tolist(),
    }
    with open(os.path.join(HERE, "crossing_bus_2x2_capacitance.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("crossing_bus_2x2", len(a), out["oracle_seconds"], "s")


if __name__ == "__main__":
    crossing_bus_2x2()
