"""Writes the stored oracle results used by the GPU parity tests.

Calls only the oracle (oracle/) and the input generators; run from the repo
root:  python tests/golden/make_golden.py [name ...]
with names among: crossing_bus_2x2, bus_3layer_5x5x5, serving_seed31 (all of
them when none is given).
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


def _write(name, out):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)


def _structure(workload, boxes, params, eps_r, what):
    a, g, c = O.mesh_boxes(boxes, **params)
    t = time.time()
    A = O.assemble(a, g)
    t_asm = time.time() - t
    C = O.capacitance_from_matrix(A, c, eps_r)
    return {
        "what": what, "workload": workload, "params": params, "n_panels": int(len(a)), "eps_r": eps_r,
        "oracle_seconds": round(time.time() - t, 1), "oracle_assembly_seconds": round(t_asm, 1),
        "threads": O.max_threads(), "C": C.tolist(),
    }


def crossing_bus_2x2():
    boxes, params = W.crossing_bus_2x2()
    out = _structure("crossing_bus_2x2", boxes, params, W.EPS_R_SIO2,
                     "Maxwell capacitance matrix (F) of the 2x2 crossing bus, eps_r 3.9, computed by the FP64 oracle")
    _write("crossing_bus_2x2_capacitance.json", out)
    print("crossing_bus_2x2", out["n_panels"], out["oracle_seconds"], "s")


def bus_3layer_5x5x5():
    boxes, params = W.bus_3layer_5x5x5()
    out = _structure("bus_3layer_5x5x5", boxes, params, W.EPS_R_SIO2,
                     "Maxwell capacitance matrix (F) of the three-layer 5x5x5 crossing bus (15 conductors), "
                     "eps_r 3.9, computed by the FP64 oracle (full assembly and Cholesky)")
    _write("bus_3layer_5x5x5_capacitance.json", out)
    print("bus_3layer_5x5x5", out["n_panels"], out["oracle_seconds"], "s")


def serving_seed31():
    """Requests 0 and 1 of the serving test's stream (seed 31, ten requests,
    N log-uniform in [400, 2500])."""
    reqs = W.serving_requests(seed=31, count=10, rate_per_s=1000.0, n_lo=400, n_hi=2500)
    outs = []
    for k in range(2):
        _, boxes, params = reqs[k]
        o = _structure(f"serving_requests(seed=31, count=10, rate_per_s=1000, n_lo=400, n_hi=2500)[{k}]",
                       boxes, params, W.EPS_R_SIO2, "Maxwell capacitance matrix (F), FP64 oracle")
        o["request"] = k
        outs.append(o)
        print("serving_seed31", k, o["n_panels"], o["oracle_seconds"], "s")
    _write("serving_seed31_capacitance.json", {"requests": outs})


JOBS = {"crossing_bus_2x2": crossing_bus_2x2, "bus_3layer_5x5x5": bus_3layer_5x5x5,
        "serving_seed31": serving_seed31}

if __name__ == "__main__":
    for name in (sys.argv[1:] or list(JOBS)):
        JOBS[name]()
