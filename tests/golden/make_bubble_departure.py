"""Writes bubble_departure.json: the step at which the first bubble departs from the heated wall in the
FP64 oracle, for the bubble_departure workload (Sec. IV B: a bubble nucleates over the heated part of
the wall, grows, detaches and leaves a small attached bubble behind).

Departure is the first step after which a vapour region under the free surface no longer touches the
wall (tests.helpers.departed_bubble). The oracle is checked every 25 steps; the 25 steps before the
first detection are then replayed one at a time from a saved state. Only oracle/ computes here.

    python -m tests.golden.make_bubble_departure
"""

import copy
import json
import os
import time

from oracle import model
from paper_1709_04400_gb300 import workloads

from tests.helpers import RL, RV, TC, departed_bubble, oracle_params

COARSE, MAX_STEPS = 25, 14000


def main():
    case, rho, T = workloads.bubble_departure(TC, RV, RL)
    p = oracle_params(case)
    s = model.init_state(p, rho, T)
    t0 = time.time()
    saved = copy.deepcopy(s)
    while s.step < MAX_STEPS:
        for _ in range(COARSE):
            s = model.step(p, s)
        if departed_bubble(model.fields(p, s)[0], case["surface"]):
            break
        saved = copy.deepcopy(s)
    else:
        raise SystemExit(f"no departure within {MAX_STEPS} steps")
    s = saved
    while True:
        s = model.step(p, s)
        area = departed_bubble(model.fields(p, s)[0], case["surface"])
        if area:
            break
    out = {
        "case": case["name"],
        "departure_step": s.step,
        "departed_area": area,
        "rule": "first step after which a vapour region under the free surface no longer touches the wall",
        "source": "FP64 oracle (oracle/model.py), written by tests/golden/make_bubble_departure.py",
        "cite": "Sec. IV B: bubble nucleation on the heated wall, growth, detachment, a small attached bubble left",
        "seconds": round(time.time() - t0, 1),
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "bubble_departure.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(out)


if __name__ == "__main__":
    main()
