"""Write the stored oracle outputs used by the tests (calls only ``oracle``).

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2307_11248_gb300 import instances  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    w = instances.workload_sym12()
    out = oracle.run_walks(w["F"], w["D"], w["walks"], seed=w["seed"], descend=True)
    sub_opt, _ = oracle.brute_force(w["F"][:9, :9], w["D"][:9, :9])
    g = dict(
        workload="n=12 symmetric uniform [0,99], 2opt from 32 random starts (seed 1001)",
        F_sum=int(w["F"].sum()), D_sum=int(w["D"].sum()),
        best_cost=out["best_cost"].tolist(), moves=out["descent_moves"].tolist(),
        hash=[int(h) for h in out["descent_hash"]],
        sub9_optimum=int(sub_opt),
    )
    with open(os.path.join(HERE, "sym12_2opt.json"), "w") as f:
        json.dump(g, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
