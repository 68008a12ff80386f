"""Writes oracle_L4_two_steps.txt: the FP64 oracle's energies, PT permutation and
overlap q^{mu nu} after two steps (1 HB + 5 OR + PT each) of a seeded L = 4
sample.  A regression record of the oracle's own arithmetic: the test re-runs
the oracle and compares.  Calls only the oracle and the input generators.

    python tests/golden/make_oracle_fixture.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1204_6192_gb300 import inputs  # noqa: E402


def run():
    smp = inputs.small_sample(4, n_temps=3, h_r=0.2, disorder_seed=3)
    sim = oracle.OracleSim([smp], 2, 7)
    sim.step(2)
    m = sim.measure()[0]
    return {"E": np.asarray(sim.energies()[0]), "perm": m["perm"].ravel(), "q": m["q"].ravel()}


def main():
    vals = run()
    with open(os.path.join(HERE, "oracle_L4_two_steps.txt"), "w") as f:
        f.write("# written by make_oracle_fixture.py (FP64 oracle, L = 4, 2 replicas x 3 "
                "temperatures, seed 7, two steps)\n")
        for k, v in vals.items():
            f.write(k + " " + " ".join(repr(float(x)) for x in v) + "\n")


if __name__ == "__main__":
    main()
