"""Writes oracle_counts_1023.txt: the FP64 oracle's policy-iteration counts on
the 1023 x 1023 plain Isaacs workload (seed 2) and the wall time of that full
solve.  Calls only oracle/ (and the seeded generators); takes about three
minutes on one core.  bench.py scales its
bounded CPU sample (one policy evaluation + one improvement) by these counts.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.isaacs import isaacs_game  # noqa: E402

if __name__ == "__main__":
    t0 = time.time()
    res = oracle.policy_iteration(isaacs_game(1023, 0, seed=2))
    with open(os.path.join(HERE, "oracle_counts_1023.txt"), "w") as fh:
        fh.write("# FP64 oracle (Algorithm 2 with Algorithm 1, sparse LU) on the 1023^2 plain\n")
        fh.write("# Isaacs game, seed 2; written by make_oracle_counts.py\n")
        fh.write(f"outer {res.outer}\nsystems {res.systems}\n")
        fh.write(f"seconds {time.time() - t0:.1f}\n")
    print(f"outer {res.outer} systems {res.systems} residual {res.residual:.2e} "
          f"in {time.time() - t0:.0f} s")
