"""Write the oracle's exact top list of the d = 3 headline workload.

The workload: one task, n = 1000 samples, m = 1000 monomial columns, seed 2,
planted three-term target with sigma = 0.01 (`workloads.CONFIGS["C2"]`).  The
oracle (Sec. 2.4: every 3-tuple fitted by Householder QR on the raw centred
columns, 166,167,000 fits) ranks all tuples by (SSE, lexicographic order);
the first 128 are written so that a tie group straddling position 100 can be
judged.  Only `oracle/` and `workloads/` are called.

    python tests/golden/make_c2_top.py [--threads N]

Output: tests/golden/c2_top128.txt, one line per rank:
    rank  i  j  k  SSE (17 significant digits)  RMSE
"""

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from workloads import make_config  # noqa: E402

K_WRITTEN = 128
OUT = os.path.join(HERE, "c2_top128.txt")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    a = ap.parse_args()
    prob, d, k = make_config("C2")
    t0 = time.time()
    res = oracle.fit(prob.X, prob.y, d, K_WRITTEN, n_threads=a.threads)
    dt = time.time() - t0
    with open(OUT, "w") as f:
        f.write("# Oracle top-%d of the d=3, n=1000, m=1000 workload (seed 2, planted 3-term\n"
                "# target, sigma 0.01): exhaustive Householder-QR fits of all C(1000,3) tuples\n"
                "# (Sec. 2.4), ranked by (SSE, lexicographic order).  Written by\n"
                "# tests/golden/make_c2_top.py, which calls only oracle/ and workloads/.\n"
                "# planted columns: %s\n"
                "# columns: rank i j k SSE RMSE\n" % (K_WRITTEN, sorted(prob.planted[0])))
        for r in range(K_WRITTEN):
            t = res["tuples"][0][r]
            f.write("%d %d %d %d %.17e %.17e\n" % (r, t[0], t[1], t[2], res["score"][0][r],
                                                  res["rmse"][0][r]))
    print("wrote %s in %.1f s" % (OUT, dt))


if __name__ == "__main__":
    main()
