"""Writes prism_rules_table1.txt: the symmetric triangle rules of the paper's
prism rules (Table 1, N_Q = 6 ... 336 = (p + 1) x 3 ... 42), found by the
oracle's own search (fem_oracle.c, orc_tri_search).

For each degree p the search runs seeded continuation paths and keeps every
distinct positive-interior rule; the stored one has the largest smallest
barycentric coordinate.  Only the oracle is called.

    python oracle/make_prism_rules.py        (about 15 minutes on 8 cores)
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402

TRIALS = {1: 2000, 2: 5000, 3: 20000, 4: 50000, 5: 100000, 6: 400000, 7: 1500000}
SEED = 1310


def main(path=os.path.join(HERE, "prism_rules_table1.txt")):
    lines = ["# Fully symmetric positive-interior triangle rules of degree 2p behind the",
             "# paper's prism rules (Table 1: N_Q = (p + 1) x n_points), found by",
             "# oracle.tri_search (written by oracle/make_prism_rules.py).",
             "# rule p n_points n0 n1 n2 n_found params...: orbit parameters in barycentric",
             "# coordinates -- centroid: w; S21 (a, a, 1-2a): a, w; S111 (a, b, 1-a-b): a, b, w.",
             "# found p trials seed n_found smallest barycentric coordinate of each rule found"]
    shapes = {1: (0, 1, 0), 2: (0, 2, 0), 3: (0, 2, 1), 4: (1, 3, 1), 5: (1, 2, 3), 6: (0, 5, 3), 7: (0, 6, 4)}
    for p in range(1, 8):
        t0 = time.time()
        sol, mb = oracle.tri_search(p, TRIALS[p], SEED)
        if len(sol) == 0:
            raise RuntimeError("no rule found for p = %d" % p)
        n0, n1, n2 = shapes[p]
        lines.append("found %d %d %d %d %s" % (p, TRIALS[p], SEED, len(sol), " ".join("%.10f" % v for v in mb)))
        lines.append("rule %d %d %d %d %d %d %s" % (p, n0 + 3 * n1 + 6 * n2, n0, n1, n2, len(sol),
                                                   " ".join("%.17g" % v for v in sol[0])))
        print("p=%d: %d rules, %.1f s" % (p, len(sol), time.time() - t0), flush=True)
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
