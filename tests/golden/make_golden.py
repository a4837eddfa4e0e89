"""Write the stored expected values under tests/golden/ from the FP64 oracle.

Only the oracle and the seeded input generators are called here.  Each
fixture names the passage of Kuzma et al. it comes from.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2305_18236_gb300 import inputs  # noqa: E402


def listing1():
    """The tile product of Listing 1 (Section 3.2): an 8x5 ATile times a
    5x16 BTile gives an 8x16 result (mr = 8, kr = 5, nr = 16).  Integer
    inputs make every entry exact in FP32; alpha = 1.5, beta = 0.5 exercise
    Algorithm 1's scaling."""
    A = inputs.integers((8, 5), 101)
    B = inputs.integers((5, 16), 102)
    C0 = inputs.integers((8, 16), 103)
    C, _, _ = oracle.gemm(A, B, 1.5, 0.5, C0)
    return {
        "cite": "Kuzma et al., Section 3.2, Listing 1 (8x5 . 5x16 tile); Algorithm 1 (alpha, beta)",
        "M": 8, "N": 16, "K": 5, "alpha": 1.5, "beta": 0.5,
        "A": A.tolist(), "B": B.tolist(), "C0": C0.tolist(), "C": C.tolist(),
    }


def main():
    path = os.path.join(HERE, "listing1_8x5x16.json")
    with open(path, "w") as f:
        g = listing1()
        rows = []
        for k, v in g.items():
            if isinstance(v, list):
                rows.append(" %s: [\n%s\n ]" % (json.dumps(k), ",\n".join("  " + json.dumps(r) for r in v)))
            else:
                rows.append(" %s: %s" % (json.dumps(k), json.dumps(v)))
        f.write("{\n" + ",\n".join(rows) + "\n}\n")
    print(path)


if __name__ == "__main__":
    main()
