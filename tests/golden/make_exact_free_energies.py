"""Write exact ln Z(beta) of the periodic L x L Ising model (Kaufman's closed form, evaluated by
the oracle) for the learned-schedule evaluation: tests/golden/exact_lnZ.json.

    python tests/golden/make_exact_free_energies.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

BETAS = [0.25, 0.5, 0.75, 1.0]
LS = [8, 16, 32, 64, 128]

if __name__ == "__main__":
    out = {"source": "Kaufman / Ferdinand-Fisher closed form for the periodic L x L lattice, "
                     "oracle/exact_ising.c (pinned against enumeration and the transfer matrix)",
           "lnZ": {str(L): {repr(b): oracle.kaufman_lnZ(L, b) for b in BETAS} for L in LS}}
    with open(os.path.join(HERE, "exact_lnZ.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
