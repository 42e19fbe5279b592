"""Writes tests/golden/water_dfjk.json from the oracle alone (the paper prints
no worked example for this path).  Run: python tests/golden/make_golden.py"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2404_09452_gb300 import inputs as I  # noqa: E402


def main():
    m = I.water()
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, 5, 3000), S)
    r = O.dfjk(m.orb, m.aux, m.coords, C)
    out = {
        "what": "DF-J/K of the 3-atom water input (nao 18, naux 30, nocc 5), FP64 oracle",
        "E_J": r["E_J"],
        "E_K": r["E_K"],
        "J": r["J"].tolist(),
        "K": r["K"].tolist(),
    }
    with open(os.path.join(HERE, "water_dfjk.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
