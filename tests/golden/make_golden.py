"""Writes the regression fixtures in this folder. Calls only the oracle package.

Run from the repository root:  python tests/golden/make_golden.py
maxwell.json: equal-area coexistence of the Peng-Robinson EOS (Eq. 10, a = 2/49, b = 2/21, R = 1,
acentric factor 0.344, Sec. 2.2) and of Carnahan-Starling (a = 1, b = 4) at the listed reduced
temperatures.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    rows = []
    for eos, Tr in [(0, 0.6), (0, 0.7), (0, 0.8), (1, 0.7)]:
        m = oracle.maxwell(eos, Tr)
        rows.append({"eos": eos, "Tr": Tr, **{k: float(v) for k, v in m.items()}})
    with open(os.path.join(HERE, "maxwell.json"), "w") as f:
        json.dump({"source": "oracle.maxwell (equal-area construction, Eq. 10-11)",
                   "rows": rows}, f, indent=1)


if __name__ == "__main__":
    main()
