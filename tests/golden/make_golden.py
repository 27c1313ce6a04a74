"""Writes tests/golden/filters.txt from the oracle only.

The paper prints no filter coefficient and no worked example, so the stored
values are the oracle's own derivation (80-digit arithmetic, rounded once to
FP64), kept to catch any drift of that derivation across machines or edits.
Run: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle.filters as F  # noqa: E402


def main():
    w, k0 = F.magic()
    lines = ["# Daubechies-16 least-asymmetric filters (oracle derivation), FP64 hex",
             "# h_j, g_j: j = -7..8 (Eq. refinement); w_k: k = k0..k0+15 "
             "(Eq. magicfilter); a_l: l = -14..14 (Eqs. kiner, fprod)",
             f"k0 {k0}"]
    for name, arr in (("h", F.h()), ("g", F.g()), ("w", w), ("a", F.kinetic_a())):
        lines.append(name + " " + " ".join(float(v).hex() for v in arr))
    with open(os.path.join(HERE, "filters.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
