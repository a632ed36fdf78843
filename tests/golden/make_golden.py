"""Write the stored expected values under tests/golden/ from the oracle only.

The paper prints no worked numerical example for the projection, so the stored
values are the oracle's own, kept as a regression lock:
  bounds_alpha0.9.txt   cS per side L = 1..12 at alpha = 0.9 for the per-window
                        fourth-root rule of Sec. 2.1 and for the exact chi^2
                        quantile (pinned separately against scipy in the tests).
Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    sides = list(range(1, 13))
    per = oracle.bounds(sides, 0.9, oracle.PERSET)
    chi = oracle.bounds(sides, 0.9, oracle.CHI2)
    with open(os.path.join(HERE, "bounds_alpha0.9.txt"), "w") as f:
        f.write("# cS = 1/c_s(alpha) per window side L at alpha = 0.9 (Sec. 2.1)\n")
        f.write("# columns: L  perset=(Phi^-1(alpha)*sigma_s+mu_s)^4  chi2=chi2_{L^2} quantile\n")
        for L, a, b in zip(sides, per, chi):
            f.write(f"{L} {a:.15e} {b:.15e}\n")


if __name__ == "__main__":
    main()
