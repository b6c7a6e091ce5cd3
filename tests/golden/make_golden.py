"""Writes the stored expected values under tests/golden/ from the oracle alone.

  python tests/golden/make_golden.py

zolotarev_n12_1e-5.txt: Zolotarev's best relative approximation of x^-1/2 on
[1e-5, 1] with 12 poles (the rational approximation of Sec. 4.2 in the range
the heavy-doublet benchmark uses), from oracle.rational.zolotarev_inv_sqrt,
whose construction is pinned by Chebyshev alternation in
tests/test_oracle_rational.py.  Columns: a0 on the first line, then
(a_k, sigma_k) per pole, then delta.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import rational as RA  # noqa: E402


def main():
    a0, a, sigma, delta = RA.zolotarev_inv_sqrt(12, 1e-5, 1.0)
    with open(os.path.join(HERE, "zolotarev_n12_1e-5.txt"), "w") as f:
        f.write("# x^-1/2 on [1e-5, 1], 12 poles: a0 / (a_k sigma_k) x 12 / delta; oracle.rational\n")
        f.write(f"{a0:.17e}\n")
        for ak, sk in zip(a, sigma):
            f.write(f"{ak:.17e} {sk:.17e}\n")
        f.write(f"{delta:.17e}\n")


if __name__ == "__main__":
    main()
