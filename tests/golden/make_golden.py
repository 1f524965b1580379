"""Writes exact_logz.txt from oracle.exact only (transfer matrix, brute force,
Kac-Ward determinant).

Run from the repository root:  python tests/golden/make_golden.py
Each line: name Lx Ly beta couplings seed method logZ
The config-1 value (6x6 ferromagnet, beta = 0.44) is the exact transfer-matrix
ln Z of the Ising partition function of Sec. 7.1; the config-2 values (32x32
Gaussian spin glass, beta = 0.5, instances 0..7, seed 2 * 10^6 + i) are the
Kac-Ward determinant's.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exact  # noqa: E402
from workloads import ising  # noqa: E402

CASES = [
    ("config1_6x6_ferro", 6, 6, 0.44, "ferro", 0, "tm"),
    ("lattice_4x4_ferro", 4, 4, 0.44, "ferro", 0, "bf"),
    ("lattice_2x2_ferro", 2, 2, 0.44, "ferro", 0, "bf"),
    ("glass_4x5_gauss_b0.5", 4, 5, 0.5, "gauss", 2000017, "bf"),
    ("glass_6x6_gauss_b0.5", 6, 6, 0.5, "gauss", 2000000, "tm"),
    ("glass_8x6_pm1_b0.7", 8, 6, 0.7, "pm1", 11, "tm"),
] + [(f"config2_32x32_gauss_i{i}", 32, 32, 0.5, "gauss", 2000000 + i, "kw") for i in range(8)]


def main():
    lines = ["# name Lx Ly beta couplings seed method logZ   (written by make_golden.py)"]
    for name, Lx, Ly, beta, cp, seed, method in CASES:
        w = ising.lattice2d(Lx, Ly, beta, cp, seed=seed)
        if method == "tm":
            z = exact.ising_logz_transfer_matrix(Lx, Ly, w["edges"], w["J"], beta)
        elif method == "kw":
            z = exact.ising_logz_kac_ward(Lx, Ly, w["edges"], w["J"], beta)
        else:
            z = exact.ising_logz_bruteforce(w["n"], w["edges"], w["J"], beta)
        lines.append(f"{name} {Lx} {Ly} {beta} {cp} {seed} {method} {z!r}")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exact_logz.txt")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
