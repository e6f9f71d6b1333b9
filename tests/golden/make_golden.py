"""Writes the stored expected values of this folder from ``oracle/`` only.

Run from the repository root:  python tests/golden/make_golden.py
"""
import pathlib
import sys

ROOT = pathlib.Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

from oracle import closed_forms as CF  # noqa: E402


def main():
    here = pathlib.Path(__file__).resolve().parent
    row = CF.disc_row((0.5, 0.0), 32, 0.0)
    with open(here / "poisson_disc_arcs.txt", "w") as f:
        f.write("# mu_x(arc j), unit disc, K = I, x = (0.5, 0), 32 arcs of\n")
        f.write("# [2 pi j / 32, 2 pi (j+1) / 32); Poisson kernel of the ball\n")
        f.write("# (paper Sec. 1) integrated in closed form.\n")
        for j, v in enumerate(row):
            f.write(f"{j:2d} {v:.15f}\n")


if __name__ == "__main__":
    main()
