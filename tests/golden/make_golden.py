"""Writes the golden fixtures of this folder.  Calls only the oracle package.

    python tests/golden/make_golden.py

example1_laplace_8x6_10it.txt
    Example 1 of Sec. III-A (the CharmStencil 2D Laplace program) scaled
    down: boundary ring = 1 (set once by slice assignment and held),
    interior initially 0 (a fresh array), update
    u2[1:-1,1:-1] = 0.25*(N + S + W + E) for the 10 iterations the example
    runs, arrays swapped after each.  Interior 8 rows x 6 columns (the
    example's 16384^2 shrunk to a size that prints), evaluated in exact
    rational arithmetic; values are dyadic, so they are written as exact
    fractions p/q.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.exact import sweep_exact_2d  # noqa: E402


def main():
    ny, nx, iters = 8, 6, 10
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    u = sweep_exact_2d([[0] * nx for _ in range(ny)], offs, ["1/4"] * 4, 1, iters)
    path = os.path.join(HERE, "example1_laplace_8x6_10it.txt")
    with open(path, "w") as f:
        f.write("# Example 1 (Sec. III-A): 2D Laplace Jacobi, boundary 1, interior 0,\n")
        f.write("# weights 1/4 on N,S,W,E, 10 iterations; interior 8x6 after 10 steps.\n")
        f.write("# Written by tests/golden/make_golden.py (exact rationals).\n")
        for row in u:
            f.write(" ".join(f"{v.numerator}/{v.denominator}" for v in row) + "\n")


if __name__ == "__main__":
    main()
