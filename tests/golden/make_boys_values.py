"""Writes boys_mpmath.txt: the Boys function
    F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt
(Boys 1950) for m = 0..8 on a grid of T in [0, 200], by the oracle's mpmath
quadrature of that definition at 40 significant digits.  The grid covers
T = 0, tiny T, both sides of interpolation-table boundaries (multiples of
1/32 near 0, 1 and 10; 39.97-40.03) and the asymptotic range up to 200.

  python tests/golden/make_boys_values.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import boys_quadrature  # noqa: E402

T_GRID = ([0.0, 1e-14, 1e-9, 1e-6, 1e-4, 0.01, 0.0312, 0.03125, 0.0313, 0.0625, 0.09, 0.5, 0.999,
           1.0, 1.03125, 2.5, 5.0, 7.7, 10.0, 10.03125, 15.0, 20.0, 25.3, 29.9, 30.0, 30.1, 35.0,
           39.97, 39.99, 40.0, 40.01, 40.03, 45.0, 60.0, 80.0, 120.0, 200.0])


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "boys_mpmath.txt")
    with open(out, "w") as fh:
        fh.write("# Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt, mpmath quadrature at 40 digits\n")
        fh.write("# written by make_boys_values.py (oracle.boys_quadrature); columns: T m F_m(T)\n")
        for T in T_GRID:
            for m in range(9):
                fh.write(f"{T!r} {m} {boys_quadrature(m, T)}\n")


if __name__ == "__main__":
    main()
