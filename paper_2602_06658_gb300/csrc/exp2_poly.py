"""Coefficients of the polynomial used for part of the exp2 evaluations in the
tensor-core softmin (instead of the MUFU unit).

2^x = 2^n * 2^f with n = round(x), f = x - n in [-1/2, 1/2].  2^f is
approximated by the degree-5 polynomial that interpolates it at the six
Chebyshev nodes of [-1/2, 1/2] (Chebyshev interpolation, a near-minimax
method; e.g. Trefethen, "Approximation Theory and Approximation Practice",
ch. 4 and 16).  The factor 2^n is applied by adding n to the exponent field.

Run `python exp2_poly.py` to print the coefficients (lowest degree first) as
they appear in gw_softmin_tc.cu, and their maximum relative error in FP32
Horner evaluation.
"""

import numpy as np

DEGREE = 5


def coefficients(degree: int = DEGREE) -> np.ndarray:
    k = np.arange(degree + 1)
    nodes = 0.5 * np.cos((2 * k + 1) * np.pi / (2 * (degree + 1)))
    V = np.vander(nodes, degree + 1, increasing=True)
    return np.linalg.solve(V, 2.0 ** nodes)


def horner32(c, f):
    c32 = np.asarray(c, np.float32)
    f32 = np.asarray(f, np.float32)
    p = np.full_like(f32, c32[-1])
    for ci in c32[-2::-1]:
        p = (p * f32 + ci).astype(np.float32)
    return p


def max_rel_error(c) -> float:
    f = np.linspace(-0.5, 0.5, 400001)
    return float(np.abs(horner32(c, f).astype(np.float64) / 2.0 ** f - 1.0).max())


if __name__ == "__main__":
    c = coefficients()
    print(", ".join(f"{np.float32(v)!r}f".replace("np.float32(", "").replace(")", "") for v in c))
    print("max relative error:", max_rel_error(c))
