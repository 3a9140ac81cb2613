"""Why there is no FP8 cost-tile mode: the exponent of the Sinkhorn operator
on c_Gamma (Eq. sinkhorn_operators with the bilinear cost of the Remark after
Theorem 3.2) is z_ij = (h_j + 16 <X_i, V_j> + 4 s_i t_j) / eps.  With X and
V = Gamma Y rounded to e4m3 (3 mantissa bits) under a per-tile scale (one
scale per 16 rows across the feature dimension, the finest tile a block-
scaled FP8 MMA takes), every product X_ik V_jk carries a relative error of
about 2 x 2^-4, so on lifted features the exponent of each plan entry is off
by whole units already at eps = 0.1, and the error grows as 1 / eps.  The
split f16 form the library runs (hi + lo halves, three products) stays below
1e-3 units on the same data.

CPU only: the oracle's Kernel PCA features and its softmin, with the operand
rounding applied in the test."""

import numpy as np

import oracle as O
import workloads as W

LOG2E = 1.4426950408889634


def round_e4m3(x):
    """Round to the nearest e4m3 value (bias 7: normals down to 2^-6 with 3
    mantissa bits, subnormals in steps of 2^-9, largest finite 448); ties to
    even.  |x| <= 448 is assumed (the per-tile scale guarantees it)."""
    ax = np.abs(x)
    e = np.maximum(np.floor(np.log2(np.maximum(ax, 2.0 ** -9))), -6.0)
    step = 2.0 ** (e - 3.0)
    return np.sign(x) * np.minimum(np.round(ax / step) * step, 448.0)


def per_tile_e4m3(A, rows=16):
    """A rounded to e4m3 with one scale per tile of `rows` rows (max |tile|
    mapped to 448), then scaled back."""
    out = np.empty_like(A)
    for r0 in range(0, A.shape[0], rows):
        T = A[r0:r0 + rows]
        mx = np.abs(T).max()
        sc = 448.0 / mx if mx > 0 else 1.0
        out[r0:r0 + rows] = round_e4m3(T * sc) / sc
    return out


def split_f16(A):
    """hi = f16(A), lo = f16(A - hi): the library's split 16-bit operands."""
    hi = A.astype(np.float16).astype(np.float64)
    lo = (A - hi).astype(np.float16).astype(np.float64)
    return hi, lo


def test_e4m3_rounding_grid():
    assert round_e4m3(np.array([1.0, 1.0625, 1.0626, 1.1875, 448.0, 2.0 ** -9, 3 * 2.0 ** -10]))\
        .tolist() == [1.0, 1.0, 1.125, 1.25, 448.0, 2.0 ** -9, 2.0 ** -8]
    # every normal binade holds 8 values (1.94 and above round up to 2)
    v = np.unique(round_e4m3(np.linspace(1.0, 1.93, 1000)))
    assert len(v) == 8 and v.max() == 1.875


def lifted_case(n=500, D=32, seed=0):
    """Kernel PCA features of ||x - x'|| on the 8-blob clouds and the Gamma
    of an annealed oracle solve (6 outer steps, eps 0.1 -> 0.01)."""
    w = W.gmm_rigid(n, seed=seed)
    a = np.full(n, 1.0 / n)
    X = O.lift(w["x"], a, "power", 1.0, D=D)["X"]
    Y = O.lift(w["y"], a, "power", 1.0, D=D)["X"]
    res = O.cnt_gw(a, a, X, Y, 0.1, 6, 40, eps_final=0.01, symmetric=True, record=False)
    return X, Y, res["Gamma"], a


def test_fp8_exponent_error_is_whole_units_and_grows_as_one_over_eps():
    X, Y, Gamma, a = lifted_case()
    V = Y @ Gamma.T
    exact = X @ V.T
    Xq, Vq = per_tile_e4m3(X), per_tile_e4m3(V)
    d8 = np.abs(Xq @ Vq.T - exact)
    Xh, Xl = split_f16(X)
    Vh, Vl = split_f16(V)
    d16 = np.abs(Xh @ Vh.T + Xh @ Vl.T + Xl @ Vh.T - exact)
    for eps in (0.1, 0.01, 0.001):
        alpha = 16.0 * LOG2E / eps                  # base-2 units of the exponent
        rms8 = alpha * np.sqrt(np.mean(d8 ** 2))
        rms16 = alpha * np.sqrt(np.mean(d16 ** 2))
        assert rms16 < 1e-5 * (0.1 / eps), (eps, rms16)        # ~2.3e-6 units at eps = 0.1
        assert rms8 > 0.1 * (0.1 / eps), (eps, rms8)           # ~0.16 units at 0.1, ~16 at 1e-3
        assert rms8 > 1e4 * rms16


def test_fp8_softmin_misses_the_fp32_bar():
    """The row softmin at eps = 0.01 with e4m3 operands misses the derived
    FP32 bound by more than three orders of magnitude."""
    from helpers import softmin_tolerance
    X, Y, Gamma, a = lifted_case()
    V = Y @ Gamma.T
    s, t = (X * X).sum(1), (Y * Y).sum(1)
    eps = 0.01
    h = np.zeros(len(Y))
    logw = np.log(a)
    C = -16.0 * X @ V.T - 4.0 * np.outer(s, t)
    Cq = -16.0 * per_tile_e4m3(X) @ per_tile_e4m3(V).T - 4.0 * np.outer(s, t)
    f = O.softmin(eps, logw, h, C)
    fq = O.softmin(eps, logw, h, Cq)
    tol = softmin_tolerance(X, V, s, t, h, logw, eps)
    assert np.abs(fq - f).max() > 1e3 * tol.max()
