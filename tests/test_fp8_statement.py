"""The FP8 mode's rounding model and its error statement, on the CPU.

GW_PREC_FP8 rounds the feature operands of the softmin's exponent
z_ij = (h_j + 16 <X_i, V_j> + 4 s_i t_j) / eps (the Sinkhorn operator on
c_Gamma, Eq. sinkhorn_operators with the bilinear cost of the Remark after
Theorem 3.2) to e4m3 (3 mantissa bits) under one power-of-two scale per
source row and per 128-row tile of V.  The GPU parity tests compare the mode
with the oracle on operands rounded by helpers.fp8_operands; these tests pin
that emulation to the e4m3 format's definition, and state the error the
rounding itself costs: every product X_ik V_jk carries a relative error of
about 2 x 2^-4, so on lifted features the exponent of each plan entry is off
by whole units already at eps = 0.1 and the error grows as 1 / eps, while the
split f16 form stays below 1e-3 units on the same data.

CPU only: the oracle's Kernel PCA features and its softmin, with the operand
rounding applied in the test."""

import numpy as np

import oracle as O
import workloads as W
from helpers import e4m3_group_scale, fp8_operands, round_e4m3

LOG2E = 1.4426950408889634


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


def test_e4m3_group_scale_is_the_largest_power_of_two():
    for m in (448.0, 449.0, 224.0, 392.0, 393.0, 1.0, 3.5e-3, 7.0e4, 2.0 ** -60):
        c = e4m3_group_scale(m)
        assert c == 2.0 ** round(np.log2(c))                 # a power of two
        if 2.0 ** -30 <= m <= 2.0 ** 30:                    # away from the clamp
            assert m * c <= 448.0 < 2.0 * m * c, (m, c)
    assert e4m3_group_scale(448.0) == 1.0 and e4m3_group_scale(449.0) == 0.5
    assert e4m3_group_scale(392.0) == 1.0 and e4m3_group_scale(0.875) == 512.0
    assert e4m3_group_scale(0.0) == 1.0 and e4m3_group_scale(np.inf) == 1.0
    assert e4m3_group_scale(2.0 ** -60) == 2.0 ** 40           # clamped


def e4m3_codes():
    """Every finite e4m3 value with its code, decoded from the bit layout:
    sign, 4 exponent bits (bias 7), 3 mantissa bits; exponent field 0 is
    subnormal (m / 8 * 2^-6); S.1111.111 is NaN.  (+0 and -0 both map to 0.)"""
    out = {}
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        out.setdefault(-v if s else v, code)
    return out


def e4m3_table():
    return np.array(sorted(e4m3_codes()))


def test_round_e4m3_is_the_nearest_table_value():
    T = e4m3_table()
    assert len(T) == 253 and T.max() == 448.0 and T[T > 0].min() == 2.0 ** -9
    g = W.rng(11)
    x = np.concatenate([g.uniform(-448, 448, 4000), g.uniform(-0.05, 0.05, 4000),
                        (T[:-1] + T[1:]) / 2.0])               # every midpoint: a tie
    r = round_e4m3(x)
    assert np.isin(r, T).all()
    d = np.abs(x[:, None] - T[None, :])
    best = d.min(axis=1)
    assert np.all(np.abs(r - x) == best)
    # ties go to the even mantissa (code's lowest bit 0)
    codes = e4m3_codes()
    mids = (T[:-1] + T[1:]) / 2.0
    for v, a, b in zip(round_e4m3(mids), T[:-1], T[1:]):
        assert v in (a, b) and codes[v] % 2 == 0, (a, b, v)


def test_fp8_operands_follow_the_format():
    """Scaled back, every operand value is an e4m3 table value, the nearest
    one to the scaled input; each 128-row group reaches at least 224 (its
    power-of-two scale is the largest); a matrix rounds the same on either
    side of the product."""
    T = e4m3_table()
    g = W.rng(3)
    A = np.asarray(g.standard_normal((300, 20)) * np.exp(g.uniform(-6, 2, (300, 1))), np.float32)
    B = np.asarray(g.standard_normal((300, 20)) * 0.1, np.float32)
    Ah, Bh, ca, cb = fp8_operands(A, B, 0.05, scales=True)
    Bh2, Ah2 = fp8_operands(B, A, 0.01)
    assert np.array_equal(Ah, Ah2) and np.array_equal(Bh, Bh2)
    groups = np.arange(300) // 128
    for X, Xh, c in ((A, Ah, ca), (B, Bh, cb)):
        q8 = Xh * c[:, None]                                   # the e4m3 values
        assert np.isin(q8, T).all()
        x = np.asarray(X, np.float64) * c[:, None]
        nearest = np.abs(x[..., None] - T).min(axis=-1)
        assert np.allclose(np.abs(q8 - x), nearest, rtol=1e-6, atol=1e-12)
        for q in np.unique(groups):
            mx = np.abs(q8[groups == q]).max()
            assert 224.0 <= mx <= 448.0, (q, mx)
            assert len(np.unique(c[groups == q])) == 1


def test_fp8_exponent_error_is_whole_units_and_grows_as_one_over_eps():
    X, Y, Gamma, a = lifted_case()
    V = Y @ Gamma.T
    exact = X @ V.T
    Xq, Vq = per_tile_e4m3(X), per_tile_e4m3(V)
    d8 = np.abs(Xq @ Vq.T - exact)
    # the scheme the mode runs (one scale per row of X and per 128 rows of V)
    Xm, Vm = fp8_operands(X, V, 0.01)
    dm = np.abs(Xm @ Vm.T - exact)
    Xh, Xl = split_f16(X)
    Vh, Vl = split_f16(V)
    d16 = np.abs(Xh @ Vh.T + Xh @ Vl.T + Xl @ Vh.T - exact)
    for eps in (0.1, 0.01, 0.001):
        alpha = 16.0 * LOG2E / eps                  # base-2 units of the exponent
        rms8 = alpha * np.sqrt(np.mean(d8 ** 2))
        rmsm = alpha * np.sqrt(np.mean(dm ** 2))
        rms16 = alpha * np.sqrt(np.mean(d16 ** 2))
        assert rms16 < 1e-5 * (0.1 / eps), (eps, rms16)        # ~2.3e-6 units at eps = 0.1
        assert rms8 > 0.1 * (0.1 / eps), (eps, rms8)           # ~0.16 units at 0.1, ~16 at 1e-3
        assert rmsm > 0.1 * (0.1 / eps), (eps, rmsm)
        assert rms8 > 1e4 * rms16 and rmsm > 1e4 * rms16


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
