"""The exp2 polynomial of the tensor-core softmin (csrc/exp2_poly.py): its
coefficients in the kernel source equal the generator's, and the full FP32
emulation (rounding shift, Horner, exponent insertion) stays within the error
bound of ex2.approx (2^-22 relative) against 2^x in float64."""

import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2602_06658_gb300", "csrc")


def gen():
    spec = importlib.util.spec_from_file_location("exp2_poly", os.path.join(CSRC, "exp2_poly.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def kernel_coefficients():
    src = open(os.path.join(CSRC, "gw_softmin_tc.cu")).read()
    body = src[src.index("uint64_t exp2_fma_pair"):]
    body = body[: body.index("float p0, p1")]
    vals = re.findall(r"pack2\(([0-9.e-]+)f, \1f\)", body)
    # Horner order in the kernel: highest degree first
    return np.array([float(v) for v in vals if v not in ("-1.0",)], np.float64)[::-1]


def test_kernel_constants_match_generator():
    c = np.asarray(gen().coefficients(), np.float32).astype(np.float64)
    k = kernel_coefficients()
    assert len(k) == len(c)
    assert np.allclose(k, c, rtol=2e-7, atol=0)


def emulate(x):
    """The kernel's steps in numpy float32 / int32."""
    c = np.asarray(gen().coefficients(), np.float32)
    x = np.clip(np.asarray(x, np.float32), np.float32(-126.0), np.float32(126.0))
    shift = np.float32(12582912.0)
    t = (x + shift).astype(np.float32)
    n = (t - shift).astype(np.float32)
    f = (x - n).astype(np.float32)
    p = np.full_like(f, c[-1])
    for ci in c[-2::-1]:
        p = (p * f + ci).astype(np.float32)
    ni = t.view(np.int32) - np.int32(0x4B400000)
    return (p.view(np.int32) + (ni << 23)).view(np.float32)


def test_emulation_error_bound():
    x = np.concatenate([np.linspace(-126.0, 126.0, 2_000_001), np.linspace(-2, 2, 400_001)])
    y = emulate(x).astype(np.float64)
    rel = np.abs(y / 2.0 ** x.astype(np.float32).astype(np.float64) - 1.0)
    assert rel.max() <= 2.0 ** -21, rel.max()
    assert gen().max_rel_error(gen().coefficients()) <= 2.0 ** -21


def test_emulation_clamps_out_of_range():
    y = emulate(np.array([-5000.0, -127.5, 130.0, 1e6], np.float32))
    assert y[0] > 0 and y[0] < 1e-37 and y[1] < 1e-37 and y[2] >= 2.0 ** 125 and np.isfinite(y[3])
