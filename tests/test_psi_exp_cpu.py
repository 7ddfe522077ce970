"""The FP32 kernels evaluate psi(rho) = rho0 (1 - e^{-t}), t = rho/rho0, with
their own exponential (lb_common.cuh: one_minus_exp_neg): Cody-Waite reduction
t = k ln2 + r, the degree-7 Taylor polynomial of 1 - e^{-r}, and
(1 - 2^-k) + 2^-k (1 - e^{-r}).  This checks those steps, carried out in FP32
with one rounding per operation (numpy), against the exact value: the error
bound the kernels rely on.  The GPU parity tests check the kernels themselves
against the FP64 oracle."""
import math

import numpy as np

f32 = np.float32
LOG2E, ROUND = f32(1.44269504088896340736), f32(12582912.0)
LN2_HI, LN2_LO = f32(0.693145751953125), f32(1.42860682030941723212e-6)
D = [f32((-1) ** (n + 1) / math.factorial(n)) for n in range(1, 8)]


def fma(a, b, c):
    # float32 inputs: the product is exact in float64; the sum rounds twice,
    # which differs from one rounding only in rare ties (far below the bound)
    return (a.astype(np.float64) * b + c).astype(f32)


def one_minus_exp_neg(t):
    t = np.minimum(t.astype(f32), f32(80.0))
    km = fma(t, LOG2E, ROUND)
    k = (km - ROUND).astype(f32)
    r = fma(k, -LN2_HI, t)
    r = fma(k, -LN2_LO, r)
    q = np.full_like(t, D[6])
    for n in range(5, -1, -1):
        q = fma(q, r, D[n])
    q = (q * r).astype(f32)
    s = ((np.uint32(0x3F800000) - (km.view(np.uint32) << np.uint32(23))).astype(np.uint32)).view(f32)
    return fma(s, q, (f32(1.0) - s).astype(f32))


def test_one_minus_exp_neg_within_1_5_ulp():
    rs = np.random.RandomState(7)
    t = np.concatenate([np.linspace(1e-6, 0.5, 40001), np.linspace(0.5, 5.0, 40001),
                        np.linspace(5.0, 40.0, 4001), rs.uniform(0.0, 3.0, 40000),
                        2.0 ** rs.uniform(-20, -1, 5000)]).astype(f32)
    got = one_minus_exp_neg(t).astype(np.float64)
    exact = -np.expm1(-t.astype(np.float64))
    ulp = np.spacing(exact.astype(f32)).astype(np.float64)
    assert np.max(np.abs(got - exact) / ulp) <= 1.5


def test_one_minus_exp_neg_special_values():
    t = np.array([0.0, 80.0, 1000.0, 3.0e38], dtype=f32)
    got = one_minus_exp_neg(t)
    assert got[0] == 0.0  # psi(0) = 0 exactly
    assert np.all(got[1:] == 1.0)  # saturation: psi -> rho0
