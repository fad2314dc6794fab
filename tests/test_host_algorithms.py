"""The numerical methods the eigensolver and rollout kernels rest on, restated in numpy and
checked against the mathematics they replace (no GPU):

* the division-free Sturm count: the signs of the leading principal minors of T - x I, carried
  by a three-term recurrence rescaled by exact powers of two, count the eigenvalues below x
  exactly as the pivots of T - x I = L D L^T do;
* the double-word (binary32 pair) dot product with compensated accumulation (products split
  by FMA, partial sums by TwoSum): close to the exact dot product at the level of u^2 = 2^-48.
"""
from fractions import Fraction

import numpy as np
import pytest


# --------------------------------------------------------------------------- Sturm counts
def count_pivots(d, e, x, pivmin):
    """Eigenvalues of the symmetric tridiagonal (d, e) below x: negative pivots of LDL^T."""
    q = d[0] - x
    if abs(q) < pivmin:
        q = -pivmin
    cnt = int(q < 0)
    for i in range(1, len(d)):
        q = d[i] - x - e[i - 1] ** 2 / q
        if abs(q) < pivmin:
            q = -pivmin
        cnt += int(q < 0)
    return cnt


def count_minors(d, e, x):
    """The same count from the signs of the leading minors p_i = det(T_i - x I):
    p_i = (d_{i-1} - x) p_{i-1} - e_{i-2}^2 p_{i-2}, the pair (p_{i-1}, p_i) rescaled by one
    power of two when p_i leaves [2^-300, 2^300], a minor vanishing against its predecessor
    (ratio below 2^-1000, or zero) replaced by -2^-1000 p_{i-1}."""
    def expo(v):
        return np.frexp(v)[1] if v != 0 else -2000
    pm2, pm1 = 1.0, d[0] - x
    if pm1 == 0 or expo(pm1) < -1000:
        pm1 = -2.0 ** -1000
    cnt = int(pm1 < 0)
    for i in range(1, len(d)):
        p = (d[i] - x) * pm1 - e[i - 1] ** 2 * pm2
        ep = expo(p)
        if ep < -300 or ep > 300:
            em = expo(pm1)
            if p == 0 or ep < em - 1000:
                pm1 = np.ldexp(pm1, -em)
                p = -np.ldexp(pm1, -1000)
            else:
                pm1, p = np.ldexp(pm1, -ep), np.ldexp(p, -ep)
        cnt += int(np.signbit(p) != np.signbit(pm1))
        pm2, pm1 = pm1, p
    return cnt


def tridiag(n, rng, decay=1.0):
    d = rng.standard_normal(n) * decay ** np.arange(n)
    e = rng.standard_normal(n - 1) * decay ** np.arange(n - 1)
    return d, e


@pytest.mark.parametrize("seed", range(6))
def test_minor_signs_count_like_pivots_and_like_the_spectrum(seed):
    rng = np.random.default_rng(seed)
    n = 120 + 40 * seed
    d, e = tridiag(n, rng, decay=[1.0, 0.97, 1.0, 0.9, 1.0, 0.99][seed])
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    lam = np.linalg.eigvalsh(T)
    # shifts between the eigenvalues (well separated from them) and at random places
    mids = 0.5 * (lam[1:] + lam[:-1])
    xs = np.concatenate([mids[::7], rng.uniform(lam[0] - 1, lam[-1] + 1, 25)])
    gap = np.min(np.abs(xs[:, None] - lam[None, :]), axis=1)
    xs = xs[gap > 1e-9 * np.max(np.abs(lam))]
    pivmin = np.finfo(float).tiny * max(1.0, np.max(e ** 2))
    for x in xs:
        truth = int(np.sum(lam < x))
        assert count_pivots(d, e, x, pivmin) == truth
        assert count_minors(d, e, x) == truth


def test_minor_count_survives_extreme_scales_and_exact_zeros():
    rng = np.random.default_rng(9)
    d, e = tridiag(200, rng)
    lam = np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))
    x = 0.5 * (lam[80] + lam[81])
    ref = count_minors(d, e, x)
    assert ref == 81
    for s in (-400, -200, 200, 400):  # the minors overflow / underflow without the rescaling
        assert count_minors(np.ldexp(d, s), np.ldexp(e, s), np.ldexp(x, s)) == ref
    # a zero off-diagonal splits T; a shift equal to a diagonal entry gives an exact zero minor
    d2, e2 = d.copy(), e.copy()
    e2[50] = 0.0
    lam2 = np.linalg.eigvalsh(np.diag(d2) + np.diag(e2, 1) + np.diag(e2, -1))
    for x in (0.5 * (lam2[30] + lam2[31]), d2[0]):
        assert count_minors(d2, e2, x) == count_pivots(d2, e2, x, np.finfo(float).tiny)


# --------------------------------------------------------------------------- double-word dots
f32 = np.float32


def fma32(a, b, c):
    """fma in binary32: the product of two binary32 values is exact in binary64; the sum is
    rounded once to binary64 and then to binary32 (a double rounding that can differ from the
    hardware's single rounding by one ulp in rare ties, below what is checked here)."""
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def two_sum(a, b):
    s = f32(a + b)
    z = f32(s - a)
    return s, f32(f32(a - f32(s - z)) + f32(b - z))


def split(v):
    h = f32(v)
    return h, f32(v - np.float64(h))


def dw_dot(o, x):
    """sum_a o_a x_a with o, x given as binary32 pairs: the compensated accumulation of the
    rollout kernel (products split exactly by FMA, partial sums by TwoSum, errors in a second
    word), summed in order."""
    s, c = f32(0.0), f32(0.0)
    for oa, xa in zip(o, x):
        oh, ol = split(oa)
        xh, xl = split(xa)
        p = f32(oh * xh)
        err = fma32(ol, xh, fma32(oh, xl, fma32(oh, xh, -p)))
        s, t = two_sum(s, p)
        c = f32(c + f32(t + err))
    return np.float64(s) + np.float64(c)


@pytest.mark.parametrize("seed,cancel", [(0, False), (1, False), (2, True), (3, True)])
def test_double_word_dot_is_accurate_to_about_u_squared(seed, cancel):
    rng = np.random.default_rng(seed)
    n = 496  # the longest row of the r = 30 operators
    o = rng.standard_normal(n) * np.exp(rng.uniform(-3, 3, n))
    x = rng.standard_normal(n)
    if cancel:  # a result far smaller than its terms
        o[-1] = -np.dot(o[:-1], x[:-1]) / x[-1] * (1 + 1e-9)
    exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(o, x))
    got = dw_dot(o, x)
    scale = float(np.sum(np.abs(o * x)))
    err = abs(Fraction(got) - exact)
    # u^2 = 2^-48 per operation, a few hundred operations deep: 1e-12 of the terms' magnitude
    assert float(err) <= 1e-12 * scale
    # four orders of magnitude inside binary32's own rounding of the terms (2^-24 of them)
    assert float(err) <= 1e-4 * 2.0 ** -24 * scale
