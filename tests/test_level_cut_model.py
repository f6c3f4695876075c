"""The level cut's error bound, checked on an exact model of the digit arithmetic (CPU).

This does not run the kernel: it restates the scheme in exact integer arithmetic
(Python integers) and checks the bound the emulated FP64 updates rely on.  For
operand rows x (A side) and y (B side) with exponents e (max |x_k| < 2^e):

  X = rint(x 2^(7S - 1 - e)),  X = sum_t d_t 128^(S - t),  d_1 in [-64, 64],
  d_t in [-64, 63] after it, so x ~= 2^e sum_t d_t 2^(1 - 7t);
  the product of rows i and j keeps the levels l = t + u <= L of
  2^(e_i + e_j) sum_k d_t(x_ik) d_u(y_jk) 2^(2 - 7l),

with L = S + 1 without the cut and L = S + 1 - floor((E - e_i - e_j) / 7) with
it (E = max e over the A rows + max e over the B rows).  Both must stay within
K (2 + 1.01 S) 2^(E - 7S) of the exact product in every entry: the
representation error (at most 2^(e - 7S) per operand) plus the dropped levels
(at most S terms of 2^(e_i + e_j + 14 - 7l) each, from level S + 2 - q on).
A wrong cut rule (one level too many dropped) breaks the bound on the rows
with mid-range exponents, which the test plants.
"""
import math
import random
from fractions import Fraction

import pytest


def digits(x, e, S):
    """Balanced base-128 digits of rint(x 2^(7S - 1 - e)) (most significant first)."""
    v = Fraction(x) * Fraction(2) ** (7 * S - 1 - e)
    X = round(v)   # round half to even, like the device conversion
    out = []
    for _ in range(S - 1):
        d = ((X + 64) % 128) - 64
        out.append(d)
        X = (X - d) // 128
    out.append(X)
    assert abs(X) <= 64
    return out[::-1]   # d_1 .. d_S


def row_exp(row):
    m = max(abs(v) for v in row)
    return math.frexp(m)[1] if m > 0 else 0


def product(xi, yj, ei, ej, S, L):
    dx = [digits(v, ei, S) for v in xi]
    dy = [digits(v, ej, S) for v in yj]
    acc = Fraction(0)
    for a, b in zip(dx, dy):
        for t in range(1, S + 1):
            for u in range(1, S + 1):
                l = t + u
                if l <= L:
                    acc += Fraction(a[t - 1] * b[u - 1]) * Fraction(2) ** (ei + ej + 2 - 7 * l)
    return acc


def level_cut(S, E, ei, ej, planted_extra=0):
    return S + 1 - max(0, E - ei - ej) // 7 - planted_extra


def build_rows(rng, n, K):
    rows = []
    for i in range(n):
        scale = 2.0 ** (-rng.randint(0, 40))   # magnitudes spread over 40 binades, like far tiles
        rows.append([rng.uniform(-1, 1) * scale for _ in range(K)])
    return rows


@pytest.mark.parametrize("S", [5, 8])
def test_cut_and_uncut_products_within_the_bound(S):
    rng = random.Random(100 + S)
    K = 12
    A = build_rows(rng, 6, K)
    B = build_rows(rng, 6, K)
    ea = [row_exp(r) for r in A]
    eb = [row_exp(r) for r in B]
    E = max(ea) + max(eb)
    bound = Fraction(K) * (2 + Fraction(101, 100) * S) * Fraction(2) ** (E - 7 * S)
    worst = {0: Fraction(0), 1: Fraction(0)}
    for i in range(len(A)):
        for j in range(len(B)):
            exact = sum(Fraction(a) * Fraction(b) for a, b in zip(A[i], B[j]))
            for cut in (0, 1):
                L = level_cut(S, E, ea[i], eb[j]) if cut else S + 1
                err = abs(product(A[i], B[j], ea[i], eb[j], S, L) - exact)
                worst[cut] = max(worst[cut], err)
                assert err <= bound, (S, cut, i, j, float(err / bound))
    # the cut does drop work on these spread magnitudes
    assert any(level_cut(S, E, a, b) < S + 1 for a in ea for b in eb)


def test_one_level_too_many_breaks_the_bound():
    # the model is sharp enough to see a rule that drops one more level than the derivation allows
    rng = random.Random(7)
    S, K = 5, 12
    A = build_rows(rng, 6, K)
    B = build_rows(rng, 6, K)
    ea = [row_exp(r) for r in A]
    eb = [row_exp(r) for r in B]
    E = max(ea) + max(eb)
    bound = Fraction(K) * (2 + Fraction(101, 100) * S) * Fraction(2) ** (E - 7 * S)
    broken = False
    for i in range(len(A)):
        for j in range(len(B)):
            L = level_cut(S, E, ea[i], eb[j], planted_extra=1)
            if L < 2:
                continue
            exact = sum(Fraction(a) * Fraction(b) for a, b in zip(A[i], B[j]))
            if abs(product(A[i], B[j], ea[i], eb[j], S, L) - exact) > bound:
                broken = True
    assert broken
