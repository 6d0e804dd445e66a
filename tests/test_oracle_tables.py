"""Pins of the oracle's stencil tables against the paper and against first principles.

* Table 1 (interface values) is re-derived from its definition, Eq.
  (Polynomial_Construction): the polynomial of degree m+n whose cell averages
  match f on S_{j-m}^{j+n}, evaluated at x_{j+1/2}, solved in exact rationals.
* Tables 4 and 5 (delta_L, delta_R) are re-derived from Eq.
  (New_Smoothness_Indicator): the same polynomial's average over the
  neighbouring cell minus that cell's value.
* Tables 2 and 3 (modified wavenumbers) are recomputed from the Table-1 rows.
* The oracle's candidate values and indicators are probed on unit and random
  windows and compared with the exact results.
"""
import cmath
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from conftest import frac, golden_rows


def _solve(A, b):
    """Exact Gauss-Jordan solve of A x = b (lists of Fractions)."""
    n = len(A)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        piv = M[c][c]
        M[c] = [v / piv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def _cell_avg_row(k, deg):
    """Average of x^p over I_k = [k-1/2, k+1/2] (dx = 1, x_j = 0), p = 0..deg."""
    a, b = Fraction(2 * k - 1, 2), Fraction(2 * k + 1, 2)
    return [(b ** (p + 1) - a ** (p + 1)) / (p + 1) for p in range(deg + 1)]


def _poly_functionals(m, n):
    """Exact linear functionals of f_{j-m..j+n}: value at x_{j+1/2} and the
    averages over I_{j-m-1} and I_{j+n+1} of the reconstructing polynomial."""
    deg = m + n
    A = [_cell_avg_row(k, deg) for k in range(-m, n + 1)]
    ncell = deg + 1
    cols = []
    for i in range(ncell):
        e = [Fraction(int(r == i)) for r in range(ncell)]
        cols.append(_solve(A, e))          # polynomial coefficients for unit data
    half = [Fraction(1, 2) ** p for p in range(deg + 1)]
    left = _cell_avg_row(-m - 1, deg)
    right = _cell_avg_row(n + 1, deg)

    def apply(row):
        return [sum(r * c for r, c in zip(row, cols[i])) for i in range(ncell)]
    return apply(half), apply(left), apply(right)


FLUX_ROWS = {(int(r[0]), int(r[1])): (int(r[2]), [int(v) for v in r[3:]])
             for r in golden_rows("flux_table.txt")}


def _candidates(order):
    for r in golden_rows("candidate_sets.txt"):
        if int(r[0]) == order:
            return [tuple(int(x) for x in t.split(",")) for t in r[2:]]
    raise KeyError(order)


def test_flux_table_matches_polynomial_definition():
    assert len(FLUX_ROWS) == 16
    for (m, n), (den, num) in FLUX_ROWS.items():
        val, _, _ = _poly_functionals(m, n)
        assert val == [Fraction(v, den) for v in num], (m, n)


def test_indicator_tables_match_definition():
    rows = golden_rows("indicator_tables.txt")
    assert len(rows) == 8
    for r in rows:
        m, n = int(r[0]), int(r[1])
        bar = [i for i, t in enumerate(r) if t == "|"]
        Lc = [int(v) for v in r[bar[0] + 1:bar[1]]]
        Rc = [int(v) for v in r[bar[1] + 1:]]
        _, left, right = _poly_functionals(m, n)
        # delta_L functional over f_{j-m-1..j+n}: average over I_{j-m-1} minus f_{j-m-1}
        dl = [Fraction(-1)] + left
        # delta_R functional over f_{j-m..j+n+1}: average over I_{j+n+1} minus f_{j+n+1}
        dr = right + [Fraction(-1)]
        sl = 1 if dl[0] * Lc[0] > 0 else -1
        sr = 1 if dr[0] * Rc[0] > 0 else -1
        assert [sl * v for v in dl] == [Fraction(v) for v in Lc], (m, n)
        assert [sr * v for v in dr] == [Fraction(v) for v in Rc], (m, n)


def _kappa_prime(m, n, kap):
    den, num = FLUX_ROWS[(m, n)]
    s = sum(Fraction(a, den) * cmath.exp(1j * kap * (i - m)) for i, a in enumerate(num))
    return -1j * complex(s) * (1 - cmath.exp(-1j * kap))


def test_wavenumber_tables_follow_from_flux_table():
    rows = golden_rows("wavenumber_tables.txt")
    assert len(rows) == 16
    for r in rows:
        m, n = int(r[0]), int(r[1])
        s = [float(frac(v)) for v in r[3:7]]
        c = [float(frac(v)) for v in r[8:13]]
        for kap in np.linspace(0.0, math.pi, 25):
            kp = _kappa_prime(m, n, kap)
            re = sum(s[k] * math.sin((k + 1) * kap) for k in range(4))
            im = c[0] + sum(c[k] * math.cos(k * kap) for k in range(1, 5))
            assert abs(kp.real - re) < 1e-12, (m, n, kap)
            assert abs(kp.imag - im) < 1e-12, (m, n, kap)


@pytest.mark.parametrize("order", [5, 7])
def test_candidates_are_linearly_stable(order):
    # Sec. 3.2: only fluxes with Im(kappa') <= 0 for all kappa are candidates.
    for (m, n) in _candidates(order):
        for kap in np.linspace(0.0, math.pi, 200):
            assert _kappa_prime(m, n, kap).imag <= 1e-14, (m, n, kap)


def test_oracle_candidate_values_match_table(oracle_mod):
    cands = _candidates(7)
    for c, (m, n) in enumerate(cands):
        den, num = FLUX_ROWS[(m, n)]
        for i in range(9):
            w = np.zeros(9)
            w[i] = 1.0
            k = i - 4
            expect = num[k + m] / den if -m <= k <= n else 0.0
            assert oracle_mod.candidate_flux(w, c) == pytest.approx(expect, abs=1e-15), (c, k)


def test_oracle_indicators_match_definition(oracle_mod):
    rnd = random.Random(7)
    cands = _candidates(7)
    for trial in range(40):
        f = [Fraction(rnd.randint(-50, 50), rnd.randint(1, 9)) for _ in range(9)]
        w = np.array([float(v) for v in f])
        for c, (m, n) in enumerate(cands):
            dl, dr = oracle_mod.candidate_deltas(w, c)
            if m == n == 0:
                el = (abs(f[4] - f[3]) + abs(f[3] - f[2])) / 2
                er = (abs(f[4] - f[5]) + abs(f[5] - f[6])) / 2
            else:
                _, left, right = _poly_functionals(m, n)
                cells = [f[4 + k] for k in range(-m, n + 1)]
                el = abs(sum(a * b for a, b in zip(left, cells)) - f[4 - m - 1])
                er = abs(sum(a * b for a, b in zip(right, cells)) - f[4 + n + 1])
            assert dl == pytest.approx(float(el), rel=1e-13, abs=1e-12), (c, trial)
            assert dr == pytest.approx(float(er), rel=1e-13, abs=1e-12), (c, trial)
