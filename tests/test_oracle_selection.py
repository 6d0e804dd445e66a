"""Pins of the oracle's stencil selection (Sec. 3.1 properties, Sec. 3.2
principle, Appendix A tie-breaking) on windows whose answer the paper fixes."""
import math

import numpy as np
import pytest


def _window(fun, j0=0.0, h=1.0):
    """w[k] = fun at the node j0 + (k-4) h, k = 0..8."""
    return np.array([fun(j0 + (k - 4) * h) for k in range(9)])


@pytest.mark.parametrize("order", [5, 7])
def test_jump_at_the_face_falls_back_to_first_order(oracle_mod, order):
    # f_k = 0 for k <= j, 1 for k > j: only S_j^j avoids the jump, so the
    # interface value is exactly f_j (first-order upwind).
    w = np.array([0, 0, 0, 0, 0, 1, 1, 1, 1], dtype=float)
    v, idx, IS, _ = oracle_mod.face_value(w, order)
    assert v == 0.0 and idx == 0
    assert IS[0] == 0.0 and all(IS[c] >= 1.0 for c in range(1, 6 if order == 5 else 9))


@pytest.mark.parametrize("order", [5, 7])
def test_jump_one_cell_downwind_selects_upwind_stencil(oracle_mod, order):
    # centre cell c with f_{c-4..c+1} = 0 and f_{c+2..} = 1: S_{c-2}^{c+1} is the
    # highest-priority stencil that does not see the jump, giving exactly 0.
    w = np.array([0, 0, 0, 0, 0, 0, 1, 1, 1], dtype=float)
    v, idx, IS, _ = oracle_mod.face_value(w, order)
    assert v == 0.0 and idx == 3 and IS[3] == 0.0


@pytest.mark.parametrize("order", [5, 7])
def test_piecewise_constant_data_gives_an_adjacent_constant(oracle_mod, order):
    # integer levels keep every Table-1 sum exact in floating point
    rng = np.random.default_rng(3)
    for _ in range(300):
        a, b = rng.choice(np.arange(-8, 9), size=2, replace=False).astype(float)
        cut = int(rng.integers(0, 10))   # first window cell carrying b
        w = np.where(np.arange(9) < cut, a, b).astype(float)
        v, idx, _, _ = oracle_mod.face_value(w, order)
        # the face sits between window cells 4 and 5; at a jump there the
        # upwind constant (cell 4) is taken
        assert v == w[4], (a, b, cut, v, idx)


@pytest.mark.parametrize("order,top", [(5, 5), (7, 8)])
def test_smooth_data_selects_the_designed_order(oracle_mod, order, top):
    for j0 in np.linspace(0.0, 2.0, 17):
        w = _window(lambda x: math.sin(math.pi * x), j0, 0.02)
        _, idx, _, _ = oracle_mod.face_value(w, order)
        assert idx == top


def test_indicators_scale_as_dx_to_the_stencil_order(oracle_mod):
    # Sec. 3.1: IS of S_{j-m}^{j+n} is O(dx^{m+n+1}) on smooth data (S_j^j: O(dx)).
    mn = [(0, 0), (0, 1), (1, 1), (2, 1), (1, 2), (2, 2), (3, 2), (2, 3), (3, 3)]
    hs = [0.1, 0.05, 0.025]
    fun = math.exp   # every derivative positive: no accidental cancellation
    IS = np.array([oracle_mod.face_value(_window(fun, 0.3, h), 7)[2] for h in hs])
    for c, (m, n) in enumerate(mn):
        slope = math.log(IS[0, c] / IS[2, c]) / math.log(hs[0] / hs[2])
        expect = 1 if m == n == 0 else m + n + 1
        assert abs(slope - expect) < 0.1, (c, slope, expect)


def test_first_order_extremum_keeps_positive_indicator(oracle_mod):
    # Remark after Eq. (New_Smoothness_Indicator): at a first-order extremum the
    # two-difference form keeps IS_j^j away from zero.
    w = _window(lambda x: math.cos(x), 0.0, 0.1)
    _, _, IS, _ = oracle_mod.face_value(w, 5)
    assert IS[0] > 0.0
    # the one-difference form would vanish on one side at this extremum
    assert abs(w[4] - w[3]) == pytest.approx(abs(w[4] - w[5]))


@pytest.mark.parametrize("order", [5, 7])
def test_selection_principle_on_random_windows(oracle_mod, order):
    # Sec. 3.2: any IS <= delta -> the highest priority among them; else the
    # smallest IS, equal values resolved to the higher priority (Appendix A).
    nc = 6 if order == 5 else 9
    rng = np.random.default_rng(11)
    seen_threshold = seen_argmin = seen_tie = 0
    for t in range(3000):
        scale = 10.0 ** rng.uniform(-8, 0)
        if t % 3 == 0:
            w = rng.integers(-2, 3, size=9).astype(float) * scale  # frequent exact ties
        else:
            w = np.sin(rng.uniform(0.2, 3.0) * np.arange(9) + rng.uniform(0, 6)) * scale
        v, idx, IS, _ = oracle_mod.face_value(w, order)
        small = [c for c in range(nc) if IS[c] <= 1e-5]
        if small:
            seen_threshold += 1
            assert idx == max(small)
        else:
            seen_argmin += 1
            mins = [c for c in range(nc) if IS[c] == IS[:nc].min()]
            seen_tie += len(mins) > 1
            assert idx == max(mins)
        assert v == oracle_mod.candidate_flux(w, idx)
    assert seen_threshold and seen_argmin and seen_tie
