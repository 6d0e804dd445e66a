"""Spectral analysis of the oracle's ENO-AO (approximate dispersion relation,
Sec. 4.1): pins of the ADR tool's arithmetic and of what the paper states
about the curves.

* Far below the threshold delta (amplitude 1e-9) every indicator selects the
  candidate of highest order, so ENO-AO is the linear upwind-biased scheme of
  the same order, whose modified wavenumber has a closed form (from its five
  or seven interface coefficients): equal to rounding.
* At amplitude 1 the paper reports smaller dissipation than the linear
  upwind scheme for medium wavenumbers (0.4 <= kappa <= 1 for 5th order,
  0.6 <= kappa <= 1 for 7th) and larger dissipation for kappa > 1.
* Consistency: kappa' -> kappa for small kappa.
"""
import numpy as np
import pytest

from paper_2108_12742_gb300 import adr


def _oracle_adr(oracle_mod, n, order, amplitude):
    k, theta, U = adr.modes(n, amplitude)
    P = oracle_mod.make_problem((n, k.size), (0.0, 0.0), (float(n), float(k.size)),
                                system=oracle_mod.SCALAR, order=order, bc=oracle_mod.PERIODIC,
                                adv_speed=1.0)
    F, _, _ = oracle_mod.fluxes(P, U, 0, np.array([1.0, 1.0, 0.0]))
    return theta, adr.modified_wavenumber(F[0, 0], U[0, 0])


@pytest.mark.parametrize("order", [5, 7])
def test_far_below_threshold_is_the_linear_upwind_scheme(oracle_mod, order):
    theta, kp = _oracle_adr(oracle_mod, 64, order, 1e-9)
    assert np.abs(kp - adr.upwind_linear(theta, order)).max() <= 1e-13


def test_closed_form_of_the_linear_scheme():
    # the linear schemes are consistent to their order: kappa' - theta = O(theta^(p+1))
    for order, t0 in ((5, 0.02), (7, 0.1)):
        theta = np.array([t0, 2.0 * t0])
        err = np.abs(adr.upwind_linear(theta, order) - theta)
        assert err[1] / err[0] == pytest.approx(2.0 ** (order + 1), rel=0.05), order
    # the Nyquist mode is damped, not advected
    ny = adr.upwind_linear(np.array([np.pi]), 5)[0]
    assert abs(ny.real) < 1e-15 and ny.imag == pytest.approx(-16.0 / 15.0, rel=1e-14)


@pytest.mark.parametrize("order,lo", [(5, 0.4), (7, 0.6)])
def test_paper_statements_at_unit_amplitude(oracle_mod, order, lo):
    theta, kp = _oracle_adr(oracle_mod, 128, order, 1.0)
    uw = adr.upwind_linear(theta, order)
    small = theta < 0.3
    assert np.abs(kp[small] - theta[small]).max() <= 1e-3
    medium = (theta >= lo) & (theta <= 1.0)
    assert (np.abs(kp.imag[medium]) <= np.abs(uw.imag[medium])).all()
    high = theta > 1.5
    assert (np.abs(kp.imag[high]) > np.abs(uw.imag[high])).mean() >= 0.9
