"""The ADR tool on the GPU (paper_2108_12742_gb300.adr) against the oracle's:
FP64 modified wavenumbers equal to rounding wherever every stencil choice of a
mode agrees (a differing choice must be a near-tie), FP32 bulk within its
flux tolerance, and the linear regime far below the threshold."""
import numpy as np
import pytest

import oracle
import paper_2108_12742_gb300 as eno
from paper_2108_12742_gb300 import adr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12742_gb300 import build
    build.build()
    oracle.build()


def _both(n, order, amplitude, precision):
    k, theta, U = adr.modes(n, amplitude)
    rows = k.size
    with eno.Solver((n, rows), (0.0, 0.0), (float(n), float(rows)), system=eno.SCALAR_ADVECTION,
                    order=order, bc=eno.PERIODIC, adv_speed=1.0, precision=precision) as s:
        s.init_state(U)
        F, idx = s.reconstruct_fluxes(0, want_idx=True)
    P = oracle.make_problem((n, rows), (0.0, 0.0), (float(n), float(rows)), system=oracle.SCALAR,
                            order=order, bc=oracle.PERIODIC, adv_speed=1.0)
    Fo, io, gap = oracle.fluxes(P, U, 0, np.array([1.0, 1.0, 0.0]), want_idx=True)
    kp = adr.modified_wavenumber(F[0, 0], U[0, 0])
    ko = adr.modified_wavenumber(Fo[0, 0], U[0, 0])
    return theta, kp, ko, idx, io, gap


@pytest.mark.parametrize("order", [5, 7])
def test_fp64_adr_matches_oracle(order):
    theta, kp, ko, idx, io, gap = _both(256, order, 1.0, eno.FP64)
    differ = idx != io
    assert not (differ & (gap > 1e-13)).any()
    rows_ok = ~differ.any(axis=(0, 1, 2, 4))  # modes whose every choice agrees
    assert rows_ok.mean() >= 0.9
    assert np.abs(kp - ko)[rows_ok].max() <= 1e-12


@pytest.mark.parametrize("order", [5, 7])
def test_fp32_bulk_adr_and_linear_regime(order):
    theta, kp, ko, _, _, _ = _both(256, order, 1.0, eno.FP32_BULK)
    assert np.abs(kp - ko).max() <= 1e-5
    theta, kl = adr.adr(n=64, order=order, amplitude=1e-9)
    assert np.abs(kl - adr.upwind_linear(theta, order)).max() <= 1e-12
