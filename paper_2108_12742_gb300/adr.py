"""Approximate dispersion relation (ADR) of the ENO-AO reconstruction, after
the numerical technique the paper uses for its spectral analysis (Sec. 4.1,
citing Pirozzoli): the nonlinear scheme has no closed-form modified
wavenumber, so each Fourier mode is fed through the scheme and the
response's own Fourier coefficient is read back.

For linear advection u_t + u_x = 0 on a periodic grid of N cells, the
semi-discrete scheme maps the mode u_j = A cos(theta j) (theta = 2 pi k / N;
the cosine keeps the Nyquist mode k = N/2 non-zero)
to L(u)_j; the modified wavenumber is kappa' dx = i dx L^_k / u^_k (hats:
the k-th discrete Fourier coefficient), whose real part is the dispersion and
whose imaginary part (negative) the dissipation; the exact scheme gives
kappa' dx = theta.  The response depends on the amplitude A because the
selection threshold delta is absolute.

All wavenumbers run in one library call: a 2D scalar-advection problem whose
row k holds mode k, swept along x only (enoao_reconstruct_fluxes); numpy
takes the Fourier coefficients.
"""
from __future__ import annotations

import numpy as np


def modes(n: int, amplitude: float = 1.0):
    """(k, theta, U) with U[0, 0, k - 1, j] = amplitude * cos(theta_k j), k = 1 .. n/2."""
    k = np.arange(1, n // 2 + 1)
    theta = 2.0 * np.pi * k / n
    j = np.arange(n)
    U = amplitude * np.cos(theta[:, None] * j[None, :])
    return k, theta, np.ascontiguousarray(U.reshape(1, 1, k.size, n))


def modified_wavenumber(F: np.ndarray, U: np.ndarray) -> np.ndarray:
    """kappa' dx per row from interface fluxes F (rows x n+1 faces, face f between
    cells f-1 and f) of the modes U (rows x n), with dx = 1 and a = 1."""
    rows, n = U.shape
    L = -(F[:, 1:] - F[:, :-1])  # L(u)_j = -(F_{j+1/2} - F_{j-1/2}) / dx
    k = np.arange(1, rows + 1)
    Lh = np.fft.fft(L, axis=1)[np.arange(rows), k]
    Uh = np.fft.fft(U, axis=1)[np.arange(rows), k]
    return 1j * Lh / Uh


def adr(n: int = 128, order: int = 5, amplitude: float = 1.0, precision=None, delta: float = 1e-5):
    """Modified wavenumbers of ENO-AO (order 5 or 7) on the GPU: (theta, kappa' dx)."""
    import paper_2108_12742_gb300 as eno
    if precision is None:
        precision = eno.FP64
    k, theta, U = modes(n, amplitude)
    rows = k.size
    with eno.Solver((n, rows), (0.0, 0.0), (float(n), float(rows)), system=eno.SCALAR_ADVECTION,
                    order=order, bc=eno.PERIODIC, adv_speed=1.0, precision=precision,
                    delta=delta) as s:
        s.init_state(U)
        F, _ = s.reconstruct_fluxes(0)
    return theta, modified_wavenumber(F[0, 0], U[0, 0])


def upwind_linear(theta: np.ndarray, order: int = 5) -> np.ndarray:
    """kappa' dx of the linear upwind-biased scheme of the same order (the
    candidate of highest order alone), from its interface coefficients."""
    if order == 5:   # f^_{j+1/2} on cells j-2 .. j+2
        c, m0 = np.array([2.0, -13.0, 47.0, 27.0, -3.0]) / 60.0, -2
    else:            # cells j-3 .. j+3
        c, m0 = np.array([-3.0, 25.0, -101.0, 319.0, 214.0, -38.0, 4.0]) / 420.0, -3
    m = np.arange(c.size) + m0
    sym = (c[None, :] * np.exp(1j * theta[:, None] * m[None, :])).sum(axis=1)
    return -1j * (1.0 - np.exp(-1j * theta)) * sym
