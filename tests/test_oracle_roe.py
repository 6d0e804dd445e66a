"""Pins of the oracle's characteristic machinery (Sec. 4: the Roe average at the
cell face, and the eigenvectors of the Euler flux Jacobian there) by the
properties that define them, not by re-typing their formulas:

* the Roe property: A(U~) (U_R - U_L) = F(U_R) - F(U_L) for the Roe-averaged
  state U~, with A = R diag(lambda) L built from the oracle's eigenvectors;
* A(U) = R diag(lambda) L equals the flux Jacobian dF/dU, every entry, taken
  by complex-step differentiation of the Euler flux (exact to rounding);
* the normalisation of R (which matters, because the selection threshold
  delta is absolute): each column is the derivative of the conserved state
  along one simple wave -- acoustic waves with unit density change, the
  entropy wave at fixed velocity and pressure, shear waves with unit change of
  the tangential momentum -- again by complex-step differentiation;
* planted faults in a copy of the oracle's C source (arithmetic instead of
  sqrt(rho) weights, a density-weighted enthalpy, a rescaled entropy
  eigenvector with its consistent inverse) fail these checks.

The flux F(U) = [m_x, m_x u + p, m_y u, m_z u, (E + p) u] along x (momentum
along the sweep axis first) and p = (gamma - 1)(E - |m|^2 / (2 rho)) are the
ideal-gas Euler equations of Sec. 4, written here in numpy with complex
support."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

GAMMA = 1.4
H_CS = 1e-30  # complex-step size


def _flux(U, gamma=GAMMA):
    rho, m, E = U[0], U[1:-1], U[-1]
    u = m[0] / rho
    p = (gamma - 1.0) * (E - 0.5 * np.sum(m * m) / rho)
    F = np.empty_like(U)
    F[0] = m[0]
    F[1] = m[0] * u + p
    F[2:-1] = m[1:] * u
    F[-1] = (E + p) * u
    return F


def _conserved(rho, vel, p, gamma=GAMMA):
    vel = np.asarray(vel)
    return np.concatenate([[rho], rho * vel, [p / (gamma - 1.0) + 0.5 * rho * np.sum(vel * vel)]])


def _cs_jacobian(U):
    n = U.size
    J = np.empty((n, n))
    for k in range(n):
        Uc = U.astype(complex)
        Uc[k] += 1j * H_CS
        J[:, k] = _flux(Uc).imag / H_CS
    return J


def _random_state(rng, ndim):
    rho = rng.uniform(0.1, 2.0)
    vel = rng.uniform(-2.0, 2.0, size=ndim)
    p = rng.uniform(0.1, 2.0)
    return rho, vel, p


def _A(eigen, ndim, vel, H):
    R, L = eigen(ndim, GAMMA, vel, H)
    c = np.sqrt((GAMMA - 1.0) * (H - 0.5 * vel @ vel))
    lam = np.array([vel[0] - c] + [vel[0]] * ndim + [vel[0] + c])
    return R @ np.diag(lam) @ L, R, L


def _roe_residual(roe, eigen, ndim, rng, pairs=200):
    worst = 0.0
    for _ in range(pairs):
        UL = _conserved(*_random_state(rng, ndim))
        UR = _conserved(*_random_state(rng, ndim))
        vel, H = roe(ndim, GAMMA, UL, UR)
        A, _, _ = _A(eigen, ndim, vel, H)
        dF = _flux(UR) - _flux(UL)
        scale = np.abs(A).max() * np.abs(UR - UL).max() + np.abs(dF).max()
        worst = max(worst, np.abs(A @ (UR - UL) - dF).max() / scale)
    return worst


def _normalisation_residual(eigen, ndim, rng, states=50):
    """Largest deviation of R's columns from the simple-wave derivatives."""
    worst = 0.0
    for _ in range(states):
        rho, vel, p = _random_state(rng, ndim)
        c = np.sqrt(GAMMA * p / rho)
        H = c * c / (GAMMA - 1.0) + 0.5 * vel @ vel
        R, _ = eigen(ndim, GAMMA, vel, H)

        def along(drho, dvel, dp):
            Wc = _conserved(rho + 1j * H_CS * drho, vel + 1j * H_CS * np.asarray(dvel, float),
                            p + 1j * H_CS * dp)
            return Wc.imag / H_CS

        e0 = np.eye(ndim)[0]
        cols = [along(1.0, -c / rho * e0, c * c)]          # u - c wave, unit density change
        cols += [along(1.0, np.zeros(ndim), 0.0)]          # entropy wave
        for t in range(1, ndim):                            # shear waves, unit d(rho v_t)
            cols += [along(0.0, np.eye(ndim)[t] / rho, 0.0)]
        cols += [along(1.0, c / rho * e0, c * c)]           # u + c wave
        want = np.stack(cols, axis=1)
        worst = max(worst, np.abs(R - want).max() / np.abs(want).max())
    return worst


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_roe_property(oracle_mod, ndim):
    r = _roe_residual(oracle_mod.roe_average, oracle_mod.euler_eigen, ndim,
                      np.random.default_rng(100 + ndim))
    assert r <= 1e-12, r


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_eigensystem_reproduces_the_flux_jacobian(oracle_mod, ndim):
    rng = np.random.default_rng(200 + ndim)
    for _ in range(100):
        rho, vel, p = _random_state(rng, ndim)
        U = _conserved(rho, vel, p)
        # the Roe average of a state with itself is that state
        v2, H = oracle_mod.roe_average(ndim, GAMMA, U, U)
        assert np.allclose(v2, vel, rtol=1e-14, atol=1e-14)
        A, _, _ = _A(oracle_mod.euler_eigen, ndim, v2, H)
        J = _cs_jacobian(U)
        assert np.abs(A - J).max() <= 1e-12 * np.abs(J).max(), np.abs(A - J).max()


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_eigenvector_normalisation_is_the_simple_wave_one(oracle_mod, ndim):
    r = _normalisation_residual(oracle_mod.euler_eigen, ndim, np.random.default_rng(300 + ndim))
    assert r <= 1e-12, r


# ------------------------------------------------------------- planted faults

def _mutant(tmp_path, name, edits):
    """Compile a copy of the oracle with the given source edits (each must apply)."""
    import oracle
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "enoao_oracle.c")).read()
    for old, new in edits:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    d = tmp_path / name
    d.mkdir()
    (d / "enoao_oracle.c").write_text(src)
    (d / "enoao_oracle.h").write_text(open(os.path.join(here, "enoao_oracle.h")).read())
    so = d / "liboracle_mutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                    str(d / "enoao_oracle.c"), "-o", str(so), "-lm"], check=True,
                   capture_output=True)
    lib = ctypes.CDLL(str(so))
    D = ctypes.POINTER(ctypes.c_double)
    lib.or_roe_average.argtypes = [D, D, ctypes.c_int, ctypes.c_double, D, D]
    lib.or_euler_eigen.argtypes = [ctypes.c_int, ctypes.c_double, D, ctypes.c_double, D, D]
    dp = lambda a: a.ctypes.data_as(D)

    def roe(ndim, gamma, ql, qr):
        ql = np.ascontiguousarray(ql, float)
        qr = np.ascontiguousarray(qr, float)
        vel = np.zeros(ndim)
        H = ctypes.c_double()
        lib.or_roe_average(dp(ql), dp(qr), ndim, gamma, dp(vel), ctypes.byref(H))
        return vel, H.value

    def eigen(ndim, gamma, vel, H):
        nv = ndim + 2
        R, L = np.zeros((nv, nv)), np.zeros((nv, nv))
        v = np.ascontiguousarray(vel, float)
        lib.or_euler_eigen(ndim, gamma, dp(v), H, dp(R), dp(L))
        return R, L

    return roe, eigen


def test_planted_arithmetic_mean_fails_the_roe_property(tmp_path, oracle_mod):
    roe, eigen = _mutant(tmp_path, "mean", [
        ("double sl = sqrt(ql[0]), sr = sqrt(qr[0]);", "double sl = 1.0, sr = 1.0;")])
    for ndim in (1, 2, 3):
        assert _roe_residual(roe, eigen, ndim, np.random.default_rng(ndim)) > 1e-3


def test_planted_density_weighted_enthalpy_fails_the_roe_property(tmp_path, oracle_mod):
    roe, eigen = _mutant(tmp_path, "rhoH", [
        ("*H = (sl * hl + sr * hr) / (sl + sr);",
         "*H = (ql[0] * hl + qr[0] * hr) / (ql[0] + qr[0]);")])
    for ndim in (1, 2, 3):
        assert _roe_residual(roe, eigen, ndim, np.random.default_rng(ndim)) > 1e-3


def test_planted_rescaled_eigenvector_fails_the_normalisation(tmp_path, oracle_mod):
    # entropy column x 2 with its left row / 2: L R = I, the Roe property and
    # the Jacobian all still hold; only the normalisation pin sees it
    roe, eigen = _mutant(tmp_path, "scale", [
        ("R[0 * nv + e] = 1.0;", "R[0 * nv + e] = 2.0;"),
        ("R[1 * nv + e] = u;", "R[1 * nv + e] = 2.0 * u;"),
        ("R[(nv - 1) * nv + e] = 0.5 * q2;", "R[(nv - 1) * nv + e] = q2;"),
        ("R[(1 + t) * nv + e] = vel[t];", "R[(1 + t) * nv + e] = 2.0 * vel[t];"),
        ("L[e * nv + 0] = 1.0 - b2;", "L[e * nv + 0] = 0.5 * (1.0 - b2);"),
        ("L[e * nv + 1] = b1 * u;", "L[e * nv + 1] = 0.5 * b1 * u;"),
        ("L[e * nv + nv - 1] = -b1;", "L[e * nv + nv - 1] = -0.5 * b1;"),
        ("L[e * nv + 1 + t] = b1 * vel[t];", "L[e * nv + 1 + t] = 0.5 * b1 * vel[t];"),
    ])
    for ndim in (1, 2, 3):
        rng = np.random.default_rng(ndim)
        assert _roe_residual(roe, eigen, ndim, rng) <= 1e-12
        vel, H = np.array([0.3] + [0.1] * (ndim - 1)), 3.0
        R, L = eigen(ndim, GAMMA, vel, H)
        assert np.abs(L @ R - np.eye(ndim + 2)).max() < 1e-13
        assert _normalisation_residual(eigen, ndim, rng) > 0.1
