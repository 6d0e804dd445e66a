"""Seeded synthetic initial states for the ENO-AO workloads.

This module only draws and lays out input data; it holds none of the
scheme's arithmetic and is shared by the CUDA-path tests, the oracle tests
and the benchmark.  Every generator is deterministic in its seed
(``numpy.random.default_rng``).

States are float64 arrays shaped ``(nv, nz, ny, nx)`` (structure of arrays,
x fastest).  Euler states hold the conserved variables
(rho, rho*u, [rho*v], [rho*w], rho*e) with the ideal-gas total energy
rho*e = p/(gamma-1) + rho*|u|^2/2 (Sec. 4.2 of the paper).

Grids:
  * periodic advection uses the paper's node grid x_j = x_L + j*dx,
    j = 0..N-1, dx = (x_R - x_L)/N (Sec. 2; x_N coincides with x_0);
  * transmissive problems use cell centres x_j = x_L + (j + 1/2)*dx.
"""
from __future__ import annotations

import math

import numpy as np


def node_grid(n, lo, hi):
    dx = (hi - lo) / n
    return lo + dx * np.arange(n)


def centre_grid(n, lo, hi):
    dx = (hi - lo) / n
    return lo + dx * (np.arange(n) + 0.5)


def conserved(rho, vel, p, gamma):
    """Stack primitive fields (rho, [u, v, w], p) into conserved variables."""
    rho = np.asarray(rho, dtype=np.float64)
    vel = [np.asarray(v, dtype=np.float64) for v in vel]
    ke = 0.5 * rho * sum(v * v for v in vel)
    E = np.asarray(p, dtype=np.float64) / (gamma - 1.0) + ke
    return np.stack([rho] + [rho * v for v in vel] + [E])


# ---------------------------------------------------------------- advection
def advection_sine(n, lo=-1.0, hi=1.0):
    """u0 = sin(pi x) on the periodic node grid; shape (1, 1, 1, n)."""
    x = node_grid(n, lo, hi)
    return np.sin(math.pi * x).reshape(1, 1, 1, n)


def advection_square(n, seed, lo=-1.0, hi=1.0):
    """Unit square pulse on a random sub-interval of width U[0.2, 0.6]."""
    rng = np.random.default_rng(seed)
    width = rng.uniform(0.2, 0.6)
    start = rng.uniform(lo, hi - width)
    x = node_grid(n, lo, hi)
    u = ((x >= start) & (x < start + width)).astype(np.float64)
    return u.reshape(1, 1, 1, n)


def advection_random(n, seed, smooth=False):
    """Random data for parity tests: white noise, or a smooth random Fourier sum."""
    rng = np.random.default_rng(seed)
    if not smooth:
        return rng.uniform(-1.0, 1.0, size=(1, 1, 1, n))
    x = node_grid(n, -1.0, 1.0)
    u = np.zeros(n)
    for k in range(1, 5):
        u += rng.uniform(-1, 1) * np.sin(math.pi * k * x + rng.uniform(0, 2 * math.pi)) / k
    return u.reshape(1, 1, 1, n)


# ---------------------------------------------------------------- 1D Euler
def riemann_params(rng):
    """Left/right primitive states and jump position of the 1D Riemann workload."""
    left = dict(rho=rng.uniform(0.1, 1.0), u=rng.uniform(-1.0, 1.0), p=rng.uniform(0.1, 1.0))
    right = dict(rho=rng.uniform(0.1, 1.0), u=rng.uniform(-1.0, 1.0), p=rng.uniform(0.1, 1.0))
    x0 = rng.uniform(0.3, 0.7)
    k = int(rng.integers(3, 9))           # k ~ U{3..8}
    side = int(rng.integers(0, 2))        # side carrying the density wave
    return left, right, x0, k, side


def euler1d_riemann(n, seed, gamma=1.4, lo=0.0, hi=1.0, perturb=True):
    """Seeded Riemann data on [lo, hi] with rho*(1 + 0.2 sin(k pi x)) on one side."""
    rng = np.random.default_rng(seed)
    left, right, x0, k, side = riemann_params(rng)
    x = centre_grid(n, lo, hi)
    isl = x < lo + x0 * (hi - lo)
    rho = np.where(isl, left["rho"], right["rho"])
    u = np.where(isl, left["u"], right["u"])
    p = np.where(isl, left["p"], right["p"])
    if perturb:
        on = isl if side == 0 else ~isl
        rho = np.where(on, rho * (1.0 + 0.2 * np.sin(k * math.pi * x)), rho)
    return conserved(rho, [u], p, gamma).reshape(3, 1, 1, n)


def euler1d_sod(n, gamma=1.4):
    """Sod's shock tube on [0, 1], jump at 0.5 (used for exact-solution checks)."""
    x = centre_grid(n, 0.0, 1.0)
    isl = x < 0.5
    rho = np.where(isl, 1.0, 0.125)
    p = np.where(isl, 1.0, 0.1)
    return conserved(rho, [np.zeros(n)], p, gamma).reshape(3, 1, 1, n)


# ---------------------------------------------------------------- 2D Euler
def euler2d_quadrants(nx, ny, seed, gamma=1.4):
    """Four-quadrant Riemann data on [0,1]^2: rho, p ~ U[0.1, 1.5], u, v ~ U[-1, 1]
    per quadrant, split point ~ U[0.4, 0.6]^2."""
    rng = np.random.default_rng(seed)
    q = rng.uniform(size=(4, 4))
    rho_q = 0.1 + 1.4 * q[:, 0]
    p_q = 0.1 + 1.4 * q[:, 1]
    u_q = -1.0 + 2.0 * q[:, 2]
    v_q = -1.0 + 2.0 * q[:, 3]
    xs, ys = rng.uniform(0.4, 0.6, size=2)
    x = centre_grid(nx, 0.0, 1.0)[None, :]
    y = centre_grid(ny, 0.0, 1.0)[:, None]
    quad = (x >= xs).astype(int) + 2 * (y >= ys).astype(int)
    U = conserved(rho_q[quad], [u_q[quad], v_q[quad]], p_q[quad], gamma)
    return U.reshape(4, 1, ny, nx)


def euler2d_random(nx, ny, seed, gamma=1.4, amp=0.2):
    """Smooth random perturbation of a uniform flow plus a jump (parity tests)."""
    rng = np.random.default_rng(seed)
    x = centre_grid(nx, 0.0, 1.0)[None, :]
    y = centre_grid(ny, 0.0, 1.0)[:, None]
    ph = rng.uniform(0, 2 * math.pi, size=4)
    rho = 1.0 + amp * np.sin(2 * math.pi * x + ph[0]) * np.cos(2 * math.pi * y + ph[1])
    rho = rho + 0.5 * (x + 0.3 * y > 0.55)
    u = 0.3 * np.sin(2 * math.pi * y + ph[2]) + 0 * x
    v = 0.3 * np.cos(2 * math.pi * x + ph[3]) + 0 * y
    p = 1.0 + 0.3 * (x - 0.5 * y > 0.2)
    return conserved(rho, [u, v], p, gamma).reshape(4, 1, ny, nx)


# ---------------------------------------------------------------- 3D Euler
def euler3d_blast(n, seed, gamma=1.4, nmodes=8, kmax=6):
    """Periodic [0,1]^3: rho = 1 + 0.3 S with S a sum of nmodes random Fourier
    modes (integer wave-vectors, |k| <= kmax, random phases) scaled to
    max|S| = 1; u = 0; p = 10 inside a sphere of radius U[0.1, 0.2] centred
    at U[0.3, 0.7]^3, p = 1 outside."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if 0 < np.linalg.norm(k) <= kmax:
            ks.append(k)
    ph = rng.uniform(0, 2 * math.pi, size=nmodes)
    centre = rng.uniform(0.3, 0.7, size=3)
    radius = rng.uniform(0.1, 0.2)
    x = centre_grid(n, 0.0, 1.0)
    S = np.zeros((n, n, n))
    X = x[None, None, :]
    Y = x[None, :, None]
    Z = x[:, None, None]
    for k, p in zip(ks, ph):
        S += np.cos(2 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + p)
    S /= np.abs(S).max()
    rho = 1.0 + 0.3 * S
    r2 = (X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2
    p = np.where(r2 < radius * radius, 10.0, 1.0)
    zero = np.zeros_like(rho)
    return conserved(rho, [zero, zero, zero], p, gamma).reshape(5, n, n, n)


# ---------------------------------------------------------------- batched 1D
def batch_sizes(nprob, seed, nmin=256, nmax=16384):
    """Problem lengths N_i = round(exp(U[ln nmin, ln nmax]))."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), size=nprob))).astype(np.int64)


def batch_states(sizes, seed, gamma=1.4):
    """Concatenated 1D Riemann states (problem i uses seed + i), shape (3, sum N)."""
    parts = [euler1d_riemann(int(n), seed + i, gamma).reshape(3, -1) for i, n in enumerate(sizes)]
    return np.concatenate(parts, axis=1)


# ------------------------------------------------ the paper's printed cases
# Initial data exactly as printed in Sec. 4 (no random draws); the paper
# shows only figures of the results, so these cases are checked by
# invariants, by parity with the oracle and against exact solutions where one
# exists (the Lax tube).

def composite_wave(n, lo=-1.0, hi=1.0):
    """Periodic advection of Gaussians, a square wave, a triangle and a half
    ellipse on [-1, 1] (the Jiang-Shu combination of Sec. 4.1), node grid."""
    x = node_grid(n, lo, hi)
    a, z, delta, alpha = 0.5, -0.7, 0.005, 10.0
    beta = math.log(2.0) / (36.0 * delta * delta)

    def G(zc):
        return np.exp(-beta * (x - zc) ** 2)

    def F(ac):
        return np.sqrt(np.maximum(1.0 - alpha * alpha * (x - ac) ** 2, 0.0))

    u = np.zeros(n)
    m = (x >= -0.8) & (x <= -0.6)
    u[m] = ((G(z - delta) + 4.0 * G(z) + G(z + delta)) / 6.0)[m]
    u[(x >= -0.4) & (x <= -0.2)] = 1.0
    m = (x >= 0.0) & (x <= 0.2)
    u[m] = (1.0 - 10.0 * np.abs(x - 0.1))[m]
    m = (x >= 0.4) & (x <= 0.6)
    u[m] = ((F(a - delta) + 4.0 * F(a) + F(a + delta)) / 6.0)[m]
    return u.reshape(1, 1, 1, n)


def lax_tube(n, gamma=1.4):
    """Lax's shock tube on [0, 2], jump at x = 1 (Sec. 4.2), cell centres."""
    x = centre_grid(n, 0.0, 2.0)
    isl = x < 1.0
    rho = np.where(isl, 0.445, 0.5)
    u = np.where(isl, 0.698, 0.0)
    p = np.where(isl, 3.528, 0.571)
    return conserved(rho, [u], p, gamma).reshape(3, 1, 1, n)


def titarev_toro(n, gamma=1.4):
    """Mach 1.1 shock meeting a high-frequency entropy wave on [-5, 5] (the
    Titarev-Toro case of Sec. 4.2), cell centres."""
    x = centre_grid(n, -5.0, 5.0)
    isl = x < -4.5
    rho = np.where(isl, 1.515695, 1.0 + 0.1 * np.sin(20.0 * math.pi * x))
    u = np.where(isl, 0.523346, 0.0)
    p = np.where(isl, 1.805, 1.0)
    return conserved(rho, [u], p, gamma).reshape(3, 1, 1, n)


def riemann2d(config, nx, ny, gamma=1.4):
    """The two 2D Riemann configurations of Sec. 4.3 on [-1, 1]^2, cell centres:
    config 1 (four shocks) or 2 (four contact discontinuities).  Quadrant
    states (rho, u, v, p) in the order (x < 0, y < 0), (x < 0, y > 0),
    (x > 0, y > 0), (x > 0, y < 0)."""
    states = {
        1: [(0.138, 1.206, 1.206, 0.029), (0.5323, 1.206, 0.0, 0.3),
            (1.5, 0.0, 0.0, 1.5), (0.5323, 0.0, 1.206, 0.3)],
        2: [(1.0, -0.75, 0.5, 1.0), (2.0, 0.75, 0.5, 1.0),
            (1.0, 0.75, -0.5, 1.0), (3.0, -0.75, -0.5, 1.0)],
    }[config]
    x = centre_grid(nx, -1.0, 1.0)[None, :]
    y = centre_grid(ny, -1.0, 1.0)[:, None]
    xp, yp = x > 0.0, y > 0.0
    quad = np.where(~xp & ~yp, 0, np.where(~xp & yp, 1, np.where(xp & yp, 2, 3)))
    s = np.array(states)
    U = conserved(s[quad, 0], [s[quad, 1], s[quad, 2]], s[quad, 3], gamma)
    return U.reshape(4, 1, ny, nx)
