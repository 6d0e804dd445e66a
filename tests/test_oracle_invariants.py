"""Invariants that pin the oracle's multi-dimensional and characteristic code:
exact preservation of constant states, conservation, the f^- mirror rule,
eigenvector inversion, reduction of 2D to 1D and axis-swap symmetry."""
import numpy as np
import pytest

from paper_2108_12742_gb300 import inputs


def _const_state(system, shape, seed):
    rng = np.random.default_rng(seed)
    ndim = len(shape)
    full = tuple(shape) + (1,) * (3 - ndim)
    if system == 0:
        return np.full((1, full[2], full[1], full[0]), rng.uniform(-2, 2))
    vel = list(rng.uniform(-1, 1, size=ndim))
    U = inputs.conserved(rng.uniform(0.2, 2.0), vel, rng.uniform(0.2, 2.0), 1.4)
    return np.broadcast_to(U.reshape(-1, 1, 1, 1), (ndim + 2, full[2], full[1], full[0])).copy()


@pytest.mark.parametrize("system", [0, 1])
@pytest.mark.parametrize("shape", [(24,), (16, 13), (12, 11, 10)])
@pytest.mark.parametrize("order", [5, 7])
@pytest.mark.parametrize("bc", [0, 1])
def test_constant_state_is_preserved_bitwise(oracle_mod, system, shape, order, bc):
    U0 = _const_state(system, shape, seed=len(shape) * 10 + order + bc)
    P = oracle_mod.make_problem(shape, [0.0] * len(shape), [1.0] * len(shape),
                                system=system, order=order, bc=bc)
    # every interface carries the same value, so L(u) vanishes bit for bit ...
    assert not oracle_mod.rhs(P, U0).any()
    # ... and the Shu-Osher combinations (3/4, 1/4), (1/3, 2/3) only round
    U, _, _ = oracle_mod.advance(P, U0, 1.0, cfl=0.5, max_steps=2)
    assert np.abs(U - U0).max() <= 8 * np.spacing(np.abs(U0).max())


@pytest.mark.parametrize("order", [5, 7])
def test_periodic_conservation(oracle_mod, order):
    n = 32
    U0 = inputs.euler2d_random(n, n, seed=5)
    P = oracle_mod.make_problem((n, n), (0.0, 0.0), (1.0, 1.0), order=order,
                                bc=oracle_mod.PERIODIC)
    steps = 3
    U, _, k = oracle_mod.advance(P, U0, 10.0, cfl=0.4, max_steps=steps)
    assert k == steps
    eps = np.finfo(float).eps
    for v in range(4):
        bound = 10 * U0[v].size * eps * np.abs(U0[v]).max() * steps
        assert abs(U[v].sum() - U0[v].sum()) <= bound, v


@pytest.mark.parametrize("order", [5, 7])
def test_negative_speed_is_the_mirror_image(oracle_mod, order):
    # f = -u, alpha = 1 puts everything into f^-; on reflected data the result
    # must be the reflection of the f = +u run, bit for bit (Sec. 3.2 mirror rule).
    n = 40
    U0 = inputs.advection_random(n, seed=9).ravel()
    ref = np.roll(U0[::-1], 1)           # node j -> node (-j) mod n
    Pp = oracle_mod.make_problem((n,), (-1.0,), (1.0,), system=0, order=order, bc=0, adv_speed=1.0)
    Pm = oracle_mod.make_problem((n,), (-1.0,), (1.0,), system=0, order=order, bc=0, adv_speed=-1.0)
    a = oracle_mod.rhs(Pp, U0.reshape(1, 1, 1, n)).ravel()
    b = oracle_mod.rhs(Pm, ref.reshape(1, 1, 1, n)).ravel()
    assert np.array_equal(np.roll(b[::-1], 1), a)
    ua, _, _ = oracle_mod.advance(Pp, U0.reshape(1, 1, 1, n), 0.3, cfl=0.5)
    ub, _, _ = oracle_mod.advance(Pm, ref.reshape(1, 1, 1, n), 0.3, cfl=0.5)
    assert np.array_equal(np.roll(ub.ravel()[::-1], 1), ua.ravel())


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_left_eigenvectors_invert_right(oracle_mod, ndim):
    rng = np.random.default_rng(ndim)
    for _ in range(20):
        vel = rng.uniform(-2, 2, size=ndim)
        c2 = rng.uniform(0.1, 4.0)
        H = c2 / 0.4 + 0.5 * vel @ vel
        R, L = oracle_mod.euler_eigen(ndim, 1.4, vel, H)
        assert np.abs(L @ R - np.eye(ndim + 2)).max() < 1e-13
        # R's columns are eigenvectors of the flux Jacobian with eigenvalues u-c, u.., u+c
        c = np.sqrt(c2)
        lam = np.array([vel[0] - c] + [vel[0]] * ndim + [vel[0] + c])
        A = R @ np.diag(lam) @ L
        # the Jacobian's first row is (0, 1, 0.., 0) in conserved variables
        assert np.abs(A[0] - np.eye(ndim + 2)[1]).max() < 1e-12


@pytest.mark.parametrize("order", [5, 7])
def test_y_constant_2d_field_reduces_to_1d(oracle_mod, order):
    nx, ny = 48, 6
    U1 = inputs.euler1d_riemann(nx, seed=4)
    U2 = np.zeros((4, 1, ny, nx))
    U2[0] = U1[0]
    U2[1] = U1[1]
    U2[3] = U1[2]
    P1 = oracle_mod.make_problem((nx,), (0.0,), (1.0,), order=order)
    P2 = oracle_mod.make_problem((nx, ny), (0.0, 0.0), (1.0, 1.0), order=order)
    a1 = oracle_mod.alpha(P1, U1)
    a2 = oracle_mod.alpha(P2, U2)
    assert a1[0] == a2[0]
    r1 = oracle_mod.rhs(P1, U1, a1)
    r2 = oracle_mod.rhs(P2, U2, a2)
    for row in range(ny):
        assert np.array_equal(r2[0, 0, row], r1[0, 0, 0])
        assert np.array_equal(r2[1, 0, row], r1[1, 0, 0])
        assert np.array_equal(r2[3, 0, row], r1[2, 0, 0])
    assert not r2[2].any()


@pytest.mark.parametrize("order", [5, 7])
def test_axis_swap_symmetry(oracle_mod, order):
    n = 24
    U = inputs.euler2d_random(n, n, seed=8)
    T = np.stack([U[0, 0].T, U[2, 0].T, U[1, 0].T, U[3, 0].T])[:, None]
    P = oracle_mod.make_problem((n, n), (0.0, 0.0), (1.0, 1.0), order=order)
    a = oracle_mod.advance(P, U, 1.0, cfl=0.4, max_steps=2)[0]
    b = oracle_mod.advance(P, T, 1.0, cfl=0.4, max_steps=2)[0]
    bt = np.stack([b[0, 0].T, b[2, 0].T, b[1, 0].T, b[3, 0].T])[:, None]
    assert np.array_equal(a, bt)


def test_3d_axis_cycle_symmetry(oracle_mod):
    n = 12
    U = inputs.euler3d_blast(n, seed=2)
    # relabel the axes (x', y', z') = (y, z, x) together with the momenta
    def cyc(V):
        t = lambda a: np.transpose(a, (2, 0, 1))
        return np.stack([t(V[0]), t(V[2]), t(V[3]), t(V[1]), t(V[4])])
    P = oracle_mod.make_problem((n, n, n), (0.0,) * 3, (1.0,) * 3, order=7, bc=0)
    a = oracle_mod.rhs(P, U)
    b = oracle_mod.rhs(P, cyc(U))
    assert np.allclose(cyc(a), b, rtol=0, atol=1e-12 * np.abs(a).max())


# ------------------------------------------------------------- per-stage alpha
# Sec. 2 fixes alpha as the largest |f'(u)| over the mesh without saying on
# which state; the per-stage option evaluates it on each Runge-Kutta stage's
# input state (dt still from U^n).

def test_per_stage_alpha_is_inert_for_advection(oracle_mod):
    # f = a u: |f'| = |a| on every state, so both options give the same bits
    n = 64
    U0 = inputs.advection_random(n, seed=12)
    P1 = oracle_mod.make_problem((n,), (-1.0,), (1.0,), system=0, order=7, bc=0, adv_speed=0.9)
    P2 = oracle_mod.make_problem((n,), (-1.0,), (1.0,), system=0, order=7, bc=0, adv_speed=0.9,
                                 alpha_per_stage=True)
    assert np.array_equal(oracle_mod.step(P1, U0, 0.01), oracle_mod.step(P2, U0, 0.01))


def test_per_stage_alpha_where_the_fastest_cell_is_untouched(oracle_mod):
    # The fastest cells (|u| + c largest) sit in a constant stretch that no wave
    # reaches within one step, so every stage sees the same alpha: the two
    # options agree bit for bit.  With the fastest cells inside the moving
    # part, the stage alphas change and so does the result.
    n = 200
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.3, 1.0, 0.125)
    p = np.where(x < 0.3, 1.0, 0.1)
    u = np.where(x > 0.85, 1.5, 0.0)   # fast, uniform right end, far from the jump at 0.3
    U = np.stack([rho, rho * u, p / 0.4 + 0.5 * rho * u * u]).reshape(3, 1, 1, n)
    P1 = oracle_mod.make_problem((n,), (0.0,), (1.0,), order=5)
    P2 = oracle_mod.make_problem((n,), (0.0,), (1.0,), order=5, alpha_per_stage=True)
    a = oracle_mod.alpha(P1, U)
    # the max is attained in x > 0.85, where no wave arrives in one small step;
    # the velocity jump at 0.85 itself moves, so keep dt small against it
    dt = 0.1 / n / a[0]
    fast = x > 0.9
    assert np.abs(U[1, 0, 0] / U[0, 0, 0])[fast].max() + np.sqrt(1.4 * 0.1 / 0.125) == pytest.approx(a[0])
    r1, r2 = oracle_mod.step(P1, U, dt), oracle_mod.step(P2, U, dt)
    assert np.array_equal(r1[:, :, :, fast], r2[:, :, :, fast])
    # the whole step agrees only if the stage alphas did not move; they do not
    # here because the fastest cells stay bitwise constant
    assert np.array_equal(r1, r2)

    # now put the fastest gas in the compressing region: stage alphas differ
    u2 = np.where((x > 0.25) & (x < 0.35), 2.0, 0.0)
    U2 = np.stack([rho, rho * u2, p / 0.4 + 0.5 * rho * u2 * u2]).reshape(3, 1, 1, n)
    dt2 = 0.5 / n / oracle_mod.alpha(P1, U2)[0]
    s1, s2 = oracle_mod.step(P1, U2, dt2), oracle_mod.step(P2, U2, dt2)
    d = np.abs(s1 - s2).max() / np.abs(s1).max()
    assert 0.0 < d < 1e-2


@pytest.mark.parametrize("order", [5, 7])
def test_per_stage_alpha_conserves_and_keeps_constants(oracle_mod, order):
    n = 24
    U0 = inputs.euler2d_random(n, n, seed=8)
    P = oracle_mod.make_problem((n, n), (0.0, 0.0), (1.0, 1.0), order=order,
                                bc=oracle_mod.PERIODIC, alpha_per_stage=True)
    U, _, k = oracle_mod.advance(P, U0, 10.0, cfl=0.4, max_steps=2)
    assert k == 2
    eps = np.finfo(float).eps
    for v in range(4):
        assert abs(U[v].sum() - U0[v].sum()) <= 10 * U0[v].size * eps * np.abs(U0[v]).max() * 2
    C = _const_state(1, (16, 13), seed=3)
    Pc = oracle_mod.make_problem((16, 13), (0.0, 0.0), (1.0, 1.0), order=order, bc=1,
                                 alpha_per_stage=True)
    Uc, _, _ = oracle_mod.advance(Pc, C, 1.0, cfl=0.5, max_steps=2)
    assert np.abs(Uc - C).max() <= 8 * np.spacing(np.abs(C).max())
