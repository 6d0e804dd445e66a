"""Per-field (component-wise) Lax-Friedrichs splitting on the GPU against the
oracle's per-field reading (ENOAO_ALPHA_PER_FIELD): interface fluxes and
choices, whole FP64 steps to 1e-12, FP32-bulk stages on their own inputs, and
the option's limits (batched contexts, the grid-wide re-decision pass)."""
import numpy as np
import pytest

import oracle
import paper_2108_12742_gb300 as eno
from paper_2108_12742_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_FLUX = 1e-6
TOL32_STEP = 1e-7
TOL32_L1 = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12742_gb300 import build
    build.build()
    oracle.build()


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


CASES = {
    "euler1d-riemann-ao5": ((300,), eno.TRANSMISSIVE, 5, lambda: inputs.euler1d_riemann(300, seed=2)),
    "euler1d-periodic-ao7": ((150,), eno.PERIODIC, 7, lambda: inputs.euler1d_riemann(150, seed=6)),
    "euler2d-quad-ao5": ((70, 45), eno.TRANSMISSIVE, 5, lambda: inputs.euler2d_quadrants(70, 45, seed=1)),
    "euler2d-random-ao7": ((40, 37), eno.PERIODIC, 7, lambda: inputs.euler2d_random(40, 37, seed=2)),
    "euler3d-blast-ao7": ((20, 18, 16), eno.PERIODIC, 7,
                          lambda: inputs.euler3d_blast(20, seed=3)[:, :16, :18, :20].copy()),
}


def _pair(name, precision):
    shape, bc, order, init = CASES[name]
    nd = len(shape)
    lo, hi = (0.0,) * nd, (1.0,) * nd
    s = eno.Solver(shape, lo, hi, system=eno.EULER, order=order, bc=bc, precision=precision,
                   alpha_mode=eno.ALPHA_PER_FIELD)
    P = oracle.make_problem(shape, lo, hi, system=oracle.EULER, order=order, bc=bc,
                            alpha_per_field=True)
    return s, P, np.ascontiguousarray(init())


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_fluxes_and_choices_match_oracle(name):
    s, P, U0 = _pair(name, eno.FP64)
    with s:
        s.init_state(U0)
        for d in range(len(s.shape)):
            F, idx = s.reconstruct_fluxes(d, want_idx=True)
            Fo, io, gap = oracle.fluxes(P, U0, d, want_idx=True)
            differ = idx != io
            assert not (differ & (gap > 1e-13)).any(), (d, int(differ.sum()))
            face_ok = ~differ.any(axis=(0, 1))
            assert relerr(F[:, face_ok], Fo[:, face_ok]) <= TOL64, d


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_steps_match_oracle(name):
    s, P, U0 = _pair(name, eno.FP64)
    with s:
        U = U0
        for k in range(3):  # per step, from identical input states
            s.init_state(U)
            s.advance(1e9, cfl=0.5, max_steps=1)
            st = s.stats()
            got = s.get_state()
            ref = oracle.step(P, U, st.dt)
            assert relerr(got, ref) <= TOL64, (k, relerr(got, ref))
            # dt follows the one-alpha spectral radius, the largest field constant
            a = oracle.alpha_fields(P, U).max(axis=1)
            for d in range(len(s.shape)):
                assert st.alpha[d] == pytest.approx(a[d], rel=1e-14)
            U = got
        # three steps in one call (alpha and dt of steps 2 and 3 from the GPU's
        # own running maxima) against the oracle's three steps
        s.init_state(U0)
        s.advance(1e9, cfl=0.5, max_steps=3)
        ref, _, k = oracle.advance(P, U0, 1e9, cfl=0.5, max_steps=3)
        assert k == 3 and s.stats().steps == 3
        assert relerr(s.get_state(), ref) <= 1e-11
        # the option is live: the one-alpha step differs
        P1 = oracle.make_problem(s.shape, (0.0,) * len(s.shape), (1.0,) * len(s.shape),
                                 system=oracle.EULER, order=P.order, bc=P.bc[0])
        assert relerr(oracle.step(P1, U0, 1e-4), oracle.step(P, U0, 1e-4)) > 1e-9


@pytest.mark.parametrize("name", ["euler1d-riemann-ao5", "euler2d-random-ao7", "euler3d-blast-ao7"])
def test_fp32_bulk_fluxes_and_stages(name):
    # fluxes at the FP32-bulk tolerance, then each Runge-Kutta stage against the
    # oracle's operator on the stage input this path produced
    s, P, U = _pair(name, eno.FP32_BULK)
    shape = s.shape
    with s:
        s.set_redecide(eno.REDECIDE_GRID)
        assert not s.uses_grid_redecide()  # per-field splitting re-decides in the sweep
        s.init_state(U)
        agree = total = 0
        for d in range(len(shape)):
            F, idx = s.reconstruct_fluxes(d, want_idx=True)
            Fo, io, _ = oracle.fluxes(P, U, d, want_idx=True)
            agree += int((idx == io).sum())
            total += idx.size
            assert relerr(F, Fo) <= TOL32_FLUX, (d, relerr(F, Fo))
        assert agree / total >= 0.999
        af = oracle.alpha_fields(P, U)
        dt = 0.5 / sum(af[d].max() * shape[d] for d in range(len(shape)))
        G = [U]
        for k in range(3):
            s.rk_stage(k, dt)
            G.append(s.get_stage_state(k + 1) if k < 2 else s.get_state())
            Lk = oracle.rhs(P, G[k], af)
            if k == 0:
                ref = U + dt * Lk
            elif k == 1:
                ref = 0.75 * U + 0.25 * (G[1] + dt * Lk)
            else:
                ref = U / 3.0 + 2.0 / 3.0 * (G[2] + dt * Lk)
            assert relerr(G[k + 1], ref) <= TOL32_STEP, (k, relerr(G[k + 1], ref))
            assert np.abs(G[k + 1] - ref).mean() / np.abs(ref).mean() <= TOL32_L1, k


def test_tiles_do_not_change_per_field_results():
    n = (130, 75)
    U0 = inputs.euler2d_quadrants(*n, seed=3)
    for prec in (eno.FP64, eno.FP32_BULK):
        outs = []
        for tiles in (None, ((1, 31), (16, 7)), ((4, 255), (64, 15))):
            with eno.Solver(n, (0.0, 0.0), (1.0, 1.0), system=eno.EULER, order=5,
                            precision=prec, alpha_mode=eno.ALPHA_PER_FIELD) as s:
                if tiles:
                    for d, (ta, ts) in enumerate(tiles):
                        s.set_tiles(d, ta, ts)
                s.init_state(U0)
                s.advance(1e9, cfl=0.5, max_steps=3)
                outs.append(s.get_state())
        assert all(np.array_equal(outs[0], o) for o in outs[1:]), prec


def test_batched_contexts_reject_per_field():
    with pytest.raises(eno.EnoaoError):
        eno.Batch([64, 80], [0.0, 0.0], [1.0, 1.0], system=eno.EULER,
                        alpha_mode=eno.ALPHA_PER_FIELD)
