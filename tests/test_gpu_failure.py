"""Failure detection and checkpoint/resume on the GPU, in the forms that fault,
trap or hang nothing: a bounded device wait made to run out (a pass bound set
to zero), non-physical states planted on the host or reached by the flow, each
coming back as a status code with the context still usable; and a run saved
with enoao_get_state and restarted with enoao_init_state that reproduces the
uninterrupted run bit for bit."""
import numpy as np
import pytest

import paper_2108_12742_gb300 as eno
from paper_2108_12742_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12742_gb300 import build
    build.build()


def _riemann2(n, order=5, precision=eno.FP32_BULK):
    s = eno.Solver((n, n), (-1.0, -1.0), (1.0, 1.0), system=eno.EULER, order=order,
                   bc=eno.TRANSMISSIVE, precision=precision)
    return s, inputs.riemann2d(2, n, n)


def test_redecision_pass_bound_runs_out_as_a_timeout_status():
    s, U = _riemann2(160)
    with s:
        s.set_redecide(eno.REDECIDE_IN_SWEEP)
        s.init_state(U)
        s.advance_steps(3, 0.5)
        assert s.stats().fp64_fallbacks > 0  # the data has near-ties to re-decide
        s.set_redecide_pass_limit(0)
        s.init_state(U)
        with pytest.raises(eno.EnoaoError) as e:
            s.advance_steps(3, 0.5)
        assert e.value.status == 5 and "timed out" in str(e.value)
        # the wait returned and the context is usable again
        s.set_redecide_pass_limit(-1)
        s.init_state(U)
        s.advance_steps(3, 0.5)
        assert np.isfinite(s.get_state()).all()


def test_pass_limit_rejects_bad_values():
    s, U = _riemann2(32)
    with s:
        with pytest.raises(eno.EnoaoError) as e:
            s.set_redecide_pass_limit(-2)
        assert e.value.status == 1


@pytest.mark.parametrize("precision", [eno.FP64, eno.FP32_BULK])
@pytest.mark.parametrize("what", [0, 3])  # NaN density, NaN energy
def test_planted_nan_is_reported_with_its_cell(precision, what):
    n = (40, 24)
    U = inputs.euler2d_quadrants(*n, seed=4)
    x, y = 17, 9
    U[what, 0, y, x] = np.nan
    with eno.Solver(n, (0.0, 0.0), (1.0, 1.0), system=eno.EULER, order=5,
                    precision=precision) as s:
        with pytest.raises(eno.EnoaoError) as e:
            s.init_state(U)
        assert e.value.status == 4 and f"at cell {y * n[0] + x}" in str(e.value)
        s.init_state(inputs.euler2d_quadrants(*n, seed=4))   # usable again
        s.advance_steps(2, 0.5)


@pytest.mark.parametrize("precision", [eno.FP64, eno.FP32_BULK])
def test_vacuum_from_a_double_rarefaction_is_reported(precision):
    # two gases flying apart at Mach ~25 open a vacuum at x = 0.5; the
    # scheme is not positivity preserving, so the pressure there turns
    # negative within a few steps (the oracle: at step 3, cell 99)
    n = 200
    x = (np.arange(n) + 0.5) / n
    rho, u, p = np.ones(n), np.where(x < 0.5, -3.0, 3.0), np.full(n, 0.01)
    U = np.stack([rho, rho * u, p / 0.4 + 0.5 * rho * u * u]).reshape(3, 1, 1, n)
    with eno.Solver((n,), (0.0,), (1.0,), system=eno.EULER, order=5, precision=precision) as s:
        s.init_state(U)
        with pytest.raises(eno.EnoaoError) as e:
            s.advance(1.0, cfl=0.5, max_steps=20)
        assert e.value.status == 4
        cell = int(str(e.value).rsplit("at cell ", 1)[1].split()[0])
        assert 80 <= cell <= 120, cell
        s.init_state(inputs.euler1d_riemann(n, seed=1))   # usable again
        s.advance(1.0, cfl=0.5, max_steps=5)


@pytest.mark.parametrize("alpha_mode", [eno.ALPHA_PER_STEP, eno.ALPHA_PER_STAGE])
@pytest.mark.parametrize("precision", [eno.FP64, eno.FP32_BULK])
def test_checkpoint_restart_reproduces_the_run_bitwise(precision, alpha_mode):
    n, k = (96, 80), 6
    U = inputs.euler2d_quadrants(*n, seed=7)
    kw = dict(system=eno.EULER, order=5, precision=precision, alpha_mode=alpha_mode)
    with eno.Solver(n, (0.0, 0.0), (1.0, 1.0), **kw) as s:
        s.init_state(U)
        s.advance_steps(2 * k, 0.5)
        straight = s.get_state()
    with eno.Solver(n, (0.0, 0.0), (1.0, 1.0), **kw) as s:
        s.init_state(U)
        s.advance_steps(k, 0.5)
        saved = s.get_state()
    with eno.Solver(n, (0.0, 0.0), (1.0, 1.0), **kw) as s:
        s.init_state(saved)
        s.advance_steps(k, 0.5)
        resumed = s.get_state()
    assert np.array_equal(straight, resumed)


@pytest.mark.parametrize("precision", [eno.FP64, eno.FP32_BULK])
def test_batched_checkpoint_restart_is_bitwise(precision):
    sizes = inputs.batch_sizes(24, seed=5, nmin=64, nmax=1024)
    U = inputs.batch_states(sizes, seed=50)
    kw = dict(system=eno.EULER, order=5, precision=precision)
    with eno.Batch(sizes, 0.0, 1.0, **kw) as b:
        b.init_state(U)
        b.advance_steps(16, 0.5)
        straight = b.get_state()
    with eno.Batch(sizes, 0.0, 1.0, **kw) as b:
        b.init_state(U)
        b.advance_steps(8, 0.5)
        saved = b.get_state()
        b.init_state(saved)
        b.advance_steps(8, 0.5)
        resumed = b.get_state()
    assert np.array_equal(straight, resumed)
