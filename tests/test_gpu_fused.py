"""The fused 2D stage (enoao_set_fused_stage): both axes of a Runge-Kutta
stage in one launch, on 2D tiles whose x part a block stores and reads back
itself.  Every face is computed from the same window and every cell combines
the same two axis parts as with one launch per axis, so the states, alpha
and dt must be the same bits; the per-axis path is itself parity-tested
against the oracle."""
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


def _run(shape, U, steps, fused, tiles=(0, 0, 0, 0), **kw):
    with eno.Solver(shape, (0.0, 0.0), (1.0, 1.0), precision=eno.FP32_BULK, **kw) as s:
        s.init_state(U)
        if fused:
            s.set_fused_stage(True, tiles)
        s.advance_steps(steps, 0.5)
        st = s.stats()
        return s.get_state(), np.array(st.alpha[:]), st.dt, st.steps


@pytest.mark.parametrize("order", [5, 7])
@pytest.mark.parametrize("bc", [eno.TRANSMISSIVE, eno.PERIODIC])
@pytest.mark.parametrize("tiles", [(0, 0, 0, 0), (2, 32, 16, 32), (8, 128, 8, 24)])
def test_fused_stage_gives_the_per_axis_bits_euler(order, bc, tiles):
    # a grid that is not a whole number of 2D tiles along either axis
    shape = (150, 101)
    U = inputs.euler2d_quadrants(*shape, seed=5)
    ref = _run(shape, U, 4, False, system=eno.EULER, order=order, bc=bc)
    got = _run(shape, U, 4, True, tiles, system=eno.EULER, order=order, bc=bc)
    assert np.array_equal(got[0], ref[0])
    assert np.array_equal(got[1], ref[1]) and got[2] == ref[2] and got[3] == ref[3]


@pytest.mark.parametrize("order", [5, 7])
def test_fused_stage_gives_the_per_axis_bits_advection(order):
    nx, ny = 96, 70
    rng = np.random.default_rng(2)
    U = np.ascontiguousarray(rng.uniform(-1, 1, size=(1, 1, ny, nx)))
    kw = dict(system=eno.SCALAR_ADVECTION, order=order, bc=eno.PERIODIC)
    ref = _run((nx, ny), U, 3, False, **kw)
    got = _run((nx, ny), U, 3, True, **kw)
    assert np.array_equal(got[0], ref[0]) and got[2] == ref[2]


def test_fused_stage_on_evolved_data_with_re_decisions():
    # after 30 steps of the four-quadrant problem there are near-ties to re-decide
    shape = (256, 192)
    U = inputs.euler2d_quadrants(*shape, seed=1)
    ref = _run(shape, U, 30, False, system=eno.EULER, order=5)
    got = _run(shape, U, 30, True, system=eno.EULER, order=5)
    assert np.array_equal(got[0], ref[0])


def test_fused_stage_rejections():
    with eno.Solver((64,), (0.0,), (1.0,), precision=eno.FP32_BULK) as s:
        with pytest.raises(eno.EnoaoError) as e:
            s.set_fused_stage(True)
        assert e.value.status == 1
    with eno.Solver((64, 48), (0.0, 0.0), (1.0, 1.0), precision=eno.FP32_BULK) as s:
        with pytest.raises(eno.EnoaoError) as e:
            s.set_fused_stage(True, (4, 64, 8, 30))   # y cells not a multiple of x lines
        assert e.value.status == 1
        with pytest.raises(eno.EnoaoError) as e:
            s.set_fused_stage(True, (3, 64, 8, 48))   # x lines not 1, 2, 4 or 8
        assert e.value.status == 1
        s.set_fused_stage(True)
        s.set_fused_stage(False)
