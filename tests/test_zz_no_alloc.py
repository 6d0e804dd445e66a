"""enoao_step_noalloc: one Runge-Kutta step of a 1D problem that allocates no
device memory (for callers whose device memory is fully reserved up front, or
whose time loop must not pay cudaMalloc's implicit synchronisation).  Its
output must match the regular entry points (enoao_create + enoao_rk_stage) on
the same input and dt, within the parity tolerances of the other GPU tests,
on two calls in a row (the second call starts from the first one's output
and reuses the fixed scratch array the first call left behind)."""
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


def _regular_step(shape_kw, U, dt):
    with eno.Solver(**shape_kw) as s:
        s.init_state(U.reshape(s.state_shape))
        for k in range(3):
            s.rk_stage(k, dt)
        return s.get_state().reshape(U.shape)


@pytest.mark.parametrize("system,order,precision,n,bc,alpha_mode", [
    (eno.EULER, 5, eno.FP64, 2000, eno.TRANSMISSIVE, eno.ALPHA_PER_STEP),
    (eno.EULER, 7, eno.FP32_BULK, 777, eno.TRANSMISSIVE, eno.ALPHA_PER_STEP),
    (eno.SCALAR_ADVECTION, 5, eno.FP64, 200, eno.PERIODIC, eno.ALPHA_PER_STEP),
    (eno.EULER, 5, eno.FP64, 1000, eno.TRANSMISSIVE, eno.ALPHA_PER_STAGE),
])
def test_noalloc_step_matches_regular_path_twice(system, order, precision, n, bc, alpha_mode):
    import torch
    lo, hi = (0.0, 1.0) if system == eno.EULER else (-1.0, 1.0)
    kw = dict(shape=(n,), lo=(lo,), hi=(hi,), system=system, order=order, precision=precision,
              bc=bc, alpha_mode=alpha_mode)
    cfg = eno.make_config((n,), (lo,), (hi,), system=system, order=order, precision=precision,
                          bc=bc, alpha_mode=alpha_mode)
    if system == eno.EULER:
        U = inputs.euler1d_riemann(n, seed=11).reshape(3, n)
        dt = 0.2 / n
    else:
        U = inputs.advection_square(n, seed=2).reshape(1, n)
        dt = 0.5 * (hi - lo) / n
    tol = 1e-12 if precision == eno.FP64 else 1e-7
    cur = U
    for call in range(2):
        d_in = torch.from_numpy(np.ascontiguousarray(cur)).cuda()
        d_out = torch.empty_like(d_in)
        eno.step_noalloc(cfg, d_in, d_out, dt)
        got = d_out.cpu().numpy()
        ref = _regular_step(kw, cur, dt)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= tol, (call, err)
        cur = got


def test_noalloc_rejects_sizes_beyond_its_fixed_array():
    import torch
    n = (1 << 18) + 1
    cfg = eno.make_config((n,), (0.0,), (1.0,), system=eno.EULER, order=5)
    U = torch.ones((3, n), dtype=torch.float64, device="cuda")
    with pytest.raises(eno.EnoaoError) as e:
        eno.step_noalloc(cfg, U, U, 1e-4)
    assert e.value.status == 1 and "at most 262144" in str(e.value)
