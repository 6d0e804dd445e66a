"""The slab decomposition on the GPU: two or three sub-domain contexts of one
grid (enoao_create_subdomain) on the one GPU, stepped by domain.LocalGroup
with their halo layers staged through host buffers -- the stitched state must
equal the undivided grid's, bit for bit (every face is computed from the same
window either way; alpha and dt are the same maxima and quotients)."""
import numpy as np
import pytest

import paper_2108_12742_gb300 as eno
from paper_2108_12742_gb300 import domain, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12742_gb300 import build
    build.build()


def _run(shape, lo, hi, U, nslabs, steps, **kw):
    with eno.Solver(shape, lo, hi, **kw) as s:
        s.init_state(U)
        s.advance_steps(steps, 0.5)
        whole = s.get_state()
    n = shape[-1]
    order = kw.get("order", 5)
    ranges = domain.slab_ranges(n, nslabs, domain.halo_width(order))
    doms = [eno.SubDomain(shape, lo, hi, o, m, **kw) for o, m in ranges]
    try:
        axis = 4 - len(shape)  # the split axis in the (nv, nz, ny, nx) state layout
        for d, (o, m) in zip(doms, ranges):
            d.init_state(np.ascontiguousarray(np.take(U, range(o, o + m), axis=axis)))
        dx = [(hi[i] - lo[i]) / shape[i] for i in range(len(shape))]
        grp = domain.LocalGroup(doms, kw.get("bc", eno.TRANSMISSIVE), dx)
        for _ in range(steps):
            grp.step(0.5)
        parts = [d.get_state() for d in doms]
    finally:
        for d in doms:
            d.close()
    return whole, np.concatenate(parts, axis=axis)


@pytest.mark.parametrize("precision", [eno.FP64, eno.FP32_BULK])
@pytest.mark.parametrize("bc", [eno.TRANSMISSIVE, eno.PERIODIC])
@pytest.mark.parametrize("order,nslabs", [(5, 2), (7, 3)])
def test_2d_slabs_equal_the_undivided_grid(precision, bc, order, nslabs):
    shape = (70, 45)
    U = inputs.euler2d_quadrants(*shape, seed=3)
    whole, stitched = _run(shape, (0.0, 0.0), (1.0, 1.0), U, nslabs, 4, system=eno.EULER,
                           order=order, bc=bc, precision=precision)
    assert np.array_equal(whole, stitched)


@pytest.mark.parametrize("precision", [eno.FP64, eno.FP32_BULK])
def test_3d_slabs_equal_the_undivided_grid(precision):
    shape = (20, 18, 16)
    U = np.ascontiguousarray(inputs.euler3d_blast(20, seed=3)[:, :16, :18, :20])
    whole, stitched = _run(shape, (0.0,) * 3, (1.0,) * 3, U, 2, 2, system=eno.EULER, order=7,
                           bc=eno.PERIODIC, precision=precision)
    assert np.array_equal(whole, stitched)


def test_subdomain_rejections():
    shape, lo, hi = (40, 30), (0.0, 0.0), (1.0, 1.0)
    with pytest.raises(eno.EnoaoError) as e:
        eno.SubDomain(shape, lo, hi, 0, 3)           # fewer than G = 4 layers
    assert e.value.status == 1
    with pytest.raises(eno.EnoaoError) as e:
        eno.SubDomain(shape, lo, hi, 20, 11)         # beyond the grid
    assert e.value.status == 1
    with pytest.raises(eno.EnoaoError) as e:
        eno.SubDomain(shape, lo, hi, 0, 15, alpha_mode=eno.ALPHA_PER_STAGE)
    assert e.value.status == 1
    with eno.SubDomain(shape, lo, hi, 0, 15) as d:
        d.init_state(inputs.euler2d_quadrants(40, 15, seed=1))
        with pytest.raises(eno.EnoaoError) as e:
            d.advance_steps(1, 0.5)                  # steps need halo exchanges
        assert e.value.status == 1
        with pytest.raises(eno.EnoaoError) as e:
            d.halo_export(3, 0)
        assert e.value.status == 1
