"""Parity at the benchmarked sizes, on the parts the oracle can compute one by
one: the 3D Euler workload at 512^3 (periodic blast, ENO-AO7) on patches,
and the batched workload of 4096 uneven 1D problems on sampled problems.  The
2D 4096^2 workload has its patch test in test_gpu_parity.py."""
import numpy as np
import pytest

import paper_2108_12742_gb300 as eno
from paper_2108_12742_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_STEP = 1e-7
TOL32_L1 = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2108_12742_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def oracle():
    import oracle as o
    o.build()
    return o


def relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _block(dev, start, size):
    """A periodic (wrapped) block of a device state (nv, nz, ny, nx) -> numpy."""
    import torch
    nv, nz, ny, nx = dev.shape
    idx = [torch.arange(start[k], start[k] + size, device=dev.device) % dim
           for k, dim in enumerate((nx, ny, nz))]
    b = dev.index_select(3, idx[0]).index_select(2, idx[1]).index_select(1, idx[2])
    return np.ascontiguousarray(b.cpu().numpy())


N3 = 512
CORE = 16


def _corners(dev):
    # random interior patches, one across the periodic corner of the domain
    # (the wrap is part of the path), one on the edge of the pressure sphere
    import torch
    rng = np.random.default_rng(0)
    pts = [tuple(int(v) for v in rng.integers(0, N3, size=3)) for _ in range(3)]
    pts.append((N3 - CORE // 2, N3 - CORE // 2, N3 - CORE // 2))
    E = dev[4]
    jump = torch.nonzero((E[:, :, 1:] - E[:, :, :-1]).abs() > 1.0)  # p jumps 1 -> 10 there
    z, y, x = (int(v) for v in jump[len(jump) // 2])
    pts.append((x - CORE // 2, y - CORE // 2, z - CORE // 2))
    return pts


@pytest.fixture(scope="module")
def blast512():
    import torch
    U0 = inputs.euler3d_blast(N3, seed=1)
    return torch.from_numpy(U0).cuda()


def test_full_size_3d_workload_fp64_sampled_patches(oracle, blast512):
    # one FP64 step of the 512^3 workload; the oracle re-does that step on
    # patches of the same input with the GPU's alpha and dt; a patch keeps a
    # 15-cell margin (three stages x the 5-cell reach of ENO-AO7)
    import torch
    n, m = N3, 15
    with eno.Solver((n, n, n), (0.0,) * 3, (1.0,) * 3, system=eno.EULER, order=7,
                    bc=eno.PERIODIC) as s:
        s.init_state(blast512)
        s.advance(1e9, cfl=0.5, max_steps=1)
        st = s.stats()
        out = torch.empty_like(blast512)
        s.get_state(out)
    B = CORE + 2 * m
    P = oracle.make_problem((B, B, B), (0.0,) * 3, (B / n,) * 3, system=oracle.EULER, order=7,
                            bc=oracle.TRANSMISSIVE)
    a0 = oracle.alpha(oracle.make_problem((n, n, n), (0.0,) * 3, (1.0,) * 3,
                                          system=oracle.EULER, order=7, bc=oracle.PERIODIC),
                      blast512.cpu().numpy())
    assert np.allclose(st.alpha[:3], a0[:3], rtol=1e-14, atol=0)
    for c in _corners(blast512):
        blk = _block(blast512, [v - m for v in c], B)
        ref = oracle.step_alpha(P, blk, st.dt, np.array(st.alpha[:]))[:, m:m + CORE, m:m + CORE,
                                                                     m:m + CORE]
        got = _block(out, c, CORE)
        assert relerr(got, ref) <= TOL64, (c, relerr(got, ref))


def test_full_size_3d_workload_fp32_bulk_stages_on_patches(oracle, blast512):
    # FP32 bulk, stage by stage on the stage inputs this path produced (a
    # near-tie of a later stage may flip either way at FP32 rounding, so a
    # whole step is not compared cell by cell), each on patches with a 6-cell
    # margin (one stage reaches 5 cells)
    import torch
    n, m = N3, 6
    B = CORE + 2 * m
    P = oracle.make_problem((B, B, B), (0.0,) * 3, (B / n,) * 3, system=oracle.EULER, order=7,
                            bc=oracle.TRANSMISSIVE)
    corners = _corners(blast512)
    with eno.Solver((n, n, n), (0.0,) * 3, (1.0,) * 3, system=eno.EULER, order=7,
                    bc=eno.PERIODIC, precision=eno.FP32_BULK) as s:
        s.init_state(blast512)
        dt = 2e-4
        G = [blast512]
        for k in range(3):
            s.rk_stage(k, dt)
            nxt = torch.empty_like(blast512)
            if k < 2:
                s.get_stage_state(k + 1, nxt)
            else:
                s.get_state(nxt)
            alpha = np.array(s.stats().alpha[:])
            for c in corners:
                L = oracle.rhs(P, _block(G[k], [v - m for v in c], B), alpha)[
                    :, m:m + CORE, m:m + CORE, m:m + CORE]
                u0 = _block(G[0], c, CORE)
                uk = _block(G[k], c, CORE)
                if k == 0:
                    ref = u0 + dt * L
                elif k == 1:
                    ref = 0.75 * u0 + 0.25 * (uk + dt * L)
                else:
                    ref = u0 / 3.0 + 2.0 / 3.0 * (uk + dt * L)
                got = _block(nxt, c, CORE)
                assert relerr(got, ref) <= TOL32_STEP, (k, c, relerr(got, ref))
                assert np.abs(got - ref).mean() / np.abs(ref).mean() <= TOL32_L1, (k, c)
            G.append(nxt)


@pytest.mark.parametrize("precision", [eno.FP64, eno.FP32_BULK])
def test_full_batch_sampled_problems(oracle, precision):
    # the 4096-problem batch (N ~ log-uniform[256, 16384], the benchmark's
    # seeds) in one launch for one step; ten problems re-done by the oracle
    # with each problem's own alpha and dt
    sizes = inputs.batch_sizes(4096, seed=2024)
    U = inputs.batch_states(sizes, seed=10_000)
    off = np.concatenate([[0], np.cumsum(sizes)])
    rng = np.random.default_rng(3)
    picks = list(rng.choice(len(sizes), size=8, replace=False)) + [int(np.argmax(sizes)),
                                                                   int(np.argmin(sizes))]
    with eno.Batch(sizes, 0.0, 1.0, system=eno.EULER, order=5, precision=precision) as b:
        b.init_state(U)
        b.advance_steps(1, 0.5)
        got = b.get_state()
        for i in picks:
            n = int(sizes[i])
            _, a, dt = b.problem_stats(i)
            Ui = np.ascontiguousarray(U[:, off[i]:off[i + 1]]).reshape(3, 1, 1, n)
            P = oracle.make_problem((n,), (0.0,), (1.0,), system=oracle.EULER, order=5)
            a_or = oracle.alpha(P, Ui)[0]
            assert a == pytest.approx(a_or, rel=1e-14 if precision == eno.FP64 else 1e-6)
            ref = oracle.step_alpha(P, Ui, dt, np.array([a, 0.0, 0.0])).reshape(3, n)
            g = got[:, off[i]:off[i + 1]]
            if precision == eno.FP64:
                assert relerr(g, ref) <= TOL64, (i, n, relerr(g, ref))
            else:
                # L1 always; max-norm outside near-tie flips of the later stages
                assert np.abs(g - ref).mean() / np.abs(ref).mean() <= TOL32_L1, (i, n)
                over = (np.abs(g - ref) > TOL32_STEP * np.abs(ref).max(axis=1, keepdims=True))
                assert over.any(axis=0).mean() <= 1e-3, (i, n)
