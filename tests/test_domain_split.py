"""Host bookkeeping of the slab decomposition (paper_2108_12742_gb300.domain)
on the CPU: slab ranges, the exchange plan, and whole steps run as gloo ranks
(and as one process) over a numpy stand-in for a sub-domain whose operator
reaches G layers along the split axis.  The stitched slabs must equal the
undivided array stepped the same way, bit for bit, for periodic and
transmissive edges -- which holds only if every ghost layer got the right
neighbour's layers and every rank split with the global alpha."""
import os
import socket

import numpy as np
import pytest

from paper_2108_12742_gb300 import domain

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

G = 4
NV, PLANE = 2, 6
COEF = np.array([0.03, -0.11, 0.2, -0.4, 0.0, 0.41, -0.19, 0.1, -0.04])  # offsets -4..4


def toy_rhs(U, alpha):
    """L(u)_j = alpha * sum_o c_o u_{j+o} over the layers of an array that holds
    G ghost layers on each side of its interior (axis 1)."""
    n = U.shape[1] - 2 * G
    out = np.zeros((U.shape[0], n, U.shape[2]))
    for o in range(-G, G + 1):
        out = out + COEF[o + G] * U[:, G + o:G + o + n]
    return alpha * out


def toy_stage(U0, Uk, L, k, dt):
    if k == 0:
        return U0 + dt * L
    if k == 1:
        return 0.75 * U0 + 0.25 * (Uk + dt * L)
    return U0 / 3.0 + 2.0 / 3.0 * (Uk + dt * L)


class FakeSubDomain:
    """numpy stand-in for SubDomain: stage states with G ghost layers along
    axis 1 (NaN until filled), the toy operator, alpha = max |u|."""

    def __init__(self, U_local):
        n = U_local.shape[1]
        self.n = n
        self.halo_shape = (NV, G, PLANE)
        self.S = [np.full((NV, n + 2 * G, PLANE), np.nan) for _ in range(3)]
        self.S[0][:, G:G + n] = U_local
        self.alpha = None

    def interior(self, k=0):
        return self.S[k][:, G:G + self.n]

    def halo_export(self, k, side, out=None):
        lay = self.S[k][:, G:2 * G] if side == 0 else self.S[k][:, self.n:self.n + G]
        if out is None:
            return lay.copy()
        out.copy_(torch.from_numpy(np.ascontiguousarray(lay)))
        return out

    def halo_import(self, k, side, buf):
        buf = buf.numpy() if hasattr(buf, "numpy") else buf
        if side == 0:
            self.S[k][:, :G] = buf
        else:
            self.S[k][:, self.n + G:] = buf

    def halo_fill_transmissive(self, k, side):
        if side == 0:
            self.S[k][:, :G] = self.S[k][:, G:G + 1]
        else:
            self.S[k][:, self.n + G:] = self.S[k][:, self.n + G - 1:self.n + G]

    def local_alpha(self):
        return np.array([np.abs(self.interior()).max(), 0.0, 0.0])

    def set_step_alpha(self, a):
        self.alpha = np.asarray(a, dtype=np.float64)

    def rk_stage(self, k, dt):
        assert not np.isnan(self.S[k]).any(), "a ghost layer was left unfilled"
        L = toy_rhs(self.S[k], self.alpha[0])
        new = toy_stage(self.interior(0), self.interior(k), L, k, dt)
        self.S[2 if k == 1 else (1 if k == 0 else 0)][:, G:G + self.n] = new
        # every stage state must get its ghost layers anew before it is used
        nxt = self.S[0] if k == 2 else self.S[k + 1]
        nxt[:, :G] = np.nan
        nxt[:, self.n + G:] = np.nan


def undivided(U, bc, steps, cfl, dx):
    """The same steps on the whole array, ghosts by wrap or clamp."""
    n = U.shape[1]
    idx = np.arange(-G, n + G)
    idx = idx % n if bc == domain.PERIODIC else np.clip(idx, 0, n - 1)
    for _ in range(steps):
        a = np.array([np.abs(U).max(), 0.0, 0.0])
        dt = domain.step_dt(a, dx, cfl)
        Uk = U
        for k in range(3):
            Uk = toy_stage(U, Uk, toy_rhs(Uk[:, idx], a[0]), k, dt)
        U = Uk
    return U


def _global(n, seed=0):
    return np.random.default_rng(seed).uniform(-1, 1, size=(NV, n, PLANE))


def test_slab_ranges_cover_the_axis_and_respect_the_halo():
    for n, r in ((64, 2), (67, 3), (40, 8), (8, 2)):
        rng = domain.slab_ranges(n, r, G)
        assert rng[0][0] == 0 and sum(m for _, m in rng) == n
        assert all(rng[i][0] + rng[i][1] == rng[i + 1][0] for i in range(r - 1))
        assert max(m for _, m in rng) - min(m for _, m in rng) <= 1
        assert min(m for _, m in rng) >= G
    with pytest.raises(ValueError):
        domain.slab_ranges(7, 2, G)


def test_exchange_plan_pairs_every_send_with_a_receive():
    for size in (1, 2, 3, 5):
        for bc in (domain.PERIODIC, domain.TRANSMISSIVE):
            sends, recvs = [], []
            for r in range(size):
                s, v, fills = domain.exchange_plan(r, size, bc)
                sends += [(r, p, t) for p, t, _ in s]
                recvs += [(p, r, t) for p, t, _ in v]
                # two ghost sides per slab: received or filled, never both
                assert sorted([side for _, _, side in v] + fills) == [0, 1]
                if bc == domain.TRANSMISSIVE:
                    assert (0 in fills) == (r == 0) and (1 in fills) == (r == size - 1)
            assert sorted(sends) == sorted(recvs)


@pytest.mark.parametrize("bc", [domain.PERIODIC, domain.TRANSMISSIVE])
@pytest.mark.parametrize("nslabs", [1, 2, 3])
def test_local_group_equals_the_undivided_array(bc, nslabs):
    n, steps, cfl, dx = 23, 4, 0.4, (0.1, 0.05)
    U = _global(n, seed=nslabs)
    doms = [FakeSubDomain(U[:, o:o + m]) for o, m in domain.slab_ranges(n, nslabs, G)]
    grp = domain.LocalGroup(doms, bc, dx)
    for _ in range(steps):
        grp.step(cfl)
    got = np.concatenate([d.interior() for d in doms], axis=1)
    assert np.array_equal(got, undivided(U, bc, steps, cfl, dx))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, bc, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, steps, cfl, dx = 26, 3, 0.4, (0.1, 0.05)
    U = _global(n, seed=7)
    o, m = domain.slab_ranges(n, world, G)[rank]
    dom = FakeSubDomain(U[:, o:o + m])
    slab = domain.Slab(dom, domain.TorchComm("cpu"), bc, dx)
    dts = [slab.step(cfl) for _ in range(steps)]
    ref = undivided(U, bc, steps, cfl, dx)[:, o:o + m]
    out[rank] = (bool(np.array_equal(dom.interior(), ref)), dts)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("bc", [domain.PERIODIC, domain.TRANSMISSIVE])
def test_two_gloo_ranks_step_like_the_undivided_array(bc):
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, bc, out), nprocs=world, join=True)
        res = dict(out)
    assert all(res[r][0] for r in range(world)), res
    assert res[0][1] == res[1][1]  # one global alpha, one dt per step on every rank
