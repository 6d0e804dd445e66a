"""The C-ABI library builds, loads and exports every entry point of
include/enoao.h (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os

import pytest

import paper_2108_12742_gb300 as eno
from paper_2108_12742_gb300 import build as libbuild


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return eno.load()


def test_header_declares_the_boundary():
    names = eno.header_symbols()
    for required in ("enoao_create", "enoao_init_state", "enoao_reconstruct_fluxes",
                     "enoao_rk_stage", "enoao_advance", "enoao_advance_steps",
                     "enoao_get_state", "enoao_batch_create", "enoao_last_error",
                     "enoao_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in eno.header_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_config_layout_matches_header(lib):
    cfg = eno.Config()
    lib.enoao_config_default(ctypes.byref(cfg))
    assert (cfg.ndim, cfg.system, cfg.order, cfg.precision) == (1, eno.EULER, 5, eno.FP64)
    assert cfg.delta == 1e-5 and cfg.gamma == 1.4 and cfg.tie_rel == 1e-3
    assert list(cfg.n) == [1, 1, 1]
    assert ctypes.sizeof(eno.Config) == 4 * 4 + 8 * 3 + 8 * 6 + 4 * 4 + 8 * 4


def test_product_path_does_not_reach_the_oracle():
    # the package must not import, load or name the test oracle
    pkg = os.path.dirname(eno.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "liboracle" not in text, f


def test_configurations_are_validated_before_any_device_call(lib):
    # rejected on the host with ENOAO_EINVAL and a message, whether or not a GPU exists
    with pytest.raises(eno.EnoaoError) as e:
        eno.Solver((16,), (0.0,), (1.0,), alpha_mode=3)
    assert e.value.status == 1 and "alpha_mode" in str(e.value)
    with pytest.raises(eno.EnoaoError) as e:
        eno.Batch([16, 20], [0.0, 0.0], [1.0, 1.0], alpha_mode=eno.ALPHA_PER_FIELD)
    assert e.value.status == 1 and "per-field" in str(e.value)
    with pytest.raises(eno.EnoaoError) as e:
        eno.Solver((16,), (0.0,), (1.0,), order=6)
    assert e.value.status == 1


def test_noalloc_step_checks_its_buffers_before_any_device_call(lib, monkeypatch):
    # enoao_step_noalloc reads and writes nv * n doubles through raw pointers;
    # the binding rejects what the C side cannot see (size, dtype, layout,
    # host memory) before the call is made
    torch = pytest.importorskip("torch")
    called = []
    monkeypatch.setattr(lib, "enoao_step_noalloc", lambda *a: called.append(a) or 0)
    n = 64
    cfg = eno.make_config((n,), (0.0,), (1.0,), system=eno.EULER, order=5)
    good = torch.zeros((3, n), dtype=torch.float64)
    bad = [
        (torch.zeros((3, n - 1), dtype=torch.float64), "shape"),
        (torch.zeros((1, n), dtype=torch.float64), "shape"),
        (torch.zeros((3, n), dtype=torch.float32), "dtype"),
        (torch.zeros((n, 3), dtype=torch.float64).t(), "contiguous"),
        (good, "GPU"),                       # right layout, but host memory
        (good.numpy(), "CUDA torch tensor"),
    ]
    for U, what in bad:
        with pytest.raises(ValueError, match=what):
            eno.step_noalloc(cfg, U, U, 1e-4)
    assert not called
