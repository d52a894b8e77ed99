"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports every symbol
declared in include/pic.h; configuration validation and workspace sizing run on the host."""
import ctypes
import os
import re

import pytest

import paper_1502_07722_gb300 as gb
from paper_1502_07722_gb300 import _build
from paper_1502_07722_gb300.workloads import workload

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return gb.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pic.h")).read()
    return sorted(set(re.findall(r"^PIC_API\s+[\w\s\*]+?\b(pic_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(gb._SIGNATURES), "binding and header disagree"


def test_workspace_size_and_validation(lib):
    cfg = gb.make_config(workload("tiny"))
    n = gb.pic_workspace_size(cfg)
    # two particle buffers of 24 B for 2 x 16384 particles at least
    assert n > 2 * 2 * 16384 * 24
    big = gb.pic_workspace_size(gb.make_config(workload("large2d")))
    assert big > 2 * 2 * 67108864 * 24
    for bad in (dict(nx=2), dict(nz=3), dict(slab_k=65), dict(ion_charge=2.0), dict(ppc_electron=4),
                dict(tile=1), dict(pot_mode=3), dict(pot_mode=2), dict(pot_mode=2, morse_a=-1.0), dict(lattice=2),
                dict(laser_profile=2, w0=0.0), dict(cfl=1.5)):
        with pytest.raises(gb.PicError) as e:
            gb.pic_workspace_size(gb.make_config(workload("tiny"), **bad))
        assert e.value.code == gb.PIC_EINVAL
    # 3D needs ny; batches and the allocation-free energy are 2D only
    c3 = gb.make_config(workload("tiny"), dims=3, ny=32)
    assert gb.pic_workspace_size(c3) > gb.pic_workspace_size(gb.make_config(workload("tiny")))
    with pytest.raises(gb.PicError):
        gb.pic_workspace_size(gb.make_config(workload("tiny"), dims=3, ny=2))
    with pytest.raises(gb.PicError):
        gb.pic_workspace_size(gb.make_config(workload("tiny"), dims=4))
    # a batch runs one particle-kernel instance: all slabs Morse or none
    lj, mo = gb.make_config(workload("tiny")), gb.make_config(workload("tiny"), pot_mode=2, morse_a=3.0)
    assert gb.pic_batch_workspace_size([mo, mo]) > 0
    for mixed in ([lj, mo], [lj, gb.make_config(workload("tiny"), lattice=1)]):
        with pytest.raises(gb.PicError) as e:
            gb.pic_batch_workspace_size(mixed)
        assert e.value.code == gb.PIC_EINVAL
    # transport mode: neutral atoms only
    gb.pic_workspace_size(gb.make_config(workload("transport")))
    gb.pic_workspace_size(gb.make_config(workload("crater_morse")))
    gb.pic_workspace_size(gb.make_config(workload("crater_hcp")))
    gb.pic_workspace_size(gb.make_config(workload("crater3d")))
    with pytest.raises(gb.PicError):
        gb.pic_workspace_size(gb.make_config(workload("transport"), ion_charge=1.0))


def test_init_rejects_bad_workspace_without_touching_the_gpu(lib):
    cfg = gb.make_config(workload("tiny"))
    h = ctypes.c_void_p()
    n = gb.pic_workspace_size(cfg)
    assert lib.pic_init(ctypes.byref(cfg), None, n, None, ctypes.byref(h)) == gb.PIC_EINVAL
    assert lib.pic_init(ctypes.byref(cfg), 256, n - 1, None, ctypes.byref(h)) == gb.PIC_ENOMEM
    assert lib.pic_init(ctypes.byref(cfg), 257, n, None, ctypes.byref(h)) == gb.PIC_EINVAL
    assert lib.pic_step(None, 1) == gb.PIC_EINVAL
    assert lib.pic_strerror(gb.PIC_EMOVE) == b"a particle moved one cell or more in one step"


def test_config_struct_layout_matches_header(lib):
    # 10 int32 + 1 int64 + 17 double + 1 uint64 + 2 int32 + 2 int32 + 4 double
    assert ctypes.sizeof(gb.pic_config) == 10 * 4 + 8 + 17 * 8 + 8 + 2 * 4 + 2 * 4 + 4 * 8
    assert ctypes.sizeof(gb.pic_config) == lib.pic_config_bytes()
    assert gb.pic_config.morse_a.offset == ctypes.sizeof(gb.pic_config) - 8
    assert gb.pic_config.T_spot_K.offset == 10 * 4 + 8 + 17 * 8 + 8 + 4 * 4
    assert gb.pic_config.max_particles.offset == 40
    assert ctypes.sizeof(gb.pic_energy_t) == 7 * 8
    assert gb.pic_energy_t.injected.offset == 48
