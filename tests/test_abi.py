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
                dict(tile=1), dict(pot_mode=4), dict(pot_mode=2), dict(pot_mode=2, morse_a=-1.0), dict(lattice=2),
                dict(pot_mode=3, lattice=1), dict(pot_mode=3, eam_ec=0.0), dict(pot_mode=3, eam_gamma=-1.0),
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
    # 10 int32 + 1 int64 + 17 double + 1 uint64 + 2 int32 + 2 int32 + 4 double + 5 double (EAM)
    assert ctypes.sizeof(gb.pic_config) == 10 * 4 + 8 + 17 * 8 + 8 + 2 * 4 + 2 * 4 + 4 * 8 + 5 * 8
    assert ctypes.sizeof(gb.pic_config) == lib.pic_config_bytes()
    assert gb.pic_config.morse_a.offset == ctypes.sizeof(gb.pic_config) - 6 * 8
    assert gb.pic_config.eam_gamma.offset == ctypes.sizeof(gb.pic_config) - 8
    assert gb.pic_config.T_spot_K.offset == 10 * 4 + 8 + 17 * 8 + 8 + 4 * 4
    assert gb.pic_config.max_particles.offset == 40
    assert ctypes.sizeof(gb.pic_energy_t) == 7 * 8
    assert gb.pic_energy_t.injected.offset == 48


def test_fixed_point_range_is_checked_at_sizing(lib):
    """The int64 node sums stay exact while a cell holds at most 2^63 / (F * c) particles (F the
    cells whose particles reach one node, c one particle's largest contribution): in 3D with
    currents 2730 per cell (F = 64, c = 3 * 2^44), 16383 without (c = 2 * 2^42: the density while
    it is updated). A slab configured beyond that is refused with
    PIC_EOVERFLOW before any CUDA call; in 2D the J_y code resolution is lowered instead (the
    paper's 900 electrons per cell are accepted)."""
    def size(w):
        cfg = gb.make_config(w)
        n = ctypes.c_size_t(0)
        return lib.pic_workspace_size(ctypes.byref(cfg), ctypes.byref(n))
    w3 = dict(workload("3d", nx=16, ny=16, nz=16, slab_k=4))
    assert size(dict(w3, ppc_ion=1365, ppc_electron=1365)) == 0
    assert size(dict(w3, ppc_ion=1366, ppc_electron=1366)) == gb.PIC_EOVERFLOW
    assert size(dict(w3, ppc_ion=200000, ppc_electron=200000)) == gb.PIC_EOVERFLOW
    assert size(dict(w3, mode=1, ion_charge=0.0, ppc_ion=16383, ppc_electron=0)) == 0       # no currents: below 2^20 per block
    assert size(dict(w3, mode=1, ion_charge=0.0, ppc_ion=16384, ppc_electron=0)) == gb.PIC_EOVERFLOW
    assert size(dict(workload("tiny"), ppc_ion=25, ppc_electron=900)) == gb.PIC_EINVAL      # unequal in full mode
    assert size(dict(workload("tiny"), ppc_ion=900, ppc_electron=900)) == 0
    assert size(dict(workload("tiny", nx=4, nz=4, slab_k=1), ppc_ion=6_000_000, ppc_electron=6_000_000)) == \
        gb.PIC_EOVERFLOW


def test_regrid_refuses_bad_grids_before_any_cuda_call(lib):
    """pic_regrid_cells checks its arguments on the host: NULL pointers, dims other than 2 or 3,
    empty extents, non-positive cell sizes and surfaces outside 0..nz give PIC_EINVAL without a
    launch (the pointers below are never dereferenced)."""
    fake = ctypes.c_void_p(256)
    good = (8, 1, 6, 1e-8, 3)

    def call(dims=2, src=good, dst=good, s=fake, d=fake):
        return lib.pic_regrid_cells(dims, s, src[0], src[1], src[2], ctypes.c_double(src[3]), src[4], d, dst[0],
                                    dst[1], dst[2], ctypes.c_double(dst[3]), dst[4], ctypes.c_double(300.0), None)
    assert call(s=None) == gb.PIC_EINVAL
    assert call(d=None) == gb.PIC_EINVAL
    assert call(dims=1) == gb.PIC_EINVAL and call(dims=4) == gb.PIC_EINVAL
    assert call(src=(0, 1, 6, 1e-8, 3)) == gb.PIC_EINVAL
    assert call(dst=(8, 1, 0, 1e-8, 0)) == gb.PIC_EINVAL
    assert call(dims=3, src=(8, 0, 6, 1e-8, 3)) == gb.PIC_EINVAL
    assert call(src=(8, 1, 6, 0.0, 3)) == gb.PIC_EINVAL and call(dst=(8, 1, 6, -1e-8, 3)) == gb.PIC_EINVAL
    assert call(src=(8, 1, 6, 1e-8, 7)) == gb.PIC_EINVAL and call(dst=(8, 1, 6, 1e-8, -1)) == gb.PIC_EINVAL

