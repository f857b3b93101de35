"""CPU checks of the C ABI: the library builds, loads and exports every symbol
that include/amrvac.h declares; host-side mesh validation runs without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "amrvac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(amrvac_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2303_03026_gb300 import amrvac, build
    build.build()
    return amrvac.load()


def test_exports_every_declared_symbol(lib):
    from paper_2303_03026_gb300 import amrvac
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(amrvac.SYMBOLS)


def test_error_strings(lib):
    for st in range(7):
        assert lib.amrvac_error_string(st)


def _bytes(lib, W, kernel="plain"):
    from paper_2303_03026_gb300 import amrvac
    c = amrvac.make_config(W.cfg, kernel)
    inst = amrvac.make_instances(W.instances)
    meta = np.ascontiguousarray(W.block_meta, np.int32)
    n = C.c_size_t(0)
    st = lib.amrvac_workspace_bytes(C.byref(c), len(W.instances), inst, meta.shape[0],
                                    meta.ctypes.data, C.byref(n))
    return st, n.value


def test_workspace_bytes_and_mesh_validation(lib):
    W = wl.small_amr_2d()
    st, n = _bytes(lib, W)
    assert st == 0
    # at least three state buffers + scratch for the plain path
    assert n >= 3 * 9 * W.nblocks * W.ncell * 8
    bad = wl.small_amr_2d()
    bad.block_meta = bad.block_meta[1:]          # hole
    assert _bytes(lib, bad)[0] == 1
    dup = wl.small_amr_2d()
    dup.block_meta = np.concatenate([dup.block_meta, dup.block_meta[:1]])
    assert _bytes(lib, dup)[0] == 1
    # levels 0 and 2 touching across a face: not 2:1
    cfg = wl.Config(ndim=2, block_nx=(8, 8, 1))
    meta = np.array([(0, 0, 1, 0, 0), (0, 1, 0, 1, 0), (0, 1, 1, 1, 0), (0, 1, 1, 0, 0),
                     (0, 2, 0, 0, 0), (0, 2, 1, 0, 0), (0, 2, 0, 1, 0), (0, 2, 1, 1, 0)],
                    np.int32)
    unbalanced = wl.Workload("x", cfg, [wl.Instance(base_blocks=(2, 1, 1))], meta,
                             np.zeros((9, 8, 64)))
    assert _bytes(lib, unbalanced)[0] == 1
    W.cfg.courant = -1.0
    assert _bytes(lib, W)[0] == 1
    # one 4096^3 block: 2^36 cells overflow a 32-bit count; rejected, not wrapped
    big = wl.Workload("big", wl.Config(ndim=3, block_nx=(4096, 4096, 4096)),
                      [wl.Instance(base_blocks=(1, 1, 1))], np.zeros((1, 5), np.int32),
                      np.zeros((9, 1, 1)))
    assert _bytes(lib, big)[0] == 1
    # the largest accepted block: 4096^2 cells in 2D
    ok2 = wl.Workload("ok2", wl.Config(ndim=2, block_nx=(4096, 4096, 1)),
                      [wl.Instance(base_blocks=(1, 1, 1))], np.zeros((1, 5), np.int32),
                      np.zeros((9, 1, 1)))
    assert _bytes(lib, ok2)[0] == 0


def test_workspace_matches_precision(lib):
    W64 = wl.c2_orszag_tang(64)
    W32 = wl.c2_orszag_tang(64, precision="fp32")
    _, n64 = _bytes(lib, W64)
    _, n32 = _bytes(lib, W32)
    assert n32 < n64


def test_scheme_options_validated(lib):
    # the wider scheme family is accepted; values outside the enums are not
    for flux, time, lim in (("tvdlf", "ssprk43", "superbee"), ("hllc", "ssprk54", "albada"),
                            ("hlld", "ssprk3", "mcbeta"), ("hlld", "ssprk2", "woodward"),
                            ("hll", "ssprk3", "mp5"), ("hlld", "ssprk3", "weno5"),
                            ("hllc", "ssprk43", "wenoz5"), ("hlld", "ssprk3", "cada3"),
                            ("hllc", "ssprk54", "wenozp5"), ("hll", "ssprk43", "venk")):
        W = wl.small_amr_2d()
        W.cfg.flux, W.cfg.time, W.cfg.limiter = flux, time, lim
        assert _bytes(lib, W)[0] == 0, (flux, time, lim)
    from paper_2303_03026_gb300 import amrvac
    W = wl.small_amr_2d()
    for field, value in (("flux", 4), ("time", 4), ("limiter", 13), ("limiter", -1),
                         ("reflux", 2), ("fix_small_values", 3), ("level_flux", 5),
                         ("level_limiter", 14), ("level_flux", -1)):
        c = amrvac.make_config(W.cfg)
        if field.startswith("level_"):
            getattr(c, field)[2] = value
        else:
            setattr(c, field, value)
        ins = amrvac.make_instances(W.instances)
        meta = np.ascontiguousarray(W.block_meta, np.int32)
        n = C.c_size_t(0)
        st = lib.amrvac_workspace_bytes(C.byref(c), len(W.instances), ins, meta.shape[0],
                                        meta.ctypes.data, C.byref(n))
        assert st == 1, field


def test_five_point_limiters_widen_the_plain_scratch(lib):
    # three ghost layers in the plain path's padded scratch; in 3D the fused
    # kernel takes them in FP32 bulk only (a double 6-plane ring does not fit),
    # and never on a mesh mixing two- and five-point levels
    W = wl.c3_turbulence(n=32, bnx=16, precision="fp64")
    st, n2 = _bytes(lib, W, kernel="plain")
    W.cfg.limiter = "weno5"
    st5, n3 = _bytes(lib, W, kernel="plain")
    assert st == 0 and st5 == 0 and n3 > n2
    assert _bytes(lib, W, kernel="auto") == (0, n3)  # AUTO falls back to PLAIN
    assert _bytes(lib, W, kernel="fused")[0] == 1
    W.cfg.precision = "fp32"
    st, nf = _bytes(lib, W, kernel="fused")
    assert st == 0 and _bytes(lib, W, kernel="auto") == (0, nf)  # AUTO takes FUSED
    W.cfg.limiter = "vanleer"
    W.cfg.level_limiter = {0: "mp5"}
    assert _bytes(lib, W, kernel="fused")[0] == 1
    W.cfg.level_limiter = {0: "wenozp5"}
    assert _bytes(lib, W, kernel="fused")[0] == 1
    # cada3 needs two ghost layers: the fused kernels take it
    W.cfg.level_limiter = None
    W.cfg.limiter = "cada3"
    assert _bytes(lib, W, kernel="fused")[0] == 0


def test_fix_and_reflux_need_their_workspace(lib):
    W = wl.small_amr_2d()
    _, n0 = _bytes(lib, W)
    W.cfg.reflux = True
    st, n1 = _bytes(lib, W)
    assert st == 0 and n1 > n0  # flux registers of the level-change faces
    W.cfg.fix_small_values = "average"
    assert _bytes(lib, W)[0] == 1  # needs positive floors
    W.cfg.small_density, W.cfg.small_pressure = 1e-6, 1e-6
    st, n2 = _bytes(lib, W)
    assert st == 0 and n2 >= n1 + W.nblocks * W.ncell  # one flag byte per cell


def test_wall_boundaries_validated(lib):
    from paper_2303_03026_gb300 import amrvac
    W = wl.c3_turbulence(n=32, bnx=16, precision="fp32")
    W.cfg.bc = (("symmetric", "symmetric"), ("symmetric", "outflow"), ("periodic", "periodic"))
    assert _bytes(lib, W, kernel="fused")[0] == 0   # walls run on the fused kernels too
    assert _bytes(lib, W, kernel="plain")[0] == 0
    c = amrvac.make_config(W.cfg, "plain")
    ins = amrvac.make_instances(W.instances)
    meta = np.ascontiguousarray(W.block_meta, np.int32)
    n = C.c_size_t(0)
    for d, side, value in ((0, 0, 3), (1, 1, -1), (2, 0, 1)):
        c2 = amrvac.make_config(W.cfg, "plain")
        c2.bc[d][side] = value   # out of range, or periodic on one side only
        st = lib.amrvac_workspace_bytes(C.byref(c2), 1, ins, meta.shape[0], meta.ctypes.data,
                                        C.byref(n))
        assert st == 1, (d, side, value)
    assert lib.amrvac_workspace_bytes(C.byref(c), 1, ins, meta.shape[0], meta.ctypes.data,
                                      C.byref(n)) == 0
