"""CPU checks of the Python binding's marshalling (no GPU): every State method
that takes host arguments is driven against a stand-in of the library whose
functions check the call against the argument types the real library
declares (count, and pointer-or-integer kinds), and the status path raises.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2303_03026_gb300 import amrvac
from paper_2303_03026_gb300 import workloads as wl


@pytest.fixture(scope="module")
def real():
    from paper_2303_03026_gb300 import build
    build.build()
    return amrvac.load()


class _FakeFn:
    def __init__(self, name, argtypes, log, status):
        self.name, self.argtypes, self.log, self.status = name, argtypes, log, status

    def __call__(self, *args):
        assert len(args) == len(self.argtypes), (self.name, len(args), len(self.argtypes))
        for a, t in zip(args, self.argtypes):
            if t is C.c_void_p:
                assert a is None or isinstance(a, (int, C.c_void_p)) or hasattr(a, "_obj"), \
                    (self.name, a)
            elif t in (C.c_int32, C.c_int64):
                assert isinstance(a, (int, np.integer)), (self.name, a)
            elif t is C.c_double:
                assert isinstance(a, (float, int, np.floating)), (self.name, a)
        self.log.append(self.name)
        return self.status.get(self.name, 0)


class _FakeLib:
    def __init__(self, real, status=None):
        self.log = []
        self.status = status or {}
        for n in amrvac.SYMBOLS:
            setattr(self, n, _FakeFn(n, getattr(real, n).argtypes or [], self.log, self.status))


def _state(W):
    # a State without device memory: only the host-side fields the methods use
    S = object.__new__(amrvac.State)
    S.cfg, S.instances = W.cfg, list(W.instances)
    S.ninst, S.meta = len(W.instances), np.ascontiguousarray(W.block_meta, np.int32)
    S.nblocks, S.ncell = W.nblocks, W.ncell
    S.precision = wl.PRECISION[W.cfg.precision]
    S._h = C.c_void_p(1)
    return S


def test_state_methods_marshal_their_arguments(real, monkeypatch):
    fake = _FakeLib(real)
    monkeypatch.setattr(amrvac, "load", lambda path=amrvac.LIB_PATH: fake)
    W = wl.small_amr_2d()
    S = _state(W)
    S.set_time(t=0.0, t_end=1.0)
    S.set_time(t_end=2.0)
    S.set_dt(1e-3, 2.0)
    S.stage(0)
    S.step(2)
    assert S.cfl_dt().shape == (1,)
    d = S.diag()
    assert d["status"] == 0 and d["sums"].shape == (1, 9)
    S.set_tuning(2, "storage", True)
    assert set(S.get_tuning()) >= {"ctas_per_sm", "order", "dynamic"}
    S.autotune(3, cache="/nonexistent/cache")
    assert S.fix_small(0) == 0
    E, f = S.regrid_estimate(0.1, 0.2, max_level=3, weights=[0.5, 0, 0, 0, 0.5, 0, 0, 0, 0])
    assert E.shape == f.shape == (W.nblocks,)
    S.regrid_transfer(_state(W), 0, 1)
    S.save("/nonexistent/x")
    S.restore("/nonexistent/x")
    S.clear_error()
    assert isinstance(S.launches, int)
    S._h = None  # nothing to destroy
    for n in ("amrvac_set_time", "amrvac_set_dt", "amrvac_stage", "amrvac_step",
              "amrvac_cfl_dt", "amrvac_get_diag", "amrvac_set_tuning", "amrvac_get_tuning",
              "amrvac_autotune", "amrvac_fix_small_values", "amrvac_regrid_estimate",
              "amrvac_regrid_transfer", "amrvac_state_save", "amrvac_state_load",
              "amrvac_clear_error", "amrvac_launch_count"):
        assert n in fake.log, n


@pytest.mark.parametrize("name,call", [
    ("amrvac_fix_small_values", lambda S: S.fix_small(0)),
    ("amrvac_regrid_estimate", lambda S: S.regrid_estimate(0.1)),
    ("amrvac_regrid_transfer", lambda S: S.regrid_transfer(S)),
    ("amrvac_step", lambda S: S.step(1)),
])
def test_status_raises(real, monkeypatch, name, call):
    fake = _FakeLib(real, {name: 1})
    monkeypatch.setattr(amrvac, "load", lambda path=amrvac.LIB_PATH: fake)
    S = _state(wl.small_amr_2d())
    with pytest.raises(amrvac.AmrvacError):
        call(S)
    S._h = None
