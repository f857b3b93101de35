"""GPU parity of fix_small_values (Sect. 7.4 bootstrapping) with the oracle:
the repair of planted small cells through amrvac_fix_small_values (replace and
average, FP64 and FP32 bulk, single level and block AMR), and whole runs of a
near-vacuum double rarefaction with the repair after every stage.
"""
import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SD, SP = 1e-6, 1e-4


@pytest.fixture(scope="module")
def amr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2303_03026_gb300 import amrvac
    return amrvac


def _plant(orc, W, cells):
    g = W.instances[0].gamma
    for b, c, kind in cells:
        w = orc.cons_to_prim(g, W.U[:, b, c])
        if kind == "p":
            w[4] = -0.05
            W.U[:, b, c] = orc.prim_to_cons(g, w)
        else:
            W.U[0, b, c] = -1e-3


def _check_fix(amr, orc, W, method, tol):
    W.cfg.small_density, W.cfg.small_pressure = SD, SP
    W.cfg.fix_small_values = method
    fp32 = W.cfg.precision == "fp32"
    U = W.U.astype(np.float32).astype(np.float64) if fp32 else W.U
    ref, nref = orc.mesh_for(W).fix_small(U, method)
    S = amr.State.from_workload(W, kernel="plain")
    S.set_conserved(U.astype(np.float32) if fp32 else U)
    n = S.fix_small(0)
    got = S.get_conserved(0, precision=0)
    S.close()
    assert n == nref > 0
    scale = np.maximum(np.abs(ref).max(axis=(1, 2), keepdims=True), 1e-300)
    err = np.abs(got - ref) / scale
    assert err.max() <= tol, err.max(axis=(1, 2))
    changed = np.any(got != U, axis=0)
    assert changed.sum() <= nref


CELLS = [(0, 5 * 16 + 5, "p"), (0, 7 * 16 + 15, "p"), (0, 0, "p"), (1, 40, "p"),
         (1, 41, "p"), (2, 100, "rho")]


@pytest.mark.parametrize("method", ["replace", "average"])
def test_fix_parity_fp64(amr, orc, method):
    W = wl.cp_alfven(32)
    _plant(orc, W, CELLS)
    _check_fix(amr, orc, W, method, 1e-14)


@pytest.mark.parametrize("method", ["replace", "average"])
def test_fix_parity_fp32(amr, orc, method):
    W = wl.cp_alfven(32, precision="fp32")
    _plant(orc, W, CELLS)
    _check_fix(amr, orc, W, method, 1e-6)


def test_fix_parity_amr_and_3d(amr, orc):
    W = wl.small_amr_2d()
    nb, nc = W.U.shape[1], W.U.shape[2]
    _plant(orc, W, [(b, c, "p") for b in range(0, nb, 3) for c in (0, nc - 1, nc // 2)])
    _check_fix(amr, orc, W, "average", 1e-14)
    W = wl.c3_turbulence(n=32, bnx=16, precision="fp64")
    _plant(orc, W, [(b, c, "p") for b in range(8) for c in (0, 4095, 2000, 2001)])
    _check_fix(amr, orc, W, "average", 1e-14)


@pytest.mark.parametrize("method", ["replace", "average"])
def test_vacuum_run_with_fix(amr, orc, method):
    W = wl.riemann_1d((1.0, -5.0, 0, 0, 0.4, 0, 0), (1.0, 5.0, 0, 0, 0.4, 0, 0), n=200,
                      gamma=1.4, bx=0.0, t_end=0.1, flux="hll", time="ssprk3")
    W.cfg.small_density, W.cfg.small_pressure = 1e-8, 1e-8
    W.cfg.fix_small_values = method
    m = orc.mesh_for(W)
    Uo, t, ns, st = m.run(W.U, 0.1)
    assert st == 0
    S = amr.State.from_workload(W, kernel="plain")
    S.set_conserved(W.U)
    S.set_time(t=0.0, t_end=0.1)
    S.step(ns)
    d = S.diag()
    assert d["status"] == 0 and abs(d["t"][0] - t[0]) < 1e-14, d
    got = S.get_conserved(0)
    S.close()
    scale = np.abs(Uo).max(axis=(1, 2), keepdims=True)
    assert (np.abs(got - Uo) / np.maximum(scale, 1e-300)).max() < 1e-9


def test_fused_3d_run_with_fix(amr, orc):
    # a blast whose centre pressure is driven below the floor in a few cells:
    # the fused path repairs them as the oracle does
    W = wl.c4_blast_amr(base=4, levels=3, bnx=16, shell=(0.2, 0.26), precision="fp64")
    _plant(orc, W, [(b, c, "p") for b in range(0, W.U.shape[1], 17) for c in (0, 777, 4095)])
    W.cfg.small_density, W.cfg.small_pressure = SD, SP
    W.cfg.fix_small_values = "average"
    m = orc.mesh_for(W, 8)
    U0, n0 = m.fix_small(W.U, "average")
    Uo, t, ns, st = m.run(U0, 1.0, maxsteps=2)
    assert st == 0
    S = amr.State.from_workload(W, kernel="auto")
    S.set_conserved(W.U)
    assert S.fix_small(0) == n0
    S.set_time(t=0.0, t_end=1.0)
    S.step(2)
    d = S.diag()
    assert d["status"] == 0, d
    got = S.get_conserved(0)
    S.close()
    scale = np.maximum(np.abs(Uo).max(axis=(1, 2), keepdims=True), 1e-300)
    assert (np.abs(got - Uo) / scale).max() < 1e-10
