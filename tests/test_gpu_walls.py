"""GPU parity of symmetric (reflecting) walls with the oracle: stage outputs
(FP64 and FP32 bulk; 1D, 2D, 3D; uniform and AMR; with five-point limiters),
the ghost export across walls, a closed box with refluxing run to the same
state and conserving mass and energy on the device, on the plain and on the
fused kernels.
"""
import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl
from test_gpu_schemes import _scheme_stage_parity

pytestmark = pytest.mark.gpu

WALLS = (("symmetric", "symmetric"),) * 3


@pytest.fixture(scope="module")
def amr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2303_03026_gb300 import amrvac
    return amrvac


def _walled(W, sides=WALLS):
    W.cfg.bc = sides
    return W


def _cases(precision):
    mixed = (("symmetric", "outflow"), ("periodic", "periodic"), ("periodic", "periodic"))
    return [
        _walled(wl.small_amr_2d(periodic=False, precision=precision)),
        _walled(wl.cp_alfven(32, precision=precision), mixed),
        _walled(wl.c4_blast_amr(base=2, levels=3, bnx=8, shell=(0.2, 0.26),
                                precision=precision)),
        _walled(wl.riemann_1d((1.0, 0.5, 0, 0, 1.0, 1.0, 0), (0.5, -0.5, 0, 0, 0.5, -1.0, 0),
                              n=128, nblocks=4), WALLS),
    ]


def test_wall_stage_parity_fp64(amr, orc):
    for W in _cases("fp64"):
        if W.cfg.precision != "fp64":
            continue
        _scheme_stage_parity(amr, orc, W, "auto", 1e-12)


def test_wall_stage_parity_fp32(amr, orc):
    for W in _cases("fp32")[:3]:
        _scheme_stage_parity(amr, orc, W, "plain", 1e-5)


@pytest.mark.parametrize("limiter", ["mp5", "wenoz5"])
def test_wall_with_five_point_limiters(amr, orc, limiter):
    W = _walled(wl.small_amr_2d(periodic=False))
    W.cfg.limiter = limiter
    _scheme_stage_parity(amr, orc, W, "auto", 1e-12)


def test_wall_ghost_export(amr, orc):
    W = _walled(wl.small_amr_2d(periodic=False))
    S = amr.State.from_workload(W, kernel="auto")
    S.set_conserved(W.U)
    got = S.fill_ghosts(0)
    S.close()
    ref = orc.mesh_for(W).fill_ghosts(W.U)
    assert np.abs(got - ref).max() <= 1e-15 * np.abs(ref).max()


def test_closed_box_run(amr, orc):
    W = _walled(wl.small_amr_2d(periodic=False))
    W.cfg.reflux = True
    m = orc.mesh_for(W)
    s0 = m.sums(W.U)
    Uo, t, ns, st = m.run(W.U, 1e30, maxsteps=6)
    assert st == 0
    S = amr.State.from_workload(W, kernel="auto")
    S.set_conserved(W.U)
    S.step(6)
    d = S.diag()
    got = S.get_conserved(0)
    S.close()
    assert d["status"] == 0 and abs(d["t"][0] - t[0]) < 1e-14
    rel = np.abs(d["sums"][0] - s0[0]) / np.abs(s0).max()
    assert rel[0] < 1e-14 and rel[4] < 1e-14, rel
    sc = np.maximum(np.abs(Uo).max(axis=(1, 2), keepdims=True), 1e-300)
    sc = np.where(sc < 1e-9 * np.abs(Uo).max(), np.abs(Uo).max(), sc)
    assert (np.abs(got - Uo) / sc).max() < 1e-10


def _fused_cases(precision):
    mixed = (("symmetric", "outflow"), ("symmetric", "symmetric"), ("periodic", "periodic"))
    return [
        _walled(wl.c3_turbulence(n=32, bnx=16, precision=precision)),
        _walled(wl.cp_alfven(32, precision=precision), mixed),
        _walled(wl.small_amr_2d(bnx=16, periodic=False, precision=precision)),
        _walled(wl.c4_blast_amr(base=4, levels=3, bnx=16, shell=(0.2, 0.26),
                                precision=precision)),
    ]


def test_fused_walls_stage_parity_fp64(amr, orc):
    # 16^3 and 16^2 blocks: the fused kernels' mirrored reads (FULL instantiations)
    for W in _fused_cases("fp64"):
        _scheme_stage_parity(amr, orc, W, "fused", 1e-12)


def test_fused_walls_stage_parity_fp32(amr, orc):
    for W in _fused_cases("fp32")[:3]:
        _scheme_stage_parity(amr, orc, W, "fused", 1e-5)


def test_fused_closed_box_run(amr, orc):
    W = _walled(wl.small_amr_2d(bnx=16, periodic=False))
    W.cfg.reflux = True
    m = orc.mesh_for(W)
    s0 = m.sums(W.U)
    Uo, t, ns, st = m.run(W.U, 1e30, maxsteps=6)
    assert st == 0
    S = amr.State.from_workload(W, kernel="fused")
    S.set_conserved(W.U)
    S.step(6)
    d = S.diag()
    got = S.get_conserved(0)
    S.close()
    assert d["status"] == 0 and abs(d["t"][0] - t[0]) < 1e-14
    rel = np.abs(d["sums"][0] - s0[0]) / np.abs(s0).max()
    assert rel[0] < 1e-14 and rel[4] < 1e-14, rel
    sc = np.maximum(np.abs(Uo).max(axis=(1, 2), keepdims=True), 1e-300)
    sc = np.where(sc < 1e-9 * np.abs(Uo).max(), np.abs(Uo).max(), sc)
    assert (np.abs(got - Uo) / sc).max() < 1e-10
