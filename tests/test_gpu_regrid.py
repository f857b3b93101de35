"""GPU parity of dynamic regridding with the oracle (oracle/regrid.py):
the per-block estimator and flags (amrvac_regrid_estimate), the transfer into
a state built on the planned block list (amrvac_regrid_transfer: copy,
prolongation, restriction), in FP64 and FP32 bulk, 1D/2D/3D, single and
multi-level, plus a regrid followed by steps on the new mesh, conservation at
the 3D workload size (sampled blocks against the oracle) and the rejected
cases.
"""
import numpy as np
import pytest

from oracle import regrid as rg
from paper_2303_03026_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2303_03026_gb300 import amrvac
    return amrvac


def _case_1d():
    cfg = wl.Config(ndim=1, block_nx=(16, 1, 1), flux="hll", limiter="vanleer", time="ssprk3",
                    precision="fp64", glm=True, bc=(("outflow", "outflow"),) * 3)
    inst = wl.Instance(base_blocks=(8, 1, 1), gamma=1.4)
    meta = wl.uniform_meta((8, 1, 1))

    def prim(inst, x, y, z):
        zero = np.zeros_like(x)
        rho = np.where(x < 0.37, 1.0, 0.125) + 0.05 * np.sin(9 * x)
        return wl.conserved_from_primitive(inst.gamma, rho, zero, zero, zero,
                                           np.where(x < 0.37, 1.0, 0.1), 0.75 + zero,
                                           1.0 + zero, zero)
    U = wl._fill_from_function(cfg, [inst], meta, prim)
    return wl.Workload("riemann_blocks", cfg, [inst], meta, U)


def _case_3d():
    # the 3D two-level shell mesh with a density wave and a dense sphere
    W = wl.c4_blast_amr(base=2, levels=3, bnx=8, shell=(0.2, 0.26), precision="fp64")

    def prim(inst, x, y, z):
        zero = np.zeros_like(x)
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * (x + 2 * y + z)) + np.where(r < 0.23, 2.0, 0.0)
        return wl.conserved_from_primitive(inst.gamma, rho, 0.2 + zero, zero, -0.1 + zero,
                                           1.0 + zero, 0.5 + zero, 0.3 + zero, zero)
    W.U = wl._fill_from_function(W.cfg, W.instances, W.block_meta, prim)
    return W


def _cases():
    return {
        "1d": _case_1d(),
        "2d": wl.small_amr_2d(),
        "2d_outflow": wl.small_amr_2d(periodic=False, seed=9),
        "3d": _case_3d(),
    }


def _as(W, precision):
    W.cfg.precision = precision
    if precision == "fp32":
        W.U = W.U.astype(np.float32).astype(np.float64)
    return W


def _thresholds(E):
    # a threshold half way between two estimator values near the 70th
    # percentile, and a derefine level half way below the 30th, so that no
    # block sits on either
    s = np.unique(E)
    hi = len(s) * 7 // 10
    thr = 0.5 * (s[hi] + s[hi - 1])
    lo = max(len(s) * 3 // 10, 1)
    dthr = 0.5 * (s[lo] + s[lo - 1])
    return thr, dthr / thr


WEIGHTS = {
    "rho": None,
    # density and pressure (the blast quantities), and every primitive
    "rho_p": [0.5, 0, 0, 0, 0.5, 0, 0, 0, 0],
    "all": [1.0, 0.3, 0.3, 0.3, 1.0, 0.2, 0.2, 0.2, 0.1],
}


@pytest.mark.parametrize("name", ["1d", "2d", "2d_outflow", "3d"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("weights", ["rho", "rho_p", "all"])
def test_estimator_parity(amr, orc, name, precision, weights):
    W = _as(_cases()[name], precision)
    wts = WEIGHTS[weights]
    Eo = rg.estimator(orc.mesh_for(W), W.U, W.cfg, weights=wts)
    thr, ratio = _thresholds(Eo)
    S = amr.State.from_workload(W, kernel="plain")
    S.set_conserved(W.U.astype(np.float32) if precision == "fp32" else W.U)
    E, f = S.regrid_estimate(thr, ratio, max_level=3, weights=wts)
    S.close()
    # FP64: rounding of the primitive recovery and of the level-change ghost
    # operators; FP32 bulk: the ghost operators run in float
    tol = (1e-13 if weights == "rho" else 1e-12) if precision == "fp64" else 2e-5
    assert np.abs(E - Eo).max() <= tol, np.abs(E - Eo).max()
    fo = rg.flags(Eo, W.block_meta, thr, ratio, 3)
    far = (np.abs(Eo - thr) > tol) & (np.abs(Eo - ratio * thr) > tol)
    assert np.array_equal(f[far], fo[far])
    assert (f == 1).any()


def _transfer_pair(amr, orc, W, flags, precision, only=None, kernel="plain"):
    new = rg.plan(W.cfg, W.instances, W.block_meta, flags)
    ref = rg.transfer(W.cfg, W.instances, W.block_meta, W.U, orc.mesh_for(W), new, only=only)
    S = amr.State.from_workload(W, kernel=kernel)
    S.set_conserved(W.U.astype(np.float32) if precision == "fp32" else W.U)
    D = amr.State(W.cfg, W.instances, new, kernel=kernel)
    S.regrid_transfer(D, 0, 0)
    got = D.get_conserved(0, precision=0)
    S.close()
    D.close()
    return new, ref, got


def _random_flags(W, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.integers(-1, 2, W.nblocks).astype(np.int32)
    f[(W.block_meta[:, 1] == 0) & (f == -1)] = 0
    return f


@pytest.mark.parametrize("name", ["1d", "2d", "2d_outflow", "3d"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_transfer_parity(amr, orc, name, precision):
    W = _as(_cases()[name], precision)
    f = _random_flags(W, 21)
    only = None
    if name == "3d":
        # sampled new blocks (copies, children and merged parents among them)
        n_new = len(rg.plan(W.cfg, W.instances, W.block_meta, f))
        only = set(range(0, n_new, 7))
    new, ref, got = _transfer_pair(amr, orc, W, f, precision, only=only)
    assert len(new) != W.nblocks
    idx = sorted(only) if only is not None else list(range(len(new)))
    scale = np.maximum(np.abs(W.U).max(axis=(1, 2)), 1e-300)[:, None, None]
    err = np.abs(got[:, idx] - ref[:, idx]) / scale
    tol = 1e-14 if precision == "fp64" else 1e-6
    assert err.max() <= tol, err.max(axis=(1, 2))


def test_multi_instance_regrid_and_steps(amr, orc):
    # independent instances (own gamma, own clock) regridded together, then
    # stepped on the new mesh: estimator, plan, transfer and the step match
    W = wl.c5_instances(count=5, nmin=32, nmax=96, precision="fp64")
    m = orc.mesh_for(W)
    wts = [0.5, 0, 0, 0, 0.5, 0, 0, 0, 0]
    Eo = rg.estimator(m, W.U, W.cfg, weights=wts)
    thr, ratio = _thresholds(Eo)
    fo = rg.flags(Eo, W.block_meta, thr, ratio, 2)
    new = rg.plan(W.cfg, W.instances, W.block_meta, fo)
    Un = rg.transfer(W.cfg, W.instances, W.block_meta, W.U, m, new)
    assert len(new) != W.nblocks and len(set(new[:, 0].tolist())) == 5
    S = amr.State.from_workload(W, kernel="auto")
    S.set_conserved(W.U)
    E, f = S.regrid_estimate(thr, ratio, max_level=2, weights=wts)
    assert np.abs(E - Eo).max() <= 1e-12 and np.array_equal(f, fo)
    N = S.regrid(thr, ratio, max_level=2, weights=wts)
    S.close()
    assert np.array_equal(N.meta, new)
    got = N.get_conserved(0)
    scale = np.maximum(np.abs(W.U).max(axis=(1, 2), keepdims=True), 1e-300)  # psi is 0
    assert (np.abs(got - Un) / scale).max() <= 1e-14
    Wn = wl.Workload("regridded", W.cfg, W.instances, new, Un)
    Uo, t, ns, st = orc.mesh_for(Wn).run(Un, 1e30, maxsteps=2)
    assert st == 0
    N.set_time(t=0.0, t_end=1e30)
    N.step(2)
    d = N.diag()
    got = N.get_conserved(0)
    N.close()
    assert d["status"] == 0 and np.abs(d["t"] - t).max() < 1e-14
    sc = np.maximum(np.abs(Uo).max(axis=(1, 2), keepdims=True), 1e-300)
    assert (np.abs(got - Uo) / sc).max() < 1e-10


def test_transfer_without_flags_is_a_copy(amr, orc):
    W = wl.small_amr_2d()
    new, ref, got = _transfer_pair(amr, orc, W, np.zeros(W.nblocks, np.int32), "fp64")
    order = {tuple(r): b for b, r in enumerate(W.block_meta)}
    perm = [order[tuple(r)] for r in new]
    assert np.array_equal(got, W.U[:, perm])


def test_regrid_then_steps(amr, orc):
    # State.regrid (estimator, plan, transfer) and two steps on the new mesh
    # match the oracle doing the same
    W = wl.small_amr_2d()
    m = orc.mesh_for(W)
    Eo = rg.estimator(m, W.U, W.cfg)
    thr, ratio = _thresholds(Eo)
    fo = rg.flags(Eo, W.block_meta, thr, ratio, 3)
    new = rg.plan(W.cfg, W.instances, W.block_meta, fo)
    Un = rg.transfer(W.cfg, W.instances, W.block_meta, W.U, m, new)
    Wn = wl.Workload("regridded", W.cfg, W.instances, new, Un)
    Uo, t, ns, st = orc.mesh_for(Wn).run(Un, 1e30, maxsteps=2)
    assert st == 0
    S = amr.State.from_workload(W, kernel="plain")
    S.set_conserved(W.U)
    S.set_time(t=0.0, t_end=1e30)
    N = S.regrid(thr, ratio, max_level=3)
    S.close()
    assert np.array_equal(N.meta, new)
    N.set_time(t=0.0, t_end=1e30)
    N.step(2)
    d = N.diag()
    got = N.get_conserved(0)
    N.close()
    assert d["status"] == 0 and abs(d["t"][0] - t[0]) < 1e-14
    scale = np.maximum(np.abs(Uo).max(axis=(1, 2), keepdims=True), 1e-300)
    assert (np.abs(got - Uo) / scale).max() < 1e-10


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_regrid_fused_3d_conserves(amr, orc, precision):
    # the 3D blast mesh (16^3 blocks, fused update path): a regrid keeps every
    # conserved integral (device sums before and after) and sampled blocks
    # match the oracle
    W = wl.c4_blast_amr(base=4, levels=3, bnx=16, shell=(0.2, 0.26), precision=precision)
    if precision == "fp32":
        W.U = W.U.astype(np.float32).astype(np.float64)
    S = amr.State.from_workload(W, kernel="auto")
    S.set_conserved(W.U.astype(np.float32) if precision == "fp32" else W.U)
    S.step(3)
    s0 = S.diag()["sums"][0]
    E, f = S.regrid_estimate(0.05, 0.2, max_level=3, weights=WEIGHTS["rho_p"])
    assert (f == 1).any() and (f == -1).any()
    U1 = S.get_conserved(0, precision=0)
    new = amr.regrid_plan(W.cfg, W.instances, W.block_meta, f)
    D = amr.State(W.cfg, W.instances, new, kernel="auto")
    S.regrid_transfer(D, 0, 0)
    s1 = D.diag()["sums"][0]
    got = D.get_conserved(0, precision=0)
    S.close()
    D.close()
    # sums are cell-volume weighted integrals over the instance
    scale = np.abs(U1).reshape(9, -1).max(axis=1)
    tol = 1e-13 if precision == "fp64" else 2e-6
    assert np.all(np.abs(s1 - s0) <= tol * scale), (s1 - s0) / scale
    W1 = wl.Workload("stepped", W.cfg, W.instances, W.block_meta, U1)
    only = set(range(0, len(new), 41))
    ref = rg.transfer(W.cfg, W.instances, W.block_meta, U1, orc.mesh_for(W1, 8), new, only=only)
    idx = sorted(only)
    err = np.abs(got[:, idx] - ref[:, idx]) / np.maximum(scale, 1e-300)[:, None, None]
    assert err.max() <= (1e-14 if precision == "fp64" else 1e-6), err.max()


def test_regrid_rejects_mismatched_states(amr):
    W = wl.small_amr_2d()
    S = amr.State.from_workload(W, kernel="plain")
    W32 = wl.small_amr_2d(precision="fp32")
    D = amr.State.from_workload(W32, kernel="plain")
    with pytest.raises(amr.AmrvacError):
        S.regrid_transfer(D)  # precision differs
    D.close()
    W5 = wl.small_amr_2d(bnx=5)
    D5 = amr.State.from_workload(W5, kernel="plain")
    with pytest.raises(amr.AmrvacError):
        D5.regrid_transfer(D5)  # odd block size
    D5.close()
    with pytest.raises(amr.AmrvacError):
        S.regrid_estimate(0.1, 0.1, max_level=16)
    # a block list that is not one regrid away (two levels of splitting)
    f = np.ones(W.nblocks, np.int32)
    m1 = rg.plan(W.cfg, W.instances, W.block_meta, f)
    m2 = rg.plan(W.cfg, W.instances, m1, np.ones(len(m1), np.int32))
    D2 = amr.State(W.cfg, W.instances, m2, kernel="plain")
    with pytest.raises(amr.AmrvacError):
        S.regrid_transfer(D2)
    D2.close()
    S.close()


def test_regrid_with_walls(amr, orc):
    # the estimator's and the prolongation's ghost values across reflecting
    # walls are the mirrored cells with the normal components negated
    W = wl.small_amr_2d(periodic=False)
    W.cfg.bc = (("symmetric", "symmetric"),) * 3
    wts = [0.5, 0.2, 0.2, 0, 0.5, 0.1, 0.1, 0, 0]
    Eo = rg.estimator(orc.mesh_for(W), W.U, W.cfg, weights=wts)
    thr, ratio = _thresholds(Eo)
    S = amr.State.from_workload(W, kernel="auto")
    S.set_conserved(W.U)
    E, f = S.regrid_estimate(thr, ratio, max_level=3, weights=wts)
    S.close()
    assert np.abs(E - Eo).max() <= 1e-12
    f = _random_flags(W, 33)
    new, ref, got = _transfer_pair(amr, orc, W, f, "fp64")
    scale = np.maximum(np.abs(W.U).max(axis=(1, 2)), 1e-300)[:, None, None]
    assert (np.abs(got - ref) / scale).max() <= 1e-14


# ----------------------------------------------------------------------------
# the plan on the device: the same block list as the host plan and the oracle
# ----------------------------------------------------------------------------

def _flag_patterns(W, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    lev = W.block_meta[:, 1]
    out = [_random_flags(W, seed)]
    sparse = np.where(rng.random(W.nblocks) < 0.05, 1, 0)
    sparse[rng.random(W.nblocks) < 0.5] = -1
    sparse[lev == 0] = np.maximum(sparse[lev == 0], 0)
    out.append(sparse)
    allc = np.full(W.nblocks, -1)
    allc[lev == 0] = 0
    out.append(allc)                       # as many merges as 2:1 allows
    out.append(np.ones(W.nblocks, int))    # every leaf splits
    return [np.asarray(f, np.int8) for f in out]


@pytest.mark.parametrize("name", ["1d", "2d", "2d_outflow", "3d", "instances"])
def test_device_plan_equals_host_and_oracle(amr, name):
    W = (wl.c5_instances(count=5, nmin=32, nmax=96, precision="fp64") if name == "instances"
         else _cases()[name])
    S = amr.State.from_workload(W, kernel="plain")
    for seed in (3, 4):
        for f in _flag_patterns(W, seed):
            ref = rg.plan(W.cfg, W.instances, W.block_meta, f)
            host = amr.regrid_plan(W.cfg, W.instances, W.block_meta, f)
            dev = S.regrid_plan(f)
            np.testing.assert_array_equal(host, ref)
            np.testing.assert_array_equal(dev, ref)
    # flags from the device estimator, used where they are
    _, fl = S.regrid_estimate(0.05, 0.2, max_level=int(W.block_meta[:, 1].max()) + 1)
    np.testing.assert_array_equal(S.regrid_plan(), rg.plan(W.cfg, W.instances, W.block_meta, fl))
    S.close()


def test_device_plan_full_3d_blast_mesh(amr):
    # the benchmark's 3D AMR mesh (18,304 blocks over 4 levels): bit-identical
    # to the host plan, and timed against it
    import time
    W = wl.c4_blast_amr(base=6)
    S = amr.State.from_workload(W)
    for f in _flag_patterns(W, 7)[:2]:
        t0 = time.perf_counter()
        host = amr.regrid_plan(W.cfg, W.instances, W.block_meta, f)
        t_host = time.perf_counter() - t0
        S.regrid_plan(f)
        t0 = time.perf_counter()
        dev = S.regrid_plan(f)
        t_dev = time.perf_counter() - t0
        np.testing.assert_array_equal(dev, host)
        print("plan of %d -> %d blocks: host %.2f ms, device %.2f ms"
              % (W.nblocks, len(dev), 1e3 * t_host, 1e3 * t_dev))
    S.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("weights", ["rho", "rho_p", "all"])
def test_estimator_uniform_blocks(amr, orc, precision, weights):
    # the blast's initial state: uniform outside r < 0.1, so most blocks hold
    # one state bit for bit and take the estimator's uniform shortcut; their
    # estimate is exactly 0, as the oracle's, and the others match as usual
    W = _as(wl.c4_blast_amr(base=2, levels=3, bnx=8, shell=(0.2, 0.26), precision="fp64"),
            precision)
    wts = WEIGHTS[weights]
    Eo = rg.estimator(orc.mesh_for(W), W.U, W.cfg, weights=wts)
    S = amr.State.from_workload(W, kernel="plain")
    S.set_conserved(W.U.astype(np.float32) if precision == "fp32" else W.U)
    E, f = S.regrid_estimate(0.05, 0.2, max_level=3, weights=wts)
    S.close()
    tol = (1e-13 if weights == "rho" else 1e-12) if precision == "fp64" else 2e-5
    assert np.abs(E - Eo).max() <= tol, np.abs(E - Eo).max()
    # most blocks are 0 on both sides (rho alone is uniform everywhere); in FP64
    # every block the oracle finds exactly 0 is exactly 0 here too (in FP32 the
    # float ghost operators at level changes leave rounding-size estimates)
    zero = Eo == 0.0
    assert zero.sum() > W.nblocks // 2 and (E == 0.0).sum() > W.nblocks // 2
    if precision == "fp64":
        np.testing.assert_array_equal(E[zero], 0.0)
    fo = rg.flags(Eo, W.block_meta, 0.05, 0.2, 3)
    far = (np.abs(Eo - 0.05) > tol) & (np.abs(Eo - 0.01) > tol)
    np.testing.assert_array_equal(f[far], fo[far])
