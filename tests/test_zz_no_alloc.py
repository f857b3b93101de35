"""GPU test of amrvac_cfl_dt_noalloc, the CFL entry point for callers that
cannot allocate device memory (no workspace, no state: only their own input
and output buffers; the library keeps its per-block partials in a fixed
1 MiB device array).

Its result must equal that of the workspace-based amrvac_cfl_dt within the
tolerance the CFL parity tests use (1e-13 relative), and the FP64 oracle's
(1e-13 for FP64 states, 1e-5 for FP32-bulk states, whose CFL terms are formed
in float), on calls in a row over the shared array: the first call covers as
many blocks as the second but has faster signal speeds, so a partial the
second call failed to write would leave a larger stale maximum behind and
change its result.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2303_03026_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def amr():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2303_03026_gb300 import amrvac
    return amrvac


def _reference_and_noalloc(amr, orc, W, t):
    import torch
    np_dtype = np.float64 if W.cfg.precision == "fp64" else np.float32
    U = np.ascontiguousarray(W.U.astype(np_dtype))
    S = amr.State.from_workload(W, kernel="plain")
    S.set_conserved(U)
    S.set_time(t=t)
    dt = S.cfl_dt()
    ch = S.diag()["ch"]
    S.close()
    odt, och = orc.mesh_for(W).cfl(U.astype(np.float64), t=t, t_end=W.instances[0].t_end)
    dU = torch.from_numpy(U).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    amr.cfl_dt_noalloc(W.cfg, W.instances[0], dU, out, t=t)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    return got, (dt[0], ch[0]), (odt[0], och[0])


def test_noalloc_cfl_matches_workspace_entry_point_and_oracle(amr, orc):
    W1 = wl.c2_orszag_tang(256)                                  # FP64, 256 blocks, fast
    W2 = wl.cp_alfven(256, precision="fp32")                     # FP32, 256 blocks, slower
    W3 = wl.c3_turbulence(n=32, bnx=16, precision="fp32")        # FP32, 8 blocks
    W3.instances[0].t_end = 1e-4                                 # the clip binds here
    assert W2.nblocks >= W1.nblocks
    res = []
    for W, t in ((W1, 0.0), (W2, 0.0), (W3, 0.0)):
        got, ref, orac = _reference_and_noalloc(amr, orc, W, t)
        assert abs(got[0] - ref[0]) <= TOL * abs(ref[0]), (W.name, got, ref)
        assert abs(got[1] - ref[1]) <= TOL * abs(ref[1]), (W.name, got, ref)
        otol = TOL if W.cfg.precision == "fp64" else 1e-5
        assert abs(got[0] - orac[0]) <= otol * abs(orac[0]), (W.name, got, orac)
        assert abs(got[1] - orac[1]) <= otol * abs(orac[1]), (W.name, got, orac)
        res.append(got)
    # the second state's signal speeds are below the first's: stale partials
    # of the first call would have raised its c_h and lowered its dt
    assert res[1][1] < res[0][1] and res[1][0] > res[0][0]
    assert res[2][0] == 1e-4


def test_noalloc_rejects_more_blocks_than_its_array(amr):
    import torch
    cfg = wl.Config(ndim=2, block_nx=(16, 16, 1))
    inst = wl.Instance(base_blocks=(300, 300, 1))  # 90,000 blocks > 65,536
    c = amr.make_config(cfg)
    ins = amr.make_instances([inst])
    U = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = amr.load().amrvac_cfl_dt_noalloc(C.byref(c), ins, 90000, U.data_ptr(), 0.0,
                                          out.data_ptr(), None)
    assert st == 1  # AMRVAC_E_INVALID, nothing launched
    # one 4096^3 block: 2^36 cells, beyond AMRVAC_MAX_BLOCK_CELLS (and an int)
    big = amr.make_config(wl.Config(ndim=3, block_nx=(4096, 4096, 4096)))
    one = amr.make_instances([wl.Instance(base_blocks=(1, 1, 1))])
    st = amr.load().amrvac_cfl_dt_noalloc(C.byref(big), one, 1, U.data_ptr(), 0.0,
                                          out.data_ptr(), None)
    assert st == 1
    torch.cuda.synchronize()
    assert out.abs().sum().item() == 0.0
