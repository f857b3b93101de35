"""GPU test of amrvac_cfl_dt_noalloc, the CFL entry point for callers that
cannot allocate device memory (no workspace, no state: only their own input
and output buffers; the library keeps its per-block partials in a fixed
1 MiB device array).

Its result must equal that of the workspace-based amrvac_cfl_dt within the
tolerance the CFL parity tests use (1e-13 relative), on two calls in a row:
the second call covers fewer blocks than the first, so stale partials left in
the shared array by the first call would show up.
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


def _reference_and_noalloc(amr, W, t):
    import torch
    np_dtype = np.float64 if W.cfg.precision == "fp64" else np.float32
    U = np.ascontiguousarray(W.U.astype(np_dtype))
    S = amr.State.from_workload(W, kernel="plain")
    S.set_conserved(U)
    S.set_time(t=t)
    dt = S.cfl_dt()
    ch = S.diag()["ch"]
    S.close()
    dU = torch.from_numpy(U).cuda()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    amr.cfl_dt_noalloc(W.cfg, W.instances[0], dU, out, t=t)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    return got, (dt[0], ch[0])


def test_noalloc_cfl_matches_workspace_entry_point_twice(amr):
    W1 = wl.c2_orszag_tang(256)                                  # FP64, 256 blocks
    W2 = wl.c3_turbulence(n=32, bnx=16, precision="fp32")        # FP32, 8 blocks
    W2.instances[0].t_end = 1e-4                                 # the clip binds here
    for W, t in ((W1, 0.0), (W2, 0.0)):
        got, ref = _reference_and_noalloc(amr, W, t)
        assert abs(got[0] - ref[0]) <= TOL * abs(ref[0]), (W.name, got, ref)
        assert abs(got[1] - ref[1]) <= TOL * abs(ref[1]), (W.name, got, ref)
    assert got[0] == 1e-4


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
    torch.cuda.synchronize()
    assert out.abs().sum().item() == 0.0
