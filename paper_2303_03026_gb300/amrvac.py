"""Python binding of the amrvac C ABI (include/amrvac.h).

Argument marshalling only: every step of the update runs in the CUDA library
``_lib/libamrvac_gb300.so``.  PyTorch supplies the device workspace and the
stream.  There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as wl

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libamrvac_gb300.so")

STATUS = {0: "ok", 1: "invalid", 2: "nomem", 3: "cuda", 4: "small_values", 5: "timeout",
          6: "state"}
KERNEL = {"auto": 0, "plain": 1, "fused": 2}
PRESSURE = {"fp64": 0, "ff": 1}
FP64, FP32 = 0, 1

# every symbol include/amrvac.h declares
SYMBOLS = ("amrvac_workspace_bytes", "amrvac_state_create", "amrvac_state_destroy",
           "amrvac_set_conserved", "amrvac_get_conserved", "amrvac_get_primitives",
           "amrvac_set_time",
           "amrvac_fill_ghosts", "amrvac_cfl_dt", "amrvac_set_dt", "amrvac_stage",
           "amrvac_step", "amrvac_get_diag", "amrvac_clear_error", "amrvac_launch_count",
           "amrvac_error_string", "amrvac_cfl_dt_noalloc", "amrvac_state_save",
           "amrvac_state_load", "amrvac_set_tuning", "amrvac_get_tuning", "amrvac_autotune",
           "amrvac_fix_small_values", "amrvac_regrid_estimate", "amrvac_regrid_plan",
           "amrvac_regrid_transfer", "amrvac_regrid_plan_device")


class AmrvacError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        super().__init__("%s: amrvac status %d (%s)" % (what, self.status,
                                                       STATUS.get(self.status, "?")))


class Config(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("block_nx", C.c_int32 * 3), ("flux", C.c_int32),
                ("limiter", C.c_int32), ("time", C.c_int32), ("precision", C.c_int32),
                ("glm", C.c_int32), ("glm_alpha", C.c_double), ("courant", C.c_double),
                ("bc", (C.c_int32 * 2) * 3), ("small_density", C.c_double),
                ("small_pressure", C.c_double), ("check_small_values", C.c_int32),
                ("kernel", C.c_int32), ("pressure", C.c_int32),
                ("fix_small_values", C.c_int32), ("reflux", C.c_int32),
                ("level_flux", C.c_int32 * 16), ("level_limiter", C.c_int32 * 16)]


class InstanceDesc(C.Structure):
    _fields_ = [("xmin", C.c_double * 3), ("xmax", C.c_double * 3),
                ("base_blocks", C.c_int32 * 3), ("gamma", C.c_double), ("t0", C.c_double),
                ("t_end", C.c_double)]


class Tuning(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("order", C.c_int32), ("dynamic", C.c_int32),
                ("faces", C.c_int32), ("ms_per_step", C.c_double)]

    def as_dict(self):
        return {"ctas_per_sm": self.ctas_per_sm, "order": ("morton", "storage")[self.order],
                "dynamic": bool(self.dynamic), "faces": ("sides", "xy")[self.faces],
                "ms_per_step": self.ms_per_step}


class ErrorInfo(C.Structure):
    _fields_ = [("code", C.c_int32), ("block", C.c_int32), ("cell", C.c_int32),
                ("var", C.c_int32)]


_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libamrvac_gb300.so not built: run paper_2303_03026_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, dbl = C.c_void_p, C.c_int32, C.c_double
    L.amrvac_workspace_bytes.argtypes = [C.POINTER(Config), i32, C.POINTER(InstanceDesc), i32,
                                         vp, C.POINTER(C.c_size_t)]
    L.amrvac_state_create.argtypes = [C.POINTER(Config), i32, C.POINTER(InstanceDesc), i32, vp,
                                      vp, C.c_size_t, vp, C.POINTER(vp)]
    L.amrvac_state_destroy.argtypes = [vp]
    L.amrvac_set_conserved.argtypes = [vp, i32, vp, i32, i32]
    L.amrvac_get_conserved.argtypes = [vp, i32, vp, i32, i32]
    L.amrvac_get_primitives.argtypes = [vp, i32, vp]
    L.amrvac_set_time.argtypes = [vp, vp, vp]
    L.amrvac_fill_ghosts.argtypes = [vp, i32, vp]
    L.amrvac_cfl_dt.argtypes = [vp, i32, vp]
    L.amrvac_set_dt.argtypes = [vp, vp, vp]
    L.amrvac_stage.argtypes = [vp, i32]
    L.amrvac_step.argtypes = [vp, i32]
    L.amrvac_get_diag.argtypes = [vp, vp, vp, vp, vp, C.POINTER(ErrorInfo)]
    L.amrvac_clear_error.argtypes = [vp]
    L.amrvac_launch_count.argtypes = [vp]
    L.amrvac_launch_count.restype = C.c_int64
    L.amrvac_error_string.argtypes = [i32]
    L.amrvac_error_string.restype = C.c_char_p
    L.amrvac_set_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.amrvac_get_tuning.argtypes = [vp, C.POINTER(Tuning)]
    L.amrvac_autotune.argtypes = [vp, i32, C.c_char_p, C.POINTER(Tuning)]
    L.amrvac_state_save.argtypes = [vp, C.c_char_p]
    L.amrvac_state_load.argtypes = [vp, C.c_char_p]
    L.amrvac_fix_small_values.argtypes = [vp, i32, vp]
    L.amrvac_regrid_estimate.argtypes = [vp, i32, vp, dbl, dbl, i32, vp, vp]
    L.amrvac_regrid_plan.argtypes = [C.POINTER(Config), i32, C.POINTER(InstanceDesc), i32, vp,
                                     vp, i32, vp, vp]
    L.amrvac_regrid_transfer.argtypes = [vp, i32, vp, i32]
    L.amrvac_regrid_plan_device.argtypes = [vp, vp, i32, vp, vp]
    L.amrvac_cfl_dt_noalloc.argtypes = [C.POINTER(Config), C.POINTER(InstanceDesc), i32, vp, dbl,
                                        vp, vp]
    _lib = L
    return L


def make_config(cfg: wl.Config, kernel: str = "auto", pressure: str = "fp64") -> Config:
    c = Config()
    c.ndim = cfg.ndim
    for d in range(3):
        c.block_nx[d] = int(cfg.block_nx[d]) if d < cfg.ndim else 1
        c.bc[d][0] = wl.BC[cfg.bc[d][0]]
        c.bc[d][1] = wl.BC[cfg.bc[d][1]]
    c.flux = wl.FLUX[cfg.flux]
    c.limiter = wl.LIMITER[cfg.limiter]
    c.time = wl.TIME[cfg.time]
    c.precision = wl.PRECISION[cfg.precision]
    c.glm = int(bool(cfg.glm))
    c.glm_alpha = float(cfg.glm_alpha)
    c.courant = float(cfg.courant)
    c.small_density = float(cfg.small_density)
    c.small_pressure = float(cfg.small_pressure)
    c.check_small_values = int(bool(cfg.check_small_values))
    c.kernel = KERNEL[kernel]
    c.pressure = PRESSURE[pressure]
    c.fix_small_values = wl.FIX[getattr(cfg, "fix_small_values", "off")]
    c.reflux = int(bool(getattr(cfg, "reflux", False)))
    lf = getattr(cfg, "level_flux", None) or {}
    ll = getattr(cfg, "level_limiter", None) or {}
    for lev in range(16):
        c.level_flux[lev] = wl.FLUX[lf[lev]] + 1 if lev in lf else 0
        c.level_limiter[lev] = wl.LIMITER[ll[lev]] + 1 if lev in ll else 0
    return c


def make_instances(instances) -> C.Array:
    arr = (InstanceDesc * len(instances))()
    for q, inst in enumerate(instances):
        for d in range(3):
            arr[q].xmin[d] = float(inst.xmin[d])
            arr[q].xmax[d] = float(inst.xmax[d])
            arr[q].base_blocks[d] = int(inst.base_blocks[d])
        arr[q].gamma = float(inst.gamma)
        arr[q].t0 = float(inst.t0)
        arr[q].t_end = float(inst.t_end)
    return arr


def _check(st, what):
    if st != 0:
        raise AmrvacError(st, what)


class State:
    """One mesh + state on a GPU.  ``cfg``/``instances``/``block_meta`` follow
    workloads.py; the device workspace is a torch uint8 tensor."""

    def __init__(self, cfg, instances, block_meta, device="cuda:0", kernel="auto", stream=None,
                 pressure="fp64"):
        import torch
        self.torch = torch
        L = load()
        self.cfg = cfg
        self.instances = list(instances)
        self.ninst = len(self.instances)
        self._c = make_config(cfg, kernel, pressure)
        self._inst = make_instances(self.instances)
        self.meta = np.ascontiguousarray(block_meta, np.int32)
        self.nblocks = int(self.meta.shape[0])
        self.ncell = int(np.prod([cfg.block_nx[d] if d < cfg.ndim else 1 for d in range(3)]))
        self.precision = wl.PRECISION[cfg.precision]
        self.dtype = torch.float64 if self.precision == FP64 else torch.float32
        nbytes = C.c_size_t(0)
        _check(L.amrvac_workspace_bytes(C.byref(self._c), self.ninst, self._inst, self.nblocks,
                                        self.meta.ctypes.data, C.byref(nbytes)),
               "amrvac_workspace_bytes")
        self.device = torch.device(device)
        self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8,
                                     device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        h = C.c_void_p()
        _check(L.amrvac_state_create(C.byref(self._c), self.ninst, self._inst, self.nblocks,
                                     self.meta.ctypes.data, C.c_void_p(self._ws_ptr),
                                     int(nbytes.value), C.c_void_p(self.stream.cuda_stream),
                                     C.byref(h)), "amrvac_state_create")
        self._h = h

    @classmethod
    def from_workload(cls, W, **kw):
        return cls(W.cfg, W.instances, W.block_meta, **kw)

    def close(self):
        if getattr(self, "_h", None):
            load().amrvac_state_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (9, self.nblocks, self.ncell)

    # ------------------------------------------------------------- data
    def set_conserved(self, U, buffer=0):
        """U: numpy array (host) or torch tensor (host or device), [9, nblocks, ncell]."""
        torch = self.torch
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U)
            assert U.shape == self.shape, U.shape
            prec = FP64 if U.dtype == np.float64 else FP32
            assert U.dtype in (np.float64, np.float32)
            _check(load().amrvac_set_conserved(self._h, buffer, U.ctypes.data, 0, prec),
                   "amrvac_set_conserved")
            self.stream.synchronize()
            return
        assert tuple(U.shape) == self.shape and U.is_contiguous()
        prec = FP64 if U.dtype == torch.float64 else FP32
        if U.is_cuda:
            # the tensor was produced on torch's current stream
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _check(load().amrvac_set_conserved(self._h, buffer, U.data_ptr(), int(U.is_cuda), prec),
               "amrvac_set_conserved")
        if U.is_cuda:
            U.record_stream(self.stream)
        else:
            self.stream.synchronize()

    def get_conserved(self, buffer=0, out=None, numpy=True, precision=None):
        """Returns buffer as a numpy array (default) or a device tensor, or fills
        ``out`` (torch tensor on host or device)."""
        torch = self.torch
        if out is None:
            if numpy:
                dt = np.float64 if (precision if precision is not None else self.precision) == FP64 \
                    else np.float32
                arr = np.empty(self.shape, dt)
                prec = FP64 if dt == np.float64 else FP32
                _check(load().amrvac_get_conserved(self._h, buffer, arr.ctypes.data, 0, prec),
                       "amrvac_get_conserved")
                self.stream.synchronize()
                return arr
            out = torch.empty(self.shape, dtype=self.dtype, device=self.device)
        prec = FP64 if out.dtype == torch.float64 else FP32
        if out.is_cuda:
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
        _check(load().amrvac_get_conserved(self._h, buffer, out.data_ptr(), int(out.is_cuda), prec),
               "amrvac_get_conserved")
        if out.is_cuda:
            # later torch work on the result is ordered after the copy
            torch.cuda.current_stream(self.device).wait_stream(self.stream)
        else:
            self.stream.synchronize()
        return out

    @property
    def ng(self):
        """Ghost cells per block face of the ghost export: 3 when the limiter
        or a level's limiter is a five-point one (mp5, weno5, wenoz5), else 2."""
        five = {"mp5", "weno5", "wenoz5", "wenozp5"}
        lims = {self.cfg.limiter} | set((self.cfg.level_limiter or {}).values())
        return 3 if lims & five else 2

    def get_primitives(self, buffer=0):
        """Primitive variables (rho, v, p, B, psi) of buffer, as the stage
        kernels recover them, returned as a numpy array in the state's
        precision."""
        out = self.torch.empty(self.shape, dtype=self.dtype, device=self.device)
        self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
        _check(load().amrvac_get_primitives(self._h, buffer, out.data_ptr()),
               "amrvac_get_primitives")
        self.stream.synchronize()
        return out.cpu().numpy()

    def fill_ghosts(self, buffer=0):
        P = 1
        for d in range(self.cfg.ndim):
            P *= self.cfg.block_nx[d] + 2 * self.ng
        out = self.torch.zeros((9, self.nblocks, P), dtype=self.dtype, device=self.device)
        self.torch.cuda.current_stream(self.device).synchronize()
        _check(load().amrvac_fill_ghosts(self._h, buffer, out.data_ptr()), "amrvac_fill_ghosts")
        self.stream.synchronize()
        return out.cpu().numpy()

    # ------------------------------------------------------------- time
    def set_time(self, t=None, t_end=None):
        tp = None if t is None else np.ascontiguousarray(np.broadcast_to(t, (self.ninst,)), np.float64)
        te = None if t_end is None else np.ascontiguousarray(
            np.broadcast_to(t_end, (self.ninst,)), np.float64)
        _check(load().amrvac_set_time(self._h, None if tp is None else tp.ctypes.data,
                                      None if te is None else te.ctypes.data), "amrvac_set_time")

    def cfl_dt(self, buffer=0):
        dt = np.zeros(self.ninst)
        _check(load().amrvac_cfl_dt(self._h, buffer, dt.ctypes.data), "amrvac_cfl_dt")
        return dt

    def set_dt(self, dt, ch):
        dt = np.ascontiguousarray(np.broadcast_to(dt, (self.ninst,)), np.float64)
        ch = np.ascontiguousarray(np.broadcast_to(ch, (self.ninst,)), np.float64)
        _check(load().amrvac_set_dt(self._h, dt.ctypes.data, ch.ctypes.data), "amrvac_set_dt")

    def stage(self, k):
        _check(load().amrvac_stage(self._h, k), "amrvac_stage")

    def step(self, n=1):
        _check(load().amrvac_step(self._h, n), "amrvac_step")

    def diag(self, raise_on_error=False):
        t = np.zeros(self.ninst)
        dt = np.zeros(self.ninst)
        ch = np.zeros(self.ninst)
        sums = np.zeros((self.ninst, 9))
        err = ErrorInfo()
        st = load().amrvac_get_diag(self._h, t.ctypes.data, dt.ctypes.data, ch.ctypes.data,
                                    sums.ctypes.data, C.byref(err))
        if st not in (0, 4, 6) or (raise_on_error and st != 0):
            raise AmrvacError(st, "amrvac_get_diag")
        return {"t": t, "dt": dt, "ch": ch, "sums": sums, "status": st,
                "error": (err.code, err.block, err.cell, err.var)}

    def set_tuning(self, ctas_per_sm=0, order="morton", dynamic=False, faces="sides"):
        """Launch shape of the fused kernels (amrvac_tuning): faces "sides" packs
        the two sides of one face per float2 lane pair, "xy" a cell's x and y
        faces (FP32 vanleer + HLLD)."""
        t = Tuning(int(ctas_per_sm), {"morton": 0, "storage": 1}[order], int(bool(dynamic)),
                   {"sides": 0, "xy": 1}[faces], 0.0)
        _check(load().amrvac_set_tuning(self._h, C.byref(t)), "amrvac_set_tuning")

    def get_tuning(self):
        t = Tuning()
        _check(load().amrvac_get_tuning(self._h, C.byref(t)), "amrvac_get_tuning")
        return t.as_dict()

    def autotune(self, trial_steps=3, cache=None):
        t = Tuning()
        _check(load().amrvac_autotune(self._h, int(trial_steps),
                                      None if cache is None else os.fsencode(cache), C.byref(t)),
               "amrvac_autotune")
        return t.as_dict()

    def save(self, path):
        _check(load().amrvac_state_save(self._h, os.fsencode(path)), "amrvac_state_save")

    def restore(self, path):
        _check(load().amrvac_state_load(self._h, os.fsencode(path)), "amrvac_state_load")

    def fix_small(self, buffer=0):
        """fix_small_values on register ``buffer``; returns the cells repaired."""
        n = C.c_int64(0)
        _check(load().amrvac_fix_small_values(self._h, int(buffer), C.addressof(n)),
               "amrvac_fix_small_values")
        return n.value

    # -------------------------------------------------------- regridding
    def regrid_estimate(self, refine_threshold, derefine_ratio=0.125, max_level=15, buffer=0,
                        weights=None):
        """Per-block estimator and flags of register ``buffer`` (numpy float64
        [nblocks], int8 [nblocks]); ``weights``: 9 weights of the primitive
        variables (rho, v, p, B, psi), default the density alone.  See
        amrvac_regrid_estimate."""
        est = np.zeros(self.nblocks, np.float64)
        flags = np.zeros(self.nblocks, np.int8)
        wp = None
        if weights is not None:
            wv = np.ascontiguousarray(weights, np.float64)
            assert wv.shape == (9,)
            wp = wv.ctypes.data
        _check(load().amrvac_regrid_estimate(self._h, int(buffer), wp, float(refine_threshold),
                                             float(derefine_ratio), int(max_level),
                                             est.ctypes.data, flags.ctypes.data),
               "amrvac_regrid_estimate")
        return est, flags

    def regrid_plan(self, flags=None):
        """Block list after one regrid, planned on the device from this state's
        mesh (amrvac_regrid_plan_device); ``flags``: int8 [nblocks] (1 refine,
        -1 coarsen, 0 keep), default the flags of the last regrid_estimate."""
        fp = None
        if flags is not None:
            fl = np.ascontiguousarray(flags, np.int8)
            assert fl.shape == (self.nblocks,)
            fp = fl.ctypes.data
        cap = self.nblocks * (1 << self.cfg.ndim)
        out = np.zeros((cap, 5), np.int32)
        n = C.c_int32(0)
        _check(load().amrvac_regrid_plan_device(self._h, fp, cap, out.ctypes.data, C.byref(n)),
               "amrvac_regrid_plan_device")
        return out[:n.value].copy()

    def regrid_transfer(self, dst, buffer=0, dst_buffer=0):
        """Fill register ``dst_buffer`` of State ``dst`` (built on a planned block
        list) from register ``buffer`` of this state."""
        _check(load().amrvac_regrid_transfer(self._h, int(buffer), dst._h, int(dst_buffer)),
               "amrvac_regrid_transfer")

    def regrid(self, refine_threshold, derefine_ratio=0.125, max_level=15, buffer=0,
               weights=None, kernel="auto", pressure="fp64"):
        """One regrid of register ``buffer``: estimator, plan and transfer into a
        new State (returned; this one is left as it is).  Each instance's clock
        continues from this state's time."""
        _, flags = self.regrid_estimate(refine_threshold, derefine_ratio, max_level, buffer,
                                        weights)
        meta = regrid_plan(self.cfg, self.instances, self.meta, flags)
        d = self.diag()
        insts = []
        for q, inst in enumerate(self.instances):
            i2 = wl.Instance(**{**inst.__dict__, "t0": float(d["t"][q])})
            insts.append(i2)
        new = State(self.cfg, insts, meta, device=self.device, kernel=kernel,
                    pressure=pressure)
        self.regrid_transfer(new, buffer, 0)
        return new

    def clear_error(self):
        _check(load().amrvac_clear_error(self._h), "amrvac_clear_error")

    @property
    def launches(self) -> int:
        return int(load().amrvac_launch_count(self._h))


def regrid_plan(cfg, instances, block_meta, flags):
    """Block list after one regrid with per-block ``flags`` (1 refine, -1
    coarsen, 0 keep); host logic of the library (amrvac_regrid_plan)."""
    L = load()
    c = make_config(cfg)
    inst = make_instances(instances)
    meta = np.ascontiguousarray(block_meta, np.int32)
    fl = np.ascontiguousarray(flags, np.int8)
    assert fl.shape == (meta.shape[0],)
    cap = meta.shape[0] * (1 << cfg.ndim) + 16
    out = np.zeros((cap, 5), np.int32)
    n = C.c_int32(0)
    st = L.amrvac_regrid_plan(C.byref(c), len(instances), inst, meta.shape[0], meta.ctypes.data,
                              fl.ctypes.data, cap, out.ctypes.data, C.byref(n))
    _check(st, "amrvac_regrid_plan")
    return out[:n.value].copy()


def cfl_dt_noalloc(cfg, instance, U, out, t=0.0, stream=None):
    """CFL time step of a uniform single-instance state without a workspace.

    For callers that cannot allocate device memory: ``U`` is the caller's
    device tensor [9, nblocks, ncell] (float64 or float32 matching
    ``cfg.precision``), ``out`` a caller-provided device float64 tensor of 2
    elements that receives (dt, c_h).  The library uses a fixed 1 MiB device
    array (at most AMRVAC_NOALLOC_MAX_BLOCKS = 65536 blocks) and allocates
    nothing.  Asynchronous on ``stream`` (default: torch's current stream)."""
    import torch
    c = make_config(cfg)
    inst = make_instances([instance])
    s = stream if stream is not None else torch.cuda.current_stream(U.device)
    _check(load().amrvac_cfl_dt_noalloc(C.byref(c), inst, int(U.shape[1]), U.data_ptr(),
                                        float(t), out.data_ptr(), s.cuda_stream),
           "amrvac_cfl_dt_noalloc")
