"""ctypes wrapper of the FP64 CPU oracle (oracle/amrvac_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The GPU library and its
Python binding never do; the two share no source.

The oracle is a plain FP64 restatement of the update (see the header of
amrvac_oracle.c for the readings of the paper it follows).  Its parity is
pinned in tests/test_oracle_*.py against exact solutions, conservation,
Rankine-Hugoniot relations, closed forms and brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "amrvac_oracle.c")
_lock = threading.Lock()
_lib = None

NVAR = 9


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-1] + "h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Config(C.Structure):
    _fields_ = [("ndim", C.c_int), ("nx", C.c_int * 3), ("flux", C.c_int),
                ("limiter", C.c_int), ("time", C.c_int), ("glm", C.c_int),
                ("glm_alpha", C.c_double), ("courant", C.c_double),
                ("bc", (C.c_int * 2) * 3), ("small_density", C.c_double),
                ("small_pressure", C.c_double), ("check_small_values", C.c_int),
                ("fix_small_values", C.c_int), ("reflux", C.c_int),
                ("level_flux", C.c_int * 16), ("level_limiter", C.c_int * 16)]


class _Instance(C.Structure):
    _fields_ = [("xmin", C.c_double * 3), ("xmax", C.c_double * 3), ("base", C.c_int * 3),
                ("gamma", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            L.orc_create.restype = C.c_void_p
            L.orc_create.argtypes = [C.POINTER(_Config), C.c_int, C.POINTER(_Instance), C.c_int,
                                     ip, C.c_char_p, C.c_int]
            L.orc_destroy.argtypes = [C.c_void_p]
            L.orc_set_threads.argtypes = [C.c_void_p, C.c_int]
            L.orc_fill_ghosts.argtypes = [C.c_void_p, dp, dp]
            L.orc_stage.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp, dp, C.c_void_p, C.c_int]
            L.orc_stage2.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, dp, dp, dp, dp,
                                     C.c_void_p, C.c_int]
            L.orc_cfl.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
            L.orc_sums.argtypes = [C.c_void_p, dp, dp]
            L.orc_run.argtypes = [C.c_void_p, dp, dp, dp, C.c_int, C.c_double,
                                  C.POINTER(C.c_int)]
            L.orc_cons_to_prim.argtypes = [C.c_double, dp, dp]
            L.orc_prim_to_cons.argtypes = [C.c_double, dp, dp]
            L.orc_fast_speed.restype = C.c_double
            L.orc_fast_speed.argtypes = [C.c_double, dp, C.c_int]
            L.orc_reconstruct.argtypes = [C.c_int, dp, C.c_int, dp, dp]
            L.orc_reconstruct5.argtypes = [C.c_int, dp, C.c_int, C.c_double, dp, dp]
            L.orc_ghost_width.argtypes = [C.c_void_p]
            L.orc_ghost_width.restype = C.c_int
            L.orc_face_flux.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                        dp, dp, dp]
            L.orc_stage_coeffs.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]
            L.orc_stage_coeffs6.argtypes = [C.c_int, C.c_int, dp]
            L.orc_num_stages.argtypes = [C.c_int]
            L.orc_fix_small.argtypes = [C.c_void_p, dp, C.c_int]
            L.orc_fix_small.restype = C.c_long
            L.orc_num_stages.restype = C.c_int
            _lib = L
    return _lib


_FLUX = {"hll": 0, "hlld": 1, "tvdlf": 2, "hllc": 3}
_LIM = {"minmod": 0, "vanleer": 1, "koren": 2, "superbee": 3, "woodward": 4, "mcbeta": 5,
        "albada": 6, "mp5": 7, "weno5": 8, "wenoz5": 9, "cada3": 10, "wenozp5": 11,
        "venk": 12}
_FIVE = (7, 8, 9, 11)
_TIME = {"ssprk2": 0, "ssprk3": 1, "ssprk43": 2, "ssprk54": 3}
_BC = {"periodic": 0, "outflow": 1, "symmetric": 2}
_FIX = {"off": 0, "replace": 1, "average": 2}


class Mesh:
    """One oracle mesh built from a workload's config, instances and block list."""

    def __init__(self, cfg, instances, block_meta, threads: int = 1):
        L = lib()
        c = _Config()
        c.ndim = cfg.ndim
        for d in range(3):
            c.nx[d] = int(cfg.block_nx[d]) if d < cfg.ndim else 1
            c.bc[d][0] = _BC[cfg.bc[d][0]]
            c.bc[d][1] = _BC[cfg.bc[d][1]]
        c.flux = _FLUX[cfg.flux]
        c.limiter = _LIM[cfg.limiter]
        c.time = _TIME[cfg.time]
        c.glm = int(bool(cfg.glm))
        c.glm_alpha = float(cfg.glm_alpha)
        c.courant = float(cfg.courant)
        c.small_density = float(cfg.small_density)
        c.small_pressure = float(cfg.small_pressure)
        c.check_small_values = int(bool(cfg.check_small_values))
        c.fix_small_values = _FIX[getattr(cfg, "fix_small_values", "off")]
        c.reflux = int(bool(getattr(cfg, "reflux", False)))
        lf = getattr(cfg, "level_flux", None) or {}
        ll = getattr(cfg, "level_limiter", None) or {}
        for lev in range(16):
            c.level_flux[lev] = _FLUX[lf[lev]] if lev in lf else -1
            c.level_limiter[lev] = _LIM[ll[lev]] if lev in ll else -1
        arr = (_Instance * len(instances))()
        for q, inst in enumerate(instances):
            for d in range(3):
                arr[q].xmin[d] = float(inst.xmin[d])
                arr[q].xmax[d] = float(inst.xmax[d])
                arr[q].base[d] = int(inst.base_blocks[d])
            arr[q].gamma = float(inst.gamma)
        self.meta = np.ascontiguousarray(block_meta, np.int32)
        err = C.create_string_buffer(256)
        self._h = L.orc_create(C.byref(c), len(instances), arr, self.meta.shape[0],
                               self.meta, err, 256)
        if not self._h:
            raise ValueError("oracle mesh: " + err.value.decode())
        self.cfg = cfg
        self.instances = instances
        self.ninst = len(instances)
        self.nblocks = self.meta.shape[0]
        self.ncell = int(np.prod([cfg.block_nx[d] if d < cfg.ndim else 1 for d in range(3)]))
        self.set_threads(threads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_threads(self, n: int):
        self.threads = max(1, int(n))
        lib().orc_set_threads(self._h, self.threads)

    def _u(self, U):
        U = np.ascontiguousarray(U, np.float64)
        assert U.shape == (NVAR, self.nblocks, self.ncell), U.shape
        return U

    @property
    def ng(self):
        """Ghost cells per block face (3 with a five-point limiter, else 2)."""
        return lib().orc_ghost_width(self._h)

    def padded_shape(self):
        P = 1
        for d in range(self.cfg.ndim):
            P *= self.cfg.block_nx[d] + 2 * self.ng
        return (NVAR, self.nblocks, P)

    def fill_ghosts(self, U):
        out = np.zeros(self.padded_shape())
        lib().orc_fill_ghosts(self._h, self._u(U), out)
        return out

    def stage(self, k, dt, ch, U0, Uk, blocks=None, out=None):
        """Stage k; returns (out, status).  ``blocks`` restricts the blocks computed
        (other blocks of ``out`` keep their content)."""
        dt = np.ascontiguousarray(np.broadcast_to(dt, (self.ninst,)), np.float64)
        ch = np.ascontiguousarray(np.broadcast_to(ch, (self.ninst,)), np.float64)
        U0 = self._u(U0)
        Uk = self._u(Uk)
        if out is None:
            out = np.zeros_like(Uk)
        if blocks is None:
            st = lib().orc_stage(self._h, k, dt, ch, U0, Uk, out, None, 0)
        else:
            sub = np.ascontiguousarray(blocks, np.int32)
            st = lib().orc_stage(self._h, k, dt, ch, U0, Uk, out,
                                 sub.ctypes.data_as(C.c_void_p), sub.shape[0])
        return out, st

    def stage2(self, k, dt, ch, U0, Uk, U2):
        """Stage k with its second output (SSPRK(5,4) stage 3): returns
        (out, out2, status) on fresh arrays."""
        dt = np.ascontiguousarray(np.broadcast_to(dt, (self.ninst,)), np.float64)
        ch = np.ascontiguousarray(np.broadcast_to(ch, (self.ninst,)), np.float64)
        U0, Uk, U2 = self._u(U0), self._u(Uk), self._u(U2)
        out = np.zeros_like(Uk)
        out2 = np.zeros_like(Uk)
        st = lib().orc_stage2(self._h, k, dt, ch, U0, Uk, U2, out, out2, None, 0)
        return out, out2, st

    def fix_small(self, U, method):
        """fix_small_values on a copy of U; returns (U, number of cells fixed)."""
        U = self._u(U).copy()
        n = lib().orc_fix_small(self._h, U, _FIX[method])
        return U, n

    def cfl(self, U, t=None, t_end=None):
        t = np.zeros(self.ninst) if t is None else np.ascontiguousarray(
            np.broadcast_to(t, (self.ninst,)), np.float64)
        te = np.full(self.ninst, 1e300) if t_end is None else np.ascontiguousarray(
            np.broadcast_to(t_end, (self.ninst,)), np.float64)
        dt = np.zeros(self.ninst)
        ch = np.zeros(self.ninst)
        lib().orc_cfl(self._h, self._u(U), t, te, dt, ch)
        return dt, ch

    def sums(self, U):
        s = np.zeros((self.ninst, NVAR))
        lib().orc_sums(self._h, self._u(U), s)
        return s

    def run(self, U, t_end, t=None, maxsteps=10 ** 9, fixed_dt=0.0):
        """Advance a copy of U; returns (U, t, nsteps, status)."""
        U = self._u(U).copy()
        t = np.zeros(self.ninst) if t is None else np.array(
            np.broadcast_to(t, (self.ninst,)), np.float64)
        te = np.ascontiguousarray(np.broadcast_to(t_end, (self.ninst,)), np.float64)
        n = C.c_int(0)
        st = lib().orc_run(self._h, U, t, te, int(maxsteps), float(fixed_dt), C.byref(n))
        return U, t, n.value, st


def mesh_for(workload, threads: int = 1) -> Mesh:
    return Mesh(workload.cfg, workload.instances, workload.block_meta, threads)


# pointwise helpers for pin tests ---------------------------------------------

def cons_to_prim(gamma, u):
    w = np.zeros(NVAR)
    lib().orc_cons_to_prim(gamma, np.ascontiguousarray(u, np.float64), w)
    return w


def prim_to_cons(gamma, w):
    u = np.zeros(NVAR)
    lib().orc_prim_to_cons(gamma, np.ascontiguousarray(w, np.float64), u)
    return u


def fast_speed(gamma, w, d):
    return lib().orc_fast_speed(gamma, np.ascontiguousarray(w, np.float64), d)


def reconstruct(limiter, w, dx=1.0):
    """Face states of a 1D row of cell values: wl[i] at i+1/2 and wr[i] at
    i-1/2 (NaN where the stencil leaves the row); dx: the cell width, used by
    wenozp5 only."""
    w = np.ascontiguousarray(w, np.float64)
    wl = np.full_like(w, np.nan)
    wr = np.full_like(w, np.nan)
    lim = _LIM[limiter]
    if lim in _FIVE:
        lib().orc_reconstruct5(lim, w, w.shape[0], float(dx), wl, wr)
    else:
        lib().orc_reconstruct(lim, w, w.shape[0], wl, wr)
    return wl, wr


def face_flux(flux, glm, gamma, ch, d, wl, wr):
    f = np.zeros(NVAR)
    lib().orc_face_flux(_FLUX[flux], int(glm), gamma, ch, d,
                        np.ascontiguousarray(wl, np.float64),
                        np.ascontiguousarray(wr, np.float64), f)
    return f


def stage_coeffs(time, k):
    a = C.c_double()
    b = C.c_double()
    lib().orc_stage_coeffs(_TIME[time], k, C.byref(a), C.byref(b))
    return a.value, b.value


def stage_coeffs6(time, k):
    """{a, b, c, a2, b2, c2} of stage k: out = a U0 + b (Uk + c dt L(Uk)),
    out2 = a2 U2 + b2 (Uk + c2 dt L(Uk))."""
    co = np.zeros(6)
    lib().orc_stage_coeffs6(_TIME[time], k, co)
    return co


def num_stages(time):
    return lib().orc_num_stages(_TIME[time])
