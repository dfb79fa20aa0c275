"""Python side of the CPU oracle (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this package.  It loads oracle/snp_oracle.cpp, built by build() with the host
compiler, and shares no code with the CUDA simulator.  See snp_oracle.cpp for
the readings of the paper it implements.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snp_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsnp_oracle.so")
_libs = {}

_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no CUDA).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load(path: Optional[str] = None):
    """The oracle library (by default the one built from snp_oracle.cpp)."""
    path = path or build()
    if path in _libs:
        return _libs[path]
    lib = ctypes.CDLL(path)
    lib.orc_system_create.restype = ctypes.c_void_p
    lib.orc_system_create.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p]
    lib.orc_system_create_terms.restype = ctypes.c_void_p
    lib.orc_system_create_terms.argtypes = [ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p, _i32p, _i32p]
    lib.orc_system_free.argtypes = [ctypes.c_void_p]
    lib.orc_applicable.argtypes = [ctypes.c_void_p, _i32p, _u8p]
    lib.orc_psi.restype = ctypes.c_uint64
    lib.orc_psi.argtypes = [ctypes.c_void_p, _i32p]
    lib.orc_spiking_vectors.restype = ctypes.c_uint64
    lib.orc_spiking_vectors.argtypes = [ctypes.c_void_p, _i32p, ctypes.c_int64, _u8p]
    lib.orc_step.restype = ctypes.c_uint64
    lib.orc_step.argtypes = [ctypes.c_void_p, _i32p, ctypes.c_int64, _i32p, _i32p]
    lib.orc_child.restype = ctypes.c_int32
    lib.orc_child.argtypes = [ctypes.c_void_p, _i32p, ctypes.c_uint64, _i32p]
    lib.orc_explore.restype = ctypes.c_void_p
    lib.orc_explore.argtypes = [ctypes.c_void_p, _i32p, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                ctypes.c_int32]
    lib.orc_result_count.restype = ctypes.c_int64
    lib.orc_result_count.argtypes = [ctypes.c_void_p]
    lib.orc_result_ndepths.restype = ctypes.c_int32
    lib.orc_result_ndepths.argtypes = [ctypes.c_void_p]
    lib.orc_result_depth_reached.restype = ctypes.c_int32
    lib.orc_result_depth_reached.argtypes = [ctypes.c_void_p]
    lib.orc_result_error.restype = ctypes.c_int32
    lib.orc_result_error.argtypes = [ctypes.c_void_p]
    lib.orc_result_copy.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, _i32p]
    lib.orc_result_depth.argtypes = [ctypes.c_void_p, ctypes.c_int32, _i64p, _i64p, _u64p, _i32p]
    lib.orc_result_free.argtypes = [ctypes.c_void_p]
    _libs[path] = lib
    return lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


@dataclass
class DepthStats:
    new: int
    examined: int
    candidates: int  # sum of Psi over the level's parents, saturating at 2**64 - 1
    truncated: int


@dataclass
class Exploration:
    configs: np.ndarray          # int32 [n, m], discovery order
    depths: List[DepthStats]     # index 0 is the root level
    depth_reached: int
    error: int

    @property
    def per_depth_new(self) -> List[int]:
        return [d.new for d in self.depths]


class Oracle:
    """The oracle for one system (rule table and M_Pi copied in)."""

    def __init__(self, system, lib_path: Optional[str] = None):
        self.lib = _load(lib_path)
        self.m = int(system.m)
        self.R = int(system.R)
        if getattr(system, "terms", None) is not None:  # general rules: unions of terms
            self._keep = [np.ascontiguousarray(x, dtype=np.int32) for x in
                          (system.rule_neuron, *system.term_arrays(), system.M.reshape(-1))]
            self.h = self.lib.orc_system_create_terms(self.m, self.R, *[_p32(x) for x in self._keep])
        else:
            self._keep = [np.ascontiguousarray(x, dtype=np.int32) for x in
                          (system.rule_neuron, system.rule_i, system.rule_j, system.M.reshape(-1))]
            self.h = self.lib.orc_system_create(self.m, self.R, *[_p32(x) for x in self._keep])
        self.c0 = np.ascontiguousarray(system.c0, dtype=np.int32)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_system_free(self.h)
            self.h = None

    def _c(self, C) -> np.ndarray:
        C = np.ascontiguousarray(C, dtype=np.int32)
        assert C.shape == (self.m,)
        return C

    def applicable(self, C) -> np.ndarray:
        ok = np.zeros(self.R, dtype=np.uint8)
        self.lib.orc_applicable(self.h, _p32(self._c(C)), ok.ctypes.data_as(_u8p))
        return ok

    def psi(self, C) -> int:
        return int(self.lib.orc_psi(self.h, _p32(self._c(C))))

    def spiking_vectors(self, C, cap: int = 1 << 16) -> np.ndarray:
        C = self._c(C)
        n = min(self.psi(C), cap)
        S = np.zeros((max(n, 1), self.R), dtype=np.uint8)
        self.lib.orc_spiking_vectors(self.h, _p32(C), n, S.ctypes.data_as(_u8p))
        return S[:n]

    def step(self, C, cap: int = 1 << 16) -> np.ndarray:
        C = self._c(C)
        n = min(self.psi(C), cap)
        out = np.zeros((max(n, 1), self.m), dtype=np.int32)
        err = ctypes.c_int32(0)
        self.lib.orc_step(self.h, _p32(C), n, _p32(out), ctypes.byref(err))
        if err.value:
            raise OverflowError("a child leaves the int32 range")
        return out[:n]

    def child(self, C, t: int) -> Optional[np.ndarray]:
        out = np.zeros(self.m, dtype=np.int32)
        ok = self.lib.orc_child(self.h, _p32(self._c(C)), ctypes.c_uint64(int(t)), _p32(out))
        return out if ok else None

    def explore(self, depth: int, cap: int = 0, budget: int = 0, max_expand: int = -1,
                c0=None) -> Exploration:
        c0 = self.c0 if c0 is None else self._c(c0)
        r = self.lib.orc_explore(self.h, _p32(c0), int(depth), int(cap), int(budget), int(max_expand))
        try:
            n = self.lib.orc_result_count(r)
            configs = np.zeros((n, self.m), dtype=np.int32)
            if n:
                self.lib.orc_result_copy(r, 0, n, _p32(configs))
            depths = []
            for d in range(self.lib.orc_result_ndepths(r)):
                a, b, t = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
                c = ctypes.c_uint64()
                self.lib.orc_result_depth(r, d, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                          ctypes.byref(t))
                depths.append(DepthStats(a.value, b.value, c.value, t.value))
            return Exploration(configs, depths, self.lib.orc_result_depth_reached(r),
                               self.lib.orc_result_error(r))
        finally:
            self.lib.orc_result_free(r)
