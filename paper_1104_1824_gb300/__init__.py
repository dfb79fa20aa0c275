"""GB300 simulator for spiking neural P systems without delays.

A thin ctypes binding over the C ABI in include/snp.h (libsnp_gb300.so, built
by paper_1104_1824_gb300.build).  Every function with an ``snp_`` name marshals
its arguments and calls the C function of the same name; every step of the
exploration runs in the library's CUDA kernels.  There is no fallback: if the
library is missing, the first call raises ImportError.

Arrays may be numpy arrays (host memory) or objects exposing ``data_ptr()``
such as torch tensors (device memory); the library infers the copy direction.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsnp_gb300.so")

SNP_OK = 0
SNP_E_INVALID = 1
SNP_E_RANGE = 2
SNP_E_NOMEM = 3
SNP_E_CUDA = 4
SNP_E_TIMEOUT = 5
SNP_E_BUFFER = 6
SNP_E_OVERFLOW = 7
SNP_E_STATE = 8
SNP_E_INTERNAL = 9
SNP_E_CANCELLED = 10
SNP_T_SPARSE_I32 = 0
SNP_T_TC_I8 = 1
SNP_T_TC_F8 = 2
SNP_PSI_SAT = (1 << 64) - 1

ERROR_NAMES = {0: "SNP_OK", 1: "SNP_E_INVALID", 2: "SNP_E_RANGE", 3: "SNP_E_NOMEM", 4: "SNP_E_CUDA",
               5: "SNP_E_TIMEOUT", 6: "SNP_E_BUFFER", 7: "SNP_E_OVERFLOW", 8: "SNP_E_STATE",
               9: "SNP_E_INTERNAL", 10: "SNP_E_CANCELLED"}

# Every symbol include/snp.h declares.
EXPORTS = ["snp_explore_opts_init", "snp_load_system", "snp_free", "snp_step", "snp_explore", "snp_reachable",
           "snp_parents", "snp_depth_stats", "snp_last_error", "snp_abi_version", "snp_explore_static",
           "snp_explore_resume", "snp_debug_fail_allocation", "snp_system_info", "snp_debug_hold_root_slot",
           "snp_tc_peak_tops", "snp_explore_batch", "snp_batch_autotune", "snp_server_create",
           "snp_server_submit", "snp_server_poll", "snp_server_wait", "snp_server_stats", "snp_server_destroy",
           "snp_row_width"]


class SnpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


class snp_system_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("R", ctypes.c_int32),
                ("rule_neuron", ctypes.c_void_p), ("rule_i", ctypes.c_void_p), ("rule_j", ctypes.c_void_p),
                ("M", ctypes.c_void_p), ("c0", ctypes.c_void_p),
                ("rule_terms", ctypes.c_void_p), ("term_i", ctypes.c_void_p), ("term_j", ctypes.c_void_p)]


class snp_explore_opts(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int32), ("transition", ctypes.c_int32),
                ("frontier_cap", ctypes.c_int64), ("candidate_budget", ctypes.c_int64),
                ("max_expand_value", ctypes.c_int32), ("record_parents", ctypes.c_int32),
                ("chunk", ctypes.c_int64), ("stream", ctypes.c_void_p), ("kernel_timing", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("warps", ctypes.c_int32), ("timeout_ms", ctypes.c_int32),
                ("cancel", ctypes.c_void_p), ("packed", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class snp_depth_info(ctypes.Structure):
    _fields_ = [("new_configs", ctypes.c_int64), ("parents", ctypes.c_int64), ("candidates", ctypes.c_uint64),
                ("examined", ctypes.c_int64), ("truncated", ctypes.c_int32), ("chunks", ctypes.c_int32),
                ("ms", ctypes.c_float), ("expand_ms", ctypes.c_float), ("expand_bytes", ctypes.c_int64),
                ("launches", ctypes.c_int64)]


class snp_server_info(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("active", ctypes.c_int64),
                ("pending", ctypes.c_int64), ("new_configs", ctypes.c_int64), ("ticks", ctypes.c_int64),
                ("busy_ms", ctypes.c_double), ("span_ms", ctypes.c_double), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libsnp_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1104_1824_gb300.build.build() "
                          "(the simulator has no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    lib.snp_explore_opts_init.argtypes = [ctypes.POINTER(snp_explore_opts)]
    lib.snp_explore_opts_init.restype = None
    lib.snp_load_system.argtypes = [ctypes.POINTER(snp_system_desc), ctypes.POINTER(vp)]
    lib.snp_free.argtypes = [vp]
    lib.snp_debug_hold_root_slot.argtypes = [i32]
    lib.snp_system_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.snp_step.argtypes = [vp, vp, i64, vp, ctypes.POINTER(u64)]
    lib.snp_explore.argtypes = [vp, ctypes.POINTER(snp_explore_opts), ctypes.POINTER(i32), vp]
    lib.snp_reachable.argtypes = [vp, vp, i64, ctypes.POINTER(i64), vp]
    lib.snp_parents.argtypes = [vp, vp, vp, i64, ctypes.POINTER(i64)]
    lib.snp_depth_stats.argtypes = [vp, i32, ctypes.POINTER(snp_depth_info)]
    lib.snp_row_width.argtypes = [vp, ctypes.POINTER(i32)]
    lib.snp_explore_resume.argtypes = [vp, vp, i64, ctypes.POINTER(snp_depth_info), i32,
                                       ctypes.POINTER(snp_explore_opts), ctypes.POINTER(i32), vp]
    lib.snp_debug_fail_allocation.argtypes = [i64]
    lib.snp_abi_version.argtypes = []
    lib.snp_explore_static.argtypes = [vp, ctypes.POINTER(snp_explore_opts), vp, i64, ctypes.POINTER(i64),
                                       ctypes.POINTER(i32), vp]
    lib.snp_tc_peak_tops.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
    lib.snp_explore_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(snp_explore_opts), vp]
    lib.snp_server_create.argtypes = [ctypes.c_size_t, i32, ctypes.POINTER(vp)]
    lib.snp_server_submit.argtypes = [vp, vp, ctypes.POINTER(snp_explore_opts), ctypes.POINTER(u64)]
    lib.snp_server_poll.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(i32)]
    lib.snp_server_wait.argtypes = [vp]
    lib.snp_server_stats.argtypes = [vp, ctypes.POINTER(snp_server_info)]
    lib.snp_server_destroy.argtypes = [vp]
    lib.snp_batch_autotune.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(snp_explore_opts),
                                       ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.snp_last_error.restype = ctypes.c_char_p
    lib.snp_last_error.argtypes = []
    lib.snp_abi_version.restype = ctypes.c_int
    for name in EXPORTS:
        if name not in ("snp_explore_opts_init", "snp_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code: int):
    if code != SNP_OK:
        raise SnpError(code, _lib.snp_last_error().decode())


def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return int(a.data_ptr())
    if isinstance(a, np.ndarray):
        return int(a.ctypes.data)
    return int(a)


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


# --- functions named as in the C ABI ------------------------------------------------------

def snp_abi_version() -> int:
    return load_library().snp_abi_version()


def snp_last_error() -> str:
    return load_library().snp_last_error().decode()


def snp_explore_opts_init() -> snp_explore_opts:
    o = snp_explore_opts()
    load_library().snp_explore_opts_init(ctypes.byref(o))
    return o


def snp_load_system(m, rule_neuron, rule_i, rule_j, M, c0, terms=None) -> ctypes.c_void_p:
    """terms: optional (rule_terms, term_i, term_j) arrays of general (union) rule expressions."""
    lib = load_library()
    arrs = [np.ascontiguousarray(x, dtype=np.int32).reshape(-1) for x in (rule_neuron, rule_i, rule_j, M, c0)]
    targs = [np.ascontiguousarray(x, dtype=np.int32).reshape(-1) for x in terms] if terms is not None else []
    d = snp_system_desc(int(m), int(arrs[0].shape[0]), *[a.ctypes.data for a in arrs],
                        *([a.ctypes.data for a in targs] if targs else [None, None, None]))
    h = ctypes.c_void_p()
    _check(lib.snp_load_system(ctypes.byref(d), ctypes.byref(h)))
    return h


def snp_free(h) -> None:
    load_library().snp_free(h)


def snp_step(h, C, capacity: int, out) -> int:
    psi = ctypes.c_uint64()
    _check(load_library().snp_step(h, _ptr(C), int(capacity), _ptr(out), ctypes.byref(psi)))
    return psi.value


def snp_explore(h, opts: snp_explore_opts, truncated_flags: Optional[np.ndarray] = None) -> int:
    dr = ctypes.c_int32()
    _check(load_library().snp_explore(h, ctypes.byref(opts), ctypes.byref(dr), _ptr(truncated_flags)))
    return dr.value


def snp_debug_fail_allocation(k: int) -> None:
    """Testing hook: the k-th device allocation from now on fails (k <= 0: off)."""
    _check(load_library().snp_debug_fail_allocation(ctypes.c_int64(int(k))))


def snp_debug_hold_root_slot(on: bool = True) -> None:
    """Testing hook: the next exploration leaves C0's table slot being claimed
    (a candidate equal to C0 then waits until the wait bound runs out)."""
    _check(load_library().snp_debug_hold_root_slot(ctypes.c_int32(1 if on else 0)))


def snp_explore_resume(h, rows: np.ndarray, stats, opts: snp_explore_opts,
                       truncated_flags: Optional[np.ndarray] = None) -> int:
    """rows: [n, m] int32 (host array or a torch device tensor); stats: a ctypes array of snp_depth_info."""
    dr = ctypes.c_int32()
    if hasattr(rows, "data_ptr"):
        ptr, n = rows.data_ptr(), int(rows.shape[0])
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        ptr, n = rows.ctypes.data, int(rows.shape[0])
    _check(load_library().snp_explore_resume(h, ctypes.c_void_p(ptr), ctypes.c_int64(n),
                                             ctypes.cast(stats, ctypes.POINTER(snp_depth_info)),
                                             ctypes.c_int32(len(stats)), ctypes.byref(opts), ctypes.byref(dr),
                                             _ptr(truncated_flags)))
    return dr.value


def snp_reachable(h, out, capacity: int, per_depth_new: Optional[np.ndarray] = None) -> int:
    n = ctypes.c_int64()
    _check(load_library().snp_reachable(h, _ptr(out), int(capacity), ctypes.byref(n), _ptr(per_depth_new)))
    return n.value


def snp_reachable_count(h) -> int:
    n = ctypes.c_int64()
    rc = load_library().snp_reachable(h, None, 0, ctypes.byref(n), None)
    if rc not in (SNP_OK, SNP_E_BUFFER):
        _check(rc)
    return n.value


def snp_parents(h, parent, index, capacity: int) -> int:
    n = ctypes.c_int64()
    _check(load_library().snp_parents(h, _ptr(parent), _ptr(index), int(capacity), ctypes.byref(n)))
    return n.value


def snp_system_info(h) -> Tuple[int, int, int]:
    """(m, R, device) of a loaded system."""
    m, r, dev = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().snp_system_info(h, ctypes.byref(m), ctypes.byref(r), ctypes.byref(dev)))
    return m.value, r.value, dev.value


def snp_system_m(h) -> int:
    return snp_system_info(h)[0]


def snp_system_device(h) -> int:
    return snp_system_info(h)[2]


def snp_explore_static(h, opts: snp_explore_opts, out, capacity: int,
                       per_depth_new: Optional[np.ndarray] = None) -> Tuple[int, int]:
    """Exploration into the caller's device buffer `out`, allocating nothing.
    Returns (configurations written, depth reached).  `out` must be a
    contiguous int32 device tensor on the handle's device with at least
    capacity * m entries; `per_depth_new`, if given, an int64 array of at least
    opts.depth + 1 entries."""
    m = snp_system_m(h)
    if not hasattr(out, "data_ptr") or not hasattr(out, "is_cuda") or not out.is_cuda:
        raise SnpError(SNP_E_INVALID, "out must be a device (CUDA) tensor")
    if str(out.dtype) != "torch.int32" or not out.is_contiguous():
        raise SnpError(SNP_E_INVALID, "out must be a contiguous int32 tensor")
    if int(capacity) < 0 or out.numel() < int(capacity) * m:
        raise SnpError(SNP_E_INVALID, f"out holds {out.numel()} entries, capacity * m needs {int(capacity) * m}")
    if out.device.index != snp_system_device(h):
        raise SnpError(SNP_E_INVALID, f"out is on device {out.device.index}, the system on {snp_system_device(h)}")
    if per_depth_new is not None:
        if not isinstance(per_depth_new, np.ndarray) or per_depth_new.dtype != np.int64 or \
                not per_depth_new.flags["C_CONTIGUOUS"] or per_depth_new.shape[0] < opts.depth + 1:
            raise SnpError(SNP_E_INVALID, "per_depth_new must be a contiguous int64 array of depth + 1 entries")
    n = ctypes.c_int64()
    dr = ctypes.c_int32()
    _check(load_library().snp_explore_static(h, ctypes.byref(opts), _ptr(out), int(capacity), ctypes.byref(n),
                                             ctypes.byref(dr), _ptr(per_depth_new)))
    return n.value, dr.value


def snp_tc_peak_tops(iters: int = 20000) -> float:
    """Measured int8 tensor-core rate (mma.sync m16n8k32) of the current device, TOPS."""
    v = ctypes.c_double()
    rc = load_library().snp_tc_peak_tops(int(iters), ctypes.byref(v))
    if rc != 0:
        raise SnpError(SNP_E_CUDA, f"snp_tc_peak_tops returned {rc}")
    return v.value


def _handle_array(handles):
    arr = (ctypes.c_void_p * len(handles))()
    for k, h in enumerate(handles):
        arr[k] = h.value if isinstance(h, ctypes.c_void_p) else h
    return arr


def snp_explore_batch(handles, opts: snp_explore_opts, statuses: Optional[np.ndarray] = None) -> None:
    """Explores the systems of `handles` together (one launch per depth)."""
    arr = _handle_array(handles)
    _check(load_library().snp_explore_batch(arr, len(handles), ctypes.byref(opts), _ptr(statuses)))


def snp_batch_autotune(handles, opts: snp_explore_opts) -> Tuple[int, int, int]:
    """(chunk, tile, warps) that run this batch fastest."""
    arr = _handle_array(handles)
    c, t, w = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().snp_batch_autotune(arr, len(handles), ctypes.byref(opts), ctypes.byref(c), ctypes.byref(t),
                                             ctypes.byref(w)))
    return c.value, t.value, w.value


def explore_batch(systems, depth: int, cap: int, budget: int = 0, max_expand: int = -1, chunk: int = 0,
                  tile: int = 0, warps: int = 0, stream=None, transition: int = SNP_T_SPARSE_I32) -> np.ndarray:
    """Convenience: snp_explore_batch over System objects; returns the statuses."""
    o = snp_explore_opts_init()
    o.transition = int(transition)
    o.depth, o.frontier_cap, o.candidate_budget, o.max_expand_value = int(depth), int(cap), int(budget), int(max_expand)
    o.chunk, o.tile, o.warps, o.stream = int(chunk), int(tile), int(warps), _stream_handle(stream)
    st = np.zeros(len(systems), dtype=np.int32)
    snp_explore_batch([s.h for s in systems], o, st)
    for s in systems:
        s.depth_reached = max(d for d, x in enumerate(s.depth_stats()) if x.new > 0)
    return st


def snp_server_create(hbm_budget: int, max_active: int):
    srv = ctypes.c_void_p()
    _check(load_library().snp_server_create(int(hbm_budget), int(max_active), ctypes.byref(srv)))
    return srv


def snp_server_submit(srv, h, opts: snp_explore_opts) -> int:
    rid = ctypes.c_uint64()
    _check(load_library().snp_server_submit(srv, h, ctypes.byref(opts), ctypes.byref(rid)))
    return rid.value


def snp_server_poll(srv, max_n: int = 4096):
    ids = np.zeros(max_n, dtype=np.uint64)
    lat = np.zeros(max_n, dtype=np.float64)
    sts = np.zeros(max_n, dtype=np.int32)
    n = ctypes.c_int32()
    _check(load_library().snp_server_poll(srv, _ptr(ids), _ptr(lat), _ptr(sts), int(max_n), ctypes.byref(n)))
    return ids[: n.value], lat[: n.value], sts[: n.value]


def snp_server_wait(srv) -> None:
    _check(load_library().snp_server_wait(srv))


def snp_server_stats(srv) -> snp_server_info:
    info = snp_server_info()
    _check(load_library().snp_server_stats(srv, ctypes.byref(info)))
    return info


def snp_server_destroy(srv) -> None:
    load_library().snp_server_destroy(srv)


def snp_depth_stats(h, d: int) -> snp_depth_info:
    info = snp_depth_info()
    _check(load_library().snp_depth_stats(h, int(d), ctypes.byref(info)))
    return info


def snp_row_width(h) -> int:
    """Bytes per spike count of the last exploration's store (1, 2 or 4)."""
    w = ctypes.c_int32()
    _check(load_library().snp_row_width(h, ctypes.byref(w)))
    return int(w.value)


# --- convenience wrapper ------------------------------------------------------------------

@dataclass
class DepthStats:
    new: int
    parents: int
    candidates: int
    examined: int
    truncated: int
    chunks: int
    ms: float
    expand_ms: float
    expand_bytes: int
    launches: int


class System:
    """One loaded system (owns a library handle)."""

    def __init__(self, system):
        self.m = int(system.m)
        self.R = int(system.R)
        self.h = snp_load_system(self.m, system.rule_neuron, system.rule_i, system.rule_j, system.M, system.c0,
                                 terms=system.term_arrays() if getattr(system, "terms", None) is not None else None)
        self.depth_reached = None

    def close(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            snp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, C, capacity: Optional[int] = None) -> Tuple[np.ndarray, int]:
        C = np.ascontiguousarray(C, dtype=np.int32)
        if capacity is None:
            psi = snp_step(self.h, C, 0, None)
            capacity = min(psi, 1 << 22)
        out = np.zeros((max(int(capacity), 1), self.m), dtype=np.int32)
        psi = snp_step(self.h, C, int(capacity), out)
        return out[: min(psi, int(capacity))], psi

    def explore(self, depth: int, cap: int = 0, budget: int = 0, transition: int = SNP_T_SPARSE_I32,
                max_expand: int = -1, record_parents: bool = False, chunk: int = 0, stream=None,
                kernel_timing: bool = False, timeout_ms: int = 0, cancel=None, packed: bool = False) -> int:
        """cancel: a host int32 array of one element, polled between passes;
        packed: store counts in 1 or 2 bytes where the bound allows
        (row_width() tells which)."""
        o = snp_explore_opts_init()
        o.packed = 1 if packed else 0
        o.timeout_ms = int(timeout_ms)
        o.cancel = _ptr(cancel) or None
        o.depth = int(depth)
        o.transition = int(transition)
        o.frontier_cap = int(cap)
        o.candidate_budget = int(budget)
        o.max_expand_value = int(max_expand)
        o.record_parents = 1 if record_parents else 0
        o.chunk = int(chunk)
        o.stream = _stream_handle(stream)
        o.kernel_timing = 1 if kernel_timing else 0
        self.truncated = np.zeros(int(depth) + 1, dtype=np.int32)
        self.depth_reached = snp_explore(self.h, o, self.truncated)
        return self.depth_reached

    def checkpoint(self) -> Tuple[np.ndarray, np.ndarray]:
        """State at the last depth boundary: (rows [n, m] in discovery order,
        per-depth records as raw bytes) -- what resume() takes back; both can
        be written to disk as they are."""
        rows = self.reachable()
        infos = []
        d = 0
        while True:
            info = snp_depth_info()
            if load_library().snp_depth_stats(self.h, d, ctypes.byref(info)) != SNP_OK:
                break
            infos.append(info)
            d += 1
        arr = (snp_depth_info * len(infos))(*infos)
        return rows, np.frombuffer(bytes(arr), dtype=np.uint8).copy()

    def resume(self, checkpoint, depth: int, cap: int = 0, budget: int = 0, transition: int = SNP_T_SPARSE_I32,
               max_expand: int = -1, chunk: int = 0, stream=None, packed: bool = False) -> int:
        """Continues the exploration a checkpoint() was taken from up to `depth`."""
        rows, raw = checkpoint
        raw = np.ascontiguousarray(raw, dtype=np.uint8)
        k = raw.nbytes // ctypes.sizeof(snp_depth_info)
        stats = (snp_depth_info * k).from_buffer_copy(raw.tobytes())
        o = snp_explore_opts_init()
        o.depth, o.transition, o.frontier_cap, o.candidate_budget = int(depth), int(transition), int(cap), int(budget)
        o.max_expand_value, o.chunk, o.stream = int(max_expand), int(chunk), _stream_handle(stream)
        o.packed = 1 if packed else 0
        self.truncated = np.zeros(int(depth) + 1, dtype=np.int32)
        self.depth_reached = snp_explore_resume(self.h, rows, stats, o, self.truncated)
        return self.depth_reached

    def count(self) -> int:
        return snp_reachable_count(self.h)

    def row_width(self) -> int:
        """Bytes per spike count of the last exploration's store (1, 2 or 4)."""
        return snp_row_width(self.h)

    def reachable(self) -> np.ndarray:
        n = self.count()
        out = np.zeros((n, self.m), dtype=np.int32)
        snp_reachable(self.h, out, n)
        return out

    def per_depth_new(self) -> List[int]:
        pdn = np.zeros(self.depth_reached + 1, dtype=np.int64)
        n = ctypes.c_int64()
        rc = load_library().snp_reachable(self.h, None, 0, ctypes.byref(n), _ptr(pdn))
        if rc not in (SNP_OK, SNP_E_BUFFER):
            _check(rc)
        return [int(x) for x in pdn]

    def depth_stats(self) -> List[DepthStats]:
        out = []
        d = 0
        while True:
            info = snp_depth_info()
            if load_library().snp_depth_stats(self.h, d, ctypes.byref(info)) != SNP_OK:
                break
            out.append(DepthStats(info.new_configs, info.parents, info.candidates, info.examined, info.truncated,
                                  info.chunks, info.ms, info.expand_ms, info.expand_bytes, info.launches))
            d += 1
        return out

    def parents(self) -> Tuple[np.ndarray, np.ndarray]:
        n = self.count()
        par = np.zeros(n, dtype=np.int64)
        idx = np.zeros(n, dtype=np.uint64)
        snp_parents(self.h, par, idx, n)
        return par, idx

