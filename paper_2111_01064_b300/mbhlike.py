"""ctypes binding of libmbhlike (include/mbhlike.h), argument marshalling only.

Every compute step runs in the library's CUDA kernels; this module turns torch
tensors into device pointers and the current torch stream into a cudaStream_t.
There is no CPU fallback: a missing library or device raises MBHError.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Sequence

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmbhlike.so")
DEBUG_LIB_PATH = os.path.join(HERE, "libmbhlike_debug.so")

FP64, MIXED, MIXED_F32 = 0, 1, 2
_PREC = {"fp64": FP64, "mixed": MIXED, "mixed_f32": MIXED_F32, FP64: FP64, MIXED: MIXED,
         MIXED_F32: MIXED_F32}
STATUS = {0: "MBH_OK", 1: "MBH_EINVAL", 2: "MBH_ENOMEM", 3: "MBH_ECUDA", 4: "MBH_ETIMEOUT",
          5: "MBH_EBUSY"}


class MBHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("f0", C.c_double), ("df", C.c_double), ("n", C.c_int64), ("t_obs", C.c_double)]


class HetConfig(C.Structure):
    """mbh_het_config: threads per walker (1..32), block (0 = the kernel's default, or a
    multiple of 32 up to 256 for which a kernel exists), persistent (0/1)."""
    _fields_ = [("threads_per_walker", C.c_int32), ("block", C.c_int32), ("persistent", C.c_int32)]

    def as_dict(self) -> dict:
        return dict(threads_per_walker=self.threads_per_walker, block=self.block,
                    persistent=self.persistent)


def het_config(threads_per_walker=8, block=0, persistent=0) -> HetConfig:
    return HetConfig(int(threads_per_walker), int(block), int(persistent))


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_batch_walkers", C.c_int32),
                ("max_inflight_batches", C.c_int32), ("max_queue", C.c_int32),
                ("precision", C.c_int), ("config", HetConfig)]


class ServerReport(C.Structure):
    _fields_ = [("completed", C.c_int64), ("walkers", C.c_int64), ("batches", C.c_int64),
                ("rejected", C.c_int64), ("queued", C.c_int64), ("mean_batch_walkers", C.c_double),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("walkers_per_s", C.c_double), ("source_bytes", C.c_int64), ("slot_bytes", C.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class PTOpts(C.Structure):
    """mbh_pt_opts (see include/mbhlike.h)."""
    _fields_ = [("ntemps", C.c_int32), ("walkers", C.c_int32), ("a", C.c_double),
                ("probs", C.c_double * 4), ("lo", C.c_double * 11), ("hi", C.c_double * 11),
                ("seed", C.c_uint64), ("precision", C.c_int), ("het_config", HetConfig),
                ("modes", C.c_uint32), ("adapt_time", C.c_double), ("adapt_lag", C.c_double),
                ("no_fuse", C.c_int32)]


class LoadgenOpts(C.Structure):
    _fields_ = [("rate_per_s", C.c_double), ("seconds", C.c_double), ("min_walkers", C.c_int32),
                ("max_walkers", C.c_int32), ("seed", C.c_uint64)]


class LoadgenReport(C.Structure):
    _fields_ = [("offered_per_s", C.c_double), ("submitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("failed", C.c_int64), ("wall_seconds", C.c_double),
                ("completed_per_s", C.c_double), ("walkers_per_s", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("max_ms", C.c_double), ("batches", C.c_int64),
                ("mean_batch_walkers", C.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class DeviceStatus(C.Structure):
    _fields_ = [("code", C.c_int32), ("kernel", C.c_int32), ("source", C.c_int32), ("reserved", C.c_int32),
                ("index", C.c_int64), ("limit", C.c_int64)]


def grid_struct(g: dict) -> Grid:
    return Grid(float(g["f0"]), float(g["df"]), int(g["n"]), float(g["t_obs"]))


_lib = None
vp, dp, i64, i32 = C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.c_int32


def lib() -> C.CDLL:
    """Load libmbhlike.so (built in-tree by paper_2111_01064_b300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    # MBH_DEBUG_CHECKS=1 selects the debug build (in-kernel index checks, see mbh_sync_status)
    path = DEBUG_LIB_PATH if os.environ.get("MBH_DEBUG_CHECKS") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise MBHError(3, f"{path} not built: run `python -m paper_2111_01064_b300.build`"
                          f"{' --debug' if path == DEBUG_LIB_PATH else ''}")
    L = C.CDLL(path)
    gp = C.POINTER(Grid)
    sigs = {
        "mbh_last_error": (C.c_char_p, []),
        "mbh_psd_aet": (C.c_int, [gp, vp, vp]),
        "mbh_noise_aet": (C.c_int, [gp, vp, vp, i32, vp, vp]),
        "template_batch": (C.c_int, [gp, vp, i64, C.c_int, vp, vp]),
        "mbh_data_create": (C.c_int, [gp, vp, vp, vp, C.POINTER(vp)]),
        "mbh_data_dd": (C.c_double, [vp]),
        "mbh_data_free": (None, [vp]),
        "direct_loglike_batch": (C.c_int, [vp, vp, i64, C.c_int, vp, vp]),
        "direct_loglike_stored": (C.c_int, [vp, vp, i64, C.c_int, vp, vp]),
        "direct_loglike_stored_noalloc": (C.c_int, [vp, vp, i64, C.c_int, vp, vp]),
        "het_prepare_reference": (C.c_int, [vp, dp, i32, vp, C.POINTER(vp)]),
        "mbh_ref_bins": (i32, [vp]),
        "mbh_ref_read": (C.c_int, [vp, C.POINTER(C.c_int64), dp, dp, dp]),
        "mbh_ref_free": (None, [vp]),
        "het_loglike_batch": (C.c_int, [C.POINTER(vp), C.POINTER(C.c_int64), i32, vp, C.c_int, vp,
                                        vp]),
        "het_loglike_batch_cfg": (C.c_int, [C.POINTER(vp), C.POINTER(C.c_int64), i32, vp, C.c_int,
                                            C.POINTER(HetConfig), vp, vp]),
        "mbh_het_autotune": (C.c_int, [C.POINTER(vp), C.POINTER(C.c_int64), i32, vp, C.c_int, vp, i32,
                                       vp, C.POINTER(HetConfig), C.POINTER(C.c_double)]),
        "mbh_het_graph_create": (C.c_int, [C.POINTER(vp), C.POINTER(C.c_int64), i32, vp, C.c_int,
                                           C.POINTER(HetConfig), vp, vp, C.POINTER(vp)]),
        "mbh_het_graph_launch": (C.c_int, [vp, vp]),
        "mbh_het_graph_free": (None, [vp]),
        "mbh_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(vp)]),
        "mbh_server_add_source": (C.c_int, [vp, vp, C.POINTER(C.c_int32)]),
        "mbh_server_remove_source": (C.c_int, [vp, i32]),
        "mbh_server_replace_source": (C.c_int, [vp, i32, vp]),
        "mbh_server_submit": (C.c_int, [vp, i32, vp, i64, vp, C.POINTER(C.c_uint64)]),
        "mbh_server_wait": (C.c_int, [vp, C.c_uint64, i32, C.POINTER(C.c_int)]),
        "mbh_server_cancel": (C.c_int, [vp, C.c_uint64]),
        "mbh_server_pause": (C.c_int, [vp, i32]),
        "mbh_server_stats": (C.c_int, [vp, C.POINTER(ServerReport)]),
        "mbh_server_reset_stats": (C.c_int, [vp]),
        "mbh_server_free": (None, [vp]),
        "mbh_selftest_math": (C.c_int, [i32, vp, vp, i64, vp, vp, vp]),
        "mbh_ref_modes": (C.c_uint32, [vp]),
        "mbh_ref_f32_edges": (i32, [vp]),
        "template_batch_hm": (C.c_int, [gp, vp, i64, C.c_uint32, C.c_int, vp, vp]),
        "direct_loglike_batch_hm": (C.c_int, [vp, vp, i64, C.c_uint32, C.c_int, vp, vp]),
        "het_prepare_reference_hm": (C.c_int, [vp, dp, i32, C.c_uint32, vp, C.POINTER(vp)]),
        "mbh_pt_create": (C.c_int, [C.POINTER(PTOpts), vp, vp, dp, vp, vp, C.POINTER(vp)]),
        "mbh_pt_create_multi": (C.c_int, [C.POINTER(PTOpts), C.POINTER(vp), i32, vp, dp, vp, vp,
                                          C.POINTER(vp)]),
        "mbh_pt_set_ref_at": (C.c_int, [vp, i32, vp, vp]),
        "mbh_pt_best_at": (C.c_int, [vp, i32, i32, dp, dp, vp]),
        "mbh_server_loadgen": (C.c_int, [vp, C.POINTER(C.c_int32), i32, C.POINTER(dp), i64,
                                         C.POINTER(LoadgenOpts), C.POINTER(LoadgenReport)]),
        "mbh_pt_run": (C.c_int, [vp, i64, i32, vp]),
        "mbh_pt_state": (C.c_int, [vp, vp, vp, vp]),
        "mbh_pt_set_state": (C.c_int, [vp, vp, vp]),
        "mbh_pt_set_ref": (C.c_int, [vp, vp, vp]),
        "mbh_pt_set_betas": (C.c_int, [vp, dp, vp]),
        "mbh_pt_get_betas": (C.c_int, [vp, dp, vp]),
        "mbh_pt_counters": (C.c_int, [vp, C.POINTER(C.c_int64), C.POINTER(C.c_uint64), vp]),
        "mbh_pt_best": (C.c_int, [vp, i32, dp, dp, vp]),
        "mbh_pt_free": (None, [vp]),
        "mbh_sync_status": (C.c_int, [vp, C.POINTER(DeviceStatus)]),
        "mbh_debug_checks": (i32, []),
        "mbh_debug_ref_limit": (C.c_int, [vp, i32]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise MBHError(status, lib().mbh_last_error().decode())


def _require_cuda():
    if not torch.cuda.is_available():
        raise MBHError(3, "no CUDA device: the mbhlike kernels have no CPU fallback")


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: torch.Tensor, dtype, shape=None, name="tensor") -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise MBHError(1, f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise MBHError(1, f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise MBHError(1, f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise MBHError(1, f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t.data_ptr()


def _prec(p) -> int:
    try:
        return _PREC[p]
    except KeyError:
        raise MBHError(1, f"unknown precision {p!r}") from None


# ---- PSD, noise, templates ----------------------------------------------------------
def mbh_psd_aet(grid: dict, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    _require_cuda()
    if out is None:
        out = torch.empty((3, int(grid["n"])), dtype=torch.float64, device="cuda")
    g = grid_struct(grid)
    _check(lib().mbh_psd_aet(C.byref(g), _dev(out, torch.float64, (3, g.n), "out"), _stream(stream)))
    return out


def mbh_noise_aet(grid: dict, z: torch.Tensor, psd: torch.Tensor, out: torch.Tensor | None = None,
                  accumulate: bool = False, stream=None) -> torch.Tensor:
    _require_cuda()
    n = int(grid["n"])
    if out is None:
        out = torch.zeros((3, n), dtype=torch.complex128, device="cuda")
    g = grid_struct(grid)
    _check(lib().mbh_noise_aet(C.byref(g), _dev(z, torch.float64, (3, n, 2), "z"),
                               _dev(psd, torch.float64, (3, n), "psd"), 1 if accumulate else 0,
                               _dev(out, torch.complex128, (3, n), "out"), _stream(stream)))
    return out


def template_batch(grid: dict, theta: torch.Tensor, precision="fp64", out: torch.Tensor | None = None,
                   stream=None, modes: int = 1) -> torch.Tensor:
    """Templates (W, 3, n) on the grid; `modes` selects harmonic modes (1 = the (2,2) mode)."""
    _require_cuda()
    p = _prec(precision)
    W = theta.shape[1]
    n = int(grid["n"])
    dt = torch.complex128 if p == FP64 else torch.complex64
    if out is None:
        out = torch.empty((W, 3, n), dtype=dt, device="cuda")
    g = grid_struct(grid)
    _check(lib().template_batch_hm(C.byref(g), _dev(theta, torch.float64, (11, W), "theta"), W,
                                   int(modes), p, _dev(out, dt, (W, 3, n), "out"), _stream(stream)))
    return out


# ---- data and the direct likelihood ----------------------------------------------------
class Data:
    """mbh_data handle: the data d (3, n) complex128 and PSD (3, n) on one grid."""

    def __init__(self, grid: dict, d: torch.Tensor, psd: torch.Tensor, stream=None):
        _require_cuda()
        self.grid = dict(grid)
        n = int(grid["n"])
        h = vp()
        g = grid_struct(grid)
        _check(lib().mbh_data_create(C.byref(g), _dev(d, torch.complex128, (3, n), "d"),
                                     _dev(psd, torch.float64, (3, n), "psd"), _stream(stream),
                                     C.byref(h)))
        self.handle = h

    @property
    def dd(self) -> float:
        return lib().mbh_data_dd(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            lib().mbh_data_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mbh_data_create(grid: dict, d: torch.Tensor, psd: torch.Tensor, stream=None) -> Data:
    return Data(grid, d, psd, stream)


def direct_loglike_batch(data: Data, theta: torch.Tensor, precision="fp64",
                         out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    W = theta.shape[1]
    if out is None:
        out = torch.empty((3, W), dtype=torch.float64, device="cuda")
    _check(lib().direct_loglike_batch(data.handle, _dev(theta, torch.float64, (11, W), "theta"), W,
                                      _prec(precision), _dev(out, torch.float64, (3, W), "out"),
                                      _stream(stream)))
    return out


def direct_loglike_batch_hm(data: Data, theta: torch.Tensor, modes: int, precision="fp64",
                            out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Direct likelihood of templates summed over the harmonic modes of the mask."""
    W = theta.shape[1]
    if out is None:
        out = torch.empty((3, W), dtype=torch.float64, device="cuda")
    _check(lib().direct_loglike_batch_hm(data.handle, _dev(theta, torch.float64, (11, W), "theta"), W,
                                         int(modes), _prec(precision),
                                         _dev(out, torch.float64, (3, W), "out"), _stream(stream)))
    return out


def direct_loglike_stored(data: Data, h: torch.Tensor, precision="fp64",
                          out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    p = _prec(precision)
    W = h.shape[0]
    dt = torch.complex128 if p == FP64 else torch.complex64
    if out is None:
        out = torch.empty((3, W), dtype=torch.float64, device="cuda")
    _check(lib().direct_loglike_stored(data.handle, _dev(h, dt, (W, 3, data.grid["n"]), "h"), W, p,
                                       _dev(out, torch.float64, (3, W), "out"), _stream(stream)))
    return out


def direct_loglike_stored_noalloc(data: Data, h: torch.Tensor, precision="fp64", *,
                                  out: torch.Tensor, stream=None) -> torch.Tensor:
    """direct_loglike_stored for callers that cannot allocate device memory: the C
    call allocates nothing (static 8 MiB scratch shared by all calls on a device, so
    calls must not overlap on the GPU); `out` must be preallocated by the caller."""
    p = _prec(precision)
    W = h.shape[0]
    dt = torch.complex128 if p == FP64 else torch.complex64
    _check(lib().direct_loglike_stored_noalloc(data.handle, _dev(h, dt, (W, 3, data.grid["n"]), "h"),
                                               W, p, _dev(out, torch.float64, (3, W), "out"),
                                               _stream(stream)))
    return out


# ---- heterodyne ---------------------------------------------------------------------------
class Ref:
    """mbh_ref handle: one heterodyne reference (summary data resident on the device)."""

    def __init__(self, data: Data, theta0, n_bins: int, stream=None, modes: int = 1):
        th = np.ascontiguousarray(np.asarray(theta0, dtype=np.float64).reshape(11))
        h = vp()
        _check(lib().het_prepare_reference_hm(data.handle, th.ctypes.data_as(dp), int(n_bins),
                                              int(modes), _stream(stream), C.byref(h)))
        self.handle = h
        self.grid = dict(data.grid)
        self.theta0 = th.copy()

    @property
    def bins(self) -> int:
        return int(lib().mbh_ref_bins(self.handle))

    @property
    def modes(self) -> int:
        return int(lib().mbh_ref_modes(self.handle))

    @property
    def f32_edges(self) -> int:
        """Edges that MBH_MIXED evaluates with the float32 ratio (per-edge precision)."""
        return int(lib().mbh_ref_f32_edges(self.handle))

    def read(self) -> dict:
        E = self.bins
        edges = np.empty(E + 1, dtype=np.int64)
        summ = np.empty((E, 3, 6))
        h0e = np.empty((E + 1, 3), dtype=np.complex128)
        dd = np.empty(1)
        _check(lib().mbh_ref_read(self.handle, edges.ctypes.data_as(C.POINTER(C.c_int64)),
                                  summ.ctypes.data_as(dp), h0e.view(np.float64).ctypes.data_as(dp),
                                  dd.ctypes.data_as(dp)))
        return dict(E=E, edges=edges, summary=summ, h0e=h0e, dd=float(dd[0]))

    def close(self):
        if getattr(self, "handle", None):
            lib().mbh_ref_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def het_prepare_reference(data: Data, theta0, n_bins: int, stream=None, modes: int = 1) -> Ref:
    return Ref(data, theta0, n_bins, stream, modes)


def het_loglike_batch(refs: Sequence[Ref], offsets, theta: torch.Tensor, precision="mixed",
                      out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Walkers offsets[s]..offsets[s+1] of theta (11, W) use refs[s]."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    ns = len(refs)
    if off.shape != (ns + 1,):
        raise MBHError(1, f"offsets must have {ns + 1} entries")
    W = int(off[-1])
    if out is None:
        out = torch.empty((3, W), dtype=torch.float64, device="cuda")
    arr = (vp * max(ns, 1))(*[r.handle for r in refs])
    _check(lib().het_loglike_batch(arr, off.ctypes.data_as(C.POINTER(C.c_int64)), ns,
                                   _dev(theta, torch.float64, (11, W), "theta"), _prec(precision),
                                   _dev(out, torch.float64, (3, W), "out"), _stream(stream)))
    return out


def _het_args(refs, offsets, theta):
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    ns = len(refs)
    if off.shape != (ns + 1,):
        raise MBHError(1, f"offsets must have {ns + 1} entries")
    W = int(off[-1])
    arr = (vp * max(ns, 1))(*[r.handle for r in refs])
    return off, ns, W, arr


def het_loglike_batch_cfg(refs: Sequence[Ref], offsets, theta: torch.Tensor, precision="mixed",
                          cfg: HetConfig | None = None, out: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
    off, ns, W, arr = _het_args(refs, offsets, theta)
    if out is None:
        out = torch.empty((3, W), dtype=torch.float64, device="cuda")
    _check(lib().het_loglike_batch_cfg(arr, off.ctypes.data_as(C.POINTER(C.c_int64)), ns,
                                       _dev(theta, torch.float64, (11, W), "theta"), _prec(precision),
                                       C.byref(cfg) if cfg is not None else None,
                                       _dev(out, torch.float64, (3, W), "out"), _stream(stream)))
    return out


def mbh_het_autotune(refs: Sequence[Ref], offsets, theta: torch.Tensor, precision="mixed",
                     reps: int = 3, out: torch.Tensor | None = None, stream=None):
    """Fastest launch configuration for this batch: (HetConfig, ms per batch)."""
    off, ns, W, arr = _het_args(refs, offsets, theta)
    if out is None:
        out = torch.empty((3, W), dtype=torch.float64, device="cuda")
    best = HetConfig()
    ms = C.c_double()
    _check(lib().mbh_het_autotune(arr, off.ctypes.data_as(C.POINTER(C.c_int64)), ns,
                                  _dev(theta, torch.float64, (11, W), "theta"), _prec(precision),
                                  _dev(out, torch.float64, (3, W), "out"), int(reps), _stream(stream),
                                  C.byref(best), C.byref(ms)))
    return best, ms.value


class HetGraph:
    """A heterodyne batch captured in a CUDA graph: theta and out are fixed buffers; rewrite
    theta in place and call launch() for each evaluation."""

    def __init__(self, refs: Sequence[Ref], offsets, theta: torch.Tensor, out: torch.Tensor,
                 precision="mixed", cfg: HetConfig | None = None, stream=None):
        off, ns, W, arr = _het_args(refs, offsets, theta)
        self.refs, self.theta, self.out = list(refs), theta, out   # keep them alive
        h = vp()
        _check(lib().mbh_het_graph_create(arr, off.ctypes.data_as(C.POINTER(C.c_int64)), ns,
                                          _dev(theta, torch.float64, (11, W), "theta"), _prec(precision),
                                          C.byref(cfg) if cfg is not None else None,
                                          _dev(out, torch.float64, (3, W), "out"), _stream(stream),
                                          C.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        _check(lib().mbh_het_graph_launch(self.handle, _stream(stream)))
        return self.out

    def close(self):
        if getattr(self, "handle", None):
            lib().mbh_het_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """mbh_server: continuous batching of heterodyne requests (see include/mbhlike.h)."""

    def __init__(self, hbm_budget_bytes: int, max_batch_walkers: int = 16384, max_inflight_batches: int = 3,
                 max_queue: int = 4096, precision="mixed", cfg: HetConfig | None = None):
        _require_cuda()
        opts = ServerOpts(int(hbm_budget_bytes), int(max_batch_walkers), int(max_inflight_batches),
                          int(max_queue), _prec(precision), cfg if cfg is not None else HetConfig(0, 0, 0))
        h = vp()
        _check(lib().mbh_server_create(C.byref(opts), C.byref(h)))
        self.handle = h
        self.refs = {}
        self._out = {}

    def add_source(self, ref: Ref) -> int:
        sid = C.c_int32()
        _check(lib().mbh_server_add_source(self.handle, ref.handle, C.byref(sid)))
        self.refs[sid.value] = ref
        return sid.value

    def remove_source(self, sid: int):
        _check(lib().mbh_server_remove_source(self.handle, int(sid)))
        self.refs.pop(sid, None)

    def replace_source(self, sid: int, ref: Ref):
        """Hot swap of a source's reference (reference refresh); the previous Ref may be
        freed once this returns."""
        _check(lib().mbh_server_replace_source(self.handle, int(sid), ref.handle))
        self.refs[sid] = ref

    def submit(self, sid: int, theta: np.ndarray) -> int:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        W = th.shape[1]
        out = np.empty((3, W))
        rid = C.c_uint64()
        _check(lib().mbh_server_submit(self.handle, int(sid), th.ctypes.data, W, out.ctypes.data,
                                       C.byref(rid)))
        self._out[rid.value] = out
        return rid.value

    def wait(self, rid: int, timeout_ms: int = -1) -> tuple[int, np.ndarray]:
        """(request status, results (3, W)); raises MBHError(MBH_ETIMEOUT) on timeout."""
        st = C.c_int()
        _check(lib().mbh_server_wait(self.handle, C.c_uint64(rid), int(timeout_ms), C.byref(st)))
        return st.value, self._out.pop(rid)

    def cancel(self, rid: int):
        _check(lib().mbh_server_cancel(self.handle, C.c_uint64(rid)))

    def pause(self, paused: bool = True):
        _check(lib().mbh_server_pause(self.handle, 1 if paused else 0))

    def stats(self) -> dict:
        r = ServerReport()
        _check(lib().mbh_server_stats(self.handle, C.byref(r)))
        return r.as_dict()

    def loadgen(self, source_ids, pools, rate_per_s: float, seconds: float, min_walkers: int = 64,
                max_walkers: int = 4096, seed: int = 0) -> dict:
        """Native load generator (one C++ client thread per source, Poisson arrivals, open
        loop); pools: one float64 (11, P) host array per client."""
        n = len(source_ids)
        pools = [np.ascontiguousarray(np.asarray(p, dtype=np.float64)) for p in pools]
        P = pools[0].shape[1]
        if any(p.shape != (11, P) for p in pools):
            raise MBHError(1, "pools must all be (11, P)")
        ids = (C.c_int32 * n)(*[int(i) for i in source_ids])
        ptrs = (dp * n)(*[p.ctypes.data_as(dp) for p in pools])
        o = LoadgenOpts(float(rate_per_s), float(seconds), int(min_walkers), int(max_walkers), int(seed))
        rep = LoadgenReport()
        _check(lib().mbh_server_loadgen(self.handle, ids, n, ptrs, P, C.byref(o), C.byref(rep)))
        return rep.as_dict()

    def reset_stats(self):
        _check(lib().mbh_server_reset_stats(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().mbh_server_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mbh_selftest_math(kind: int, x: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    """Library float32 device math on x (and y): kind 0 -> (sin, cos), 1 -> sinc,
    2 -> sinc(x(1+y)) - sinc(x(1-y)); 3, 4: the four-term forms of 1 and 2 (small x).
    Double-float math, x as (hi, lo) pairs of shape (n, 2): kind 5 -> (sin, cos - 1) as pairs;
    kind 6 -> x y mod 2 pi as pairs, y of shape (n, 3) (triple-floats)."""
    n = x.numel() // 2 if kind >= 5 else x.numel()
    o1 = torch.empty_like(x)
    o2 = torch.empty_like(x) if kind in (0, 5) else None
    _check(lib().mbh_selftest_math(int(kind), _dev(x, torch.float32, None, "x"),
                                   _dev(y, torch.float32, None, "y") if y is not None else None, n,
                                   _dev(o1, torch.float32, None, "o1"),
                                   _dev(o2, torch.float32, None, "o2") if o2 is not None else None,
                                   _stream(stream)))
    return (o1, o2) if kind in (0, 5) else o1


class PTSampler:
    """mbh_pt: parallel-tempered ensemble sampler iterations on the device (Sec. III).

    One of ``ref`` (heterodyned likelihood), ``refs`` (one ensemble per reference, stepping
    together) and ``data`` (direct likelihood; ``n_ens`` independent ensembles of it).
    ``x``: CUDA float64 (11, n_ens*T*W) start positions in the sampler coordinates
    (ln M_T, q, a1, a2, D_L, phi_ref, cos iota, lambda, sin beta, psi, t_ref); ``betas``: (T,)
    for every ensemble or (n_ens, T)."""

    def __init__(self, x: torch.Tensor, betas, lo, hi, *, ref: Ref | None = None,
                 refs: Sequence[Ref] | None = None, data: Data | None = None, n_ens: int = 1,
                 walkers: int, a: float = 2.0, probs=(0.85, 0.04, 0.03, 0.08), seed: int = 0,
                 precision="mixed", cfg: HetConfig | None = None, modes: int = 1, adapt=None,
                 fuse: bool = True, stream=None):
        _require_cuda()
        if ref is not None:
            refs = [ref]
        if refs is not None:
            n_ens = len(refs)
        betas = np.asarray(betas, dtype=np.float64)
        T = betas.shape[-1]
        betas = np.ascontiguousarray(np.broadcast_to(betas, (n_ens, T)))
        o = PTOpts()
        o.ntemps, o.walkers, o.a = T, int(walkers), float(a)
        o.probs[:] = [float(p) for p in probs]
        o.lo[:] = [float(v) for v in lo]
        o.hi[:] = [float(v) for v in hi]
        o.seed, o.precision = int(seed), _prec(precision)
        o.het_config = cfg if cfg is not None else HetConfig(0, 0, 0)
        o.modes = int(modes)
        if adapt is not None:   # (nu, n0): ladder adaptation
            o.adapt_time, o.adapt_lag = float(adapt[0]), float(adapt[1])
        o.no_fuse = 0 if fuse else 1
        self.T, self.W, self.n_ens = T, int(walkers), int(n_ens)
        self.refs, self.data = (list(refs) if refs is not None else None), data   # keep them alive
        arr = (vp * n_ens)(*[r.handle for r in refs]) if refs is not None else None
        h = vp()
        _check(lib().mbh_pt_create_multi(C.byref(o), arr, n_ens, data.handle if data else None,
                                         betas.ctypes.data_as(dp),
                                         _dev(x, torch.float64, (11, n_ens * T * self.W), "x"),
                                         _stream(stream), C.byref(h)))
        self.handle = h

    def run(self, n_iter: int, graph: bool = True, stream=None):
        _check(lib().mbh_pt_run(self.handle, int(n_iter), 1 if graph else 0, _stream(stream)))

    def state(self, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        N = self.n_ens * self.T * self.W
        x = torch.empty((11, N), dtype=torch.float64, device="cuda")
        out = torch.empty((3, N), dtype=torch.float64, device="cuda")
        _check(lib().mbh_pt_state(self.handle, x.data_ptr(), out.data_ptr(), _stream(stream)))
        return x, out

    def set_state(self, x: torch.Tensor, stream=None):
        _check(lib().mbh_pt_set_state(self.handle,
                                      _dev(x, torch.float64, (11, self.n_ens * self.T * self.W), "x"),
                                      _stream(stream)))

    def set_ref(self, ref: Ref, ensemble: int = 0, stream=None):
        _check(lib().mbh_pt_set_ref_at(self.handle, int(ensemble), ref.handle, _stream(stream)))
        self.refs[ensemble] = ref

    def set_betas(self, betas, stream=None):
        b = np.ascontiguousarray(np.broadcast_to(np.asarray(betas, dtype=np.float64),
                                                 (self.n_ens, self.T)))
        _check(lib().mbh_pt_set_betas(self.handle, b.ctypes.data_as(dp), _stream(stream)))

    def betas(self, stream=None) -> np.ndarray:
        """(T,) for one ensemble, (n_ens, T) otherwise."""
        b = np.zeros((self.n_ens, self.T))
        _check(lib().mbh_pt_get_betas(self.handle, b.ctypes.data_as(dp), _stream(stream)))
        return b[0] if self.n_ens == 1 else b

    def counters(self, stream=None) -> tuple[np.ndarray, int]:
        """int64 [n_ens * 10 T] (see include/mbhlike.h) and the iteration counter."""
        c = np.zeros(10 * self.n_ens * self.T, dtype=np.int64)
        step = C.c_uint64(0)
        _check(lib().mbh_pt_counters(self.handle, c.ctypes.data_as(C.POINTER(C.c_int64)),
                                     C.byref(step), _stream(stream)))
        return c, int(step.value)

    def best(self, temp: int = 0, ensemble: int = 0, stream=None) -> tuple[np.ndarray, np.ndarray]:
        x, o = np.zeros(11), np.zeros(3)
        _check(lib().mbh_pt_best_at(self.handle, int(ensemble), int(temp), x.ctypes.data_as(dp),
                                    o.ctypes.data_as(dp), _stream(stream)))
        return x, o

    def close(self):
        if getattr(self, "handle", None):
            lib().mbh_pt_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mbh_sync_status(stream=None) -> tuple[int, dict]:
    """Synchronise the stream, read and clear the device status word: (status, details)."""
    info = DeviceStatus()
    st = lib().mbh_sync_status(_stream(stream), C.byref(info))
    return st, {name: getattr(info, name) for name, _ in DeviceStatus._fields_}


def mbh_debug_checks() -> bool:
    return bool(lib().mbh_debug_checks())


def mbh_debug_ref_limit(ref: "Ref", e_check: int):
    _check(lib().mbh_debug_ref_limit(ref.handle, int(e_check)))
