"""Thin Python binding of the C ABI in ``include/ldpc.h`` (argument marshalling only).

Every function has the name of the C entry point it calls. Device buffers are
PyTorch CUDA tensors (PyTorch provides memory and streams; all decoding runs
in the library's kernels). The library must be built (``build.build()``); if
it is missing or a call fails, an exception is raised -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

LDPC_MSG = {"f32": 0, "f16": 1, "bf16": 2, "i8": 3}
LDPC_RULE = {"sum_product": 0, "min_sum": 1, "sp_table": 2, "min_sum_adaptive": 3}
KERNEL_CLASSES = ("interleave", "check", "bit", "syndrome", "finalize", "other", "passes")


class LdpcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"ldpc status {status}: {message}")
        self.status = status


class ldpc_code_opts_t(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32)]


class ldpc_code_info_t(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("n", ctypes.c_int32), ("n_edges", ctypes.c_int64),
                ("max_check_degree", ctypes.c_int32), ("max_var_degree", ctypes.c_int32),
                ("mean_check_degree", ctypes.c_double), ("mean_var_degree", ctypes.c_double),
                ("n_check_bins", ctypes.c_int32), ("check_bin_max_degree", ctypes.c_int32 * 8),
                ("check_bin_count", ctypes.c_int32 * 8), ("device", ctypes.c_int32), ("ira_k", ctypes.c_int32)]


class ldpc_decode_opts_t(ctypes.Structure):
    _fields_ = [("early_exit", ctypes.c_int32), ("l_max", ctypes.c_float), ("msg_dtype", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("r_out", ctypes.c_void_p), ("frames_per_lane", ctypes.c_int32),
                ("check_schedule", ctypes.c_int32), ("streams", ctypes.c_int32), ("tile_frames", ctypes.c_int32),
                ("check_rule", ctypes.c_int32), ("rule_alpha", ctypes.c_float), ("rule_beta", ctypes.c_float)]


class ldpc_server_opts_t(ctypes.Structure):
    _fields_ = [("max_batch_frames", ctypes.c_int32), ("max_slots", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("max_pending_frames", ctypes.c_int64), ("max_iter", ctypes.c_int32), ("early_exit", ctypes.c_int32),
                ("l_max", ctypes.c_float), ("msg_dtype", ctypes.c_int32), ("check_rule", ctypes.c_int32),
                ("rule_alpha", ctypes.c_float), ("rule_beta", ctypes.c_float)]


class ldpc_server_stats_t(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("completed", ctypes.c_int64), ("frames", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("queued_frames", ctypes.c_int64), ("info_bits", ctypes.c_int64)]


class ldpc_prof_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 7), ("total_ms", ctypes.c_double * 7), ("kernels", ctypes.c_int64)]


EXPORTS = ("ldpc_code_create", "ldpc_code_create_qc", "ldpc_gen_bits", "ldpc_encode_ira", "ldpc_code_build_encoder",
           "ldpc_encode", "ldpc_decode_host_stream",
           "ldpc_code_destroy", "ldpc_code_info", "ldpc_code_set_rule_table", "ldpc_code_tables", "ldpc_decode",
           "ldpc_decode_host", "ldpc_decode_static", "ldpc_gen_awgn", "ldpc_count_errors", "ldpc_batch_create",
           "ldpc_batch_run", "ldpc_batch_tune", "ldpc_batch_info", "ldpc_batch_destroy", "ldpc_server_create",
           "ldpc_server_submit", "ldpc_server_wait", "ldpc_server_stats", "ldpc_server_destroy", "ldpc_philox4x64_10", "ldpc_prof_read", "ldpc_last_error",
           "ldpc_version", "ldpc_debug_giveup")

_LIB = None
_LOCK = threading.Lock()


def library():
    """The loaded C library (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.library_path()
            if not path.exists():
                raise RuntimeError(f"libldpc_gb300 is not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(str(path))
            vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            lib.ldpc_code_create.argtypes = [i32, i32, i64, vp, vp, ctypes.POINTER(ldpc_code_opts_t), ctypes.POINTER(vp)]
            lib.ldpc_code_create_qc.argtypes = [i32, i32, i32, i64, vp, vp, vp, ctypes.POINTER(ldpc_code_opts_t),
                                                ctypes.POINTER(vp)]
            lib.ldpc_gen_bits.argtypes = [u64, i64, i32, i32, vp, vp]
            lib.ldpc_decode_host_stream.argtypes = [vp, i32, vp, i32, i32, ctypes.POINTER(ldpc_decode_opts_t), vp, vp,
                                                    vp, vp]
            lib.ldpc_encode_ira.argtypes = [vp, vp, i32, vp, vp]
            lib.ldpc_code_build_encoder.argtypes = [vp, vp]
            lib.ldpc_encode.argtypes = [vp, vp, i32, vp, vp]
            lib.ldpc_code_destroy.argtypes = [vp]
            lib.ldpc_code_destroy.restype = None
            lib.ldpc_code_info.argtypes = [vp, ctypes.POINTER(ldpc_code_info_t)]
            lib.ldpc_code_tables.argtypes = [vp] + [vp] * 11
            lib.ldpc_code_set_rule_table.argtypes = [vp, i32, vp, vp]
            lib.ldpc_decode.argtypes = [vp, vp, i32, i32, ctypes.POINTER(ldpc_decode_opts_t), vp, vp, vp, vp, vp]
            lib.ldpc_decode_host.argtypes = [vp, vp, i32, i32, ctypes.POINTER(ldpc_decode_opts_t), vp, vp, vp, vp, vp]
            lib.ldpc_decode_static.argtypes = [vp, vp, i32, i32, ctypes.POINTER(ldpc_decode_opts_t), vp, vp, vp, vp,
                                               vp]
            lib.ldpc_gen_awgn.argtypes = [u64, i64, i32, i32, ctypes.c_float, vp, vp, vp]
            lib.ldpc_philox4x64_10.argtypes = [u64, u64, u64, u64, i64, vp, vp]
            lib.ldpc_count_errors.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp]
            lib.ldpc_batch_create.argtypes = [i32, vp, vp, i32, ctypes.POINTER(ldpc_decode_opts_t), ctypes.POINTER(vp)]
            lib.ldpc_batch_run.argtypes = [vp, vp, vp, vp, vp, vp, vp]
            lib.ldpc_batch_tune.argtypes = [vp, vp, vp]
            lib.ldpc_batch_info.argtypes = [vp, i32, vp, vp, vp, vp]
            lib.ldpc_batch_destroy.argtypes = [vp]
            lib.ldpc_batch_destroy.restype = None
            lib.ldpc_server_create.argtypes = [i32, vp, ctypes.POINTER(ldpc_server_opts_t), ctypes.POINTER(vp)]
            lib.ldpc_server_submit.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
            lib.ldpc_server_wait.argtypes = [vp, ctypes.c_uint64, i32, ctypes.POINTER(ctypes.c_double)]
            lib.ldpc_server_stats.argtypes = [vp, ctypes.POINTER(ldpc_server_stats_t)]
            lib.ldpc_server_destroy.argtypes = [vp]
            lib.ldpc_server_destroy.restype = None
            lib.ldpc_prof_read.argtypes = [vp, ctypes.POINTER(ldpc_prof_t), i32]
            lib.ldpc_debug_giveup.argtypes = [vp, i32]
            lib.ldpc_last_error.restype = ctypes.c_char_p
            lib.ldpc_version.restype = ctypes.c_char_p
            for name in ("ldpc_code_create", "ldpc_code_create_qc", "ldpc_gen_bits", "ldpc_encode_ira",
                         "ldpc_code_build_encoder", "ldpc_encode",
                         "ldpc_decode_host_stream", "ldpc_code_info", "ldpc_code_set_rule_table", "ldpc_code_tables",
                         "ldpc_decode", "ldpc_decode_host",
                         "ldpc_decode_static",
                         "ldpc_gen_awgn", "ldpc_philox4x64_10", "ldpc_prof_read", "ldpc_count_errors",
                         "ldpc_batch_create", "ldpc_batch_run", "ldpc_batch_tune", "ldpc_batch_info",
                         "ldpc_server_create", "ldpc_server_submit", "ldpc_server_wait", "ldpc_server_stats",
                         "ldpc_debug_giveup"):
                getattr(lib, name).restype = ctypes.c_int
            _LIB = lib
        return _LIB


def _check(status: int) -> None:
    if status != 0:
        raise LdpcError(status, library().ldpc_last_error().decode(errors="replace"))


def ldpc_version() -> str:
    return library().ldpc_version().decode()


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, shape, name, device):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the code is on cuda:{device}")
    return ctypes.c_void_p(t.data_ptr())


class Code:
    """Owner of an ``ldpc_code_t`` handle (released by :meth:`close` or GC)."""

    def __init__(self, handle, m, n, n_edges, device):
        self._h = handle
        self.m, self.n, self.n_edges, self.device = m, n, n_edges, device

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("code is closed")
        return self._h

    def close(self):
        if self._h is not None:
            library().ldpc_code_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ldpc_code_create(m: int, n: int, rows, cols, device: int = 0) -> Code:
    """Build a code from the COO of H (``rows``, ``cols``: int sequences)."""
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    if r.shape != c.shape or r.ndim != 1:
        raise ValueError("rows and cols must be 1-D of equal length")
    h = ctypes.c_void_p()
    opts = ldpc_code_opts_t(device=device)
    _check(library().ldpc_code_create(m, n, r.shape[0], r.ctypes.data_as(ctypes.c_void_p),
                                      c.ctypes.data_as(ctypes.c_void_p), ctypes.byref(opts), ctypes.byref(h)))
    return Code(h, m, n, int(r.shape[0]), device)


def ldpc_code_create_qc(mb: int, nb: int, Z: int, entries, device: int = 0) -> Code:
    """Lift a base matrix: ``entries`` is a sequence of (row, col, shift)
    triples, each a Z x Z circulant P^shift (row t -> column (t + shift) mod
    Z) at that block; repeated blocks with distinct shifts are parallel
    protograph edges."""
    e = np.asarray(entries, dtype=np.int64).reshape(-1, 3)
    br = np.ascontiguousarray(e[:, 0], dtype=np.int32)
    bc = np.ascontiguousarray(e[:, 1], dtype=np.int32)
    sh = np.ascontiguousarray(e[:, 2], dtype=np.int32)
    h = ctypes.c_void_p()
    opts = ldpc_code_opts_t(device=device)
    vp = ctypes.c_void_p
    _check(library().ldpc_code_create_qc(mb, nb, Z, e.shape[0], br.ctypes.data_as(vp), bc.ctypes.data_as(vp),
                                         sh.ctypes.data_as(vp), ctypes.byref(opts), ctypes.byref(h)))
    return Code(h, mb * Z, nb * Z, int(e.shape[0]) * Z, device)


def ldpc_code_info(code: Code) -> dict:
    info = ldpc_code_info_t()
    _check(library().ldpc_code_info(code.handle, ctypes.byref(info)))
    nb = info.n_check_bins
    return {"m": info.m, "n": info.n, "n_edges": info.n_edges, "max_check_degree": info.max_check_degree,
            "max_var_degree": info.max_var_degree, "mean_check_degree": info.mean_check_degree,
            "mean_var_degree": info.mean_var_degree, "check_bin_max_degree": list(info.check_bin_max_degree[:nb]),
            "check_bin_count": list(info.check_bin_count[:nb]), "device": info.device,
            "ira_k": info.ira_k}


def ldpc_code_set_rule_table(code: Code, alpha_by_degree, beta_by_degree=None) -> None:
    """Scale and offset per check degree for ``rule="min_sum_adaptive"``
    (index = check degree; degrees past the end take the last entry)."""
    a = np.ascontiguousarray(alpha_by_degree, dtype=np.float32)
    b = None if beta_by_degree is None else np.ascontiguousarray(beta_by_degree, dtype=np.float32)
    if a.ndim != 1 or (b is not None and b.shape != a.shape):
        raise ValueError("alpha_by_degree and beta_by_degree must be 1-D and of one length")
    vp = ctypes.c_void_p
    _check(library().ldpc_code_set_rule_table(code.handle, a.shape[0], a.ctypes.data_as(vp),
                                              None if b is None else b.ctypes.data_as(vp)))


TABLE_NAMES = ("v", "c", "t", "s", "u", "ebar", "vbar", "cbar", "tbar", "sbar", "ubar")


def ldpc_code_tables(code: Code) -> dict:
    """The address-iterator arrays of Tables 1-2 as numpy int32 arrays."""
    arrs = {k: np.zeros(code.n_edges, dtype=np.int32) for k in TABLE_NAMES}
    _check(library().ldpc_code_tables(code.handle, *[arrs[k].ctypes.data_as(ctypes.c_void_p) for k in TABLE_NAMES]))
    return arrs



def _opts(early_exit, l_max, msg_dtype, profile, r_out_ptr, frames_per_lane=0, check_schedule=0, streams=0,
          tile_frames=0, rule="sum_product", rule_alpha=1.0, rule_beta=0.0):
    if msg_dtype not in LDPC_MSG:
        raise ValueError(f"msg_dtype must be one of {sorted(LDPC_MSG)}")
    if rule not in LDPC_RULE:
        raise ValueError(f"rule must be one of {sorted(LDPC_RULE)}")
    return ldpc_decode_opts_t(early_exit=1 if early_exit else 0, l_max=float(l_max), msg_dtype=LDPC_MSG[msg_dtype],
                              profile=int(profile), r_out=r_out_ptr, frames_per_lane=int(frames_per_lane),
                              check_schedule=int(check_schedule), streams=int(streams), tile_frames=int(tile_frames),
                              check_rule=LDPC_RULE[rule], rule_alpha=float(rule_alpha), rule_beta=float(rule_beta))


def ldpc_decode(code: Code, llr, max_iter: int, *, early_exit: bool = True, l_max: float = 20.0,
                msg_dtype: str = "f32", profile: bool = False, want_post: bool = True, want_r: bool = False,
                out: dict | None = None, stream=None, frames_per_lane: int = 0, check_schedule: int = 0,
                streams: int = 0, tile_frames: int = 0, rule: str = "sum_product", rule_alpha: float = 1.0,
                rule_beta: float = 0.0) -> dict:
    """Decode ``llr`` (CUDA float32 [F, n]); returns CUDA tensors
    ``bits`` uint8 [F, n], ``iters`` int32 [F], ``ok`` uint8 [F] and, when
    asked, ``post`` float32 [F, n] and ``r`` float32 [F, E] (edge order)."""
    import torch
    f = int(llr.shape[0]) if llr.dim() == 2 else -1
    dev = torch.device("cuda", code.device)
    _dev_ptr(llr, torch.float32, (f, code.n), "llr", code.device)
    o = dict(out or {})
    if "bits" not in o:
        o["bits"] = torch.empty((f, code.n), dtype=torch.uint8, device=dev)
    if "iters" not in o:
        o["iters"] = torch.empty((f,), dtype=torch.int32, device=dev)
    if "ok" not in o:
        o["ok"] = torch.empty((f,), dtype=torch.uint8, device=dev)
    if want_post and "post" not in o:
        o["post"] = torch.empty((f, code.n), dtype=torch.float32, device=dev)
    if want_r and "r" not in o:
        o["r"] = torch.empty((f, code.n_edges), dtype=torch.float32, device=dev)
    r_ptr = _dev_ptr(o.get("r"), torch.float32, (f, code.n_edges), "r", code.device) if want_r else None
    opts = _opts(early_exit, l_max, msg_dtype, profile, r_ptr.value if r_ptr else None, frames_per_lane,
                 check_schedule, streams, tile_frames, rule, rule_alpha, rule_beta)
    _check(library().ldpc_decode(
        code.handle, _dev_ptr(llr, torch.float32, (f, code.n), "llr", code.device), f, max_iter, ctypes.byref(opts),
        _dev_ptr(o["bits"], torch.uint8, (f, code.n), "bits", code.device),
        _dev_ptr(o["iters"], torch.int32, (f,), "iters", code.device),
        _dev_ptr(o["ok"], torch.uint8, (f,), "ok", code.device),
        _dev_ptr(o.get("post"), torch.float32, (f, code.n), "post", code.device) if want_post else None,
        _stream_handle(stream)))
    return o


def ldpc_decode_host(code: Code, llr: np.ndarray, max_iter: int, *, early_exit: bool = True, l_max: float = 20.0,
                     msg_dtype: str = "f32", profile: bool = False, want_post: bool = False, out: dict | None = None,
                     stream=None, frames_per_lane: int = 0, check_schedule: int = 0, streams: int = 0,
                     tile_frames: int = 0) -> dict:
    """Decode host LLRs (numpy float32 [F, n], or a pinned CPU torch tensor);
    copies in and out inside the call and returns host arrays."""
    import torch
    if isinstance(llr, torch.Tensor):
        if llr.is_cuda or llr.dtype != torch.float32 or not llr.is_contiguous():
            raise ValueError("llr must be a contiguous float32 host tensor")
        f, n = llr.shape
        llr_ptr = ctypes.c_void_p(llr.data_ptr())
        mk = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=llr.is_pinned())  # noqa: E731
        dts = (torch.uint8, torch.int32, torch.uint8, torch.float32)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    else:
        llr = np.ascontiguousarray(llr, dtype=np.float32)
        f, n = llr.shape
        llr_ptr = llr.ctypes.data_as(ctypes.c_void_p)
        mk = lambda shape, dt: np.empty(shape, dtype=dt)  # noqa: E731
        dts = (np.uint8, np.int32, np.uint8, np.float32)
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    if n != code.n:
        raise ValueError("llr has the wrong code length")
    o = dict(out or {})
    o.setdefault("bits", mk((f, n), dts[0]))
    o.setdefault("iters", mk((f,), dts[1]))
    o.setdefault("ok", mk((f,), dts[2]))
    if want_post:
        o.setdefault("post", mk((f, n), dts[3]))
    opts = _opts(early_exit, l_max, msg_dtype, profile, None, frames_per_lane, check_schedule, streams, tile_frames)
    _check(library().ldpc_decode_host(code.handle, llr_ptr, f, max_iter, ctypes.byref(opts), ptr(o["bits"]),
                                      ptr(o["iters"]), ptr(o["ok"]), ptr(o["post"]) if want_post else None,
                                      _stream_handle(stream)))
    return o


def ldpc_decode_host_stream(code: Code, llrs, max_iter: int, *, early_exit: bool = True, l_max: float = 20.0,
                            msg_dtype: str = "f32", outs=None, stream=None, frames_per_lane: int = 0,
                            check_schedule: int = 0, streams: int = 0, rule: str = "sum_product",
                            rule_alpha: float = 1.0, rule_beta: float = 0.0) -> list:
    """Decode a list of host batches (contiguous float32 CPU tensors [F, n],
    pinned for overlap) with copies overlapping decodes; returns (or fills
    ``outs``) one dict of host tensors ``bits``, ``iters``, ``ok`` per batch.
    Output dicts may be shared between batches."""
    import torch
    if not llrs:
        return []
    f, n = llrs[0].shape
    if n != code.n:
        raise ValueError("llr has the wrong code length")
    for t in llrs:
        if t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != (f, n):
            raise ValueError("every batch must be a contiguous float32 host tensor of the same shape")
    if outs is None:
        pin = llrs[0].is_pinned()
        outs = [{"bits": torch.empty((f, n), dtype=torch.uint8, pin_memory=pin),
                 "iters": torch.empty((f,), dtype=torch.int32, pin_memory=pin),
                 "ok": torch.empty((f,), dtype=torch.uint8, pin_memory=pin)} for _ in llrs]
    if len(outs) != len(llrs):
        raise ValueError("one output dict per batch")
    vp = ctypes.c_void_p
    arr = lambda ts: (vp * len(ts))(*[t.data_ptr() for t in ts])  # noqa: E731
    opts = _opts(early_exit, l_max, msg_dtype, False, None, frames_per_lane, check_schedule, streams, 0, rule,
                 rule_alpha, rule_beta)
    _check(library().ldpc_decode_host_stream(code.handle, len(llrs), arr(llrs), f, max_iter, ctypes.byref(opts),
                                             arr([o["bits"] for o in outs]), arr([o["iters"] for o in outs]),
                                             arr([o["ok"] for o in outs]), _stream_handle(stream)))
    return outs


def ldpc_decode_static(code: Code, llr, max_iter: int, *, early_exit: bool = True, l_max: float = 20.0,
                       msg_dtype: str = "f32", want_post: bool = True, out: dict | None = None, stream=None,
                       frames_per_lane: int = 0, check_schedule: int = 0, rule: str = "sum_product",
                       rule_alpha: float = 1.0, rule_beta: float = 0.0) -> dict:
    """ldpc_decode for callers that may not allocate device memory while they
    decode: the library's scratch is a fixed 64 MiB device array (see
    include/ldpc.h). Output tensors are allocated here unless passed in
    ``out``; pass them in to keep the whole call allocation-free."""
    import torch
    f = int(llr.shape[0]) if llr.dim() == 2 else -1
    dev = torch.device("cuda", code.device)
    o = dict(out or {})
    if "bits" not in o:
        o["bits"] = torch.empty((f, code.n), dtype=torch.uint8, device=dev)
    if "iters" not in o:
        o["iters"] = torch.empty((f,), dtype=torch.int32, device=dev)
    if "ok" not in o:
        o["ok"] = torch.empty((f,), dtype=torch.uint8, device=dev)
    if want_post and "post" not in o:
        o["post"] = torch.empty((f, code.n), dtype=torch.float32, device=dev)
    opts = _opts(early_exit, l_max, msg_dtype, False, None, frames_per_lane, check_schedule, 0, 0, rule, rule_alpha,
                 rule_beta)
    _check(library().ldpc_decode_static(
        code.handle, _dev_ptr(llr, torch.float32, (f, code.n), "llr", code.device), f, max_iter, ctypes.byref(opts),
        _dev_ptr(o["bits"], torch.uint8, (f, code.n), "bits", code.device),
        _dev_ptr(o["iters"], torch.int32, (f,), "iters", code.device),
        _dev_ptr(o["ok"], torch.uint8, (f,), "ok", code.device),
        _dev_ptr(o.get("post"), torch.float32, (f, code.n), "post", code.device) if want_post else None,
        _stream_handle(stream)))
    return o


def ldpc_gen_awgn(seed: int, frame_offset: int, n_frames: int, n: int, sigma2: float, codewords=None, out=None,
                  device: int = 0, stream=None):
    """BPSK/AWGN channel LLRs (CUDA float32 [n_frames, n]) from the on-device
    Philox-4x64-10 generator; ``codewords`` is a CUDA uint8 [n_frames, n]
    tensor or None (all-zero word)."""
    import torch
    if out is None:
        out = torch.empty((n_frames, n), dtype=torch.float32, device=torch.device("cuda", device))
    _check(library().ldpc_gen_awgn(seed, frame_offset, n_frames, n, float(sigma2),
                                   _dev_ptr(codewords, torch.uint8, (n_frames, n), "codewords", None),
                                   _dev_ptr(out, torch.float32, (n_frames, n), "out", None), _stream_handle(stream)))
    return out


def ldpc_gen_bits(seed: int, frame_offset: int, n_frames: int, k: int, out=None, device: int = 0, stream=None):
    """Random information words (CUDA uint8 [n_frames, k], one bit per byte)
    from the on-device Philox-4x64-10 generator (key (seed, 1))."""
    import torch
    if out is None:
        out = torch.empty((n_frames, k), dtype=torch.uint8, device=torch.device("cuda", device))
    _check(library().ldpc_gen_bits(seed, frame_offset, n_frames, k,
                                   _dev_ptr(out, torch.uint8, (n_frames, k), "out", None), _stream_handle(stream)))
    return out


def ldpc_encode_ira(code: Code, info, out=None, stream=None):
    """Systematic IRA encoding on the device: CUDA uint8 info [F, k] ->
    codewords [F, n] (``k`` = ``ldpc_code_info(code)["ira_k"]``)."""
    import torch
    k = code.n - code.m
    f = int(info.shape[0])
    if out is None:
        out = torch.empty((f, code.n), dtype=torch.uint8, device=info.device)
    _check(library().ldpc_encode_ira(code.handle, _dev_ptr(info, torch.uint8, (f, k), "info", code.device), f,
                                     _dev_ptr(out, torch.uint8, (f, code.n), "out", code.device),
                                     _stream_handle(stream)))
    return out


def ldpc_code_build_encoder(code: Code) -> int:
    """Build the code's systematic encoder (any code; host GF(2) reduction of
    H, kept with the code); returns k, its number of information bits."""
    k = ctypes.c_int32()
    _check(library().ldpc_code_build_encoder(code.handle, ctypes.byref(k)))
    return k.value


def ldpc_encode(code: Code, info, out=None, stream=None):
    """Systematic encoding with the encoder ldpc_code_build_encoder built:
    CUDA uint8 info [F, k] -> codewords [F, n]."""
    import torch
    k = ldpc_code_build_encoder(code)
    f = int(info.shape[0])
    if out is None:
        out = torch.empty((f, code.n), dtype=torch.uint8, device=info.device)
    _check(library().ldpc_encode(code.handle, _dev_ptr(info, torch.uint8, (f, k), "info", code.device), f,
                                 _dev_ptr(out, torch.uint8, (f, code.n), "out", code.device), _stream_handle(stream)))
    return out


def ldpc_count_errors(bits, ref=None, iters=None, ok=None, counts=None, stream=None):
    """Accumulate [bit errors, frame errors, sum of iterations, unsatisfied
    frames] of decoded words into a CUDA int64 tensor [4] (returned)."""
    import torch
    f, n = bits.shape
    if counts is None:
        counts = torch.zeros(4, dtype=torch.int64, device=bits.device)
    _check(library().ldpc_count_errors(
        _dev_ptr(bits, torch.uint8, (f, n), "bits", None), _dev_ptr(ref, torch.uint8, (f, n), "ref", None), f, n,
        _dev_ptr(iters, torch.int32, (f,), "iters", None), _dev_ptr(ok, torch.uint8, (f,), "ok", None),
        _dev_ptr(counts, torch.int64, (4,), "counts", None), _stream_handle(stream)))
    return counts


def ldpc_philox4x64_10(key0: int, key1: int, ctr0: int, ctr1: int, count: int, device: int = 0, stream=None):
    """Raw Philox-4x64-10 blocks as a CUDA int64 tensor [count, 4] (bit pattern of uint64)."""
    import torch
    out = torch.empty((count, 4), dtype=torch.int64, device=torch.device("cuda", device))
    _check(library().ldpc_philox4x64_10(key0, key1, ctr0, ctr1, count, ctypes.c_void_p(out.data_ptr()),
                                        _stream_handle(stream)))
    return out


def ldpc_debug_giveup(code: Code, cta: int) -> None:
    """Arm the bounded-wait test hook for the next decode of ``code``: warp 0
    of CTA ``cta`` of its first later check pass takes the give-up path after
    its rows have landed (-1 disarms)."""
    _check(library().ldpc_debug_giveup(code.handle, int(cta)))


def ldpc_prof_read(code: Code, reset: bool = True) -> dict:
    """Per kernel class: profiled launches and total CUDA-event milliseconds;
    ``kernels``: all library kernels enqueued for the code since the last reset."""
    p = ldpc_prof_t()
    _check(library().ldpc_prof_read(code.handle, ctypes.byref(p), 1 if reset else 0))
    out = {k: {"launches": int(p.launches[i]), "total_ms": float(p.total_ms[i])} for i, k in enumerate(KERNEL_CLASSES)}
    out["kernels"] = int(p.kernels)
    return out


class Batch:
    """Owner of an ``ldpc_batch_t``: several codes decoded as one CUDA graph.

    Keeps references to its codes (the batch borrows their tables) and to the
    buffers of the last run (the captured graph points at them)."""

    def __init__(self, handle, codes, frames):
        self._h = handle
        self.codes = list(codes)
        self.frames = list(frames)
        self._keep = None

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("batch is closed")
        return self._h

    def close(self):
        if self._h is not None:
            library().ldpc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr_array(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def ldpc_batch_create(codes, n_frames, max_iter: int, *, early_exit: bool = True, l_max: float = 20.0,
                      msg_dtype: str = "f32", frames_per_lane: int = 0, check_schedule: int = 0,
                      rule: str = "sum_product", rule_alpha: float = 1.0, rule_beta: float = 0.0) -> Batch:
    """A mixed-code batch over ``codes`` (``Code`` handles on one device)."""
    hs = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])
    fr = (ctypes.c_int32 * len(codes))(*[int(f) for f in n_frames])
    opts = _opts(early_exit, l_max, msg_dtype, False, None, frames_per_lane, check_schedule, 0, 0, rule, rule_alpha,
                 rule_beta)
    h = ctypes.c_void_p()
    _check(library().ldpc_batch_create(len(codes), hs, fr, max_iter, ctypes.byref(opts), ctypes.byref(h)))
    return Batch(h, codes, n_frames)


def ldpc_batch_run(batch: Batch, llrs, outs=None, want_post: bool = False, stream=None):
    """Decode every item (llrs: CUDA float32 [F_i, n_i] tensors). Returns a
    list of output dicts; pass the same ``outs`` again to replay the graph."""
    import torch
    if outs is None:
        outs = []
        for c, f in zip(batch.codes, batch.frames):
            dev = torch.device("cuda", c.device)
            o = {"bits": torch.empty((f, c.n), dtype=torch.uint8, device=dev),
                 "iters": torch.empty((f,), dtype=torch.int32, device=dev),
                 "ok": torch.empty((f,), dtype=torch.uint8, device=dev)}
            if want_post:
                o["post"] = torch.empty((f, c.n), dtype=torch.float32, device=dev)
            outs.append(o)
    for c, f, l in zip(batch.codes, batch.frames, llrs):
        _dev_ptr(l, torch.float32, (f, c.n), "llr", c.device)
    posts = [o.get("post") for o in outs]
    _check(library().ldpc_batch_run(batch.handle, _ptr_array(llrs), _ptr_array([o["bits"] for o in outs]),
                                    _ptr_array([o["iters"] for o in outs]), _ptr_array([o["ok"] for o in outs]),
                                    _ptr_array(posts) if any(p is not None for p in posts) else None,
                                    _stream_handle(stream)))
    batch._keep = (llrs, outs)
    return outs


def ldpc_batch_tune(batch: Batch, llrs, stream=None) -> None:
    _check(library().ldpc_batch_tune(batch.handle, _ptr_array(llrs), _stream_handle(stream)))


def ldpc_batch_info(batch: Batch, item: int) -> dict:
    v, s, st, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(library().ldpc_batch_info(batch.handle, item, ctypes.byref(v), ctypes.byref(s), ctypes.byref(st),
                                     ctypes.byref(k)))
    return {"frames_per_lane": v.value, "check_schedule": s.value, "streams": st.value, "kernels_per_run": k.value}


class Server:
    """Owner of an ``ldpc_server_t`` (continuous request batching)."""

    def __init__(self, handle, codes):
        self._h = handle
        self.codes = list(codes)
        self._live = {}  # request id -> tensors kept alive until waited

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("server is closed")
        return self._h

    def close(self):
        if self._h is not None:
            library().ldpc_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ldpc_server_create(codes, *, max_batch_frames: int = 1024, max_slots: int = 4, memory_budget: int = 0,
                       max_pending_frames: int = 0, max_iter: int = 50, early_exit: bool = True, l_max: float = 20.0,
                       msg_dtype: str = "f16", rule: str = "sum_product", rule_alpha: float = 1.0,
                       rule_beta: float = 0.0) -> Server:
    hs = (ctypes.c_void_p * len(codes))(*[c.handle.value for c in codes])
    o = ldpc_server_opts_t(max_batch_frames=max_batch_frames, max_slots=max_slots, memory_budget=memory_budget,
                           max_pending_frames=max_pending_frames, max_iter=max_iter, early_exit=1 if early_exit else 0,
                           l_max=float(l_max), msg_dtype=LDPC_MSG[msg_dtype], check_rule=LDPC_RULE[rule],
                           rule_alpha=float(rule_alpha), rule_beta=float(rule_beta))
    h = ctypes.c_void_p()
    _check(library().ldpc_server_create(len(codes), hs, ctypes.byref(o), ctypes.byref(h)))
    return Server(h, codes)


def ldpc_server_submit(server: Server, code_index: int, llr, out: dict | None = None, want_post: bool = False) -> tuple:
    """Queue ``llr`` (CUDA float32 [F, n]) for code ``code_index``; returns
    (request id, output dict filled when the request completes)."""
    import torch
    if not 0 <= code_index < len(server.codes):
        raise ValueError(f"code_index {code_index} outside [0, {len(server.codes)})")
    c = server.codes[code_index]
    f = int(llr.shape[0])
    dev = torch.device("cuda", c.device)
    o = dict(out or {})
    o.setdefault("bits", torch.empty((f, c.n), dtype=torch.uint8, device=dev))
    o.setdefault("iters", torch.empty((f,), dtype=torch.int32, device=dev))
    o.setdefault("ok", torch.empty((f,), dtype=torch.uint8, device=dev))
    if want_post:
        o.setdefault("post", torch.empty((f, c.n), dtype=torch.float32, device=dev))
    rid = ctypes.c_uint64()
    _check(library().ldpc_server_submit(
        server.handle, code_index, _dev_ptr(llr, torch.float32, (f, c.n), "llr", c.device), f,
        _dev_ptr(o["bits"], torch.uint8, (f, c.n), "bits", c.device),
        _dev_ptr(o["iters"], torch.int32, (f,), "iters", c.device), _dev_ptr(o["ok"], torch.uint8, (f,), "ok", c.device),
        _dev_ptr(o.get("post"), torch.float32, (f, c.n), "post", c.device) if want_post else None, ctypes.byref(rid)))
    server._live[rid.value] = (llr, o)
    return rid.value, o


def ldpc_server_wait(server: Server, request_id: int, timeout_ms: int = -1) -> float:
    """Wait for a request; returns its submit-to-completion latency in ms."""
    lat = ctypes.c_double()
    _check(library().ldpc_server_wait(server.handle, request_id, timeout_ms, ctypes.byref(lat)))
    server._live.pop(request_id, None)
    return lat.value


def ldpc_server_stats(server: Server) -> dict:
    st = ldpc_server_stats_t()
    _check(library().ldpc_server_stats(server.handle, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in ldpc_server_stats_t._fields_}


def code_from_inputs(code, device: int = 0) -> Code:
    """Convenience: an ``ldpc_code_t`` from an ``inputs.Code``."""
    return ldpc_code_create(code.m, code.n, code.rows, code.cols, device=device)
