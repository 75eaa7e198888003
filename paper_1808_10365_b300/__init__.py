"""B300 spectral-kurtosis RFI detector (Taylor et al., arXiv:1808.10365).

Python binding of the C ABI in ``include/sk.h``.  Every function here has the
name of the C entry point it calls and does argument marshalling only; all
arithmetic runs in ``libsk.so`` (hand-written sm_103a CUDA).  Device buffers
and streams come from PyTorch (tensors' ``data_ptr()``, ``torch.cuda.Stream``),
or are given as raw integers.  There is no CPU fallback: if the library is
missing, importing the binding's functions raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SK_DEBUG_LIBRARY=1 loads the debug build (bounds-checked loads and stores)
LIB_PATH = os.path.join(HERE, "libsk_debug.so" if os.environ.get("SK_DEBUG_LIBRARY") == "1"
                        else "libsk.so")
# tile choices measured on B300 by autotune.py; a caller's SK_AUTOTUNE_CACHE wins
os.environ.setdefault("SK_AUTOTUNE_CACHE", os.path.join(HERE, "tiles_b300.txt"))

SK_OK = 0
SK_ERR_INVALID_ARG = 1
SK_ERR_UNSUPPORTED = 2
SK_ERR_OOM = 3
SK_ERR_CUDA = 4
SK_ERR_BUSY = 5
SK_ERR_TIMEOUT = 6
SK_ERR_NOT_READY = 7
SK_ERR_CLOSED = 8
SK_LAYOUT_TIME_MAJOR = 0
SK_LAYOUT_INPUT_MAJOR = 1
SK_RUNNING_OFFSET = 0x1
SK_THRESH_PEARSON3 = 0x2
SK_RUNNING_MU = 0x4
SK_OFFSET_BUCKETS = 4096
SK_MAX_INPUTS = 4096
SK_MAX_TIME = 4096
SK_PATH_AUTO = 0
SK_PATH_TEAM = 1
SK_PATH_WARP_SLICE = 2
SK_PATH_ROW_BALANCED = 3
SK_PATH_GENERAL = 4
SK_PATH_PER_INPUT = 5
SK_PATH_STREAM = 6
SK_NOALLOC_MAX_BYTES = 16 * 1024 * 1024
SK_NOALLOC_MAX_FRAMES = 65536

EXPORTED = [
    "sk_plan_create", "sk_plan_destroy", "sk_plan_thresholds", "sk_plan_offset_table",
    "sk_plan_set_tiles", "sk_plan_get_tiles", "sk_plan_set_config", "sk_plan_get_config",
    "sk_compute", "sk_flag", "sk_flag_host",
    "sk_flag_host_noalloc", "sk_compute_inputs", "sk_finish",
    "sk_batch_create", "sk_batch_run", "sk_batch_launches", "sk_batch_destroy", "sk_server_create",
    "sk_server_destroy", "sk_stream_open", "sk_stream_submit", "sk_stream_submit_ref",
    "sk_ticket_wait",
    "sk_stream_drain", "sk_stream_get_state", "sk_stream_set_state", "sk_stream_close",
    "sk_server_stats", "sk_stream_stats", "sk_server_replay", "sk_digitisation_offset",
    "sk_selftest_conversions", "sk_selftest_slot_wait", "sk_last_error",
]


class SkError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"sk status {status}: {message}")
        self.status = status
        self.message = message


class sk_params_t(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int32), ("n_time", ctypes.c_int32),
                ("layout", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("n_sigma", ctypes.c_double), ("mean_offset", ctypes.c_double),
                ("offset_table", ctypes.c_void_p)]


class sk_launch_config_t(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("path", ctypes.c_int32), ("team_log2", ctypes.c_int32),
                ("prefetch", ctypes.c_int32), ("batch_path", ctypes.c_int32),
                ("last_path", ctypes.c_int32)]


class sk_batch_item_t(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("d_in", ctypes.c_void_p),
                ("n_frames", ctypes.c_int64), ("d_sk", ctypes.c_void_p),
                ("d_mask", ctypes.c_void_p)]


class sk_replay_t(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("streams", ctypes.c_void_p), ("frames", ctypes.c_void_p),
                ("pool_frames", ctypes.c_void_p), ("frames_per_stream", ctypes.c_int64),
                ("cadence_s", ctypes.c_double), ("jitter_mean_s", ctypes.c_double),
                ("paced", ctypes.c_int32), ("by_reference", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class sk_replay_result_t(ctypes.Structure):
    _fields_ = [("wall_s", ctypes.c_double), ("frames", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("busy_retries", ctypes.c_int64),
                ("bytes", ctypes.c_double), ("latency_p50_us", ctypes.c_double),
                ("latency_p99_us", ctypes.c_double), ("submit_p50_us", ctypes.c_double),
                ("submit_p99_us", ctypes.c_double)]


class sk_stream_stats_t(ctypes.Structure):
    _fields_ = [("frames_done", ctypes.c_int64), ("frames_flagged", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("outstanding", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("latency_p50_us", ctypes.c_double),
                ("latency_p99_us", ctypes.c_double)]


class sk_server_stats_t(ctypes.Structure):
    _fields_ = [("frames_done", ctypes.c_int64), ("frames_flagged", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("latency_p50_us", ctypes.c_double), ("latency_p99_us", ctypes.c_double),
                ("hbm_in_use", ctypes.c_size_t)]


_lib = None


def library():
    """The loaded libsk.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsk.so not built ({LIB_PATH}); run paper_1808_10365_b300/build.py")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U8 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint8
    st = ctypes.c_int
    sig = {
        "sk_plan_create": [ctypes.POINTER(sk_params_t), ctypes.c_int, ctypes.POINTER(P)],
        "sk_plan_destroy": [P],
        "sk_plan_thresholds": [P, P, P],
        "sk_plan_offset_table": [P, P],
        "sk_plan_set_tiles": [P, I32, I32],
        "sk_plan_get_tiles": [P, ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "sk_plan_set_config": [P, ctypes.POINTER(sk_launch_config_t)],
        "sk_plan_get_config": [P, ctypes.POINTER(sk_launch_config_t)],
        "sk_compute": [P, P, I64, P, P, P, P, P, P],
        "sk_flag": [P, P, I64, P, P, P],
        "sk_flag_host": [P, P, I64, P, P, P],
        "sk_flag_host_noalloc": [P, P, I64, P, P, P],
        "sk_compute_inputs": [P, P, I64, P, P, P, P, P],
        "sk_batch_create": [ctypes.POINTER(sk_batch_item_t), I32, ctypes.c_int, ctypes.POINTER(P)],
        "sk_batch_run": [P, P],
        "sk_batch_launches": [P, ctypes.POINTER(I32)],
        "sk_batch_destroy": [P],
        "sk_server_create": [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(P)],
        "sk_server_destroy": [P],
        "sk_stream_open": [P, ctypes.POINTER(sk_params_t), I32, ctypes.POINTER(I32)],
        "sk_stream_submit": [P, I32, P, I64, ctypes.POINTER(I64)],
        "sk_stream_submit_ref": [P, I32, P, I64, ctypes.POINTER(I64)],
        "sk_ticket_wait": [P, I64, I64, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(U8)],
        "sk_stream_drain": [P, I32, I64],
        "sk_stream_get_state": [P, I32, P, ctypes.POINTER(ctypes.c_size_t)],
        "sk_stream_set_state": [P, I32, P, ctypes.c_size_t],
        "sk_stream_close": [P, I32],
        "sk_server_stats": [P, ctypes.POINTER(sk_server_stats_t)],
        "sk_stream_stats": [P, I32, ctypes.POINTER(sk_stream_stats_t)],
        "sk_server_replay": [P, ctypes.POINTER(sk_replay_t), ctypes.POINTER(sk_replay_result_t)],
        "sk_digitisation_offset": [ctypes.c_double, ctypes.POINTER(ctypes.c_double)],
        "sk_selftest_conversions": [ctypes.c_int, ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "sk_selftest_slot_wait": [P, I32, ctypes.POINTER(I32), P],
        "sk_finish": [P, P, P, I64, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = st
    L.sk_last_error.argtypes = []
    L.sk_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status: int):
    if status != SK_OK:
        raise SkError(status, library().sk_last_error().decode(errors="replace"))


def _ptr(x):
    """Raw address of a torch tensor, numpy array, int, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


# (N, M) of the plans and served streams created through this binding, so that
# buffer sizes can be checked before a kernel ever sees them
_plan_shape = {}
_stream_shape = {}


def _buf(x, nbytes, where, what):
    """Raw address of x after checking it.  A torch tensor or numpy array must be
    contiguous, hold at least nbytes (when the shape is known) and live where the
    call reads it: 'device' (a CUDA tensor, or a page-locked CPU tensor the device
    can read) or 'host' (numpy, or a CPU tensor).  Plain integers pass unchecked."""
    if x is None or isinstance(x, int):
        return _ptr(x)
    if isinstance(x, np.ndarray):
        if where == "device":
            raise SkError(SK_ERR_INVALID_ARG, f"{what}: a numpy array is host memory; "
                                              "this call reads device memory")
        if not x.flags.c_contiguous:
            raise SkError(SK_ERR_INVALID_ARG, f"{what}: array is not contiguous")
        size = x.nbytes
    else:
        if not x.is_contiguous():
            raise SkError(SK_ERR_INVALID_ARG, f"{what}: tensor is not contiguous")
        if where == "device" and not (x.is_cuda or x.is_pinned()):
            raise SkError(SK_ERR_INVALID_ARG, f"{what}: tensor is in pageable host memory; "
                                              "this call reads device memory")
        if where == "host" and x.is_cuda:
            raise SkError(SK_ERR_INVALID_ARG, f"{what}: CUDA tensor given to a host-buffer call")
        size = x.numel() * x.element_size()
    if nbytes is not None and size < nbytes:
        raise SkError(SK_ERR_INVALID_ARG, f"{what}: {size} bytes, the call needs {nbytes}")
    return _ptr(x)


def _sizes(shape, n_frames, per_frame):
    """Bytes of each buffer for n_frames frames (None if the shape is unknown)."""
    if shape is None or n_frames < 0:
        return [None] * len(per_frame)
    N, M = shape
    return [int(n_frames) * f(N, M) for f in per_frame]


def _stream(s):
    if s is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _params(n_inputs, n_time, n_sigma, mean_offset, layout, flags, offset_table):
    p = sk_params_t()
    p.n_inputs = int(n_inputs)
    p.n_time = int(n_time)
    p.layout = int(layout)
    p.flags = int(flags)
    p.n_sigma = float(n_sigma)
    p.mean_offset = float(mean_offset)
    keep = None
    if offset_table is not None:
        keep = np.ascontiguousarray(offset_table, dtype=np.int64)
        if keep.size != SK_OFFSET_BUCKETS:
            raise ValueError("offset_table needs SK_OFFSET_BUCKETS entries")
        p.offset_table = keep.ctypes.data
    return p, keep


# ------------------------------------------------------------------ plans

def sk_plan_create(n_inputs, n_time, n_sigma=3.0, mean_offset=0.0, layout=0, flags=0,
                   offset_table=None, device=0) -> int:
    p, keep = _params(n_inputs, n_time, n_sigma, mean_offset, layout, flags, offset_table)
    h = ctypes.c_void_p()
    _check(library().sk_plan_create(ctypes.byref(p), int(device), ctypes.byref(h)))
    _plan_shape[h.value] = (int(n_inputs), int(n_time))
    return h.value


def sk_plan_destroy(plan):
    _check(library().sk_plan_destroy(plan))
    _plan_shape.pop(plan, None)


def sk_plan_thresholds(plan, n_inputs):
    lo = np.zeros(n_inputs + 1, dtype=np.int64)
    hi = np.zeros(n_inputs + 1, dtype=np.int64)
    _check(library().sk_plan_thresholds(plan, lo.ctypes.data, hi.ctypes.data))
    return lo, hi


def sk_plan_offset_table(plan):
    e = np.zeros(SK_OFFSET_BUCKETS, dtype=np.int64)
    _check(library().sk_plan_offset_table(plan, e.ctypes.data))
    return e


def sk_plan_set_tiles(plan, rows_per_batch, grid_ctas=0):
    _check(library().sk_plan_set_tiles(plan, int(rows_per_batch), int(grid_ctas)))


def sk_plan_get_tiles(plan):
    r = ctypes.c_int32()
    g = ctypes.c_int32()
    _check(library().sk_plan_get_tiles(plan, ctypes.byref(r), ctypes.byref(g)))
    return r.value, g.value


def sk_plan_get_config(plan) -> dict:
    """The plan's launch configuration (sk_launch_config_t) as a dict."""
    c = sk_launch_config_t()
    _check(library().sk_plan_get_config(plan, ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in sk_launch_config_t._fields_}


def sk_plan_set_config(plan, rows=16, grid_ctas=0, path=SK_PATH_AUTO, team_log2=0, prefetch=0,
                       batch_path=SK_PATH_AUTO):
    c = sk_launch_config_t(int(rows), int(grid_ctas), int(path), int(team_log2), int(prefetch),
                           int(batch_path), 0)
    _check(library().sk_plan_set_config(plan, ctypes.byref(c)))


def sk_compute(plan, d_in, n_frames, s1=None, s2=None, q=None, sk=None, neff=None, stream=None):
    F = int(n_frames)
    b_in, b_s, b_q, b_4 = _sizes(_plan_shape.get(plan), F, [
        lambda N, M: M * N, lambda N, M: 4 * N, lambda N, M: 8, lambda N, M: 4])
    _check(library().sk_compute(plan, _buf(d_in, b_in, "device", "d_in"), F,
                                _buf(s1, b_s, "device", "s1"), _buf(s2, b_s, "device", "s2"),
                                _buf(q, b_q, "device", "q"), _buf(sk, b_4, "device", "sk"),
                                _buf(neff, b_4, "device", "neff"), _stream(stream)))


def sk_compute_inputs(plan, d_in, n_frames, sk_in, mask_in=None, sk=None, mask=None,
                      stream=None):
    F = int(n_frames)
    b_in, b_ski, b_mi, b_sk, b_m = _sizes(_plan_shape.get(plan), F, [
        lambda N, M: M * N, lambda N, M: 4 * N, lambda N, M: N, lambda N, M: 4,
        lambda N, M: 1])
    _check(library().sk_compute_inputs(plan, _buf(d_in, b_in, "device", "d_in"), F,
                                       _buf(sk_in, b_ski, "device", "sk_in"),
                                       _buf(mask_in, b_mi, "device", "mask_in"),
                                       _buf(sk, b_sk, "device", "sk"),
                                       _buf(mask, b_m, "device", "mask"), _stream(stream)))


def sk_flag(plan, d_in, n_frames, sk, mask, stream=None):
    F = int(n_frames)
    b_in, b_sk, b_m = _sizes(_plan_shape.get(plan), F, [
        lambda N, M: M * N, lambda N, M: 4, lambda N, M: 1])
    _check(library().sk_flag(plan, _buf(d_in, b_in, "device", "d_in"), F,
                             _buf(sk, b_sk, "device", "sk"), _buf(mask, b_m, "device", "mask"),
                             _stream(stream)))


def sk_finish(plan, d_q, d_neff, n_frames, sk, mask, stream=None):
    """SK and mask per frame from Q and neff summed over input shards, with the
    whole array's plan (input sharding; see sharding.py)."""
    F = int(n_frames)
    b_q, b_n, b_sk, b_m = _sizes(_plan_shape.get(plan), F, [
        lambda N, M: 8, lambda N, M: 4, lambda N, M: 4, lambda N, M: 1])
    _check(library().sk_finish(plan, _buf(d_q, b_q, "device", "q"),
                               _buf(d_neff, b_n, "device", "neff"), F,
                               _buf(sk, b_sk, "device", "sk"), _buf(mask, b_m, "device", "mask"),
                               _stream(stream)))


def _host_call(fn, plan, h_in, n_frames, h_sk, h_mask, stream):
    F = int(n_frames)
    b_in, b_sk, b_m = _sizes(_plan_shape.get(plan), F, [
        lambda N, M: M * N, lambda N, M: 4, lambda N, M: 1])
    _check(fn(plan, _buf(h_in, b_in, "host", "h_in"), F, _buf(h_sk, b_sk, "host", "h_sk"),
              _buf(h_mask, b_m, "host", "h_mask"), _stream(stream)))


def sk_flag_host(plan, h_in, n_frames, h_sk, h_mask, stream=None):
    _host_call(library().sk_flag_host, plan, h_in, n_frames, h_sk, h_mask, stream)


def sk_flag_host_noalloc(plan, h_in, n_frames, h_sk, h_mask, stream=None):
    """sk_flag_host for callers that cannot allocate device memory: stages through a
    fixed array inside the library (at most SK_NOALLOC_MAX_BYTES input bytes and
    SK_NOALLOC_MAX_FRAMES frames per call)."""
    _host_call(library().sk_flag_host_noalloc, plan, h_in, n_frames, h_sk, h_mask, stream)


# ---------------------------------------------------------------- batched

def sk_batch_create(items, device=0) -> int:
    """items: sequence of (plan, d_in, n_frames, d_sk, d_mask)."""
    arr = (sk_batch_item_t * len(items))()
    for k, (plan, d_in, n, sk, mask) in enumerate(items):
        b_in, b_sk, b_m = _sizes(_plan_shape.get(plan), int(n), [
            lambda N, M: M * N, lambda N, M: 4, lambda N, M: 1])
        arr[k].plan = plan
        arr[k].d_in = _buf(d_in, b_in, "device", f"item {k} d_in")
        arr[k].n_frames = int(n)
        arr[k].d_sk = _buf(sk, b_sk, "device", f"item {k} sk")
        arr[k].d_mask = _buf(mask, b_m, "device", f"item {k} mask")
    h = ctypes.c_void_p()
    _check(library().sk_batch_create(arr, len(items), int(device), ctypes.byref(h)))
    return h.value


def sk_batch_run(batch, stream=None):
    _check(library().sk_batch_run(batch, _stream(stream)))


def sk_batch_launches(batch) -> int:
    n = ctypes.c_int32()
    _check(library().sk_batch_launches(batch, ctypes.byref(n)))
    return n.value


def sk_batch_destroy(batch):
    _check(library().sk_batch_destroy(batch))


# ---------------------------------------------------------------- serving

def sk_server_create(device=0, hbm_budget_bytes=1 << 34) -> int:
    h = ctypes.c_void_p()
    _check(library().sk_server_create(int(device), int(hbm_budget_bytes), ctypes.byref(h)))
    return h.value


def sk_server_destroy(server):
    _check(library().sk_server_destroy(server))
    for key in [k for k in _stream_shape if k[0] == server]:
        del _stream_shape[key]


def sk_stream_open(server, n_inputs, n_time, ring_frames=16, n_sigma=3.0, mean_offset=0.0,
                   flags=0, offset_table=None, layout=0) -> int:
    p, keep = _params(n_inputs, n_time, n_sigma, mean_offset, layout, flags, offset_table)
    sid = ctypes.c_int32()
    _check(library().sk_stream_open(server, ctypes.byref(p), int(ring_frames), ctypes.byref(sid)))
    _stream_shape[(server, sid.value)] = (int(n_inputs), int(n_time))
    return sid.value


def sk_stream_submit(server, stream_id, frame, frame_index=0) -> int:
    """frame: host bytes (numpy uint8 or CPU tensor) of one frame; returns the ticket."""
    (nb,) = _sizes(_stream_shape.get((server, int(stream_id))), 1, [lambda N, M: M * N])
    t = ctypes.c_int64()
    _check(library().sk_stream_submit(server, int(stream_id), _buf(frame, nb, "host", "frame"),
                                      int(frame_index), ctypes.byref(t)))
    return t.value


def sk_stream_submit_ref(server, stream_id, frame, frame_index=0) -> int:
    """frame: a CUDA tensor or a page-locked CPU tensor, read where it is (no copy);
    it must stay unchanged until the ticket completes.  Returns the ticket."""
    (nb,) = _sizes(_stream_shape.get((server, int(stream_id))), 1, [lambda N, M: M * N])
    t = ctypes.c_int64()
    _check(library().sk_stream_submit_ref(server, int(stream_id),
                                          _buf(frame, nb, "device", "frame"),
                                          int(frame_index), ctypes.byref(t)))
    return t.value


def sk_ticket_wait(server, ticket, timeout_us=-1):
    sk = ctypes.c_float()
    m = ctypes.c_uint8()
    _check(library().sk_ticket_wait(server, int(ticket), int(timeout_us), ctypes.byref(sk),
                                    ctypes.byref(m)))
    return sk.value, m.value


def sk_stream_drain(server, stream_id, timeout_us=-1):
    _check(library().sk_stream_drain(server, int(stream_id), int(timeout_us)))


def sk_stream_get_state(server, stream_id) -> bytes:
    n = ctypes.c_size_t(0)
    _check(library().sk_stream_get_state(server, int(stream_id), None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(library().sk_stream_get_state(server, int(stream_id), buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def sk_stream_set_state(server, stream_id, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(library().sk_stream_set_state(server, int(stream_id), buf, len(state)))


def sk_stream_close(server, stream_id):
    _check(library().sk_stream_close(server, int(stream_id)))
    _stream_shape.pop((server, int(stream_id)), None)


def sk_server_stats(server) -> dict:
    s = sk_server_stats_t()
    _check(library().sk_server_stats(server, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in sk_server_stats_t._fields_}


def sk_stream_stats(server, stream_id) -> dict:
    s = sk_stream_stats_t()
    _check(library().sk_stream_stats(server, int(stream_id), ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in sk_stream_stats_t._fields_ if k != "pad"}


def sk_server_replay(server, stream_ids, pools, frames_per_stream, cadence_s, jitter_mean_s,
                     paced=True, threads=8, seed=1, by_reference=False):
    """Replay frame pools (one uint8 array [pool, M*N] per stream) into open streams.
    by_reference: submit with sk_stream_submit_ref; the pools must then be page-locked
    CPU tensors or CUDA tensors (2-D, contiguous)."""
    n = len(stream_ids)
    if by_reference:
        for p in pools:
            _buf(p, None, "device", "pool")
        ptrs = (ctypes.c_void_p * n)(*[p.data_ptr() for p in pools])
        npool = (ctypes.c_int32 * n)(*[int(p.shape[0]) for p in pools])
    else:
        pools = [np.ascontiguousarray(p, dtype=np.uint8) for p in pools]
        ptrs = (ctypes.c_void_p * n)(*[p.ctypes.data for p in pools])
        npool = (ctypes.c_int32 * n)(*[p.shape[0] for p in pools])
    ids = (ctypes.c_int32 * n)(*stream_ids)
    r = sk_replay_t(n, int(threads), ctypes.cast(ids, ctypes.c_void_p).value,
                    ctypes.cast(ptrs, ctypes.c_void_p).value,
                    ctypes.cast(npool, ctypes.c_void_p).value, int(frames_per_stream),
                    float(cadence_s), float(jitter_mean_s), 1 if paced else 0,
                    1 if by_reference else 0, int(seed))
    out = sk_replay_result_t()
    _check(library().sk_server_replay(server, ctypes.byref(r), ctypes.byref(out)))
    return {k: getattr(out, k) for k, _ in sk_replay_result_t._fields_}


# ------------------------------------------------------------------- misc

def sk_digitisation_offset(sigma) -> float:
    d = ctypes.c_double()
    _check(library().sk_digitisation_offset(float(sigma), ctypes.byref(d)))
    return d.value


def sk_selftest_conversions(device: int = 0):
    """(cases checked, mismatches) of the kernels' exact conversions against CUDA's
    conversion intrinsics on `device`."""
    n = ctypes.c_int64()
    bad = ctypes.c_int64()
    _check(library().sk_selftest_conversions(int(device), ctypes.byref(n), ctypes.byref(bad)))
    return n.value, bad.value


def sk_selftest_slot_wait(plan, spin_limit: int = 16, stream=None) -> bool:
    """Runs the kernels' bounded slot wait against a slot that is never freed, with
    a bound of spin_limit polls; True if the wait gave up and raised the plan's
    error word (the plan's next call then reports SK_ERR_TIMEOUT)."""
    out = ctypes.c_int32()
    _check(library().sk_selftest_slot_wait(plan, int(spin_limit), ctypes.byref(out),
                                           _stream(stream)))
    return bool(out.value)


def sk_last_error() -> str:
    return library().sk_last_error().decode(errors="replace")
