"""Thin Python binding of libhd.so.

The ``hd_*`` functions mirror the C ABI of ``include/hd.h`` one to one (plain
integers for pointers and the CUDA stream).  ``decode``/``encode`` add only
argument marshalling for PyTorch tensors: device pointers, sizes and the
current CUDA stream.  Every step of the decode runs in the library's kernels;
there is no fallback of any kind, and a missing library raises.
"""
from __future__ import annotations

import ctypes
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libhd.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "hd.h")

HD_OK = 0
HD_ERR_INVALID_N = 1
HD_ERR_NULL = 2
HD_ERR_SIZE = 3
HD_ERR_ALIGN = 4
HD_ERR_CAPACITY = 5
HD_ERR_TIMEOUT = 6
HD_ERR_CUDA = 7
HD_ERR_INVALID_ARG = 8

SYN_NONE, SYN_U8, SYN_U16 = 0, 1, 2

_lib = None

_c = ctypes
_vp, _u32, _u64, _i32 = _c.c_void_p, _c.c_uint32, _c.c_uint64, _c.c_int

class VariantInfo(ctypes.Structure):
    """Mirror of hd_variant_info."""
    _fields_ = [("index", _u32), ("n", _u32), ("syn_type", _u32), ("codewords_per_thread", _u32),
                ("threads", _u32), ("stages", _u32), ("inplace", _u32), ("smem_bytes", _u32),
                ("chunk_codewords", _u64), ("blocks_per_sm", _c.c_int32), ("measured_us", _c.c_float),
                ("table_lookup", _u32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_VIP = _c.POINTER(VariantInfo)


class Packet(ctypes.Structure):
    """Mirror of hd_packet."""
    _fields_ = [("in_", _vp), ("out", _vp), ("syndromes", _vp), ("num_codewords", _u64), ("n", _u32),
                ("syn_type", _u32)]


class PlanInfo(ctypes.Structure):
    """Mirror of hd_plan_info."""
    _fields_ = [("num_packets", _u32), ("num_tiles", _u32), ("full_tiles", _u32), ("warps_per_cta", _u32),
                ("stages", _u32), ("smem_bytes", _u32), ("variant", _u32), ("num_variants", _u32),
                ("codewords", _u64), ("in_bytes", _u64), ("out_bytes", _u64), ("syn_bytes", _u64),
                ("measured_us", _c.c_float), ("table_lookup", _u32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class StreamJob(ctypes.Structure):
    """Mirror of hd_stream_job."""
    _fields_ = [("stream", _vp), ("out_bits", _vp), ("syndromes", _vp), ("err_count", _vp),
                ("num_codewords", _u64), ("n", _u32), ("syn_type", _u32)]


class HostJob(ctypes.Structure):
    _fields_ = [("host_stream", _c.c_void_p), ("host_out", _c.c_void_p), ("host_syndromes", _c.c_void_p),
                ("host_err_count", _c.c_void_p), ("num_codewords", _c.c_uint64), ("n", _c.c_uint32),
                ("syn_type", _c.c_uint32)]


class ServerConfig(ctypes.Structure):
    """Mirror of hd_server_config."""
    _fields_ = [("max_waves", _u32), ("max_wave_packets", _u32), ("max_wave_tiles", _u32),
                ("queue_capacity", _u32), ("mem_cap_bytes", _u64), ("host_staging_bytes", _u64)]


class Completion(ctypes.Structure):
    """Mirror of hd_completion."""
    _fields_ = [("tag", _u64), ("err_count", _u64), ("t_submit_ns", _u64), ("t_admit_ns", _u64),
                ("t_done_ns", _u64), ("status", _c.c_int32)]


class ServerStats(ctypes.Structure):
    """Mirror of hd_server_stats."""
    _fields_ = [("submitted", _u64), ("completed", _u64), ("rejected", _u64), ("waves", _u64),
                ("max_resident_bytes", _u64), ("mean_wave_packets", _c.c_double), ("p50_latency_us", _c.c_double),
                ("p99_latency_us", _c.c_double), ("max_latency_us", _c.c_double), ("duration_s", _c.c_double),
                ("backpressure_waits", _u64), ("host_waves", _u64), ("mean_t_in_us", _c.c_double),
                ("mean_t_decode_us", _c.c_double), ("mean_t_out_us", _c.c_double),
                ("p999_latency_us", _c.c_double), ("max_submit_lag_us", _c.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_PKP = _c.POINTER(Packet)
_PIP = _c.POINTER(PlanInfo)
_SCP = _c.POINTER(ServerConfig)
_CMP = _c.POINTER(Completion)
_SSP = _c.POINTER(ServerStats)

# name -> (restype, argtypes); every entry is declared in include/hd.h
SIGNATURES = {
    "hd_variant_count": (_i32, [_u32, _i32, _c.POINTER(_u32)]),
    "hd_variant_info_get": (_i32, [_u32, _i32, _u32, _VIP]),
    "hd_variant_select": (_i32, [_u32, _i32, _c.c_int32]),
    "hd_variant_current": (_i32, [_u32, _i32, _VIP]),
    "hd_autotune": (_i32, [_u32, _i32, _u64, _u32, _vp, _VIP]),
    "hd_decode": (_i32, [_vp, _u64, _u32, _u64, _vp, _vp, _i32, _vp, _vp]),
    "hd_decode_streams": (_i32, [_c.POINTER(StreamJob), _u32, _vp]),
    "hd_plan_create": (_i32, [_PKP, _u32, _c.POINTER(_vp)]),
    "hd_plan_launch": (_i32, [_vp, _vp, _vp]),
    "hd_plan_autotune": (_i32, [_vp, _u32, _vp, _PIP]),
    "hd_plan_select": (_i32, [_vp, _u32]),
    "hd_plan_get_info": (_i32, [_vp, _PIP]),
    "hd_plan_destroy": (None, [_vp]),
    "hd_decode_batch": (_i32, [_PKP, _u32, _vp, _vp]),
    "hd_decode_batch_noalloc": (_i32, [_PKP, _u32, _vp, _vp]),
    "hd_batch_tiles": (_i32, [_PKP, _u32, _c.POINTER(_u64)]),
    "hd_server_create": (_i32, [_SCP, _c.POINTER(_vp)]),
    "hd_server_submit": (_i32, [_vp, _PKP, _u64]),
    "hd_server_submit_host": (_i32, [_vp, _PKP, _u64]),
    "hd_server_inject_launch_failures": (_i32, [_vp, _u32]),
    "hd_server_poll": (_i32, [_vp, _CMP, _u32, _c.POINTER(_u32)]),
    "hd_server_drain": (_i32, [_vp, _u64]),
    "hd_server_get_stats": (_i32, [_vp, _SSP]),
    "hd_server_destroy": (None, [_vp]),
    "hd_serve_trace": (_i32, [_SCP, _PKP, _c.POINTER(_c.c_double), _u32, _CMP, _SSP]),
    "hd_serve_trace_host": (_i32, [_SCP, _PKP, _c.POINTER(_c.c_double), _u32, _CMP, _SSP]),
    "hd_encode": (_i32, [_vp, _u32, _u64, _vp, _vp]),
    "hd_short_params": (_i32, [_u32, _c.POINTER(_u32), _c.POINTER(_u32)]),
    "hd_segment_params": (_i32, [_u32, _u32, _c.POINTER(_u32), _c.POINTER(_u32), _c.POINTER(_u32)]),
    "hd_decode_short": (_i32, [_vp, _u64, _u32, _u64, _vp, _vp, _i32, _vp, _vp, _vp]),
    "hd_encode_short": (_i32, [_vp, _u32, _u64, _vp, _vp]),
    "hd_short_plan_create": (_i32, [_u32, _c.POINTER(_vp)]),
    "hd_decode_short_plan": (_i32, [_vp, _vp, _u64, _u64, _vp, _vp, _i32, _vp, _vp, _vp]),
    "hd_short_plan_destroy": (None, [_vp]),
    "hd_short_variant_count": (_i32, [_c.POINTER(_u32)]),
    "hd_short_variant_select": (_i32, [_c.c_int32]),
    "hd_short_autotune": (_i32, [_u32, _u64, _u32, _vp, _c.POINTER(_c.c_int32)]),
    "hd_decode_secded": (_i32, [_vp, _u64, _u32, _u64, _vp, _vp, _i32, _vp, _vp, _vp]),
    "hd_encode_secded": (_i32, [_vp, _u32, _u64, _vp, _vp]),
    "hd_decode_host_batch": (_i32, [_c.POINTER(HostJob), _u32, _u64, _u32]),
    "hd_decode_host": (_i32, [_vp, _u64, _u32, _u64, _vp, _vp, _i32, _c.POINTER(_c.c_ulonglong), _u64, _u32]),
    "hd_secded_variant_count": (_i32, [_u32, _i32, _c.POINTER(_u32)]),
    "hd_secded_variant_info_get": (_i32, [_u32, _i32, _u32, _VIP]),
    "hd_secded_variant_select": (_i32, [_u32, _i32, _c.c_int32]),
    "hd_set_max_ctas": (_i32, [_u32]),
    "hd_get_max_ctas": (_u32, []),
    "hd_status_string": (_c.c_char_p, [_i32]),
    "hd_device_status": (_i32, [_c.POINTER(_u32)]),
    "hd_launch_count": (_u64, []),
    "hd_version": (_i32, []),
}


class HDError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__(f"{what}: {status_string(status)}" if what else status_string(status))


def lib() -> ctypes.CDLL:
    """Load libhd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1412_6862_gb300.build` "
                               "(the decoder has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions declared in include/hd.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hd_[a-z0-9_]+)\s*\(", text)))


def status_string(status: int) -> str:
    try:
        return lib().hd_status_string(int(status)).decode()
    except RuntimeError:
        return f"hd_status {status}"


def check(status: int, what: str = "") -> None:
    if status != HD_OK:
        raise HDError(status, what)


# ----------------------------------------------------------------------------
# C-ABI mirrors
# ----------------------------------------------------------------------------
def hd_decode(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count, cuda_stream) -> int:
    return lib().hd_decode(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count,
                           cuda_stream)


def stream_jobs(jobs) -> ctypes.Array:
    """ctypes array of hd_stream_job from (stream_ptr, n, num_codewords, out_ptr, syn_ptr, syn_type, err_ptr)."""
    arr = (StreamJob * max(1, len(jobs)))()
    for i, (a, n, N, o, sy, st, e) in enumerate(jobs):
        arr[i] = StreamJob(a, o, sy, e, N, n, st if sy else SYN_NONE)
    return arr


def hd_decode_streams(jobs_array, num_jobs: int, cuda_stream) -> int:
    return lib().hd_decode_streams(jobs_array, num_jobs, cuda_stream)


def hd_decode_host(host_stream, in_bits, n, num_codewords, host_out, host_syndromes, syn_type, chunk_codewords=0,
                   depth=0):
    """C-ABI mirror taking host pointers (ints); returns (status, err_count)."""
    err = _c.c_ulonglong(0)
    rc = lib().hd_decode_host(host_stream, in_bits, n, num_codewords, host_out, host_syndromes, syn_type,
                              ctypes.byref(err), chunk_codewords, depth)
    return rc, int(err.value)


def hd_decode_host_batch(jobs, chunk_codewords: int = 0, depth: int = 0):
    """jobs: list of (host_stream_ptr, n, num_codewords, host_out_ptr, host_syn_ptr or None, syn_type).
    Returns (status, [err_count per job])."""
    arr = (HostJob * max(1, len(jobs)))()
    errs = (_c.c_ulonglong * max(1, len(jobs)))()
    for i, (hs, n, N, ho, hsyn, st) in enumerate(jobs):
        arr[i] = HostJob(hs, ho, hsyn, ctypes.addressof(errs) + 8 * i, N, n, st)
    rc = lib().hd_decode_host_batch(arr, len(jobs), chunk_codewords, depth)
    return rc, [int(errs[i]) for i in range(len(jobs))]


def decode_host(stream_words, n: int, num_codewords: int, syn_type: int = SYN_U8, out=None, syndromes=None,
                chunk_codewords: int = 0, depth: int = 0):
    """Decode host (numpy or CPU-tensor) words; pinned buffers overlap the copies.
    Returns (out words, syndromes or None, err_count)."""
    import numpy as np
    m, k = code_params(n)
    src = stream_words
    if out is None:
        out = np.zeros(max(1, words_for(num_codewords * k)), dtype=np.uint32)
    if syndromes is None and syn_type != SYN_NONE:
        syndromes = np.zeros(max(1, num_codewords), dtype=np.uint8 if syn_type == SYN_U8 else np.uint16)

    def ptr(a):
        if a is None:
            return None
        return int(a.data_ptr()) if hasattr(a, "data_ptr") else int(a.ctypes.data)

    rc, err = hd_decode_host(ptr(src), n * num_codewords, n, num_codewords, ptr(out),
                             ptr(syndromes) if syn_type != SYN_NONE else None, syn_type, chunk_codewords, depth)
    check(rc, "hd_decode_host")
    return out, syndromes, err


def hd_encode(data_bits, n, num_codewords, stream, cuda_stream) -> int:
    return lib().hd_encode(data_bits, n, num_codewords, stream, cuda_stream)


def hd_variant_count(n: int, syn_type: int) -> int:
    c = _u32(0)
    check(lib().hd_variant_count(n, syn_type, ctypes.byref(c)), "hd_variant_count")
    return int(c.value)


def hd_variant_info_get(n: int, syn_type: int, ordinal: int) -> dict:
    info = VariantInfo()
    check(lib().hd_variant_info_get(n, syn_type, ordinal, ctypes.byref(info)), "hd_variant_info_get")
    return info.as_dict()


def hd_variant_select(n: int, syn_type: int, ordinal: int) -> None:
    check(lib().hd_variant_select(n, syn_type, ordinal), "hd_variant_select")


def hd_variant_current(n: int, syn_type: int) -> dict:
    info = VariantInfo()
    check(lib().hd_variant_current(n, syn_type, ctypes.byref(info)), "hd_variant_current")
    return info.as_dict()


def hd_secded_variant_count(n: int, syn_type: int) -> int:
    c = _u32(0)
    check(lib().hd_secded_variant_count(n, syn_type, ctypes.byref(c)), "hd_secded_variant_count")
    return int(c.value)


def hd_secded_variant_info_get(n: int, syn_type: int, ordinal: int) -> dict:
    info = VariantInfo()
    check(lib().hd_secded_variant_info_get(n, syn_type, ordinal, ctypes.byref(info)), "hd_secded_variant_info_get")
    return info.as_dict()


def hd_secded_variant_select(n: int, syn_type: int, ordinal: int) -> None:
    check(lib().hd_secded_variant_select(n, syn_type, ordinal), "hd_secded_variant_select")


def hd_set_max_ctas(max_ctas: int) -> None:
    check(lib().hd_set_max_ctas(max_ctas), "hd_set_max_ctas")


def hd_get_max_ctas() -> int:
    return int(lib().hd_get_max_ctas())


def hd_autotune(n: int, syn_type: int, num_codewords: int, reps: int = 5, cuda_stream=None) -> dict:
    info = VariantInfo()
    check(lib().hd_autotune(n, syn_type, num_codewords, reps, _stream_handle(cuda_stream), ctypes.byref(info)),
          "hd_autotune")
    return info.as_dict()


def packet_table(packets) -> ctypes.Array:
    """ctypes array of hd_packet from (in_ptr, out_ptr, syn_ptr, num_codewords, n, syn_type) tuples."""
    arr = (Packet * max(1, len(packets)))()
    for i, (a, b, c, N, n, st) in enumerate(packets):
        arr[i] = Packet(a, b, c, N, n, st)
    return arr


def hd_plan_create(table, num_packets: int) -> int:
    plan = _vp()
    check(lib().hd_plan_create(table, num_packets, ctypes.byref(plan)), "hd_plan_create")
    return plan.value


def hd_plan_launch(plan: int, err_counts, cuda_stream) -> int:
    return lib().hd_plan_launch(plan, err_counts, cuda_stream)


def hd_plan_autotune(plan: int, reps: int = 3, cuda_stream=None) -> dict:
    info = PlanInfo()
    check(lib().hd_plan_autotune(plan, reps, _stream_handle(cuda_stream), ctypes.byref(info)), "hd_plan_autotune")
    return info.as_dict()


def hd_plan_select(plan: int, variant: int) -> None:
    check(lib().hd_plan_select(plan, variant), "hd_plan_select")


def hd_plan_get_info(plan: int) -> dict:
    info = PlanInfo()
    check(lib().hd_plan_get_info(plan, ctypes.byref(info)), "hd_plan_get_info")
    return info.as_dict()


def hd_plan_destroy(plan: int) -> None:
    lib().hd_plan_destroy(plan)


def hd_decode_batch(table, num_packets: int, err_counts, cuda_stream) -> int:
    return lib().hd_decode_batch(table, num_packets, err_counts, cuda_stream)


def hd_decode_batch_noalloc(table, num_packets: int, err_counts, cuda_stream) -> int:
    return lib().hd_decode_batch_noalloc(table, num_packets, err_counts, cuda_stream)


def hd_batch_tiles(table, num_packets: int) -> int:
    """Tiles the packets are cut into (host-only)."""
    t = _u64(0)
    check(lib().hd_batch_tiles(table, num_packets, ctypes.byref(t)), "hd_batch_tiles")
    return int(t.value)


def server_config(max_waves=4, max_wave_packets=4096, max_wave_tiles=65536, queue_capacity=1 << 16,
                  mem_cap_bytes=4 << 30, host_staging_bytes=0) -> ServerConfig:
    return ServerConfig(max_waves, max_wave_packets, max_wave_tiles, queue_capacity, mem_cap_bytes,
                        host_staging_bytes)


def hd_serve_trace(cfg: ServerConfig, table, arrival_s, num: int, host: bool = False):
    """Replay an arrival trace (host=True: the packets' buffers are pinned host
    memory, hd_serve_trace_host); returns (completions array, stats dict)."""
    import numpy as np
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    comps = (Completion * max(1, num))()
    st = ServerStats()
    fn = lib().hd_serve_trace_host if host else lib().hd_serve_trace
    check(fn(ctypes.byref(cfg), table, arr.ctypes.data_as(_c.POINTER(_c.c_double)), num, comps, ctypes.byref(st)),
          "hd_serve_trace_host" if host else "hd_serve_trace")
    return comps, st.as_dict()


class Server:
    """A continuous-batching server (hd_server_*)."""

    def __init__(self, cfg: ServerConfig | None = None):
        self.cfg = cfg or server_config()
        h = _vp()
        check(lib().hd_server_create(ctypes.byref(self.cfg), ctypes.byref(h)), "hd_server_create")
        self.handle = h.value

    def submit(self, in_ptr, out_ptr, syn_ptr, num_codewords, n, syn_type, tag) -> int:
        pk = Packet(in_ptr, out_ptr, syn_ptr, num_codewords, n, syn_type if syn_ptr else SYN_NONE)
        return lib().hd_server_submit(self.handle, ctypes.byref(pk), tag)

    def submit_host(self, in_ptr, out_ptr, syn_ptr, num_codewords, n, syn_type, tag) -> int:
        """Queue a packet whose buffers are pinned host memory."""
        pk = Packet(in_ptr, out_ptr, syn_ptr, num_codewords, n, syn_type if syn_ptr else SYN_NONE)
        return lib().hd_server_submit_host(self.handle, ctypes.byref(pk), tag)

    def inject_launch_failures(self, count: int) -> None:
        check(lib().hd_server_inject_launch_failures(self.handle, count), "hd_server_inject_launch_failures")

    def poll(self, max_n: int = 4096):
        buf = (Completion * max_n)()
        c = _u32(0)
        rc = lib().hd_server_poll(self.handle, buf, max_n, ctypes.byref(c))
        return rc, [buf[i] for i in range(c.value)]

    def drain(self, timeout_s: float = 60.0) -> int:
        return lib().hd_server_drain(self.handle, int(timeout_s * 1e9))

    def stats(self) -> dict:
        st = ServerStats()
        check(lib().hd_server_get_stats(self.handle, ctypes.byref(st)), "hd_server_get_stats")
        return st.as_dict()

    def close(self) -> None:
        if self.handle:
            lib().hd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A batched-decode plan over device tensors.  ``packets`` holds
    (in, out, syndromes or None, num_codewords, n, syn_type) with tensors."""

    def __init__(self, packets):
        self._keep = packets
        self.table = packet_table([(_ptr(a), _ptr(b), _ptr(c), N, n, st if c is not None else SYN_NONE)
                                   for a, b, c, N, n, st in packets])
        self.handle = hd_plan_create(self.table, len(packets))
        self.num_packets = len(packets)

    def launch(self, err_counts=None, cuda_stream=None) -> None:
        check(hd_plan_launch(self.handle, _ptr(err_counts), _stream_handle(cuda_stream)), "hd_plan_launch")

    def autotune(self, reps: int = 3, cuda_stream=None) -> dict:
        return hd_plan_autotune(self.handle, reps, cuda_stream)

    def select(self, variant: int) -> None:
        hd_plan_select(self.handle, variant)

    def info(self) -> dict:
        return hd_plan_get_info(self.handle)

    def close(self) -> None:
        if self.handle:
            hd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hd_device_status() -> int:
    v = _u32(0)
    check(lib().hd_device_status(ctypes.byref(v)), "hd_device_status")
    return int(v.value)


def hd_launch_count() -> int:
    return int(lib().hd_launch_count())


def hd_version() -> int:
    return int(lib().hd_version())


# ----------------------------------------------------------------------------
# PyTorch marshalling
# ----------------------------------------------------------------------------
def code_params(n: int) -> tuple[int, int]:
    """(m, k) for n = 2^m - 1, 2 <= m <= 8."""
    for m in range(2, 9):
        if n == (1 << m) - 1:
            return m, n - m
    raise HDError(HD_ERR_INVALID_N, f"n={n}")


def words_for(bits: int) -> int:
    return (int(bits) + 31) // 32


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def decode(stream_words, n: int, num_codewords: int, syn_type: int = SYN_U8, out=None, syndromes=None,
           err_count=None, cuda_stream=None):
    """Decode a device tensor of packed stream words (int32/uint32, 16-byte aligned).

    Returns (out_words int32 tensor, syndromes tensor or None, err_count int64
    tensor of one element).  Outputs are allocated when not given."""
    import torch
    m, k = code_params(n)
    dev = stream_words.device
    if out is None:
        out = torch.empty(max(1, words_for(num_codewords * k)), dtype=torch.int32, device=dev)
    if syndromes is None and syn_type != SYN_NONE:
        dt = torch.uint8 if syn_type == SYN_U8 else torch.int16
        syndromes = torch.empty(max(1, num_codewords), dtype=dt, device=dev)
    if err_count is None:
        err_count = torch.empty(1, dtype=torch.int64, device=dev)
    rc = hd_decode(_ptr(stream_words), n * num_codewords, n, num_codewords, _ptr(out),
                   _ptr(syndromes) if syn_type != SYN_NONE else None, syn_type, _ptr(err_count),
                   _stream_handle(cuda_stream))
    check(rc, "hd_decode")
    return out, syndromes, err_count


def hd_short_params(n: int) -> tuple[int, int]:
    """(r, k) of the shortened code of length n."""
    r, k = _u32(0), _u32(0)
    check(lib().hd_short_params(n, ctypes.byref(r), ctypes.byref(k)), f"hd_short_params n={n}")
    return int(r.value), int(k.value)


def hd_segment_params(packet_bytes: int, t: int) -> tuple[int, int, int]:
    """(n, k, r) of the segments of a packet of packet_bytes bytes split into t."""
    n, k, r = _u32(0), _u32(0), _u32(0)
    check(lib().hd_segment_params(packet_bytes, t, ctypes.byref(n), ctypes.byref(k), ctypes.byref(r)),
          f"hd_segment_params M={packet_bytes} t={t}")
    return int(n.value), int(k.value), int(r.value)


def hd_decode_short(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count, detected_count,
                    cuda_stream) -> int:
    return lib().hd_decode_short(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count,
                                 detected_count, cuda_stream)


def hd_encode_short(data_bits, n, num_codewords, stream, cuda_stream) -> int:
    return lib().hd_encode_short(data_bits, n, num_codewords, stream, cuda_stream)


def hd_short_variant_count() -> int:
    c = _u32(0)
    check(lib().hd_short_variant_count(ctypes.byref(c)), "hd_short_variant_count")
    return int(c.value)


def hd_short_variant_select(ordinal: int) -> None:
    check(lib().hd_short_variant_select(ordinal), "hd_short_variant_select")


def hd_short_autotune(n: int, num_codewords: int, reps: int = 5, cuda_stream=None) -> int:
    """Time every tile configuration for length n; returns the chosen ordinal (-1: single kernel)."""
    chosen = _c.c_int32(-2)
    check(lib().hd_short_autotune(n, num_codewords, reps, _stream_handle(cuda_stream), ctypes.byref(chosen)),
          "hd_short_autotune")
    return int(chosen.value)


def decode_short(stream_words, n: int, num_codewords: int, syn_type: int = SYN_U16, out=None, syndromes=None,
                 counts=None, cuda_stream=None):
    """Decode a device tensor of shortened-code segments of length n.

    Returns (out_words, syndromes or None, counts) where counts is an int64
    tensor of two elements: [nonzero syndromes, syndromes past n]."""
    import torch
    r, k = hd_short_params(n)
    dev = stream_words.device
    if out is None:
        out = torch.empty(max(4, words_for(num_codewords * k)), dtype=torch.int32, device=dev)
    if syndromes is None and syn_type != SYN_NONE:
        dt = torch.uint8 if syn_type == SYN_U8 else torch.int16
        syndromes = torch.empty(max(16, num_codewords), dtype=dt, device=dev)
    if counts is None:
        counts = torch.empty(2, dtype=torch.int64, device=dev)
    rc = hd_decode_short(_ptr(stream_words), n * num_codewords, n, num_codewords, _ptr(out),
                         _ptr(syndromes) if syn_type != SYN_NONE else None, syn_type, _ptr(counts),
                         _ptr(counts) + 8, _stream_handle(cuda_stream))
    check(rc, "hd_decode_short")
    return out, syndromes, counts


class ShortPlan:
    """The tables of one shortened-code length (hd_short_plan_*): decodes with
    it allocate nothing and may run inside a stream capture."""

    def __init__(self, n: int):
        h = _vp()
        check(lib().hd_short_plan_create(n, ctypes.byref(h)), "hd_short_plan_create")
        self.handle, self.n = h.value, n

    def decode(self, stream_words, num_codewords: int, syn_type: int = SYN_U16, out=None, syndromes=None,
               counts=None, cuda_stream=None):
        """As decode_short(); returns (out_words, syndromes or None, counts)."""
        import torch
        r, k = hd_short_params(self.n)
        dev = stream_words.device
        if out is None:
            out = torch.empty(max(4, words_for(num_codewords * k)), dtype=torch.int32, device=dev)
        if syndromes is None and syn_type != SYN_NONE:
            dt = torch.uint8 if syn_type == SYN_U8 else torch.int16
            syndromes = torch.empty(max(16, num_codewords), dtype=dt, device=dev)
        if counts is None:
            counts = torch.empty(2, dtype=torch.int64, device=dev)
        rc = lib().hd_decode_short_plan(self.handle, _ptr(stream_words), self.n * num_codewords, num_codewords,
                                        _ptr(out), _ptr(syndromes) if syn_type != SYN_NONE else None, syn_type,
                                        _ptr(counts), _ptr(counts) + 8, _stream_handle(cuda_stream))
        check(rc, "hd_decode_short_plan")
        return out, syndromes, counts

    def close(self) -> None:
        if self.handle:
            lib().hd_short_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode_short(data_words, n: int, num_codewords: int, out=None, cuda_stream=None):
    """Encode a device tensor of packed messages into segments of length n."""
    import torch
    if out is None:
        out = torch.empty(max(4, words_for(num_codewords * n)), dtype=torch.int32, device=data_words.device)
    check(hd_encode_short(_ptr(data_words), n, num_codewords, _ptr(out), _stream_handle(cuda_stream)),
          "hd_encode_short")
    return out


def hd_decode_secded(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count, detected_count,
                     cuda_stream) -> int:
    return lib().hd_decode_secded(stream, in_bits, n, num_codewords, out_bits, syndromes, syn_type, err_count,
                                  detected_count, cuda_stream)


def hd_encode_secded(data_bits, n, num_codewords, stream, cuda_stream) -> int:
    return lib().hd_encode_secded(data_bits, n, num_codewords, stream, cuda_stream)


def decode_secded(stream_words, n: int, num_codewords: int, syn_type: int = SYN_U16, out=None, syndromes=None,
                  counts=None, cuda_stream=None):
    """Decode a device tensor of SECDED codewords (n + 1 bits each).  Returns
    (out_words, syndromes or None, counts) with counts = [nonzero syndromes, detected]."""
    import torch
    m, k = code_params(n)
    dev = stream_words.device
    if out is None:
        out = torch.empty(max(4, words_for(num_codewords * k)), dtype=torch.int32, device=dev)
    if syndromes is None and syn_type != SYN_NONE:
        dt = torch.uint8 if syn_type == SYN_U8 else torch.int16
        syndromes = torch.empty(max(16, num_codewords), dtype=dt, device=dev)
    if counts is None:
        counts = torch.empty(2, dtype=torch.int64, device=dev)
    rc = hd_decode_secded(_ptr(stream_words), (n + 1) * num_codewords, n, num_codewords, _ptr(out),
                          _ptr(syndromes) if syn_type != SYN_NONE else None, syn_type, _ptr(counts),
                          _ptr(counts) + 8, _stream_handle(cuda_stream))
    check(rc, "hd_decode_secded")
    return out, syndromes, counts


def encode_secded(data_words, n: int, num_codewords: int, out=None, cuda_stream=None):
    """Encode a device tensor of packed messages into SECDED codewords."""
    import torch
    if out is None:
        out = torch.empty(max(4, words_for(num_codewords * (n + 1))), dtype=torch.int32, device=data_words.device)
    check(hd_encode_secded(_ptr(data_words), n, num_codewords, _ptr(out), _stream_handle(cuda_stream)),
          "hd_encode_secded")
    return out


def encode(data_words, n: int, num_codewords: int, out=None, cuda_stream=None):
    """Encode a device tensor of packed message bits; returns the stream words."""
    import torch
    if out is None:
        out = torch.empty(max(1, words_for(num_codewords * n)), dtype=torch.int32, device=data_words.device)
    check(hd_encode(_ptr(data_words), n, num_codewords, _ptr(out), _stream_handle(cuda_stream)), "hd_encode")
    return out
