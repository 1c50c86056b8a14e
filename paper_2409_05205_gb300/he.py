"""ctypes binding of libhe (include/he.h), one Python function per C entry point,
with the same names.  It only marshals arguments: device buffers are passed as
raw device addresses (an int, or any object with ``data_ptr()`` such as a
torch tensor), streams as raw ``cudaStream_t`` values (an int, or an object
with ``cuda_stream``).  Every step of the server path runs in the CUDA
library; if the library is missing, every call raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhe.so")

HE_OK, HE_ERR_ARG, HE_ERR_SHAPE, HE_ERR_UNSUPPORTED, HE_ERR_NOMEM, HE_ERR_CUDA, HE_ERR_TIMEOUT = range(7)
HE_COEFF, HE_NTT = 0, 1
HE_OUT_EXTRACTED, HE_OUT_PER_CHANNEL, HE_OUT_EXTRACTED_UNFOLDED = 0, 1, 2
HE_MAX_LIMBS = 16
HE_MAX_INTERLEAVE = 128
HE_DEVICE_NONE = -1
HE_FORM_PLAIN, HE_FORM_MASKED, HE_FORM_CLIENT = range(3)
HE_PHASE_NTT, HE_PHASE_REST, HE_PHASE_MAC, HE_PHASE_FINISH, HE_PHASE_RESCALE, HE_PHASE_FIN = range(6)

_STATUS = {0: "HE_OK", 1: "HE_ERR_ARG", 2: "HE_ERR_SHAPE", 3: "HE_ERR_UNSUPPORTED",
           4: "HE_ERR_NOMEM", 5: "HE_ERR_CUDA", 6: "HE_ERR_TIMEOUT"}


class HEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class he_conv_desc(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("ci", "co", "h", "w", "fh", "fw", "stride", "pad")]


class he_conv_layout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("s", "G", "H", "P", "hp", "h_out", "w_out", "M", "off_mult")]


class he_fc_layout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("n_in", "n_in_p", "n_out", "rows_per_poly", "P_fc")]


class he_layer_call(ctypes.Structure):
    _fields_ = [("filters", ctypes.c_void_p), ("d_in", ctypes.c_void_p), ("in_domain", ctypes.c_int),
                ("d_out", ctypes.c_void_p), ("B", ctypes.c_uint32), ("d_share", ctypes.c_void_p),
                ("d_share_out", ctypes.c_void_p), ("d_rescaled", ctypes.c_void_p)]


class he_op_counts(ctypes.Structure):
    _fields_ = [("fwd_ntts", ctypes.c_uint64), ("inv_ntts", ctypes.c_uint64), ("inv_len", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("cwms", ctypes.c_uint64), ("rotations", ctypes.c_uint64)]


class he_plan_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("split", "mac_item_kb", "mac_ctas_per_sm", "fused_max_nj",
                                               "tc_min_batch", "fc_direct", "groups", "fin_parts",
                                               "tw_smem", "mac_pdl", "l2_hints")]


class he_plan_info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("kernels_per_run", "ntt_items", "mac_items", "mac_ctas",
                                               "finish_items", "fused_items", "fc_items", "split_calls")] + \
               [("workspace_bytes", ctypes.c_uint64), ("tuning", he_plan_tuning)] + \
               [(n, ctypes.c_uint32) for n in ("tc_items", "tc_ctas", "tc_calls", "rescale_items",
                                              "rescale_fused_calls")]


class he_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("streams", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32)]


class he_request_stats(ctypes.Structure):
    _fields_ = [("arrive_ms", ctypes.c_double), ("done_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class he_server_report_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "finished", "failed", "batches", "batched_calls",
                                               "lanes", "bytes_in_use", "bytes_peak", "evictions")] + \
               [("batch_hist", ctypes.c_uint64 * 4)]


_lib = None

_vp, _u32, _i32, _sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_int, ctypes.c_size_t
_SIGS = {
    "he_params_create": [_u32, _u32, _vp, _u32, _i32, ctypes.POINTER(_vp)],
    "he_params_primes": [_vp, _vp],
    "he_params_psi": [_vp, _vp],
    "he_params_delta": [_vp, _vp],
    "he_params_reserve": [_vp, _sz],
    "he_conv_workspace_bytes": [_vp, ctypes.POINTER(he_conv_desc), _u32, ctypes.POINTER(_sz)],
    "he_fc_workspace_bytes": [_vp, _u32, ctypes.POINTER(_sz)],
    "he_params_destroy": [_vp],
    "he_conv_layout_query": [_vp, ctypes.POINTER(he_conv_desc), ctypes.POINTER(he_conv_layout)],
    "he_fc_layout_query": [_vp, _u32, _u32, ctypes.POINTER(he_fc_layout)],
    "he_conv_op_counts": [_vp, ctypes.POINTER(he_conv_desc), _i32, _i32, _u32, ctypes.POINTER(he_op_counts)],
    "he_fc_op_counts": [_vp, _u32, _u32, _i32, _i32, _u32, ctypes.POINTER(he_op_counts)],
    "he_pack_filters": [_vp, ctypes.POINTER(he_conv_desc), _vp, ctypes.POINTER(_vp)],
    "he_pack_filters_for_batch": [_vp, ctypes.POINTER(he_conv_desc), _vp, _u32, ctypes.POINTER(_vp)],
    "he_filters_tensor_core": [_vp, ctypes.POINTER(_u32)],
    "he_pack_masked": [_vp, ctypes.POINTER(he_conv_desc), _vp, _vp, ctypes.POINTER(_vp)],
    "he_conv_layer_masked": [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _u32, _vp],
    "he_pack_client": [_vp, ctypes.POINTER(he_conv_desc), _vp, _vp, ctypes.POINTER(_vp)],
    "he_rescale": [_vp, _vp, _vp, _u32, _vp],
    "he_conv_client": [_vp, _vp, _vp, _vp, _vp, _u32, _vp],
    "he_pack_fc": [_vp, _u32, _u32, _vp, _vp, ctypes.POINTER(_vp)],
    "he_pack_fc_masked": [_vp, _u32, _u32, _vp, _vp, _vp, ctypes.POINTER(_vp)],
    "he_fc_layer_masked": [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _u32, _vp],
    "he_pack_fc_client": [_vp, _u32, _u32, _vp, _vp, ctypes.POINTER(_vp)],
    "he_fc_client": [_vp, _vp, _vp, _vp, _vp, _u32, _vp],
    "he_filters_destroy": [_vp],
    "he_conv_layer": [_vp, _vp, _vp, _i32, _vp, _i32, _u32, _vp],
    "he_conv_layer_noalloc": [_vp, _vp, _vp, _i32, _vp, _i32, _u32, _vp],
    "he_fc_layer": [_vp, _vp, _vp, _i32, _vp, _i32, _u32, _vp],
    "he_bench_butterflies": [_vp, _u32, _u32, _vp, _vp],
    "he_ntt_forward": [_vp, _vp, _vp, _u32, _vp],
    "he_ntt_inverse": [_vp, _vp, _vp, _u32, _vp],
    "he_plan_create": [ctypes.POINTER(he_layer_call), _u32, ctypes.POINTER(_vp)],
    "he_plan_tuning_default": [ctypes.POINTER(he_plan_tuning)],
    "he_plan_create_tuned": [ctypes.POINTER(he_layer_call), _u32, ctypes.POINTER(he_plan_tuning), ctypes.POINTER(_vp)],
    "he_plan_workspace_bytes": [ctypes.POINTER(he_layer_call), _u32, ctypes.POINTER(_sz)],
    "he_plan_set_wait_limit": [_vp, _u32],
    "he_plan_set_checks": [_vp, _i32],
    "he_plan_autotune": [ctypes.POINTER(he_layer_call), _u32, _u32, _vp, ctypes.POINTER(he_plan_tuning),
                         ctypes.POINTER(_vp)],
    "he_plan_autotune_inflight": [ctypes.POINTER(he_layer_call), _u32, _u32, _u32, _vp,
                                  ctypes.POINTER(he_plan_tuning), ctypes.POINTER(_vp)],
    "he_plan_run": [_vp, _vp],
    "he_plan_run_host": [_vp, _vp, _vp, _vp],
    "he_plan_host_words": [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                           ctypes.POINTER(_u32)],
    "he_plan_run_phase": [_vp, _i32, _vp],
    "he_plan_query": [_vp, ctypes.POINTER(he_plan_info), _vp],
    "he_plan_check": [_vp],
    "he_plan_destroy": [_vp],
    "he_server_create": [ctypes.POINTER(he_server_config), ctypes.POINTER(_vp)],
    "he_server_add_model": [_vp, ctypes.POINTER(_vp), _u32, ctypes.POINTER(_u32)],
    "he_server_submit": [_vp, _u32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_uint64)],
    "he_server_wait": [_vp, ctypes.c_uint64, _u32, ctypes.POINTER(he_request_stats)],
    "he_server_report": [_vp, ctypes.POINTER(he_server_report_t)],
    "he_server_latencies": [_vp, _i32, ctypes.POINTER(ctypes.c_double), ctypes.c_uint64,
                            ctypes.POINTER(ctypes.c_uint64)],
    "he_server_destroy": [_vp],
    "he_sync": [_vp],
    "he_last_error": [],
}
_VOID = {"he_params_destroy", "he_filters_destroy", "he_plan_destroy", "he_server_destroy"}


def lib() -> ctypes.CDLL:
    """The loaded libhe.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it first (__graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = None if name in _VOID else (ctypes.c_char_p if name == "he_last_error" else ctypes.c_int)
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != HE_OK:
        raise HEError(status, lib().he_last_error().decode(errors="replace"))


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError(f"cannot take a device address of {type(x)}")


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _desc(d) -> he_conv_desc:
    if isinstance(d, he_conv_desc):
        return d
    return he_conv_desc(d["ci"], d["co"], d["h"], d["w"], d.get("fh", 3), d.get("fw", 3),
                        d.get("stride", 1), d.get("pad", 1))


# ----------------------------------------------------------------------------
# entry points
# ----------------------------------------------------------------------------

def he_last_error() -> str:
    return lib().he_last_error().decode(errors="replace")


def he_params_create(N: int, L: int, primes=None, t: int = 65537, device: int = 0) -> int:
    out = _vp()
    arr = None
    if primes is not None:
        arr = np.ascontiguousarray(primes, dtype=np.uint32)
        assert arr.size == L
    _check(lib().he_params_create(N, L, None if arr is None else arr.ctypes.data, t, device,
                                  ctypes.byref(out)))
    return out.value


def _limb_query(fn, p, L):
    a = np.zeros(L, dtype=np.uint32)
    _check(fn(p, a.ctypes.data))
    return [int(x) for x in a]


def he_params_primes(p: int, L: int) -> list[int]:
    return _limb_query(lib().he_params_primes, p, L)


def he_params_psi(p: int, L: int) -> list[int]:
    return _limb_query(lib().he_params_psi, p, L)


def he_params_delta(p: int, L: int) -> list[int]:
    return _limb_query(lib().he_params_delta, p, L)


def he_params_reserve(p: int, nbytes: int) -> None:
    _check(lib().he_params_reserve(p, nbytes))


def he_conv_workspace_bytes(p: int, desc, B: int) -> int:
    out = _sz()
    d = _desc(desc)
    _check(lib().he_conv_workspace_bytes(p, ctypes.byref(d), B, ctypes.byref(out)))
    return out.value


def he_fc_workspace_bytes(p: int, B: int) -> int:
    out = _sz()
    _check(lib().he_fc_workspace_bytes(p, B, ctypes.byref(out)))
    return out.value


def he_params_destroy(p: int) -> None:
    lib().he_params_destroy(p)


def he_conv_layout_query(p: int, desc) -> dict:
    out = he_conv_layout()
    d = _desc(desc)
    _check(lib().he_conv_layout_query(p, ctypes.byref(d), ctypes.byref(out)))
    return {n: getattr(out, n) for n, _ in he_conv_layout._fields_}


def he_fc_layout_query(p: int, n_in: int, n_out: int) -> dict:
    out = he_fc_layout()
    _check(lib().he_fc_layout_query(p, n_in, n_out, ctypes.byref(out)))
    return {n: getattr(out, n) for n, _ in he_fc_layout._fields_}


def he_pack_filters(p: int, desc, w: np.ndarray) -> int:
    d = _desc(desc)
    w = np.ascontiguousarray(w, dtype=np.int8)
    assert w.size == d.co * d.ci * d.fh * d.fw
    out = _vp()
    _check(lib().he_pack_filters(p, ctypes.byref(d), w.ctypes.data, ctypes.byref(out)))
    return out.value


def _op_counts(c: he_op_counts) -> dict:
    return {n: getattr(c, n) for n, _ in he_op_counts._fields_ if n != "pad"}


def he_conv_op_counts(p: int, desc, form: int, in_domain: int, B: int = 1) -> dict:
    d = _desc(desc)
    c = he_op_counts()
    _check(lib().he_conv_op_counts(p, ctypes.byref(d), form, in_domain, B, ctypes.byref(c)))
    return _op_counts(c)


def he_fc_op_counts(p: int, n_in: int, n_out: int, form: int, in_domain: int, B: int = 1) -> dict:
    c = he_op_counts()
    _check(lib().he_fc_op_counts(p, n_in, n_out, form, in_domain, B, ctypes.byref(c)))
    return _op_counts(c)


def he_pack_filters_for_batch(p: int, desc, w: np.ndarray, B: int) -> int:
    d = _desc(desc)
    w = np.ascontiguousarray(w, dtype=np.int8)
    assert w.size == d.co * d.ci * d.fh * d.fw
    out = _vp()
    _check(lib().he_pack_filters_for_batch(p, ctypes.byref(d), w.ctypes.data, B, ctypes.byref(out)))
    return out.value


def he_pack_masked(p: int, desc, w: np.ndarray, rho: np.ndarray) -> int:
    d = _desc(desc)
    w = np.ascontiguousarray(w, dtype=np.int8)
    assert w.size == d.co * d.ci * d.fh * d.fw
    rho = np.ascontiguousarray(rho, dtype=np.uint32)
    out = _vp()
    _check(lib().he_pack_masked(p, ctypes.byref(d), w.ctypes.data, rho.ctypes.data, ctypes.byref(out)))
    return out.value


def he_conv_layer_masked(p: int, f: int, d_c0, d_sh, d_shp, in_domain: int, d_out, B: int, stream=None) -> None:
    _check(lib().he_conv_layer_masked(p, f, _ptr(d_c0), _ptr(d_sh), _ptr(d_shp), in_domain, _ptr(d_out), B,
                                      _stream(stream)))


def he_pack_client(p: int, desc, p1: np.ndarray, p2: np.ndarray) -> int:
    d = _desc(desc)
    p1 = np.ascontiguousarray(p1, dtype=np.uint32)
    p2 = np.ascontiguousarray(p2, dtype=np.uint32)
    out = _vp()
    _check(lib().he_pack_client(p, ctypes.byref(d), p1.ctypes.data, p2.ctypes.data, ctypes.byref(out)))
    return out.value


def he_conv_client(p: int, f: int, d_v, d_ish, d_out, B: int, stream=None) -> None:
    _check(lib().he_conv_client(p, f, _ptr(d_v), _ptr(d_ish), _ptr(d_out), B, _stream(stream)))


def he_bench_butterflies(p: int, blocks: int, iters: int, d_sink, stream=None) -> None:
    """Launches the butterfly-peak kernel (blocks * 256 * 8 * iters forward
    butterflies in registers); the caller times it."""
    _check(lib().he_bench_butterflies(p, blocks, iters, _ptr(d_sink), _stream(stream)))


def he_rescale(p: int, d_in, d_out, count: int, stream=None) -> None:
    _check(lib().he_rescale(p, _ptr(d_in), _ptr(d_out), count, _stream(stream)))


def he_filters_tensor_core(f: int) -> int:
    tc = _u32()
    _check(lib().he_filters_tensor_core(f, ctypes.byref(tc)))
    return tc.value


def he_pack_fc(p: int, n_in: int, n_out: int, W: np.ndarray, bias: np.ndarray | None = None) -> int:
    W = np.ascontiguousarray(W, dtype=np.int8)
    assert W.shape == (n_out, n_in)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.int32)
    out = _vp()
    _check(lib().he_pack_fc(p, n_in, n_out, W.ctypes.data, None if b is None else b.ctypes.data,
                            ctypes.byref(out)))
    return out.value


def he_pack_fc_masked(p: int, n_in: int, n_out: int, W: np.ndarray, bias: np.ndarray | None,
                      rho: np.ndarray) -> int:
    W = np.ascontiguousarray(W, dtype=np.int8)
    assert W.shape == (n_out, n_in)
    b = None if bias is None else np.ascontiguousarray(bias, dtype=np.int32)
    rho = np.ascontiguousarray(rho, dtype=np.uint32)
    out = _vp()
    _check(lib().he_pack_fc_masked(p, n_in, n_out, W.ctypes.data, None if b is None else b.ctypes.data,
                                   rho.ctypes.data, ctypes.byref(out)))
    return out.value


def he_fc_layer_masked(p: int, f: int, d_c0, d_sh, d_shp, in_domain: int, d_out, B: int, stream=None) -> None:
    _check(lib().he_fc_layer_masked(p, f, _ptr(d_c0), _ptr(d_sh), _ptr(d_shp), in_domain, _ptr(d_out), B,
                                    _stream(stream)))


def he_pack_fc_client(p: int, n_in: int, n_out: int, p1: np.ndarray, p2: np.ndarray) -> int:
    p1 = np.ascontiguousarray(p1, dtype=np.uint32)
    p2 = np.ascontiguousarray(p2, dtype=np.uint32)
    out = _vp()
    _check(lib().he_pack_fc_client(p, n_in, n_out, p1.ctypes.data, p2.ctypes.data, ctypes.byref(out)))
    return out.value


def he_fc_client(p: int, f: int, d_v, d_ish, d_out, B: int, stream=None) -> None:
    _check(lib().he_fc_client(p, f, _ptr(d_v), _ptr(d_ish), _ptr(d_out), B, _stream(stream)))


def he_filters_destroy(f: int) -> None:
    lib().he_filters_destroy(f)


def he_conv_layer(p: int, f: int, d_in, in_domain: int, d_out, out_mode: int, B: int,
                  stream=None) -> None:
    _check(lib().he_conv_layer(p, f, _ptr(d_in), in_domain, _ptr(d_out), out_mode, B, _stream(stream)))


def he_conv_layer_noalloc(p: int, f: int, d_in, in_domain: int, d_out, out_mode: int, B: int,
                          stream=None) -> None:
    """he_conv_layer without any device allocation: coefficient-domain
    inputs are transformed in a fixed 8 MiB per-device scratch array
    (B * G * 2 * L * N <= 2**21 words).  Calls that may overlap race on that
    scratch; order them on one stream."""
    _check(lib().he_conv_layer_noalloc(p, f, _ptr(d_in), in_domain, _ptr(d_out), out_mode, B,
                                       _stream(stream)))


def he_fc_layer(p: int, f: int, d_in, in_domain: int, d_out, out_mode: int, B: int,
                stream=None) -> None:
    _check(lib().he_fc_layer(p, f, _ptr(d_in), in_domain, _ptr(d_out), out_mode, B, _stream(stream)))


def he_ntt_forward(p: int, d_in, d_out, count: int, stream=None) -> None:
    _check(lib().he_ntt_forward(p, _ptr(d_in), _ptr(d_out), count, _stream(stream)))


def he_ntt_inverse(p: int, d_in, d_out, count: int, stream=None) -> None:
    _check(lib().he_ntt_inverse(p, _ptr(d_in), _ptr(d_out), count, _stream(stream)))


def _calls(calls):
    """(filters, d_in, in_domain, d_out, B[, d_share[, d_share_out[,
    d_rescaled]]]) tuples or dicts with those keys."""
    arr = (he_layer_call * len(calls))()
    for i, c in enumerate(calls):
        if isinstance(c, dict):
            c = (c["filters"], c["d_in"], c.get("in_domain", HE_COEFF), c["d_out"], c["B"], c.get("d_share"),
                 c.get("d_share_out"), c.get("d_rescaled"))
        f, d_in, dom, d_out, B = c[:5]
        extra = [(_ptr(c[k]) if len(c) > k else None) for k in (5, 6, 7)]
        arr[i] = he_layer_call(f, _ptr(d_in), dom, _ptr(d_out), B, *extra)
    return arr


def _tuning_dict(t: he_plan_tuning) -> dict:
    return {n: getattr(t, n) for n, _ in he_plan_tuning._fields_}


def he_plan_create(calls) -> int:
    """calls: sequence of (filters, d_in, in_domain, d_out, B[, d_share[,
    d_share_out[, d_rescaled]]]) tuples or dicts (the shares for masked and
    client banks; d_rescaled for an output rescaled by the last prime)."""
    out = _vp()
    _check(lib().he_plan_create(_calls(calls), len(calls), ctypes.byref(out)))
    return out.value


def he_plan_tuning_default() -> dict:
    t = he_plan_tuning()
    _check(lib().he_plan_tuning_default(ctypes.byref(t)))
    return _tuning_dict(t)


def he_plan_create_tuned(calls, tuning: dict) -> int:
    """tuning: knob -> value; knobs it leaves out keep their default."""
    t = he_plan_tuning(**dict(he_plan_tuning_default(), **tuning))
    out = _vp()
    _check(lib().he_plan_create_tuned(_calls(calls), len(calls), ctypes.byref(t), ctypes.byref(out)))
    return out.value


def he_plan_workspace_bytes(calls) -> int:
    """Workspace he_plan_create would allocate for these calls (d_in / d_out
    may be None); allocates nothing."""
    out = _sz()
    _check(lib().he_plan_workspace_bytes(_calls(calls), len(calls), ctypes.byref(out)))
    return out.value


HE_WAIT_POLLS_DEFAULT = 1 << 20


def he_plan_set_wait_limit(plan: int, polls: int) -> None:
    _check(lib().he_plan_set_wait_limit(plan, polls))


def he_plan_set_checks(plan: int, on: bool) -> None:
    _check(lib().he_plan_set_checks(plan, 1 if on else 0))


def he_plan_autotune(calls, iters: int = 5, stream=None) -> tuple[int, dict]:
    """(plan, chosen tuning).  Runs the calls while timing candidates."""
    t = he_plan_tuning()
    out = _vp()
    _check(lib().he_plan_autotune(_calls(calls), len(calls), iters, _stream(stream), ctypes.byref(t),
                                  ctypes.byref(out)))
    return out.value, _tuning_dict(t)


def he_plan_autotune_inflight(calls, iters: int = 5, in_flight: int = 2, stream=None) -> tuple[int, dict]:
    """(plan, chosen tuning) for `in_flight` runs in flight at once."""
    t = he_plan_tuning()
    out = _vp()
    _check(lib().he_plan_autotune_inflight(_calls(calls), len(calls), iters, in_flight, _stream(stream),
                                           ctypes.byref(t), ctypes.byref(out)))
    return out.value, _tuning_dict(t)


def he_plan_run(plan: int, stream=None) -> None:
    _check(lib().he_plan_run(plan, _stream(stream)))


def he_plan_run_host(plan: int, h_in, h_out, stream=None) -> None:
    """he_plan_run with host buffers (host addresses, or objects with
    data_ptr(), e.g. pinned torch tensors): inputs of every call in call
    order in h_in, outputs in h_out (sizes: he_plan_host_words)."""
    _check(lib().he_plan_run_host(plan, _ptr(h_in), _ptr(h_out), _stream(stream)))


def he_plan_host_words(plan: int) -> dict:
    """{"in_words", "out_words", "copies"} of he_plan_run_host."""
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), _u32()
    _check(lib().he_plan_host_words(plan, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"in_words": a.value, "out_words": b.value, "copies": c.value}


def he_plan_run_phase(plan: int, phase: int, stream=None) -> None:
    _check(lib().he_plan_run_phase(plan, phase, _stream(stream)))


def he_plan_query(plan: int, ncalls: int | None = None) -> dict:
    """The plan's he_plan_info as a dict; with ncalls, also "split": the
    per-call split-form (scalar MAC kernel) flags, and "form": per call 0
    (fused channel kernel), 1 (split form, scalar MAC kernel) or 2
    (tensor-core MAC kernel)."""
    info = he_plan_info()
    sp = None if ncalls is None else np.zeros(ncalls, dtype=np.uint8)
    _check(lib().he_plan_query(plan, ctypes.byref(info), None if sp is None else sp.ctypes.data))
    out = {n: getattr(info, n) for n, _ in he_plan_info._fields_ if n != "tuning"}
    out["tuning"] = _tuning_dict(info.tuning)
    if sp is not None:
        out["split"] = [int(x) == 1 for x in sp]
        out["form"] = [int(x) for x in sp]
    return out


def he_plan_check(plan: int) -> None:
    _check(lib().he_plan_check(plan))


def he_plan_destroy(plan: int) -> None:
    lib().he_plan_destroy(plan)


def he_server_create(device: int = 0, hbm_budget_bytes: int = 120 << 30, max_batch: int = 8, streams: int = 8,
                     max_inflight: int = 16) -> int:
    cfg = he_server_config(device, hbm_budget_bytes, max_batch, streams, max_inflight)
    out = _vp()
    _check(lib().he_server_create(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def he_server_add_model(s: int, layers) -> int:
    arr = (_vp * len(layers))(*layers)
    mid = _u32()
    _check(lib().he_server_add_model(s, arr, len(layers), ctypes.byref(mid)))
    return mid.value


def he_server_submit(s: int, model_id: int, h_in, h_out) -> int:
    """h_in, h_out: per-layer HOST buffers (addresses or objects with
    data_ptr(), e.g. pinned torch tensors)."""
    ins = (_vp * len(h_in))(*[_ptr(x) for x in h_in])
    outs = (_vp * len(h_out))(*[_ptr(x) for x in h_out])
    t = ctypes.c_uint64()
    _check(lib().he_server_submit(s, model_id, ins, outs, ctypes.byref(t)))
    return t.value


def he_server_wait(s: int, ticket: int, timeout_ms: int = 60000) -> dict:
    st = he_request_stats()
    _check(lib().he_server_wait(s, ticket, timeout_ms, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in he_request_stats._fields_}


def he_server_report(s: int) -> dict:
    r = he_server_report_t()
    _check(lib().he_server_report(s, ctypes.byref(r)))
    d = {n: getattr(r, n) for n, _ in he_server_report_t._fields_}
    d["batch_hist"] = {str(1 << i): int(r.batch_hist[i]) for i in range(4)}
    return d


def he_server_latencies(s: int, which: int) -> np.ndarray:
    n = ctypes.c_uint64()
    _check(lib().he_server_latencies(s, which, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=np.float64)
    _check(lib().he_server_latencies(s, which, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n.value,
                                     ctypes.byref(n)))
    return out[: n.value]


def he_server_destroy(s: int) -> None:
    lib().he_server_destroy(s)


def he_sync(stream=None) -> None:
    _check(lib().he_sync(_stream(stream)))
