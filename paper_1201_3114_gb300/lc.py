"""Python binding of liblorenzcipher (include/lc.h).

Argument marshalling only: every step of the cipher runs in the library's
CUDA kernels.  Functions keep the C names (lc_encrypt, lc_decrypt,
lc_run_batch, ...); device buffers are PyTorch CUDA tensors (or raw device
addresses) and streams are ``torch.cuda.Stream`` objects (or raw
``cudaStream_t`` values).  There is no CPU fallback: if the shared library
cannot be built or loaded, :func:`load` raises.
"""
import ctypes as C
import os
import re
import threading

from . import build as _build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lc.h")

LC_OK, LC_ERR_ARG, LC_ERR_PASSWORD, LC_ERR_LENGTH, LC_ERR_INTEGRITY = 0, 1, 2, 3, 4
LC_ERR_CUDA, LC_ERR_TIMEOUT, LC_ERR_NOMEM = 5, 6, 7
LC_PARALLEL, LC_SEQUENTIAL = 0, 1
LC_ENCRYPT, LC_DECRYPT = 0, 1
LC_HOST_INFLIGHT = 3

# objects a submitted host batch reads or writes after the call returns,
# kept alive until its ticket is waited for: {(ctx, ticket): refs}
_host_inflight = {}
_host_lock = threading.Lock()


class lc_params(C.Structure):
    _fields_ = [
        ("sigma", C.c_double),
        ("rho", C.c_double),
        ("beta", C.c_double),
        ("dt", C.c_double),
        ("n_warm", C.c_uint32),
        ("steps_per_byte", C.c_uint32),
        ("lam", C.c_double * 3),
        ("k", C.c_uint32 * 3),
        ("block_len", C.c_uint32),
        ("tag_len", C.c_uint32),
        ("eta", C.c_double),
        ("omega_alpha_shift", C.c_uint32),
        ("reserved", C.c_uint32),
    ]


class lc_req(C.Structure):
    _fields_ = [
        ("pw", C.c_void_p),
        ("pw_len", C.c_uint32),
        ("dir", C.c_uint32),
        ("inp", C.c_void_p),
        ("in_len", C.c_size_t),
        ("out", C.c_void_p),
        ("out_cap", C.c_size_t),
    ]


LC_KEY_LAMBDA, LC_KEY_K = 1, 2


class lc_req_ex(C.Structure):
    _fields_ = [
        ("req", lc_req),
        ("key_flags", C.c_uint32),
        ("k", C.c_uint32 * 3),
        ("lam", C.c_double * 3),
    ]


class lc_launch(C.Structure):
    _fields_ = [
        ("threads_per_cta", C.c_uint32),
        ("ctas_per_sm", C.c_uint32),
        ("smem_staging", C.c_uint32),
        ("small_batch_rows", C.c_uint32),
        ("host_chunk_mib", C.c_uint32),
        ("dense_build", C.c_uint32),
        ("full_grid_rows", C.c_uint32),
        ("split_rows", C.c_uint32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class lc_tune_entry(C.Structure):
    _fields_ = [("launch", lc_launch), ("median_ms", C.c_double)]


class lc_key_info_t(C.Structure):
    _fields_ = [
        ("aprime", C.c_double * 3),
        ("mu", C.c_uint32 * 3),
        ("omega", C.c_uint32 * 3),
        ("L", C.c_uint32),
        ("D", C.c_uint32),
    ]


class lc_pipe_rates(C.Structure):
    _fields_ = [
        ("dadd_gops", C.c_double),
        ("dmul_gops", C.c_double),
        ("cvt_gops", C.c_double),
        ("imad_gops", C.c_double),
        ("ialu_gops", C.c_double),
        ("ffma_gops", C.c_double),
        ("sm_clock_mhz", C.c_double),
        ("sm_count", C.c_uint32),
        ("reserved", C.c_uint32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


LC_STATS_MAX_LAG = 8


class lc_byte_stats_t(C.Structure):
    _fields_ = [
        ("n", C.c_uint64),
        ("hist", C.c_uint64 * 256),
        ("sum", C.c_uint64),
        ("sum_sq", C.c_uint64),
        ("lag_sum", C.c_uint64 * LC_STATS_MAX_LAG),
    ]


class lc_digit_stats_t(C.Structure):
    _fields_ = [
        ("states", C.c_uint64),
        ("int_part", (C.c_uint64 * 128) * 3),
        ("digits", ((C.c_uint64 * 100) * 3) * 3),
        ("out_of_range", C.c_uint64 * 3),
    ]

    def arrays(self):
        """(int_part [3, 128], digits [3, 3, 100], out_of_range [3]) as numpy."""
        import numpy as np
        ip = np.array([list(self.int_part[c]) for c in range(3)], dtype=np.uint64)
        dg = np.array([[list(self.digits[c][j]) for j in range(3)] for c in range(3)], dtype=np.uint64)
        return ip, dg, np.array(list(self.out_of_range), dtype=np.uint64)


class LcError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        detail = ""
        if status in (LC_ERR_CUDA, LC_ERR_NOMEM):
            detail = " [%s]" % load().lc_last_cuda_error().decode()
        super().__init__("%s: %s (status %d)%s" % (what, status_string(status), status, detail))


_lib = None
_lock = threading.Lock()

_SIGNATURES = {
    "lc_version": (C.c_uint32, []),
    "lc_status_string": (C.c_char_p, [C.c_int]),
    "lc_last_cuda_error": (C.c_char_p, []),
    "lc_params_default": (C.c_int, [C.POINTER(lc_params)]),
    "lc_ctx_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "lc_ctx_destroy": (None, [C.c_void_p]),
    "lc_ctx_set_params": (C.c_int, [C.c_void_p, C.POINTER(lc_params)]),
    "lc_ctx_get_params": (C.c_int, [C.c_void_p, C.POINTER(lc_params)]),
    "lc_ciphertext_len": (C.c_size_t, [C.c_void_p, C.c_size_t, C.c_int]),
    "lc_plaintext_len": (C.c_int, [C.c_void_p, C.c_size_t, C.c_int, C.POINTER(C.c_size_t)]),
    "lc_encrypt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                             C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]),
    "lc_decrypt": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p, C.c_size_t,
                             C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]),
    "lc_run_batch": (C.c_int, [C.c_void_p, C.POINTER(lc_req), C.c_size_t, C.c_void_p, C.c_int,
                               C.c_void_p]),
    "lc_run_batch_host": (C.c_int, [C.c_void_p, C.POINTER(lc_req), C.c_size_t, C.c_void_p,
                                    C.c_int, C.c_void_p]),
    "lc_build_flags": (C.c_uint32, []),
    "lc_submit_batch_host": (C.c_int, [C.c_void_p, C.POINTER(lc_req), C.c_size_t, C.c_void_p,
                                       C.c_int, C.c_void_p, C.POINTER(C.c_uint64)]),
    "lc_wait_batch_host": (C.c_int, [C.c_void_p, C.c_uint64]),
    "lc_ctx_get_launch": (C.c_int, [C.c_void_p, C.POINTER(lc_launch)]),
    "lc_ctx_set_launch": (C.c_int, [C.c_void_p, C.POINTER(lc_launch)]),
    "lc_tune": (C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(lc_launch)]),
    "lc_tune_report": (C.c_int, [C.c_void_p, C.POINTER(lc_tune_entry), C.c_size_t,
                                 C.POINTER(C.c_size_t)]),
    "lc_ctx_timing": (C.c_int, [C.c_void_p, C.c_int]),
    "lc_ctx_kernel_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_uint64)]),
    "lc_ctx_launch_count": (C.c_uint64, [C.c_void_p]),
    "lc_key_info": (C.c_int, [C.POINTER(lc_params), C.c_void_p, C.c_size_t,
                              C.POINTER(lc_key_info_t)]),
    "lc_plan_batch": (C.c_int, [C.POINTER(lc_params), C.POINTER(lc_req), C.c_size_t, C.c_int,
                                C.c_void_p, C.POINTER(C.c_uint64)]),
    "lc_probe_pipes": (C.c_int, [C.c_int, C.POINTER(lc_pipe_rates)]),
    "lc_run_batch_noalloc": (C.c_int, [C.POINTER(lc_req), C.c_size_t, C.c_void_p, C.c_int,
                                       C.c_void_p]),
    "lc_softfp_eval": (C.c_int, [C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_size_t, C.c_void_p]),
    "lc_emu_mask": (C.c_uint32, []),
    "lc_warm_mask": (C.c_uint32, []),
    "lc_partial_mask": (C.c_uint32, []),
    "lc_probe_fp64_warp": (C.c_int, [C.c_int, C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(C.c_double)]),
    "lc_byte_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_uint32,
                                C.POINTER(lc_byte_stats_t), C.c_void_p]),
    "lc_synth_uniform": (C.c_int, [C.c_void_p, C.c_size_t, C.c_uint64, C.c_uint64, C.c_void_p]),
    "lc_ctx_digit_stats": (C.c_int, [C.c_void_p, C.c_int]),
    "lc_run_batch_ex": (C.c_int, [C.c_void_p, C.POINTER(lc_req_ex), C.c_size_t, C.c_void_p, C.c_int,
                                  C.c_void_p]),
    "lc_plan_batch_ex": (C.c_int, [C.POINTER(lc_params), C.POINTER(lc_req_ex), C.c_size_t, C.c_int,
                                   C.c_void_p, C.POINTER(C.c_uint64)]),
    "lc_ctx_get_digit_stats": (C.c_int, [C.c_void_p, C.POINTER(lc_digit_stats_t)]),
    "lc_ctx_ciphertext_stats": (C.c_int, [C.c_void_p, C.c_int]),
    "lc_ctx_get_ciphertext_stats": (C.c_int, [C.c_void_p, C.POINTER(lc_byte_stats_t)]),
}


def header_symbols():
    """Every function the public header declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lc_[a-z0-9_]+)\s*\(", text)))


def load():
    """Build if needed and load the shared library (raises on failure)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("LC_LIBRARY") or _build.build()
            if not os.path.exists(path):
                raise RuntimeError("liblorenzcipher.so is missing at %s" % path)
            lib = C.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def library_path():
    return _build.LIB_PATH


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(x):
    """Device/host address of a tensor, or an int address, or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() else None
    if hasattr(x, "ctypes"):
        return x.ctypes.data if x.size else None
    raise TypeError("cannot take the address of %r" % type(x))


def _nbytes(x):
    if hasattr(x, "numel"):
        return x.numel() * x.element_size()
    if hasattr(x, "nbytes"):
        return x.nbytes
    raise TypeError("cannot size %r" % type(x))


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _pwbuf(pw):
    if isinstance(pw, str):
        pw = pw.encode("latin-1")
    pw = bytes(pw)
    buf = C.create_string_buffer(pw, max(1, len(pw)))
    return buf, len(pw)


def status_string(status: int) -> str:
    return load().lc_status_string(status).decode()


def check(status, what="liblorenzcipher"):
    if status != LC_OK:
        raise LcError(status, what)
    return status


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------

def lc_version() -> int:
    return load().lc_version()


LC_BUILD_CHECKED = 1


def lc_build_flags() -> int:
    return load().lc_build_flags()


def lc_status_string(status: int) -> str:
    return status_string(status)


def lc_last_cuda_error() -> str:
    return load().lc_last_cuda_error().decode()


def lc_params_default() -> lc_params:
    p = lc_params()
    check(load().lc_params_default(C.byref(p)), "lc_params_default")
    return p


def params(**over) -> lc_params:
    """Default parameters with field overrides (``lam``/``k`` take 3-sequences)."""
    p = lc_params_default()
    for k, v in over.items():
        if k in ("lam", "k"):
            arr = getattr(p, k)
            for i in range(3):
                arr[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def lc_ctx_create(device: int = 0) -> int:
    h = C.c_void_p()
    check(load().lc_ctx_create(device, C.byref(h)), "lc_ctx_create")
    return h.value


def lc_ctx_destroy(ctx) -> None:
    load().lc_ctx_destroy(ctx)
    with _host_lock:
        for key in [k for k in _host_inflight if k[0] == ctx]:
            del _host_inflight[key]


def lc_ctx_set_params(ctx, p: lc_params) -> int:
    return load().lc_ctx_set_params(ctx, C.byref(p))


def lc_ctx_get_params(ctx) -> lc_params:
    p = lc_params()
    check(load().lc_ctx_get_params(ctx, C.byref(p)), "lc_ctx_get_params")
    return p


def lc_ciphertext_len(ctx, n: int, mode: int = LC_PARALLEL) -> int:
    return load().lc_ciphertext_len(ctx, n, mode)


def lc_plaintext_len(ctx, c_len: int, mode: int = LC_PARALLEL):
    n = C.c_size_t()
    st = load().lc_plaintext_len(ctx, c_len, mode, C.byref(n))
    return n.value if st == LC_OK else None


def lc_encrypt(ctx, pw, P, n, Cbuf, c_cap, mode=LC_PARALLEL, stream=None) -> int:
    buf, L = _pwbuf(pw)
    return load().lc_encrypt(ctx, buf, L, _ptr(P), n, _ptr(Cbuf), c_cap, mode, _stream(stream))


def lc_decrypt(ctx, pw, Cbuf, c_len, P, p_cap, mode=LC_PARALLEL, stream=None) -> int:
    buf, L = _pwbuf(pw)
    return load().lc_decrypt(ctx, buf, L, _ptr(Cbuf), c_len, _ptr(P), p_cap, mode, _stream(stream))


class Batch:
    """An lc_req array plus the password buffers it points to."""

    def __init__(self, items):
        """items: iterable of (pw, dir, in, in_len, out, out_cap)."""
        items = list(items)
        self._pw = []
        self.reqs = (lc_req * max(1, len(items)))()
        self.count = len(items)
        for i, (pw, d, inp, in_len, out, out_cap) in enumerate(items):
            buf, L = _pwbuf(pw)
            self._pw.append(buf)
            r = self.reqs[i]
            r.pw = C.cast(buf, C.c_void_p)
            r.pw_len = L
            r.dir = d
            r.inp = _ptr(inp)
            r.in_len = in_len
            r.out = _ptr(out)
            r.out_cap = out_cap


class BatchEx:
    """An lc_req_ex array (requests with their own key material) plus the
    password buffers it points to."""

    def __init__(self, items):
        """items: iterable of (pw, dir, in, in_len, out, out_cap, lam, k), where
        lam and k are 3-sequences or None (the context's value)."""
        items = list(items)
        self._pw = []
        self.reqs = (lc_req_ex * max(1, len(items)))()
        self.count = len(items)
        for i, (pw, d, inp, in_len, out, out_cap, lam, k) in enumerate(items):
            buf, L = _pwbuf(pw)
            self._pw.append(buf)
            e = self.reqs[i]
            r = e.req
            r.pw = C.cast(buf, C.c_void_p)
            r.pw_len = L
            r.dir = d
            r.inp = _ptr(inp)
            r.in_len = in_len
            r.out = _ptr(out)
            r.out_cap = out_cap
            e.key_flags = (LC_KEY_LAMBDA if lam is not None else 0) | (LC_KEY_K if k is not None else 0)
            for j in range(3):
                e.lam[j] = lam[j] if lam is not None else 0.0
                e.k[j] = k[j] if k is not None else 0


def lc_run_batch_ex(ctx, batch: BatchEx, status_dev, mode=LC_PARALLEL, stream=None) -> int:
    return load().lc_run_batch_ex(ctx, batch.reqs, batch.count, _ptr(status_dev), mode, _stream(stream))


def lc_plan_batch_ex(batch: BatchEx, mode=LC_PARALLEL, p: lc_params = None):
    """(status, per-request init statuses, parts) of a host-only validation."""
    import numpy as np
    st = np.zeros(max(1, batch.count), dtype=np.int32)
    rows = C.c_uint64(0)
    rc = load().lc_plan_batch_ex(C.byref(p) if p is not None else None, batch.reqs, batch.count, mode,
                                 st.ctypes.data, C.byref(rows))
    return rc, st[:batch.count], rows.value


def lc_run_batch(ctx, batch: Batch, status_dev, mode=LC_PARALLEL, stream=None) -> int:
    return load().lc_run_batch(ctx, batch.reqs, batch.count, _ptr(status_dev), mode, _stream(stream))


def lc_run_batch_noalloc(batch: Batch, status_dev, mode=LC_PARALLEL, stream=None) -> int:
    return load().lc_run_batch_noalloc(batch.reqs, batch.count, _ptr(status_dev), mode,
                                       _stream(stream))


def lc_run_batch_host(ctx, batch: Batch, status_host, mode=LC_PARALLEL, stream=None) -> int:
    return load().lc_run_batch_host(ctx, batch.reqs, batch.count, _ptr(status_host), mode,
                                    _stream(stream))


def lc_submit_batch_host(ctx, batch: Batch, status_host, mode=LC_PARALLEL, stream=None):
    """(status, ticket).  The host buffers of ``batch`` and ``status_host``
    must stay alive and unchanged until lc_wait_batch_host(ctx, ticket)."""
    t = C.c_uint64(0)
    st = load().lc_submit_batch_host(ctx, batch.reqs, batch.count, _ptr(status_host), mode,
                                     _stream(stream), C.byref(t))
    if st == LC_OK:
        with _host_lock:
            _host_inflight[(ctx, t.value)] = (batch, status_host)
    return st, t.value


def lc_wait_batch_host(ctx, ticket) -> int:
    st = load().lc_wait_batch_host(ctx, ticket)
    if st != LC_ERR_ARG:
        with _host_lock:
            for key in [k for k in _host_inflight if k[0] == ctx and k[1] <= ticket]:
                del _host_inflight[key]
    return st


def lc_ctx_get_launch(ctx) -> lc_launch:
    l = lc_launch()
    check(load().lc_ctx_get_launch(ctx, C.byref(l)), "lc_ctx_get_launch")
    return l


def lc_ctx_set_launch(ctx, threads_per_cta=256, ctas_per_sm=0, smem_staging=0,
                      small_batch_rows=0, host_chunk_mib=0, dense_build=0, full_grid_rows=0,
                      split_rows=0) -> int:
    l = lc_launch(threads_per_cta, ctas_per_sm, smem_staging, small_batch_rows, host_chunk_mib,
                  dense_build, full_grid_rows, split_rows)
    return load().lc_ctx_set_launch(ctx, C.byref(l))


def lc_tune(ctx, probe_bytes=0, stream=None) -> lc_launch:
    l = lc_launch()
    check(load().lc_tune(ctx, probe_bytes, _stream(stream), C.byref(l)), "lc_tune")
    return l


def lc_tune_report(ctx):
    """[(launch dict, median ms)] of the last lc_tune call, in the order tried."""
    n = C.c_size_t(0)
    check(load().lc_tune_report(ctx, None, 0, C.byref(n)), "lc_tune_report")
    arr = (lc_tune_entry * max(1, n.value))()
    check(load().lc_tune_report(ctx, arr, n.value, C.byref(n)), "lc_tune_report")
    return [(arr[i].launch.as_dict(), arr[i].median_ms) for i in range(n.value)]


def lc_ctx_timing(ctx, enable: bool) -> int:
    return load().lc_ctx_timing(ctx, 1 if enable else 0)


def lc_ctx_kernel_time(ctx):
    ms = C.c_double()
    n = C.c_uint64()
    check(load().lc_ctx_kernel_time(ctx, C.byref(ms), C.byref(n)), "lc_ctx_kernel_time")
    return ms.value, n.value


def lc_ctx_launch_count(ctx) -> int:
    return load().lc_ctx_launch_count(ctx)


def lc_key_info(pw, p: lc_params = None):
    buf, L = _pwbuf(pw)
    out = lc_key_info_t()
    st = load().lc_key_info(C.byref(p) if p is not None else None, buf, L, C.byref(out))
    return st, out


def lc_plan_batch(batch: Batch, mode=LC_PARALLEL, p: lc_params = None):
    import numpy as np
    st = np.zeros(max(1, batch.count), dtype=np.int32)
    rows = C.c_uint64()
    rc = load().lc_plan_batch(C.byref(p) if p is not None else None, batch.reqs, batch.count, mode,
                              st.ctypes.data, C.byref(rows))
    return rc, st[:batch.count], rows.value


def lc_probe_pipes(device: int = 0) -> lc_pipe_rates:
    r = lc_pipe_rates()
    check(load().lc_probe_pipes(device, C.byref(r)), "lc_probe_pipes")
    return r


(LC_SFP_ADD, LC_SFP_SUB, LC_SFP_MUL, LC_SFP_MUL10, LC_SFP_MUL28, LC_SFP_FLOOR13, LC_SFP_MULDT, LC_SFP_MULBETA,
 LC_SFP_ADD_KICK, LC_SFP_ADD_Z) = range(10)


def lc_softfp_eval(op, a_dev, b_dev, sw_dev, hw_dev, n, stream=None) -> int:
    return load().lc_softfp_eval(op, _ptr(a_dev), _ptr(b_dev), _ptr(sw_dev), _ptr(hw_dev), n,
                                 _stream(stream))


def lc_byte_stats(ctx, data_dev, n, max_lag=LC_STATS_MAX_LAG, stream=None) -> lc_byte_stats_t:
    out = lc_byte_stats_t()
    check(load().lc_byte_stats(ctx, _ptr(data_dev), n, max_lag, C.byref(out), _stream(stream)),
          "lc_byte_stats")
    return out


def entropy_bits(stats: lc_byte_stats_t) -> float:
    """Shannon entropy (bits per byte) of the histogram (Sec. 4)."""
    import math
    n = stats.n
    return -sum((h / n) * math.log2(h / n) for h in stats.hist if h) if n else 0.0


def autocorrelation(stats: lc_byte_stats_t, max_lag=LC_STATS_MAX_LAG):
    """Lag-k auto-correlation coefficients from the exact sums: the covariance
    of (x_i, x_{i+k}) over the variance, using the whole-sequence mean."""
    n = stats.n
    if n < 2:
        return [0.0] * max_lag
    mean = stats.sum / n
    var = stats.sum_sq / n - mean * mean
    out = []
    for k in range(1, max_lag + 1):
        m = n - k
        cov = stats.lag_sum[k - 1] / m - mean * mean if m > 0 else 0.0
        out.append(cov / var if var > 0 else 0.0)
    return out


def lc_ctx_digit_stats(ctx, enable: bool) -> int:
    return load().lc_ctx_digit_stats(ctx, 1 if enable else 0)


def lc_ctx_get_digit_stats(ctx) -> lc_digit_stats_t:
    out = lc_digit_stats_t()
    check(load().lc_ctx_get_digit_stats(ctx, C.byref(out)), "lc_ctx_get_digit_stats")
    return out


def lc_ctx_ciphertext_stats(ctx, enable: bool) -> int:
    return load().lc_ctx_ciphertext_stats(ctx, 1 if enable else 0)


def lc_ctx_get_ciphertext_stats(ctx) -> lc_byte_stats_t:
    out = lc_byte_stats_t()
    check(load().lc_ctx_get_ciphertext_stats(ctx, C.byref(out)), "lc_ctx_get_ciphertext_stats")
    return out


def lc_emu_mask() -> int:
    return load().lc_emu_mask()


def lc_warm_mask() -> int:
    return load().lc_warm_mask()


def lc_partial_mask() -> int:
    return load().lc_partial_mask()


def lc_probe_fp64_warp(device, warps, chains, lanes) -> float:
    v = C.c_double()
    check(load().lc_probe_fp64_warp(device, warps, chains, lanes, C.byref(v)), "lc_probe_fp64_warp")
    return v.value


def lc_synth_uniform(dst, n, seed, offset=0, stream=None) -> int:
    return load().lc_synth_uniform(_ptr(dst), n, seed & ((1 << 64) - 1), offset, _stream(stream))


# ---------------------------------------------------------------------------
# convenience layer over the same entry points
# ---------------------------------------------------------------------------

class Context:
    """Owns an lc_ctx; encrypt/decrypt PyTorch CUDA uint8 tensors."""

    def __init__(self, device: int = 0, params_: lc_params = None):
        self.handle = lc_ctx_create(device)
        self.device = device
        if params_ is not None:
            check(lc_ctx_set_params(self.handle, params_), "lc_ctx_set_params")

    def close(self):
        if self.handle:
            lc_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def ciphertext_len(self, n, mode=LC_PARALLEL):
        return lc_ciphertext_len(self.handle, n, mode)

    def plaintext_len(self, c_len, mode=LC_PARALLEL):
        return lc_plaintext_len(self.handle, c_len, mode)

    def encrypt(self, pw, P, mode=LC_PARALLEL, stream=None, out=None):
        import torch
        n = P.numel()
        c_len = self.ciphertext_len(n, mode)
        if out is None:
            out = torch.empty(c_len, dtype=torch.uint8, device=P.device if n else "cuda")
        check(lc_encrypt(self.handle, pw, P, n, out, _nbytes(out), mode, stream), "lc_encrypt")
        return out

    def decrypt(self, pw, Cbuf, mode=LC_PARALLEL, stream=None, out=None):
        """(status, plaintext tensor); status LC_ERR_INTEGRITY leaves it zeroed."""
        import torch
        c_len = Cbuf.numel()
        n = self.plaintext_len(c_len, mode)
        if n is None:
            raise LcError(LC_ERR_LENGTH, "lc_decrypt")
        if out is None:
            out = torch.empty(max(n, 0), dtype=torch.uint8, device=Cbuf.device)
        st = lc_decrypt(self.handle, pw, Cbuf, c_len, out, _nbytes(out), mode, stream)
        if st not in (LC_OK, LC_ERR_INTEGRITY):
            raise LcError(st, "lc_decrypt")
        return st, out
