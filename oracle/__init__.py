"""ctypes binding of the CPU oracle (oracle/lco.c).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow definition of the
Lorenz-attractor chaotic cipher (arXiv 1201.3114) that the CUDA library is
checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm may import this package.  The
product library never imports it and shares no code with it.

ctypes drops the GIL during each foreign call, so several Python threads can
run independent parts of a message through the oracle at once (the
multi-core CPU baseline does this).
"""
import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

ENCRYPT, DECRYPT = 0, 1
PARALLEL, SEQUENTIAL = 0, 1
OK, ERR_ARG, ERR_PASSWORD, ERR_LENGTH, ERR_INTEGRITY = 0, 1, 2, 3, 4


class Params(C.Structure):
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


class Key(C.Structure):
    _fields_ = [
        ("a_lo", C.c_uint64 * 3),
        ("a_hi", C.c_uint64 * 3),
        ("L", C.c_uint32),
        ("D", C.c_uint32),
        ("aprime", C.c_double * 3),
        ("mu", C.c_uint32 * 3),
        ("omega", C.c_uint32 * 3),
    ]

    @property
    def a(self):
        return tuple((self.a_hi[i] << 64) | self.a_lo[i] for i in range(3))


class State(C.Structure):
    _fields_ = [
        ("r", C.c_double * 3),
        ("alpha", C.c_double * 3),
        ("mu", C.c_uint32 * 3),
        ("omega", C.c_uint32 * 3),
    ]

    def copy(self):
        s = State()
        C.memmove(C.byref(s), C.byref(self), C.sizeof(State))
        return s


class Stats(C.Structure):
    _fields_ = [
        ("max_abs_r", C.c_double),
        ("r1_hist", C.c_uint64 * 256),
        ("steps", C.c_uint64),
        ("int_part", (C.c_uint64 * 128) * 3),
        ("digits", ((C.c_uint64 * 100) * 3) * 3),
        ("out_of_range", C.c_uint64 * 3),
    ]

    def digit_arrays(self):
        """(int_part [3, 128], digits [3, 3, 100], out_of_range [3]) as numpy."""
        ip = np.array([list(self.int_part[c]) for c in range(3)], dtype=np.uint64)
        dg = np.array([[list(self.digits[c][j]) for j in range(3)] for c in range(3)], dtype=np.uint64)
        return ip, dg, np.array(list(self.out_of_range), dtype=np.uint64)


_lib = None
_lock = threading.Lock()
_u8p = C.POINTER(C.c_uint8)


def lib():
    """Load (building first if needed) the oracle shared object.  The
    environment variable LCO_LIBRARY names another build of the same source
    to load instead (used by the test that plants mistakes in copies of the
    oracle and requires the pins to catch them)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("LCO_LIBRARY") or _build.build_oracle()
            L = C.CDLL(path)
            P, K, S, ST = C.POINTER(Params), C.POINTER(Key), C.POINTER(State), C.POINTER(Stats)
            sig = {
                "lco_params_v1": (None, [P]),
                "lco_params_check": (C.c_int, [P]),
                "lco_sha256": (None, [_u8p, C.c_size_t, _u8p]),
                "lco_key_schedule": (C.c_int, [P, _u8p, C.c_size_t, K]),
                "lco_euler_step": (None, [P, C.POINTER(C.c_double)]),
                "lco_sat_floor_i64": (C.c_int64, [C.c_double]),
                "lco_rbyte": (C.c_uint32, [C.c_double, C.c_uint32]),
                "lco_encode_byte": (C.c_uint32, [C.c_uint32, C.c_uint32, C.c_uint32]),
                "lco_decode_byte": (C.c_uint32, [C.c_uint32, C.c_uint32, C.c_uint32]),
                "lco_block_begin": (None, [P, K, C.c_uint64, S]),
                "lco_step_byte": (C.c_uint32, [P, K, S, C.c_uint32, C.c_int, ST]),
                "lco_nblocks": (C.c_size_t, [P, C.c_size_t, C.c_int]),
                "lco_ciphertext_len": (C.c_size_t, [P, C.c_size_t, C.c_int]),
                "lco_plaintext_len": (C.c_int, [P, C.c_size_t, C.c_int, C.POINTER(C.c_size_t)]),
                "lco_encrypt": (C.c_int, [P, _u8p, C.c_size_t, _u8p, C.c_size_t, _u8p, C.c_int]),
                "lco_decrypt": (C.c_int, [P, _u8p, C.c_size_t, _u8p, C.c_size_t, _u8p, C.c_int]),
                "lco_encrypt_blocks": (C.c_int, [P, K, _u8p, C.c_size_t, _u8p, C.c_size_t, C.c_size_t, ST]),
                "lco_decrypt_blocks": (C.c_int, [P, K, _u8p, C.c_size_t, _u8p, C.c_size_t, C.c_size_t, _u8p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def params(**over) -> Params:
    """The v1 parameters of the method, with optional field overrides
    (``lam`` and ``k`` take 3-sequences)."""
    p = Params()
    lib().lco_params_v1(C.byref(p))
    for k, v in over.items():
        if k in ("lam", "k"):
            arr = getattr(p, k)
            for i in range(3):
                arr[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def _buf(data):
    """(pointer, keepalive array) for bytes / numpy uint8 input."""
    arr = np.ascontiguousarray(np.frombuffer(bytes(data), dtype=np.uint8)
                               if isinstance(data, (bytes, bytearray)) else data,
                               dtype=np.uint8)
    if arr.size == 0:
        arr = np.zeros(1, dtype=np.uint8)[:0]
    return arr.ctypes.data_as(_u8p), arr


def _pw(pw):
    if isinstance(pw, str):
        pw = pw.encode("latin-1")
    return bytes(pw)


def sha256(msg: bytes) -> bytes:
    out = (C.c_uint8 * 32)()
    p, keep = _buf(msg)
    lib().lco_sha256(p, len(msg), out)
    return bytes(out)


def key_schedule(pw, prm: Params = None) -> Key:
    prm = prm or params()
    pw = _pw(pw)
    key = Key()
    p, keep = _buf(pw)
    rc = lib().lco_key_schedule(C.byref(prm), p if len(pw) else None, len(pw), C.byref(key))
    if rc:
        raise ValueError("password rejected (status %d)" % rc)
    return key


def euler_step(r, prm: Params = None):
    prm = prm or params()
    arr = (C.c_double * 3)(*r)
    lib().lco_euler_step(C.byref(prm), arr)
    return tuple(arr)


def sat_floor(v: float) -> int:
    return lib().lco_sat_floor_i64(v)


def rbyte(alpha: float, omega: int) -> int:
    return lib().lco_rbyte(alpha, omega)


def encode_byte(x, r1, r2) -> int:
    return lib().lco_encode_byte(x, r1, r2)


def decode_byte(y, r1, r2) -> int:
    return lib().lco_decode_byte(y, r1, r2)


def block_begin(key: Key, b: int, prm: Params = None) -> State:
    prm = prm or params()
    st = State()
    lib().lco_block_begin(C.byref(prm), C.byref(key), b, C.byref(st))
    return st


def step_byte(key: Key, st: State, x: int, direction: int = ENCRYPT,
              prm: Params = None, stats: Stats = None) -> int:
    prm = prm or params()
    return lib().lco_step_byte(C.byref(prm), C.byref(key), C.byref(st), x, direction,
                               C.byref(stats) if stats is not None else None)


def nblocks(n: int, mode: int = PARALLEL, prm: Params = None) -> int:
    prm = prm or params()
    return lib().lco_nblocks(C.byref(prm), n, mode)


def ciphertext_len(n: int, mode: int = PARALLEL, prm: Params = None) -> int:
    prm = prm or params()
    return lib().lco_ciphertext_len(C.byref(prm), n, mode)


def plaintext_len(c_len: int, mode: int = PARALLEL, prm: Params = None):
    """n, or None when no plaintext length maps to c_len."""
    prm = prm or params()
    n = C.c_size_t(0)
    rc = lib().lco_plaintext_len(C.byref(prm), c_len, mode, C.byref(n))
    return None if rc else n.value


def encrypt(pw, P, mode: int = PARALLEL, prm: Params = None) -> np.ndarray:
    prm = prm or params()
    pw = _pw(pw)
    pp, pkeep = _buf(P)
    n = pkeep.size
    out = np.zeros(ciphertext_len(n, mode, prm), dtype=np.uint8)
    wp, wkeep = _buf(pw)
    rc = lib().lco_encrypt(C.byref(prm), wp, len(pw), pp, n,
                           out.ctypes.data_as(_u8p), mode)
    if rc:
        raise ValueError("oracle encrypt failed (status %d)" % rc)
    return out


def decrypt(pw, Cbuf, mode: int = PARALLEL, prm: Params = None):
    """(status, plaintext).  status is OK or ERR_INTEGRITY (plaintext zeroed)
    or ERR_LENGTH / ERR_PASSWORD (plaintext None)."""
    prm = prm or params()
    pw = _pw(pw)
    cp, ckeep = _buf(Cbuf)
    n = plaintext_len(ckeep.size, mode, prm)
    if n is None:
        return ERR_LENGTH, None
    out = np.zeros(n, dtype=np.uint8)
    wp, wkeep = _buf(pw)
    rc = lib().lco_decrypt(C.byref(prm), wp, len(pw), cp, ckeep.size,
                           out.ctypes.data_as(_u8p), mode)
    if rc in (OK, ERR_INTEGRITY):
        return rc, out
    return rc, None


def encrypt_blocks(key: Key, P: np.ndarray, n: int, Cbuf: np.ndarray, b0: int, b1: int,
                   prm: Params = None, stats: Stats = None):
    """Parallel-mode parts [b0, b1) of a message of n bytes.  P is the whole
    plaintext (n bytes), Cbuf the whole ciphertext buffer; both numpy uint8."""
    prm = prm or params()
    assert P.dtype == np.uint8 and Cbuf.dtype == np.uint8
    assert P.flags.c_contiguous and Cbuf.flags.c_contiguous
    rc = lib().lco_encrypt_blocks(C.byref(prm), C.byref(key), P.ctypes.data_as(_u8p), n,
                                  Cbuf.ctypes.data_as(_u8p), b0, b1,
                                  C.byref(stats) if stats is not None else None)
    if rc:
        raise ValueError("oracle encrypt_blocks failed (status %d)" % rc)


def decrypt_blocks(key: Key, Cbuf: np.ndarray, n: int, P: np.ndarray, b0: int, b1: int,
                   prm: Params = None) -> np.ndarray:
    """Parallel-mode parts [b0, b1); returns the per-part tag verdicts."""
    prm = prm or params()
    ok = np.zeros(max(0, b1 - b0), dtype=np.uint8)
    rc = lib().lco_decrypt_blocks(C.byref(prm), C.byref(key), Cbuf.ctypes.data_as(_u8p), n,
                                  P.ctypes.data_as(_u8p), b0, b1, ok.ctypes.data_as(_u8p))
    if rc:
        raise ValueError("oracle decrypt_blocks failed (status %d)" % rc)
    return ok
