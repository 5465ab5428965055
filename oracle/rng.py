"""ctypes wrapper around ``oracle/rng.c`` (test infrastructure only).

The shared object is compiled on first use with ``gcc -O2 -ffp-contract=off``
so every binary32 step is the exact IEEE operation written in the source.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rng.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_rng.so")
_lock = threading.Lock()
_lib = None

# Streams of the Philox field (counter word 3, low byte).
STREAM_SKETCH_U = 0      # S^t, U-half (Section 3.2, eq. sketched_u)
STREAM_SKETCH_V = 1      # S'^t, V-half (eq. sketched_v)
STREAM_INIT_U = 2        # U^0 (Alg. 2 line 1)
STREAM_INIT_V = 3        # V^0


def build(force=False):
    """Compile rng.c into _build/liboracle_rng.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            f32p = ctypes.POINTER(ctypes.c_float)
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.ora_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.ora_uniform_open.argtypes = [ctypes.c_uint32]
            L.ora_uniform_open.restype = ctypes.c_float
            L.ora_uniform01.argtypes = [ctypes.c_uint32]
            L.ora_uniform01.restype = ctypes.c_float
            L.ora_lnf.argtypes = [ctypes.c_float]
            L.ora_lnf.restype = ctypes.c_float
            L.ora_sincos_turn.argtypes = [ctypes.c_uint32, f32p, f32p]
            L.ora_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, f32p, f32p]
            L.ora_field_words.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                          ctypes.c_int64, ctypes.c_int64, u32p]
            L.ora_gaussian_field.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                             ctypes.c_int64, ctypes.c_int64, ctypes.c_float, f32p]
            L.ora_uniform_field.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_int64, ctypes.c_int64, f32p]
            L.ora_feistel_half_bits.argtypes = [ctypes.c_int64]
            L.ora_feistel_half_bits.restype = ctypes.c_int
            L.ora_feistel_once.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                           ctypes.c_int, ctypes.c_uint32]
            L.ora_feistel_once.restype = ctypes.c_uint32
            L.ora_subsample.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                        ctypes.c_int64, ctypes.c_int64, i32p]
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: 4 counter words, 2 key words -> 4 output words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().ora_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def field_words(seed, stream, t, rows, cols):
    out = np.empty((rows, cols), dtype=np.uint32)
    lib().ora_field_words(seed, stream, t, rows, cols, _ptr(out, ctypes.c_uint32))
    return out


def lnf(u):
    return np.float32(lib().ora_lnf(float(np.float32(u))))


def sincos_turn(w):
    s = ctypes.c_float()
    c = ctypes.c_float()
    lib().ora_sincos_turn(int(w), ctypes.byref(s), ctypes.byref(c))
    return np.float32(s.value), np.float32(c.value)


def uniform_open(w):
    return np.float32(lib().ora_uniform_open(int(w)))


def box_muller(wa, wb):
    a = ctypes.c_float()
    b = ctypes.c_float()
    lib().ora_box_muller(int(wa), int(wb), ctypes.byref(a), ctypes.byref(b))
    return np.float32(a.value), np.float32(b.value)


def gaussian_scale(d):
    """1/sqrt(d) rounded once to binary32 (the scale of Section 3.4)."""
    return np.float32(1.0 / np.sqrt(np.float64(d)))


def gaussian_field(seed, stream, t, rows, cols, scale):
    """rows x cols binary32 Gaussian field times ``scale`` (exact bits)."""
    out = np.empty((rows, cols), dtype=np.float32)
    lib().ora_gaussian_field(seed, stream, t, rows, cols, float(np.float32(scale)),
                             _ptr(out, ctypes.c_float))
    return out


def rademacher_field(seed, stream, t, rows, cols, scale):
    """rows x cols binary32 field of +-scale: the sign is the top bit of the
    entry's Philox word (set bit: -scale)."""
    w = field_words(seed, stream, t, rows, cols)
    sc = np.float32(scale)
    return np.where((w >> np.uint32(31)) != 0, -sc, sc).astype(np.float32)


STREAM_COUNT = 0x30     # count sketch hashes (| side)


def count_buckets(seed, side, t, n, d):
    """Bucket h(i) in [0, d) and sign s(i) of each of the n rows of a count
    sketch: w = the field word of (row i, column 0) of stream 0x30 | side;
    h = ((w >> 1) * d) >> 31 (integer arithmetic), s = -1 if w is odd else +1."""
    w = field_words(seed, STREAM_COUNT | side, t, n, 1)[:, 0].astype(np.uint64)
    h = ((w >> np.uint64(1)) * np.uint64(d)) >> np.uint64(31)
    sgn = np.where((w & np.uint64(1)) != 0, -1.0, 1.0).astype(np.float32)
    return h.astype(np.int64), sgn


def count_field(seed, side, t, n, d):
    """The n x d count sketch as binary32: S[i][h(i)] = s(i), zero elsewhere."""
    h, sgn = count_buckets(seed, side, t, n, d)
    S = np.zeros((n, d), dtype=np.float32)
    S[np.arange(n), h] = sgn
    return S


STREAM_SRHT = 0x40      # SRHT row signs (| side); its column subset uses side 0x40 | side


def srht_pad(n):
    """Order of the Walsh-Hadamard matrix of an SRHT over n rows: the least
    power of two >= n (the rows are padded with zeros up to it)."""
    p = 1
    while p < n:
        p *= 2
    return p


def srht_signs(seed, side, t, n):
    """Diagonal D of the SRHT: -1 where the field word of (row i, column 0) of
    stream 0x40 | side has its top bit set, else +1."""
    w = field_words(seed, STREAM_SRHT | side, t, n, 1)[:, 0]
    return np.where((w >> np.uint32(31)) != 0, -1.0, 1.0)


def srht_columns(seed, side, t, n, d):
    """The d Hadamard columns R picks, drawn without replacement from
    {0..srht_pad(n)-1} by the subsampling draw with side 0x40 | side; ascending."""
    return subsample_indices(seed, STREAM_SRHT | side, t, srht_pad(n), d)


def _parity(x):
    """Parity of the set bits of each entry of a non-negative int array (< 2^32)."""
    x = np.asarray(x, dtype=np.uint64).copy()
    for sh in (16, 8, 4, 2, 1):
        x ^= x >> np.uint64(sh)
    return (x & np.uint64(1)).astype(np.int64)


def srht_field(seed, side, t, n, d, scale):
    """The n x d subsampled randomized Hadamard transform S = sqrt(p/d) D H R
    (Section 3.4's SRHT; p = srht_pad(n), H the p x p Walsh-Hadamard matrix of
    Sylvester's construction normalised by 1/sqrt(p), R the columns
    srht_columns) restricted to its first n rows, as binary32: entry (i, j) =
    D_i (-1)^popcount(i & J_j) * scale, with scale = float32(1/sqrt(d)) for
    the SRHT itself (sqrt(p/d) / sqrt(p)), or 1 for the unit draws."""
    D = srht_signs(seed, side, t, n)
    J = srht_columns(seed, side, t, n, d).astype(np.int64)
    i = np.arange(n, dtype=np.int64)
    H = 1.0 - 2.0 * _parity(i[:, None] & J[None, :])
    return (D[:, None] * H * np.float64(np.float32(scale))).astype(np.float32)


def uniform_field(seed, stream, t, rows, cols):
    out = np.empty((rows, cols), dtype=np.float32)
    lib().ora_uniform_field(seed, stream, t, rows, cols, _ptr(out, ctypes.c_float))
    return out


def feistel_half_bits(n):
    return int(lib().ora_feistel_half_bits(n))


def feistel_once(seed, side, t, h, x):
    return int(lib().ora_feistel_once(seed, side, t, h, x))


def subsample_indices(seed, side, t, n, d):
    """The d sampled indices of {0..n-1}, sorted ascending (Section 3.4)."""
    J = np.empty(d, dtype=np.int32)
    lib().ora_subsample(seed, side, t, n, d, _ptr(J, ctypes.c_int32))
    return np.sort(J)


def subsample_scale(n, d):
    """sqrt(n/d) rounded once to binary32 (makes E[S S^T] = I, Assumption 1)."""
    return np.float32(np.sqrt(np.float64(n) / np.float64(d)))
