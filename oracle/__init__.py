"""ACEAPEX CPU oracle — TEST INFRASTRUCTURE ONLY.

Python access to ``oracle.c``: a plain, sequential encoder and decoder of the
archive format, written from the paper's §2 (absolute offsets,
global match search, fixed blocks, four streams), §4.1 (read-to-block index)
and §5 (64-bit fields, range decode). Only the tests, the package smoke
check and the benchmark's CPU-baseline leg may import this package; the GPU
library neither imports it nor shares code with it.

Pins (tests/test_oracle_*.py): round trip on random, structured and
adversarial inputs; a hand-derived worked example (tests/golden/abab_archive.txt); brute-force
enumeration of every legal command list on tiny inputs; the rANS final-state
invariant and the zero-order entropy bound; CRC-32 against zlib; the paper's
printed block and index arithmetic (§4.1, §5); record starts by brute force.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ECORRUPT, ENOMEM, ERANGE = 0, 1, 2, 3, 6
SYM_MAX = 16384

u8p = ctypes.POINTER(ctypes.c_uint8)
u64p = ctypes.POINTER(ctypes.c_uint64)
u32p = ctypes.POINTER(ctypes.c_uint32)


class Cmd(ctypes.Structure):
    _fields_ = [("lit_len", ctypes.c_uint32), ("mlen", ctypes.c_uint32), ("src", ctypes.c_uint64)]


class Info(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("n", "n_segments", "n_blocks", "n_deps", "n_reads", "D",
                                               "payload_bytes", "total_bytes")] + \
               [(k, ctypes.c_uint32) for k in ("log2_B", "log2_S", "W", "min_match", "max_level")]


CMD_DTYPE = np.dtype([("lit_len", np.uint32), ("mlen", np.uint32), ("src", np.uint64)])


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C, portable flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.orc_crc32.argtypes = [ctypes.c_uint32, u8p, ctypes.c_uint64]
            lib.orc_crc32.restype = ctypes.c_uint32
            lib.orc_crc32_bitwise.argtypes = [ctypes.c_uint32, u8p, ctypes.c_uint64]
            lib.orc_crc32_bitwise.restype = ctypes.c_uint32
            lib.orc_normalize.argtypes = [u64p, ctypes.POINTER(ctypes.c_uint16)]
            lib.orc_parse.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(ctypes.POINTER(Cmd)),
                                      ctypes.POINTER(u64p)]
            lib.orc_parse.restype = ctypes.c_int64
            lib.orc_serialize.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                          ctypes.c_uint64, ctypes.POINTER(Cmd), u64p, u64p, ctypes.c_uint64,
                                          ctypes.POINTER(u8p)]
            lib.orc_serialize.restype = ctypes.c_int64
            lib.orc_encode.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_uint32, u64p, ctypes.c_uint64, ctypes.POINTER(u8p)]
            lib.orc_encode.restype = ctypes.c_int64
            lib.orc_free.argtypes = [ctypes.c_void_p]
            lib.orc_decode.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint64]
            lib.orc_decode.restype = ctypes.c_int
            lib.orc_decode_wavefront.argtypes = [u8p, ctypes.c_uint64, u8p, ctypes.c_uint64, ctypes.c_int]
            lib.orc_decode_wavefront.restype = ctypes.c_int
            lib.orc_decode_stream.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.c_uint64, u32p, ctypes.c_uint64]
            lib.orc_decode_stream.restype = ctypes.c_int
            lib.orc_info.argtypes = [u8p, ctypes.c_uint64, ctypes.POINTER(Info)]
            lib.orc_info.restype = ctypes.c_int
            lib.orc_segment_info.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(Cmd), u64p, u8p,
                                             u64p, u32p]
            lib.orc_segment_info.restype = ctypes.c_int
            lib.orc_geometry.argtypes = [ctypes.c_uint64, ctypes.c_uint32, u64p, u64p, u32p, u32p]
            lib.orc_geometry.restype = ctypes.c_int
            lib.orc_fastq_record_starts.argtypes = [u8p, ctypes.c_uint64, u64p, ctypes.c_uint64]
            lib.orc_fastq_record_starts.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _buf(data) -> np.ndarray:
    if isinstance(data, np.ndarray):
        return np.ascontiguousarray(data, dtype=np.uint8).reshape(-1)
    return np.frombuffer(bytes(data), dtype=np.uint8).copy()


def _p8(a: np.ndarray):
    return a.ctypes.data_as(u8p)


def _take(ptr, n: int) -> np.ndarray:
    lib = _load()
    out = np.ctypeslib.as_array(ptr, shape=(n,)).copy() if n else np.empty(0, dtype=np.uint8)
    lib.orc_free(ptr)
    return out


# ------------------------------------------------------------------ encode

def parse(data, log2_B: int = 14, min_match: int = 8, max_level: int = 8, D: int = 0, chain: int = 16):
    """Encoder match search. Returns (commands as CMD_DTYPE array, cmd_ptr)."""
    lib = _load()
    buf = _buf(data)
    cp = ctypes.POINTER(Cmd)()
    pp = u64p()
    k = lib.orc_parse(_p8(buf), buf.size, log2_B, min_match, max_level, D, chain, ctypes.byref(cp), ctypes.byref(pp))
    if k < 0:
        raise OracleError(-k, "orc_parse")
    n_seg = (buf.size + (1 << min(log2_B, 14)) - 1) >> min(log2_B, 14)
    cmds = np.empty(k, dtype=CMD_DTYPE)
    if k:
        ctypes.memmove(cmds.ctypes.data, cp, k * CMD_DTYPE.itemsize)
    ptr = np.ctypeslib.as_array(pp, shape=(n_seg + 1,)).copy()
    lib.orc_free(cp)
    lib.orc_free(pp)
    return cmds, ptr


def serialize(data, cmds: np.ndarray, cmd_ptr: np.ndarray, log2_B: int = 14, min_match: int = 8,
              max_level: int = 8, D: int = 0, reads=None) -> np.ndarray:
    """Archive from explicit commands (the format's symbol message, rANS coding and layout)."""
    lib = _load()
    buf = _buf(data)
    cmds = np.ascontiguousarray(cmds, dtype=CMD_DTYPE)
    ptr = np.ascontiguousarray(cmd_ptr, dtype=np.uint64)
    r = np.ascontiguousarray(reads if reads is not None else np.empty(0), dtype=np.uint64)
    out = u8p()
    n = lib.orc_serialize(_p8(buf), buf.size, log2_B, min_match, max_level, D,
                          cmds.ctypes.data_as(ctypes.POINTER(Cmd)), ptr.ctypes.data_as(u64p),
                          r.ctypes.data_as(u64p), r.size, ctypes.byref(out))
    if n < 0:
        raise OracleError(-n, "orc_serialize")
    return _take(out, n)


def encode(data, log2_B: int = 14, min_match: int = 8, max_level: int = 8, D: int = 0, chain: int = 16,
           reads=None) -> np.ndarray:
    """Encode ``data`` (global match search + rANS) into an archive."""
    lib = _load()
    buf = _buf(data)
    r = np.ascontiguousarray(reads if reads is not None else np.empty(0), dtype=np.uint64)
    out = u8p()
    n = lib.orc_encode(_p8(buf), buf.size, log2_B, min_match, max_level, D, chain, r.ctypes.data_as(u64p),
                       r.size, ctypes.byref(out))
    if n < 0:
        raise OracleError(-n, "orc_encode")
    return _take(out, n)


# ------------------------------------------------------------------ decode

def info(arc) -> dict:
    lib = _load()
    a = _buf(arc)
    inf = Info()
    rc = lib.orc_info(_p8(a), a.size, ctypes.byref(inf))
    if rc:
        raise OracleError(rc, "orc_info")
    return {k: getattr(inf, k) for k, _ in Info._fields_}


def decode_status(arc, out: np.ndarray | None = None):
    """(status, output) without raising."""
    lib = _load()
    a = _buf(arc)
    n = 0
    if a.size >= 24:
        n = int(np.frombuffer(a[16:24].tobytes(), dtype="<u8")[0])
    if out is None:
        out = np.zeros(max(min(n, 1 << 36), 1), dtype=np.uint8)
    rc = lib.orc_decode(_p8(a), a.size, _p8(out), out.size)
    return rc, out[:n] if rc == OK else out


def decode(arc) -> np.ndarray:
    rc, out = decode_status(arc)
    if rc:
        raise OracleError(rc, "orc_decode")
    return out


def decode_wavefront(arc, threads: int) -> np.ndarray:
    """The segment decoder run level by level on `threads` host threads."""
    lib = _load()
    a = _buf(arc)
    n = info(a)["n"]
    out = np.zeros(max(n, 1), dtype=np.uint8)
    rc = lib.orc_decode_wavefront(_p8(a), a.size, _p8(out), out.size, threads)
    if rc:
        raise OracleError(rc, "orc_decode_wavefront")
    return out[:n]


def decode_stream_crcs(arc, lo: int, hi: int, window: int) -> np.ndarray:
    """One CRC-32 per window of [lo, hi), decoding through a ring (D > 0)."""
    lib = _load()
    a = _buf(arc)
    nw = max(1, (hi - lo + window - 1) // window)
    crcs = np.zeros(nw, dtype=np.uint32)
    rc = lib.orc_decode_stream(_p8(a), a.size, lo, hi, window, crcs.ctypes.data_as(u32p), nw)
    if rc:
        raise OracleError(rc, "orc_decode_stream")
    return crcs[: (hi - lo + window - 1) // window]


def segment_info(arc, s: int):
    """(status, commands, symbols, final lane states) of segment s."""
    lib = _load()
    a = _buf(arc)
    cmds = (Cmd * SYM_MAX)()
    nc = ctypes.c_uint64(0)
    sym = np.zeros(SYM_MAX, dtype=np.uint8)
    ns = ctypes.c_uint64(0)
    st = np.zeros(32, dtype=np.uint32)
    rc = lib.orc_segment_info(_p8(a), a.size, s, cmds, ctypes.byref(nc), _p8(sym), ctypes.byref(ns),
                              st.ctypes.data_as(u32p))
    c = np.frombuffer(bytes(cmds)[: nc.value * CMD_DTYPE.itemsize], dtype=CMD_DTYPE).copy()
    return rc, c, sym[: ns.value].copy(), st


def crc32(data, crc: int = 0) -> int:
    lib = _load()
    b = _buf(data)
    return int(lib.orc_crc32(crc, _p8(b), b.size))


def crc32_bitwise(data, crc: int = 0) -> int:
    lib = _load()
    b = _buf(data)
    return int(lib.orc_crc32_bitwise(crc, _p8(b), b.size))


def normalize(counts) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(counts, dtype=np.uint64)
    f = np.zeros(256, dtype=np.uint16)
    lib.orc_normalize(c.ctypes.data_as(u64p), f.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)))
    return f


def geometry(n: int, log2_B: int) -> dict:
    """Segment count, block count, offset width and segment exponent for n bytes."""
    lib = _load()
    ns, nb, w, ls = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32()
    rc = lib.orc_geometry(n, log2_B, ctypes.byref(ns), ctypes.byref(nb), ctypes.byref(w), ctypes.byref(ls))
    if rc:
        raise OracleError(rc, "orc_geometry")
    return {"n_segments": ns.value, "n_blocks": nb.value, "W": w.value, "log2_S": ls.value}


def fastq_record_starts(data) -> np.ndarray:
    lib = _load()
    b = _buf(data)
    n = lib.orc_fastq_record_starts(_p8(b), b.size, None, 0)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    lib.orc_fastq_record_starts(_p8(b), b.size, out.ctypes.data_as(u64p), n)
    return out[:n]


# ------------------------------------------------------- archive section views

def sections(arc) -> dict:
    """Raw header fields and section arrays of an archive (the format's section layout)."""
    a = _buf(arc)
    h = a[:128].tobytes()
    u64 = lambda o: int.from_bytes(h[o:o + 8], "little")
    n_seg, n_deps, n_reads = u64(40), u64(48), u64(56)
    off_dir, off_dep_ptr, off_deps, off_reads = u64(72), u64(80), u64(88), u64(96)
    d = a[off_dir: off_dir + 24 * n_seg]
    dirrec = np.frombuffer(d.tobytes(), dtype=np.dtype([("payload_off", "<u8"), ("n_words", "<u4"),
                                                         ("n_cmd", "<u4"), ("n_lit", "<u4"),
                                                         ("level", "<u2"), ("pad", "<u2")]))
    return {
        "N": u64(16), "log2_B": h[24], "log2_S": h[25], "W": h[26], "min_match": h[27], "max_level": h[30],
        "D": u64(32), "n_segments": n_seg, "n_deps": n_deps, "n_reads": n_reads,
        "off_payload": u64(104), "payload_bytes": u64(112), "total_bytes": u64(120),
        "tables": np.frombuffer(a[128:128 + 2048].tobytes(), dtype="<u2").reshape(4, 256),
        "dir": dirrec,
        "dep_ptr": np.frombuffer(a[off_dep_ptr: off_dep_ptr + 8 * (n_seg + 1)].tobytes(), dtype="<u8"),
        "deps": np.frombuffer(a[off_deps: off_deps + 4 * n_deps].tobytes(), dtype="<u4"),
        "reads": np.frombuffer(a[off_reads: off_reads + 8 * n_reads].tobytes(), dtype="<u8"),
    }
