"""Seeded synthetic genomic inputs shared by the oracle tests, the GPU tests
and the benchmark.

This package produces decompressed bytes only; it contains none of the
codec's arithmetic. The generators are C (``synth.c``) behind ctypes so that
the 1 GiB and 50 GB workloads generate in seconds; each function
states its recipe. Every function takes explicit seeds and is deterministic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_SRC = os.path.join(_HERE, "synth.c")
_lock = threading.Lock()
_lib = None

u64 = ctypes.c_uint64
u8p = ctypes.POINTER(ctypes.c_uint8)
u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (host C, portable flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.synth_reference.argtypes = [u64, u64, u64, ctypes.c_uint32, ctypes.c_uint32, u8p]
            lib.synth_reference.restype = ctypes.c_int
            lib.synth_fastq.argtypes = [u8p, u64, u64, u64, ctypes.c_int, ctypes.c_int, u64, u64,
                                        ctypes.c_int, u8p, u64p]
            lib.synth_fastq.restype = ctypes.c_int64
            lib.synth_fasta_new.argtypes = [u64, u64, u64, ctypes.c_int]
            lib.synth_fasta_new.restype = ctypes.c_void_p
            lib.synth_fasta_free.argtypes = [ctypes.c_void_p]
            lib.synth_fasta_read.argtypes = [ctypes.c_void_p, u8p, u64]
            lib.synth_fasta_read.restype = u64
            lib.synth_fasta_fill.argtypes = [u64, u64, u64, ctypes.c_int, ctypes.c_int, u8p]
            lib.synth_fasta_fill.restype = ctypes.c_int
            lib.synth_loguniform_sizes.argtypes = [u64, u64, u64, ctypes.c_double, ctypes.c_double, u64p]
            lib.synth_uniform.argtypes = [u64, u64, u64, u64, u64p]
            lib.synth_bytes.argtypes = [u64, u64, u64, u8p, ctypes.c_int, u8p]
            lib.synth_poisson_gaps.argtypes = [u64, u64, u64, ctypes.c_double, u64p]
            lib.synth_qualities.argtypes = [u64, u64, u64, u64, u8p]
            _lib = lib
    return _lib


def _p8(a: np.ndarray):
    return a.ctypes.data_as(u8p)


def _p64(a: np.ndarray):
    return a.ctypes.data_as(u64p)


def reference(seed_a: int, seed_b: int, length: int, repeat_frac: float = 0.0,
              n_families: int = 50) -> np.ndarray:
    """Random ACGT reference; optionally pasted with diverged repeat copies."""
    lib = _load()
    out = np.empty(length, dtype=np.uint8)
    rc = lib.synth_reference(seed_a, seed_b, length, int(round(repeat_frac * 1e6)), n_families, _p8(out))
    if rc != 0:
        raise MemoryError("synth_reference failed")
    return out


def fastq(ref: np.ndarray, seed_a: int, seed_b: int, *, paired: bool, max_bytes: int,
          max_units: int = 0, read_len: int = 150, truncate: bool = False):
    """FASTQ records sampled from ``ref``. Returns (bytes as uint8 array, units)."""
    lib = _load()
    out = np.empty(max_bytes, dtype=np.uint8)
    n_units = u64(0)
    n = lib.synth_fastq(_p8(ref), ref.size, seed_a, seed_b, int(paired), read_len, max_bytes,
                        max_units, int(truncate), _p8(out), ctypes.byref(n_units))
    if n < 0:
        raise MemoryError("synth_fastq failed")
    return out[:n].copy() if n < max_bytes // 2 else out[:n], int(n_units.value)


# ---------------------------------------------------------------- workloads

def tiny_fastq(seed: int = 1) -> np.ndarray:
    """2,000 single-end 150 bp reads from a 200 kb reference (about 0.7 MB)."""
    ref = reference(seed, 0, 200_000)
    data, n = fastq(ref, seed, 1, paired=False, max_bytes=4 << 20, max_units=2000)
    assert n == 2000
    return data


def pe_fastq(nbytes: int = 1 << 30, seed: int = 2, ref_len: int = 50_000_000) -> np.ndarray:
    """Interleaved paired-end FASTQ, last full pair within ``nbytes``; the
    reference carries 5% interspersed repeats (50 families)."""
    ref = reference(seed, 0, ref_len, repeat_frac=0.05, n_families=50)
    data, _ = fastq(ref, seed, 1, paired=True, max_bytes=nbytes)
    return data


def batch_sizes(n: int = 4096, seed: int = 3, lo: int = 16384, hi: int = 1 << 24) -> np.ndarray:
    """Log-uniform archive sizes in [lo, hi)."""
    lib = _load()
    out = np.empty(n, dtype=np.uint64)
    lib.synth_loguniform_sizes(seed, 0, n, float(lo), float(hi), _p64(out))
    return out


def batch_fastq(sizes, seed: int = 3, ref_len: int = 50_000_000, threads: int = 0):
    """One paired-end FASTQ per size, each cut to exactly its size; all share
    one reference drawn from ``seed`` and draw reads from seed (seed, 1000 + i).
    Archives are generated in parallel threads (the C generator releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor

    ref = reference(seed, 0, ref_len, repeat_frac=0.05, n_families=50)

    def one(i):
        d, _ = fastq(ref, seed, 1000 + i, paired=True, max_bytes=int(sizes[i]), truncate=True)
        return d.copy()

    with ThreadPoolExecutor(threads or (os.cpu_count() or 1)) as ex:
        return list(ex.map(one, range(len(sizes))))


class FastaStream:
    """Streaming FASTA genome of exactly ``total_bytes`` bytes."""

    def __init__(self, total_bytes: int, seed: int = 4, n_chrom: int = 24):
        self._lib = _load()
        self._h = self._lib.synth_fasta_new(seed, 0, total_bytes, n_chrom)
        if not self._h:
            raise ValueError("bad FASTA parameters")
        self.total = total_bytes

    def read_into(self, out: np.ndarray) -> int:
        return int(self._lib.synth_fasta_read(self._h, _p8(out), out.size))

    def read(self, n: int) -> np.ndarray:
        out = np.empty(n, dtype=np.uint8)
        k = self.read_into(out)
        return out[:k]

    def close(self):
        if self._h:
            self._lib.synth_fasta_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fasta(total_bytes: int, seed: int = 4, n_chrom: int = 24, threads: int = 0) -> np.ndarray:
    """The whole genome file; chromosomes are generated in parallel (same
    bytes as FastaStream)."""
    lib = _load()
    out = np.empty(total_bytes, dtype=np.uint8)
    threads = threads or min(64, os.cpu_count() or 1)
    if lib.synth_fasta_fill(seed, 0, total_bytes, n_chrom, threads, _p8(out)) != 0:
        raise ValueError("bad FASTA parameters")
    return out


def uniform(seed_a: int, seed_b: int, n: int, bound: int) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.uint64)
    lib.synth_uniform(seed_a, seed_b, n, bound, _p64(out))
    return out


def random_bytes(seed_a: int, seed_b: int, n: int, alphabet: bytes = bytes(range(256))) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.uint8)
    alpha = np.frombuffer(alphabet, dtype=np.uint8).copy()
    lib.synth_bytes(seed_a, seed_b, n, _p8(alpha), len(alphabet), _p8(out))
    return out


def qualities(n: int, seed: int = 6, read_len: int = 150) -> np.ndarray:
    """n bytes of back-to-back Phred+33 quality strings (the FASTQ quality
    model) with nothing between them: a literal-only symbol stream."""
    lib = _load()
    out = np.empty(n, dtype=np.uint8)
    lib.synth_qualities(seed, 0, n, read_len, _p8(out))
    return out


def poisson_gaps_ns(seed_a: int, seed_b: int, n: int, rate: float) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.uint64)
    lib.synth_poisson_gaps(seed_a, seed_b, n, rate, _p64(out))
    return out
