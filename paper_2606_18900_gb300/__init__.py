"""GB300-native device-resident decoder for the absolute-offset LZ77 block
format of arXiv 2606.18900 ("Compressed-Resident Genomics").

This module is a thin ctypes binding over ``libaceapex.so`` (C ABI in
``include/aceapex.h``): it marshals arguments and nothing else. Every step of
the decode path runs in the library's CUDA kernels; PyTorch only provides
device memory and streams. There is no CPU fallback: when the library is
missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_SO_PLAIN = os.path.join(_HERE, "libaceapex.so")
_SO_PHASES = os.path.join(_HERE, "libaceapex_phases.so")
# ACEAPEX_LIBRARY=phases selects the build with per-phase cycle counters
# (bench.py's phase-split leg); any other value is the path of a library build.
_SO = {None: _SO_PLAIN, "": _SO_PLAIN, "phases": _SO_PHASES}.get(os.environ.get("ACEAPEX_LIBRARY"),
                                                                os.environ.get("ACEAPEX_LIBRARY"))
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
_SOURCES = ["kernels.cu", "gpu_encoder.cu", "host.cpp", "encoder.cpp", "server.cpp"]
_lock = threading.Lock()
_lib = None

OK, EINVAL, ECORRUPT, ENOMEM, ECUDA, ETIMEOUT, ERANGE, EBUSY = range(8)
STATUS = {0: "OK", 1: "EINVAL", 2: "ECORRUPT", 3: "ENOMEM", 4: "ECUDA", 5: "ETIMEOUT", 6: "ERANGE", 7: "EBUSY"}

ARCH = "-gencode=arch=compute_103a,code=sm_103a"


class AceapexError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {STATUS.get(code, code)}")
        self.code = code


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libaceapex.so in-tree for sm_103a (the translation units in
    parallel, then one link), and beside it libaceapex_phases.so, the same
    library with per-phase cycle counters in the decode kernels."""
    srcs = [os.path.join(_CSRC, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_CSRC, h) for h in ("format.h", "kernels.h", "archive.h", "encoder_rules.h")] + [os.path.join(_INCLUDE, "aceapex.h")]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and all(os.path.exists(p) and os.path.getmtime(p) >= newest for p in (_SO_PLAIN, _SO_PHASES)):
        return _SO_PLAIN
    nvcc = _nvcc()
    bdir = os.path.join(_HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + _CSRC, "-I" + _INCLUDE]

    def compile_one(job):
        src, obj, extra = job
        cmd = [nvcc, "-c", src, "-o", obj] + common + extra
        if src.endswith(".cu"):
            cmd += [ARCH, "-lineinfo", "-Xptxas", "-v" if verbose else "-O3"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    jobs = [(s, os.path.join(bdir, os.path.basename(s) + ".o"), []) for s in srcs]
    kern = os.path.join(_CSRC, "kernels.cu")
    jobs.append((kern, os.path.join(bdir, "kernels_phases.cu.o"), ["-DACEAPEX_PHASE_CLOCKS"]))
    with ThreadPoolExecutor(len(jobs)) as ex:
        objs = list(ex.map(compile_one, jobs))
    plain = objs[: len(srcs)]
    phased = [objs[-1] if os.path.basename(o) == "kernels.cu.o" else o for o in plain]
    for target, parts in ((_SO_PLAIN, plain), (_SO_PHASES, phased)):
        tmp = target + f".tmp{os.getpid()}"
        r = subprocess.run([nvcc, "-shared", ARCH, "-o", tmp] + parts + ["-lpthread"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, target)
    return _SO_PLAIN


class Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("decoded_bytes", "compressed_bytes", "match_bytes", "literal_bytes",
                                               "n_commands", "n_segments", "n_blocks", "n_deps", "n_reads")] + \
               [(k, ctypes.c_uint32) for k in ("max_level", "log2_B", "log2_S", "W")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class EncodeStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("ms_total", "ms_h2d", "ms_chains", "ms_match", "ms_parse",
                                               "ms_entropy", "ms_d2h")] + \
               [(k, ctypes.c_uint64) for k in ("input_bytes", "archive_bytes", "n_segments", "n_deps", "windows",
                                               "kernel_launches")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "refused", "batches", "bytes_served",
                                               "max_batch", "max_inflight", "queued", "slot_segments")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    """The loaded library (built first when out of date)."""
    global _lib
    with _lock:
        if _lib is None:
            if _SO in (_SO_PLAIN, _SO_PHASES) and not os.path.exists(_SO):
                build()
            L = ctypes.CDLL(_SO)
            vp, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.aceapex_open.argtypes = [vp, u64, i32, ctypes.POINTER(vp)]
            L.aceapex_close.argtypes = [vp]
            L.aceapex_close.restype = None
            L.aceapex_release_cached_memory.argtypes = [i32]
            L.aceapex_decoded_size.argtypes = [vp]
            L.aceapex_decoded_size.restype = u64
            L.aceapex_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
            L.aceapex_level_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_uint32]
            L.aceapex_decode_all.argtypes = [vp, vp, u64, vp, ctypes.POINTER(Stats)]
            L.aceapex_decode_range.argtypes = [vp, u64, u64, vp, u64, vp]
            L.aceapex_read_lookup.argtypes = [vp, u64, u64p, u64p]
            L.aceapex_range_closure.argtypes = [vp, u64, u64, u64p, ctypes.POINTER(ctypes.c_uint32)]
            L.aceapex_range_closure.restype = i32
            L.aceapex_last_error.argtypes = [vp, i32, vp]
            L.aceapex_set_wait_limit.argtypes = [vp, u64]
            L.aceapex_debug_block_segments.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), u32]
            L.aceapex_stream_range.argtypes = [vp, u64, u64, u64, u64, vp, vp]
            L.aceapex_decode_batch.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), vp]
            L.aceapex_encode.argtypes = [vp, u64, u32, u32, u32, u64, u64p, u64, i32, ctypes.POINTER(vp), u64p]
            L.aceapex_set_launch.argtypes = [vp, u32, u32, u32]
            L.aceapex_set_launch.restype = i32
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.aceapex_get_launch.argtypes = [vp, u32p, u32p, u32p, u32p]
            L.aceapex_get_launch.restype = i32
            L.aceapex_server_create.argtypes = [ctypes.POINTER(vp), i32, u64, i32, ctypes.POINTER(vp)]
            L.aceapex_server_create.restype = i32
            L.aceapex_server_destroy.argtypes = [vp]
            L.aceapex_server_destroy.restype = None
            L.aceapex_server_submit.argtypes = [vp, i32, u64, u64, vp, u64, u64p]
            L.aceapex_server_submit.restype = i32
            L.aceapex_server_poll.argtypes = [vp, u64, i32, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
            L.aceapex_server_poll.restype = i32
            L.aceapex_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
            L.aceapex_server_replay.argtypes = [vp, u64, ctypes.POINTER(i32), u64p, u64p, ctypes.POINTER(vp), u64p,
                                                u64p, u64p, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_double)]
            L.aceapex_server_replay.restype = i32
            L.aceapex_server_get_stats.restype = i32
            L.aceapex_decode_all_noalloc.argtypes = [vp, u64, vp, u64, vp, vp]
            L.aceapex_decode_all_noalloc.restype = i32
            L.aceapex_free.argtypes = [vp]
            L.aceapex_free.restype = None
            L.aceapex_fastq_index.argtypes = [vp, u64, u64p, u64]
            L.aceapex_fastq_index.restype = u64
            L.aceapex_decode_all_to_host.argtypes = [vp, vp, u64, u64, vp]
            L.aceapex_decode_host.argtypes = [vp, u64, i32, vp, u64, u64]
            L.aceapex_fastq_split.argtypes = [vp, u64, vp, u64p]
            L.aceapex_fastq_split.restype = u64
            L.aceapex_decode_fastq_streams.argtypes = [ctypes.POINTER(vp), vp, u64, vp]
            L.aceapex_fasta_index.argtypes = [vp, u64, u64p, u64, ctypes.POINTER(ctypes.c_uint32)]
            L.aceapex_fasta_index.restype = u64
            L.aceapex_region_lookup.argtypes = [vp, u64, u64, u64, ctypes.c_uint32, u64p, u64p]
            L.aceapex_decode_region.argtypes = [vp, u64, u64, u64, ctypes.c_uint32, vp, u64, vp]
            L.aceapex_gpu_encoder_create.argtypes = [i32, ctypes.POINTER(vp)]
            L.aceapex_gpu_encoder_create.restype = i32
            L.aceapex_gpu_encoder_destroy.argtypes = [vp]
            L.aceapex_gpu_encoder_destroy.restype = None
            L.aceapex_gpu_encode.argtypes = [vp, vp, i32, u64, u32, u32, u32, u64, u64p, u64, ctypes.POINTER(vp), u64p,
                                             ctypes.POINTER(EncodeStats)]
            L.aceapex_gpu_encode.restype = i32
            for f in ("aceapex_open", "aceapex_get_stats", "aceapex_decode_all", "aceapex_decode_range",
                      "aceapex_read_lookup", "aceapex_last_error", "aceapex_set_wait_limit",
                      "aceapex_debug_block_segments", "aceapex_stream_range", "aceapex_decode_batch",
                      "aceapex_encode"):
                getattr(L, f).restype = i32
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        raise AceapexError(rc, what)


def _ptr(x) -> int:
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return s.cuda_stream  # torch.cuda.Stream


def _as_u8(data) -> np.ndarray:
    if isinstance(data, np.ndarray):
        return np.ascontiguousarray(data.reshape(-1).view(np.uint8))
    return np.frombuffer(bytes(data), dtype=np.uint8)


# -------------------------------------------------------------------- host API

def encode(data, log2_B: int = 14, min_match: int = 0, max_level: int = 8, dist_bound: int = 0,
           reads=None, threads: int = 0) -> np.ndarray:
    """Host encoder of the library: returns the archive bytes (uint8 array)."""
    L = lib()
    buf = _as_u8(data)
    r = np.ascontiguousarray(reads if reads is not None else np.empty(0), dtype=np.uint64)
    out = ctypes.c_void_p()
    n = ctypes.c_uint64()
    rc = L.aceapex_encode(buf.ctypes.data if buf.size else None, buf.size, log2_B, min_match, max_level, dist_bound,
                          r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if r.size else None, r.size, threads,
                          ctypes.byref(out), ctypes.byref(n))
    _check(rc, "aceapex_encode")
    arr = np.empty(n.value, dtype=np.uint8)
    ctypes.memmove(arr.ctypes.data, out.value, n.value)
    L.aceapex_free(out)
    return arr


class GpuEncoder:
    """The GPU encoder on one device: the same archive as encode(), byte for
    byte, with the match search, parse and entropy coding in CUDA kernels.
    Keeps its device scratch between calls; close() (or a with block) frees
    it. last_stats holds the phase times of the latest call."""

    def __init__(self, device: int = 0):
        self._h = ctypes.c_void_p()
        _check(lib().aceapex_gpu_encoder_create(int(device), ctypes.byref(self._h)), "aceapex_gpu_encoder_create")
        self.device = int(device)
        self.last_stats = None

    def encode(self, data, log2_B: int = 14, min_match: int = 0, max_level: int = 8, dist_bound: int = 0,
               reads=None) -> np.ndarray:
        """Archive bytes (uint8 array) of data: a numpy array / bytes in host
        memory, or a contiguous uint8 torch tensor on this encoder's device."""
        if not self._h:
            raise ValueError("encoder is closed")
        on_dev = hasattr(data, "data_ptr") and getattr(data, "is_cuda", False)
        if on_dev:
            if not data.is_contiguous() or data.element_size() != 1:
                raise ValueError("device input must be a contiguous uint8 tensor")
            ptr, n, keep = data.data_ptr(), data.numel(), data
        else:
            keep = _as_u8(data)
            ptr, n = (keep.ctypes.data if keep.size else None), keep.size
        r = np.ascontiguousarray(reads if reads is not None else np.empty(0), dtype=np.uint64)
        out = ctypes.c_void_p()
        ln = ctypes.c_uint64()
        st = EncodeStats()
        rc = lib().aceapex_gpu_encode(self._h, ptr, 1 if on_dev else 0, n, log2_B, min_match, max_level, dist_bound,
                                      r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)) if r.size else None, r.size,
                                      ctypes.byref(out), ctypes.byref(ln), ctypes.byref(st))
        del keep
        _check(rc, "aceapex_gpu_encode")
        arr = np.empty(ln.value, dtype=np.uint8)
        ctypes.memmove(arr.ctypes.data, out.value, ln.value)
        lib().aceapex_free(out)
        self.last_stats = st.as_dict()
        return arr

    def close(self):
        if self._h:
            lib().aceapex_gpu_encoder_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fastq_index(data) -> np.ndarray:
    L = lib()
    buf = _as_u8(data)
    n = L.aceapex_fastq_index(buf.ctypes.data, buf.size, None, 0)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    L.aceapex_fastq_index(buf.ctypes.data, buf.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n)
    return out[:n]


def decode_host(archive, out, device: int = 0, window: int = 0):
    """Decode a host archive (numpy array or CPU tensor; pinned memory lets
    its upload overlap) into host memory `out` (CPU tensor or numpy array of
    at least the decoded size) in one call: aceapex_decode_host (open, upload
    overlapped with the window decodes and copies back, close)."""
    nbytes = archive.nbytes if isinstance(archive, np.ndarray) else archive.numel() * archive.element_size()
    cap = out.nbytes if isinstance(out, np.ndarray) else out.numel() * out.element_size()
    _check(lib().aceapex_decode_host(_ptr(archive), nbytes, int(device), _ptr(out), cap, window),
           "aceapex_decode_host")


def release_cached_memory(device: int = 0):
    """Return the device memory that the library keeps for reuse after
    closes on `device` (aceapex_release_cached_memory)."""
    _check(lib().aceapex_release_cached_memory(int(device)), "aceapex_release_cached_memory")


def fastq_split(data):
    """The four line streams of a FASTQ (headers, sequences, '+' lines,
    qualities) and its record count."""
    L = lib()
    buf = _as_u8(data)
    out = np.empty(max(buf.size, 1), dtype=np.uint8)
    lens = (ctypes.c_uint64 * 4)()
    n = L.aceapex_fastq_split(buf.ctypes.data, buf.size, out.ctypes.data, lens)
    cuts = np.cumsum([0] + [int(x) for x in lens])
    return [out[cuts[k]:cuts[k + 1]] for k in range(4)], int(n)


def decode_fastq_streams(parts, out, stream=None):
    """Reassemble a FASTQ from the Archives of its four line streams into out."""
    hs = (ctypes.c_void_p * 4)(*[p._h for p in parts])
    _check(lib().aceapex_decode_fastq_streams(hs, _ptr(out), out.numel() * out.element_size(), _stream(stream)),
           "aceapex_decode_fastq_streams")


def fasta_index(data):
    """(coordinate index, line width) of a FASTA buffer: for every record the
    offset of its '>' and of its first sequence byte."""
    L = lib()
    buf = _as_u8(data)
    w = ctypes.c_uint32(0)
    n = L.aceapex_fasta_index(buf.ctypes.data, buf.size, None, 0, None)
    out = np.zeros(max(n, 1), dtype=np.uint64)
    L.aceapex_fasta_index(buf.ctypes.data, buf.size, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), n,
                          ctypes.byref(w))
    return out[:n], int(w.value)


# ------------------------------------------------------------------- archives

class Archive:
    """A device-resident archive (aceapex_open / aceapex_close)."""

    def __init__(self, archive_bytes, device: int = 0):
        L = lib()
        buf = _as_u8(archive_bytes)
        h = ctypes.c_void_p()
        _check(L.aceapex_open(buf.ctypes.data, buf.size, device, ctypes.byref(h)), "aceapex_open")
        self._h = h
        self.device = device

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().aceapex_close(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def size(self) -> int:
        return int(lib().aceapex_decoded_size(self._h))

    def stats(self) -> dict:
        st = Stats()
        _check(lib().aceapex_get_stats(self._h, ctypes.byref(st)), "aceapex_get_stats")
        return st.as_dict()

    def level_counts(self) -> list:
        """Number of segments at each dependency level 0 .. max_level."""
        n = self.stats()["max_level"] + 1
        h = (ctypes.c_uint64 * n)()
        _check(lib().aceapex_level_counts(self._h, h, n), "aceapex_level_counts")
        return [int(x) for x in h]

    def decode_all(self, out, stream=None):
        """Decode the whole archive into device buffer ``out`` (async)."""
        cap = out.numel() * out.element_size() if hasattr(out, "numel") else int(out[1])
        _check(lib().aceapex_decode_all(self._h, _ptr(out if hasattr(out, "numel") else out[0]), cap,
                                        _stream(stream), None), "aceapex_decode_all")

    def decode_all_to_host(self, host_out, window: int = 0, stream=None):
        """Decode the whole archive into a (preferably pinned) host tensor,
        copying windows out while the next ones decode (async)."""
        cap = host_out.numel() * host_out.element_size()
        _check(lib().aceapex_decode_all_to_host(self._h, host_out.data_ptr(), cap, window, _stream(stream)),
               "aceapex_decode_all_to_host")

    def decode_range(self, lo: int, hi: int, out, stream=None):
        cap = out.numel() * out.element_size()
        _check(lib().aceapex_decode_range(self._h, lo, hi, _ptr(out), cap, _stream(stream)), "aceapex_decode_range")

    def range_closure(self, lo: int, hi: int):
        """(segments decoded, deepest level) of a range decode of [lo, hi)."""
        n, lv = ctypes.c_uint64(), ctypes.c_uint32()
        _check(lib().aceapex_range_closure(self._h, lo, hi, ctypes.byref(n), ctypes.byref(lv)),
               "aceapex_range_closure")
        return n.value, lv.value

    def read_lookup(self, read_id: int):
        lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().aceapex_read_lookup(self._h, read_id, ctypes.byref(lo), ctypes.byref(hi)), "aceapex_read_lookup")
        return lo.value, hi.value

    def region_lookup(self, chrom: int, pos: int, length: int, line_width: int = 60):
        """Byte range covering bases [pos, pos + length) of FASTA record chrom."""
        lo, hi = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().aceapex_region_lookup(self._h, chrom, pos, length, line_width, ctypes.byref(lo),
                                           ctypes.byref(hi)), "aceapex_region_lookup")
        return lo.value, hi.value

    def decode_region(self, chrom: int, pos: int, length: int, out, line_width: int = 60, stream=None):
        """Bases [pos, pos + length) of FASTA record chrom into out (newlines dropped)."""
        cap = out.numel() * out.element_size()
        _check(lib().aceapex_decode_region(self._h, chrom, pos, length, line_width, _ptr(out), cap,
                                           _stream(stream)), "aceapex_decode_region")

    def stream_range(self, lo: int, hi: int, ring_bytes: int, window: int, crc_out, stream=None):
        _check(lib().aceapex_stream_range(self._h, lo, hi, ring_bytes, window, _ptr(crc_out), _stream(stream)),
               "aceapex_stream_range")

    def last_error(self, sync: bool = True, stream=None) -> int:
        return int(lib().aceapex_last_error(self._h, int(sync), _stream(stream)))

    def check(self, stream=None):
        """Synchronise and raise if a kernel latched an error."""
        _check(self.last_error(True, stream), "device error")

    def set_wait_limit(self, ns: int):
        _check(lib().aceapex_set_wait_limit(self._h, ns), "aceapex_set_wait_limit")

    def set_launch(self, ctas: int = 0, warps_per_cta: int = 0, stage_bytes: int = 0):
        """Launch knobs of later decode calls (0 = default): persistent CTAs,
        working warps per CTA, shared staging bytes per warp."""
        _check(lib().aceapex_set_launch(self._h, ctas, warps_per_cta, stage_bytes), "aceapex_set_launch")

    def get_launch(self) -> dict:
        v = [ctypes.c_uint32() for _ in range(4)]
        _check(lib().aceapex_get_launch(self._h, *[ctypes.byref(x) for x in v]), "aceapex_get_launch")
        return dict(zip(("ctas", "max_ctas", "warps_per_cta", "stage_bytes"), [x.value for x in v]))

    def debug_block_segments(self, segs):
        a = np.ascontiguousarray(segs, dtype=np.uint32)
        _check(lib().aceapex_debug_block_segments(
            self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)) if a.size else None, a.size),
            "aceapex_debug_block_segments")


class Server:
    """Continuous-batching serving engine over device-resident archives
    (aceapex_server_*). Results land in caller-owned device buffers."""

    def __init__(self, archives, mem_budget: int = 2 << 30, slots: int = 4):
        self.archives = list(archives)          # keep the handles alive
        hs = (ctypes.c_void_p * len(self.archives))(*[a.handle for a in self.archives])
        h = ctypes.c_void_p()
        _check(lib().aceapex_server_create(hs, len(self.archives), mem_budget, slots, ctypes.byref(h)),
               "aceapex_server_create")
        self._h = h

    def submit(self, arc: int, lo: int, hi: int, out) -> int:
        """Queue [lo, hi) of archive `arc` into device tensor `out`; returns a ticket."""
        t = ctypes.c_uint64()
        _check(lib().aceapex_server_submit(self._h, arc, lo, hi, _ptr(out), out.numel() * out.element_size(),
                                           ctypes.byref(t)), "aceapex_server_submit")
        return t.value

    def replay(self, reqs, outs, gaps_ns):
        """Offer requests [(arc, lo, hi), ...] into device tensors `outs` with
        the given inter-arrival gaps (ns) from the library's own thread
        (aceapex_server_replay). Returns (tickets, status codes, seconds from
        the call to the last submission); a refused request has ticket 0."""
        n = len(reqs)
        arc = (ctypes.c_int * n)(*[r[0] for r in reqs])
        lo = (ctypes.c_uint64 * n)(*[r[1] for r in reqs])
        hi = (ctypes.c_uint64 * n)(*[r[2] for r in reqs])
        dst = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
        cap = (ctypes.c_uint64 * n)(*[o.numel() * o.element_size() for o in outs])
        gap = (ctypes.c_uint64 * n)(*[int(g) for g in gaps_ns])
        tk = (ctypes.c_uint64 * n)()
        stt = (ctypes.c_int * n)()
        secs = ctypes.c_double()
        _check(lib().aceapex_server_replay(self._h, n, arc, lo, hi, dst, cap, gap, tk, stt, ctypes.byref(secs)),
               "aceapex_server_replay")
        return list(tk), list(stt), secs.value

    def poll(self, ticket: int, wait: bool = False):
        """None while pending; else the latency in ms (raises on a failed request)."""
        done = ctypes.c_int()
        lat = ctypes.c_double()
        rc = lib().aceapex_server_poll(self._h, ticket, int(wait), ctypes.byref(done), ctypes.byref(lat))
        if not done.value:
            _check(rc, "aceapex_server_poll")
            return None
        _check(rc, "served request")
        return lat.value

    def wait(self, ticket: int) -> float:
        return self.poll(ticket, True)

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().aceapex_server_get_stats(self._h, ctypes.byref(st)), "aceapex_server_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().aceapex_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def decode_all_noalloc(d_archive, nbytes: int, out, status, stream=None) -> int:
    """aceapex_decode_all_noalloc: the archive is already in device memory
    (d_archive), nothing is allocated; returns the call's status code."""
    cap = out.numel() * out.element_size()
    return int(lib().aceapex_decode_all_noalloc(_ptr(d_archive), nbytes, _ptr(out), cap, _ptr(status),
                                                _stream(stream)))


def decode_batch(archives, outs, stream=None):
    """One persistent launch over several archives (aceapex_decode_batch)."""
    n = len(archives)
    hs = (ctypes.c_void_p * n)(*[a.handle for a in archives])
    ps = (ctypes.c_void_p * n)(*[_ptr(o) for o in outs])
    _check(lib().aceapex_decode_batch(hs, n, ps, _stream(stream)), "aceapex_decode_batch")
