"""Host-side checks of libaceapex.so that need no GPU: the library builds and
exports every entry point declared in include/aceapex.h; its encoder's
archives decode exactly under the oracle (an independent implementation of
the archive format); archive validation rejects damaged headers before any device
work."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2606_18900_gb300 as ace
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(aceapex_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = ace.lib()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_no_cpu_fallback_in_binding():
    """The binding forwards to the library only (no numpy/torch decode path)."""
    src = open(os.path.join(ROOT, "paper_2606_18900_gb300", "__init__.py")).read()
    assert "import oracle" not in src and "from oracle" not in src


@pytest.mark.parametrize("make", ["tiny", "random", "runs", "fasta"])
@pytest.mark.parametrize("log2_B", [3, 10, 14, 20])
def test_library_encoder_roundtrip_under_oracle(make, log2_B):
    if make == "tiny":
        d = synth.tiny_fastq()[:300_000]
    elif make == "random":
        d = synth.random_bytes(1, log2_B, 50_001, b"ACGT")
    elif make == "runs":
        d = np.repeat(np.frombuffer(b"ACGTN", np.uint8), [10000, 1, 30000, 7, 20000])
    else:
        d = synth.fasta(200_000, seed=2, n_chrom=2)
    mm = 2 if log2_B == 3 else 0
    a = ace.encode(d, log2_B=log2_B, min_match=mm)
    assert np.array_equal(oracle.decode(a), d)
    s = oracle.sections(a)
    assert s["dir"]["level"].max(initial=0) <= s["max_level"]


def test_library_encoder_params():
    d = synth.tiny_fastq()
    reads = ace.fastq_index(d)
    assert np.array_equal(reads, oracle.fastq_record_starts(d))
    for cap in (0, 1, 3, 8):
        a = ace.encode(d, max_level=cap, reads=reads, min_match=16)
        s = oracle.sections(a)
        assert s["dir"]["level"].max(initial=0) <= cap
        assert np.array_equal(s["reads"], reads)
        assert np.array_equal(oracle.decode(a), d)
    f = synth.fasta(500_000, seed=5, n_chrom=3)
    a = ace.encode(f, log2_B=12, dist_bound=40_000, min_match=12)
    s = oracle.sections(a)
    assert s["D"] == 40_000
    assert np.array_equal(oracle.decode(a), f)


@pytest.mark.parametrize("mm", [32, 48])
def test_library_encoder_sampled_long_matches(mm):
    """Long minimum matches switch the encoder to content-defined anchors with
    backward extension; archives still decode exactly under the oracle and
    respect every format rule (checked by the oracle's decoder)."""
    f = synth.fasta(3_000_000, seed=7, n_chrom=3)
    for D in (0, 1 << 20):
        a = ace.encode(f, min_match=mm, dist_bound=D)
        assert np.array_equal(oracle.decode(a), f)
        assert ace.encode(f, min_match=mm, dist_bound=D, threads=1).tobytes() == a.tobytes()
    assert a.size < f.size / 2


def test_library_encoder_deterministic_across_threads():
    d = synth.pe_fastq(4 << 20, ref_len=2_000_000)
    a1 = ace.encode(d, threads=1, min_match=16)
    a8 = ace.encode(d, threads=8, min_match=16)
    assert np.array_equal(a1, a8)


def test_fasta_coordinate_index():
    """Record and sequence starts of every FASTA record, and the line width,
    against a plain scan of the lines."""
    f = synth.fasta(1_500_000, seed=9, n_chrom=5)
    idx, width = ace.fasta_index(f)
    text = f.tobytes()
    want, pos = [], 0
    for line in text.split(b"\n")[:-1]:
        if line.startswith(b">"):
            want += [pos, pos + len(line) + 1]
        pos += len(line) + 1
    if not text.endswith(b"\n"):
        want.append(len(text) - 1)  # marks an unterminated last line
    assert idx.tolist() == want and len(want) in (10, 11)
    assert width == 60


def test_fastq_split_streams():
    """Line k of the FASTQ lands in stream k mod 4, in order; the streams hold
    every byte once; a FASTQ cut inside a record splits the same way."""
    d = synth.tiny_fastq()
    for cut in (d.size, d.size - 1, d.size - 200):
        x = d[:cut]
        streams, n_rec = ace.fastq_split(x)
        lines = x.tobytes().split(b"\n")
        if lines[-1] == b"":
            lines = lines[:-1]
            ends = [b"\n"] * len(lines)
        else:
            ends = [b"\n"] * (len(lines) - 1) + [b""]
        want = [b"".join(l + e for i, (l, e) in enumerate(zip(lines, ends)) if i % 4 == k) for k in range(4)]
        assert [s.tobytes() for s in streams] == want
        assert n_rec == (len(lines) + 3) // 4
        assert sum(s.size for s in streams) == x.size


@pytest.fixture(scope="module")
def encoder_emulation(tmp_path_factory):
    """tests/support/encoder_emulation.cu built for the host (nvcc)."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    csrc = os.path.join(ROOT, "paper_2606_18900_gb300", "csrc")
    exe = str(tmp_path_factory.mktemp("emul") / "encoder_emulation")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-I" + csrc, "-I" + os.path.join(ROOT, "include"),
                        "-gencode", "arch=compute_103a,code=sm_103a",
                        os.path.join(ROOT, "tests", "support", "encoder_emulation.cu"),
                        os.path.join(csrc, "encoder.cpp"), "-o", exe, "-lpthread"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


@pytest.mark.parametrize("make,cases", [
    ("tiny", ["14,16,8,0", "14,0,8,0", "12,8,3,0", "14,40,8,0", "14,16,8,5000", "10,6,8,0", "14,1,8,0",
              "2,3,8,0", "6,3,8,7", "20,16,0,0"]),
    ("fasta", ["14,32,8,1048576", "14,12,8,0"]),
    ("random", ["14,0,8,0"]),
    ("runs", ["14,0,8,0", "14,4,2,0"]),
])
def test_gpu_encoder_logic_equals_cpu_encoder(encoder_emulation, tmp_path, make, cases):
    """The GPU encoder's match search, parse, flattening and dependency lists
    (its __host__ __device__ functions, run on the host over a stable sort)
    give the CPU encoder's archive byte for byte: sampled and full hashing,
    distance bounds, 4-byte to 1 MiB blocks, level caps 0-8, min_match 1."""
    import subprocess
    data = {"tiny": lambda: synth.tiny_fastq(),
            "fasta": lambda: synth.fasta(3_000_000, seed=41),
            "random": lambda: synth.random_bytes(43, 1, 300_001),
            "runs": lambda: np.full(200_003, ord("A"), dtype=np.uint8)}[make]()
    f = tmp_path / "in.bin"
    data.tofile(f)
    r = subprocess.run([encoder_emulation, str(f)] + cases, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("same") == len(cases)


def test_gpu_encoder_fails_loudly_without_a_device():
    """No CPU fallback: without a CUDA device the GPU encoder cannot be made."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present (covered by the GPU tests)")
    with pytest.raises(ace.AceapexError):
        ace.GpuEncoder(0)


def test_empty_input():
    a = ace.encode(np.zeros(0, np.uint8))
    assert oracle.decode(a).size == 0


def _open_status(buf):
    lib = ace.lib()
    h = ctypes.c_void_p()
    b = np.ascontiguousarray(buf, dtype=np.uint8)
    return lib.aceapex_open(b.ctypes.data, b.size, 0, ctypes.byref(h))


def test_open_rejects_damaged_archives():
    a = ace.encode(synth.tiny_fastq()[:200_000], min_match=16)
    assert _open_status(a[:-16]) == ace.ECORRUPT
    for off, val in [(0, 0), (8, 2), (26, 7), (28, 11), (29, 16), (40, 99)]:
        b = a.copy()
        b[off] = val
        assert _open_status(b) == ace.ECORRUPT, off
    b = a.copy()
    b[128 + 1] ^= 4          # table sum
    assert _open_status(b) == ace.ECORRUPT
    s = oracle.sections(a)
    if s["n_deps"]:
        b = a.copy()         # level of a segment with dependencies
        seg = int(np.nonzero(np.diff(s["dep_ptr"]))[0][0])
        b[128 + 2048 + 24 * seg + 20] ^= 1
        assert _open_status(b) == ace.ECORRUPT
    lib = ace.lib()
    assert lib.aceapex_open(None, 10, 0, ctypes.byref(ctypes.c_void_p())) == ace.EINVAL


def test_decode_host_host_checks():
    """aceapex_decode_host runs the host checks before any device work: a
    null or empty archive is EINVAL and a damaged header or table ECORRUPT
    (without a GPU the checks still run; a sound archive then fails with
    ECUDA or decodes)."""
    lib = ace.lib()
    a = ace.encode(synth.tiny_fastq()[:200_000], min_match=16)
    out = np.zeros(200_000, np.uint8)

    def status(buf):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        return lib.aceapex_decode_host(b.ctypes.data, b.size, 0, out.ctypes.data, out.size, 0)

    assert lib.aceapex_decode_host(None, 10, 0, out.ctypes.data, out.size, 0) == ace.EINVAL
    assert lib.aceapex_decode_host(a.ctypes.data, 0, 0, out.ctypes.data, out.size, 0) == ace.EINVAL
    for off, val in [(0, 0), (8, 2), (26, 7), (40, 99)]:
        b = a.copy()
        b[off] = val
        assert status(b) == ace.ECORRUPT, off
    b = a.copy()
    b[128 + 1] ^= 4          # table sum
    assert status(b) == ace.ECORRUPT
    assert status(a) in (ace.OK, ace.ECUDA)
