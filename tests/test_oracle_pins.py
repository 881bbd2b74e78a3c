"""Pins of the CPU oracle against facts that do not come from the oracle
itself: the hand-derived worked example of the format, zlib's CRC-32, the
paper's printed arithmetic, the rANS final-state invariant and entropy bound,
round trips, and brute-force record scanning."""
import json
import math
import os
import zlib

import numpy as np
import pytest

import oracle
import synth
from conftest import GOLDEN, load_hex_fixture


# --------------------------------------------------------------- worked example

def test_worked_example_decodes():
    arc, meta = load_hex_fixture("abab_archive.txt")
    out = oracle.decode(arc)
    assert bytes(out) == bytes.fromhex(meta["output"][0])


def test_worked_example_serializer_bytes():
    """The encoder half must produce exactly the hand-derived bytes."""
    arc, meta = load_hex_fixture("abab_archive.txt")
    data = bytes.fromhex(meta["output"][0])
    cmds = np.array([tuple(int(v) for v in c.split(",")) for c in meta["commands"]], dtype=oracle.CMD_DTYPE)
    params = dict(kv.split("=") for kv in meta["params"])
    got = oracle.serialize(data, cmds, np.array([0, len(cmds)]), log2_B=int(params["log2_B"]),
                           min_match=int(params["min_match"]), max_level=int(params["max_level"]),
                           D=int(params["D"]))
    assert got.tobytes() == arc.tobytes()


def test_worked_example_state_arithmetic():
    """Lane states of the example follow from one rANS step (the format's rANS coding)."""
    rc, cmds, sym, states = oracle.segment_info(load_hex_fixture("abab_archive.txt")[0], 0)
    assert rc == oracle.OK
    assert list(sym) == [2, 0, 0, 0, 0, 0, 2, 0, 0, 0, 65, 66]
    assert [(c["lit_len"], c["mlen"], c["src"]) for c in cmds] == [(2, 2, 0), (0, 4, 0)]
    assert all(s == 65536 for s in states)


def test_renorm_order_example_decodes():
    """Second hand-derived archive: lanes 0 and 2 renormalise in the same step
    and take their words in ascending lane order (fixture comments)."""
    arc, meta = load_hex_fixture("renorm_order_archive.txt")
    want = bytes.fromhex(meta["output"][0])
    assert bytes(oracle.decode(arc)) == want
    rc, cmds, sym, states = oracle.segment_info(arc, 0)
    assert rc == oracle.OK and len(cmds) == 0
    assert bytes(sym) == want
    assert all(s == 65536 for s in states)


def test_renorm_order_example_discriminates_word_order():
    """With the two words swapped (what a descending-lane decoder would read)
    the archive still passes the final-state check but decodes differently,
    so the fixture pins the order and not only the states."""
    arc, meta = load_hex_fixture("renorm_order_archive.txt")
    swapped = arc.copy()
    swapped[2352:2356] = [0xFF, 0x0F, 0xFE, 0x0F]
    out = bytes(oracle.decode(swapped))
    want = bytes.fromhex(meta["output"][0])
    assert out != want and out[32] == ord("Y") and out[34] == ord("X") and out[:32] == want[:32]


# ------------------------------------------------------------------------ CRC

@pytest.mark.parametrize("n", [0, 1, 7, 64, 1000, 65537])
def test_crc32_equals_zlib(n):
    data = synth.random_bytes(11, n, n)
    assert oracle.crc32(data) == zlib.crc32(data.tobytes())
    assert oracle.crc32_bitwise(data) == zlib.crc32(data.tobytes())
    # chaining
    h = n // 2
    assert oracle.crc32(data[h:], oracle.crc32(data[:h])) == zlib.crc32(data.tobytes())


# ----------------------------------------------------------- paper arithmetic

def _paper():
    with open(os.path.join(GOLDEN, "paper_arithmetic.json")) as f:
        return json.load(f)


def test_paper_block_count_50gb():
    p = _paper()["blocks_50gb"]
    g = oracle.geometry(p["N"], p["log2_B"])
    assert g["n_blocks"] == p["n_blocks"]
    assert g["n_segments"] == p["n_blocks"]          # 16 KiB blocks are single segments
    assert g["W"] == 5                               # 5e10 < 2^40: 64-bit offsets need 5 bytes
    g2 = oracle.geometry(p["N"], 20)                 # 1 MiB blocks: 64 segments each
    assert g2["n_segments"] == p["n_blocks"] and g2["n_blocks"] == math.ceil(p["N"] / (1 << 20))


def test_paper_read_index_size():
    p = _paper()["index_5m_reads"]
    assert p["n_reads"] * p["bytes_per_read"] == p["index_bytes"]
    # the archive's read index section is exactly 8 bytes per read
    data = synth.tiny_fastq()
    reads = oracle.fastq_record_starts(data)
    a = oracle.encode(data, reads=reads)
    a0 = oracle.encode(data)
    s, s0 = oracle.sections(a), oracle.sections(a0)
    assert s["off_payload"] - s0["off_payload"] == pytest.approx(8 * len(reads), abs=15)
    q = _paper()["index_vs_fai"]
    assert q["fai_bytes"] / p["index_bytes"] == pytest.approx(q["ratio_printed"], abs=0.051)  # 6.25 printed as 6.3


def test_paper_timing_arithmetic():
    p = _paper()
    s = p["seek_speedup"]
    assert round(s["full_ms"] / s["seek_ms"]) == s["speedup_printed"]
    ph = p["phase_split"]
    assert ph["entropy_ms"] + ph["match_ms"] == pytest.approx(ph["total_ms"])
    assert ph["bytes"] / (ph["total_ms"] * 1e-3) / 1e9 == pytest.approx(ph["gbs_printed"], abs=0.1)


# ------------------------------------------------------------------ round trips

def _roundtrip(data, **kw):
    a = oracle.encode(data, **kw)
    out = oracle.decode(a)
    assert out.size == len(data)
    assert np.array_equal(out, np.asarray(data, dtype=np.uint8))
    return a


@pytest.mark.parametrize("n", [0, 1, 2, 255, 256, 257, 16383, 16384, 16385, 70001])
@pytest.mark.parametrize("alpha", [b"ab", b"ACGT", bytes(range(256))])
def test_roundtrip_random(n, alpha):
    data = synth.random_bytes(5, n + len(alpha), n, alpha)
    _roundtrip(data, log2_B=14, min_match=4 if len(alpha) > 2 else 8)


@pytest.mark.parametrize("log2_B", [2, 3, 4, 9, 14, 16])
def test_roundtrip_block_sizes(log2_B):
    data = synth.random_bytes(6, log2_B, 5000, b"ACGT")
    data[2000:3000] = data[100:1100]
    _roundtrip(data, log2_B=log2_B, min_match=2 if log2_B < 5 else 4)


def test_roundtrip_structured():
    runs = np.full(40000, ord("N"), dtype=np.uint8)
    a = _roundtrip(runs, min_match=8)
    # a run is coded as non-overlapping copies of earlier run bytes, so it compresses
    assert a.size < 10000
    periodic = np.frombuffer((b"ACGTTGCA" * 5000), dtype=np.uint8).copy()
    _roundtrip(periodic)
    _roundtrip(synth.tiny_fastq(), min_match=8)
    _roundtrip(synth.fasta(300_000, seed=9, n_chrom=3), min_match=9)


@pytest.mark.parametrize("cap", [0, 1, 2, 8])
def test_level_cap_and_deps(cap):
    data = synth.tiny_fastq()[:200_000]
    a = _roundtrip(data, max_level=cap)
    s = oracle.sections(a)
    assert s["dir"]["level"].max(initial=0) <= cap
    if cap == 0:
        assert s["n_deps"] == 0
    # stored deps are ascending and below their segment
    for seg in range(s["n_segments"]):
        d = s["deps"][s["dep_ptr"][seg]: s["dep_ptr"][seg + 1]]
        assert np.all(np.diff(d.astype(np.int64)) > 0) and np.all(d < seg)


def test_distance_bound():
    data = synth.fasta(400_000, seed=3, n_chrom=2)
    D = 50_000
    a = _roundtrip(data, D=D, min_match=9)
    s = oracle.sections(a)
    S = 1 << s["log2_S"]
    for seg in range(s["n_segments"]):
        rc, cmds, _, _ = oracle.segment_info(a, seg)
        assert rc == oracle.OK
        p = seg * S
        for c in cmds:
            p += int(c["lit_len"])
            assert p - int(c["src"]) <= D
            p += int(c["mlen"])


def test_encoder_deterministic():
    data = synth.tiny_fastq()
    assert np.array_equal(oracle.encode(data), oracle.encode(data))


# ------------------------------------------------------- format invariants

def test_invariants_fastq():
    """Every offset is below its output position (src + len <= dst), lengths
    sum to the segment size, every lane's final rANS state is 2^16 and every
    word is consumed; levels agree with the dependency lists."""
    data = synth.tiny_fastq()
    a = oracle.encode(data, min_match=8)
    s = oracle.sections(a)
    S = 1 << s["log2_S"]
    N = s["N"]
    levels = s["dir"]["level"]
    for seg in range(s["n_segments"]):
        rc, cmds, sym, states = oracle.segment_info(a, seg)
        assert rc == oracle.OK
        assert np.all(states == 65536)
        p = seg * S
        end = min(N, p + S)
        total = 0
        deps = set()
        for c in cmds:
            p += int(c["lit_len"])
            assert int(c["src"]) + int(c["mlen"]) <= p
            assert int(c["mlen"]) >= s["min_match"]
            for q in range(int(c["src"]) // S, (int(c["src"]) + int(c["mlen"]) - 1) // S + 1):
                if q != seg:
                    deps.add(q)
            p += int(c["mlen"])
            total += int(c["lit_len"]) + int(c["mlen"])
        n_trail = end - p
        assert n_trail >= 0
        assert total + n_trail == end - seg * S
        stored = s["deps"][s["dep_ptr"][seg]: s["dep_ptr"][seg + 1]]
        assert sorted(deps) == list(stored)
        assert levels[seg] == (0 if not deps else 1 + max(levels[d] for d in deps))


def test_entropy_bound():
    """Coded size stays within the rANS bound: the information content of the
    symbols under the stored tables plus at most 48 bits of state/flush slack
    per lane and segment; and the tables lose little against the empirical
    zero-order entropy of each class."""
    data = synth.tiny_fastq()
    a = oracle.encode(data, min_match=8)
    s = oracle.sections(a)
    tables = s["tables"].astype(np.float64)
    info_bits = 0.0
    counts = np.zeros((4, 256))
    for seg in range(s["n_segments"]):
        rc, cmds, sym, _ = oracle.segment_info(a, seg)
        n = len(cmds)
        W = s["W"]
        cls = np.concatenate([np.zeros(2 * n, int), np.ones(2 * n, int), np.full(W * n, 2),
                              np.full(len(sym) - (4 + W) * n, 3)])
        info_bits += float(np.sum(-np.log2(tables[cls, sym] / 4096.0)))
        np.add.at(counts, (cls, sym), 1)
        coded_bits = 16 * int(s["dir"]["n_words"][seg]) + 32 * 32
        assert coded_bits <= float(np.sum(-np.log2(tables[cls, sym] / 4096.0))) + 32 * 48
    h0 = 0.0
    for c in range(4):
        tot = counts[c].sum()
        if tot:
            p = counts[c][counts[c] > 0] / tot
            h0 += float(-(p * np.log2(p)).sum() * tot)
    assert info_bits <= h0 * 1.01 + 64
    words_bits = 16 * int(s["dir"]["n_words"].sum())
    assert words_bits <= h0 * 1.01 + 64


def test_normalize_rules():
    rng = np.random.default_rng(0)
    for trial in range(50):
        counts = np.zeros(256, dtype=np.uint64)
        k = int(rng.integers(1, 256))
        idx = rng.choice(256, size=k, replace=False)
        counts[idx] = rng.integers(1, 10**6, size=k).astype(np.uint64)
        f = oracle.normalize(counts)
        assert int(f.sum()) == 4096
        assert np.all((f > 0) == (counts > 0))
    assert int(oracle.normalize(np.zeros(256)).sum()) == 0


# ------------------------------------------------------------ corruption

def test_corruption_rejected():
    data = synth.tiny_fastq()[:100_000]
    a = oracle.encode(data, min_match=8)
    s = oracle.sections(a)

    def bad(mut):
        b = a.copy()
        mut(b)
        rc, _ = oracle.decode_status(b, np.zeros(200_000, np.uint8))
        return rc

    assert bad(lambda b: b.__setitem__(0, 0)) == oracle.ECORRUPT                   # magic
    assert bad(lambda b: b.__setitem__(26, 5)) == oracle.ECORRUPT                  # W
    assert bad(lambda b: b.__setitem__(128 + 2, b[128 + 2] ^ 1)) == oracle.ECORRUPT  # table sum
    off_payload = s["off_payload"]
    # an initial state below 2^16 is outside the state interval
    assert bad(lambda b: b.__setitem__(slice(off_payload, off_payload + 4), 0)) == oracle.ECORRUPT
    assert bad(lambda b: b.__setitem__(slice(off_payload + 2, off_payload + 4), 0)) == oracle.ECORRUPT
    rc, _ = oracle.decode_status(a[:-16], np.zeros(200_000, np.uint8))               # truncated
    assert rc == oracle.ECORRUPT
    # directory: payload offset of segment 1
    assert bad(lambda b: b.__setitem__(128 + 2048 + 24, b[128 + 2048 + 24] ^ 16)) == oracle.ECORRUPT
    # total length field
    assert bad(lambda b: b.__setitem__(120, b[120] ^ 1)) == oracle.ECORRUPT
    # level field of a segment that has deps
    if s["n_deps"]:
        seg = int(np.nonzero(np.diff(s["dep_ptr"]))[0][0])
        off = 128 + 2048 + 24 * seg + 20
        assert bad(lambda b: b.__setitem__(off, b[off] ^ 1)) == oracle.ECORRUPT


# -------------------------------------------------------------- read index

def test_state_perturbation_resynchronises():
    """A low-bit flip of an initial state may pass the final-state check (rANS
    re-synchronises), but the decoded bytes then differ from the input: the
    decoder's status alone is not a content check."""
    data = synth.tiny_fastq()[:100_000]
    a = oracle.encode(data, min_match=8)
    off = oracle.sections(a)["off_payload"]
    b = a.copy()
    b[off] ^= 1
    rc, out = oracle.decode_status(b, np.zeros(200_000, np.uint8))
    assert rc == oracle.ECORRUPT or not np.array_equal(out[:data.size], data)


def test_record_starts_bruteforce():
    data = synth.tiny_fastq()
    text = data.tobytes()
    starts, pos = [], 0
    for i, line in enumerate(text.split(b"\n")[:-1]):
        if i % 4 == 0:
            starts.append(pos)
        pos += len(line) + 1
    got = oracle.fastq_record_starts(data)
    assert list(got) == starts
    assert len(got) == 2000
    assert all(text[o] == ord("@") for o in got)


# ----------------------------------------------------------- streaming CRC

@pytest.mark.parametrize("D", [0, 20_000])
def test_stream_crcs_equal_zlib(D):
    data = synth.fasta(300_000, seed=8, n_chrom=2)
    a = oracle.encode(data, log2_B=12, D=D, min_match=9)
    for lo, hi, w in [(0, 300_000, 65536), (12345, 250_001, 10_000), (0, 1, 7), (5000, 5000 + 4096, 4096)]:
        crcs = oracle.decode_stream_crcs(a, lo, hi, w)
        ref = [zlib.crc32(data[b:min(hi, b + w)].tobytes()) for b in range(lo, hi, w)]
        assert list(crcs) == ref


def test_wavefront_decoder_equals_sequential():
    """The all-core baseline (the oracle's segment decoder run level by level
    on several threads) gives the sequential decoder's bytes, for many levels
    and for intra-segment chains."""
    import paper_2606_18900_gb300 as ace
    cases = [synth.pe_fastq(2 << 20, ref_len=300_000), synth.random_bytes(14, 2, 30_000, b"ab")]
    for d, kw in ((cases[0], dict(min_match=12)), (cases[1], dict(log2_B=6, min_match=2))):
        a = ace.encode(d, **kw)
        for t in (1, 3, 8):
            assert np.array_equal(oracle.decode_wavefront(a, t), d)


def _rans_decode_py(a: np.ndarray, sec: dict, seg: int):
    """rANS decode of one segment written out from the definition (Duda,
    arXiv:1311.2540; the interleaving rule of the format): symbol q belongs to
    lane q mod 32 and class c(q); slot = x mod 4096 selects the symbol s with
    cum[s] <= slot < cum[s] + f[s]; x <- f[s] * (x div 4096) + slot - cum[s];
    while x < 2^16 the lane shifts in the next 16-bit word."""
    d = sec["dir"][seg]
    nc, nl, nw, W = int(d["n_cmd"]), int(d["n_lit"]), int(d["n_words"]), int(sec["W"])
    n_sym = (4 + W) * nc + nl
    base = sec["off_payload"] + int(d["payload_off"])
    x = [int.from_bytes(a[base + 4 * j: base + 4 * j + 4].tobytes(), "little") for j in range(32)]
    words = a[base + 128: base + 128 + 2 * nw].view("<u2").astype(np.int64)
    freq = sec["tables"].astype(np.int64)
    cum = np.concatenate([np.zeros((4, 1), np.int64), np.cumsum(freq, axis=1)], axis=1)
    out = np.empty(n_sym, np.uint8)
    p = 0
    for q in range(n_sym):
        j = q % 32
        c = 0 if q < 2 * nc else 1 if q < 4 * nc else 2 if q < (4 + W) * nc else 3
        slot = x[j] % 4096
        sym = int(np.searchsorted(cum[c], slot, side="right")) - 1
        out[q] = sym
        x[j] = int(freq[c, sym]) * (x[j] // 4096) + slot - int(cum[c, sym])
        if x[j] < (1 << 16):
            x[j] = (x[j] << 16) + int(words[p])
            p += 1
    return out, x, p


def test_rans_against_an_independent_decoder():
    """The oracle's rANS (C) and a plain Python decoder written from the rANS
    definition give the same symbols, the final states 2^16 and every word
    consumed, on segments of archives from both encoders."""
    import paper_2606_18900_gb300 as ace
    d = synth.tiny_fastq()[:120_000]
    for a in (oracle.encode(d), ace.encode(d, min_match=16)):
        sec = oracle.sections(a)
        for seg in range(sec["n_segments"]):
            rc, cmds, sym, states = oracle.segment_info(a, seg)
            assert rc == 0
            got, x, p = _rans_decode_py(a, sec, seg)
            assert np.array_equal(got, sym), seg
            assert x == [1 << 16] * 32 and p == int(sec["dir"][seg]["n_words"])
