"""GPU parity: every decode path of libaceapex.so (called through its C ABI)
must reproduce the oracle's decoded bytes exactly (integer work: bit-exact).
Archives come from the oracle encoder and from the library encoder; expected
bytes come from the oracle decoder and from the generator's original input."""
import zlib

import numpy as np
import pytest

import oracle
import paper_2606_18900_gb300 as ace
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def gpu_decode_all(arc_bytes, stream=None):
    with ace.Archive(arc_bytes) as a:
        n = a.size
        out = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        a.decode_all(out, stream)
        a.check(stream)
        return out[:n].cpu().numpy()


def assert_same(got, want):
    assert got.size == want.size
    if not np.array_equal(got, want):
        bad = np.nonzero(got != want)[0]
        raise AssertionError(f"{bad.size} bytes differ, first at {bad[0]} (of {want.size})")


# ------------------------------------------------------------------ whole file

def test_tiny_fastq_oracle_archive():
    d = synth.tiny_fastq()
    a = oracle.encode(d, reads=oracle.fastq_record_starts(d))
    want = oracle.decode(a)
    assert_same(want, d)
    assert_same(gpu_decode_all(a), want)


def test_tiny_fastq_library_archive():
    d = synth.tiny_fastq()
    a = ace.encode(d, min_match=16)
    assert_same(gpu_decode_all(a), oracle.decode(a))


def test_worked_example():
    from conftest import load_hex_fixture
    arc, meta = load_hex_fixture("abab_archive.txt")
    assert gpu_decode_all(arc).tobytes() == bytes.fromhex(meta["output"][0])


def test_renorm_order_example():
    """Hand-derived archive in which two lanes renormalise in one step: the
    words go to the lanes in ascending lane order."""
    from conftest import load_hex_fixture
    arc, meta = load_hex_fixture("renorm_order_archive.txt")
    assert gpu_decode_all(arc).tobytes() == bytes.fromhex(meta["output"][0])


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 255, 16383, 16384, 16385, 100_003])
def test_sizes_and_ragged_tails(n):
    d = synth.random_bytes(3, n, n, b"ACGT")
    if n > 200:
        d[n // 2: n // 2 + 100] = d[10:110]
    for enc in (oracle.encode, ace.encode):
        a = enc(d, min_match=4)
        assert_same(gpu_decode_all(a), oracle.decode(a))


@pytest.mark.parametrize("log2_B", [2, 3, 4, 6, 9, 12])
def test_small_blocks_many_segments(log2_B):
    """Tiny segments: many levels, intra-segment chains and sources that span
    two segments."""
    d = synth.random_bytes(4, log2_B, 20_000, b"ab")
    for enc, kw in ((oracle.encode, dict(chain=64)), (ace.encode, {})):
        a = enc(d, log2_B=log2_B, min_match=2, max_level=8, **kw)
        assert_same(gpu_decode_all(a), oracle.decode(a))


@pytest.mark.parametrize("alpha", [b"a", b"ab", b"ACGT", bytes(range(256))])
def test_alphabets(alpha):
    d = synth.random_bytes(5, len(alpha), 70_000, alpha)
    a = oracle.encode(d, min_match=4)
    assert_same(gpu_decode_all(a), d)


def test_runs_and_periodic():
    d = np.concatenate([np.full(50_000, 78, np.uint8), np.frombuffer(b"ACGTTGCA" * 9000, np.uint8),
                        np.full(3, 65, np.uint8)])
    for enc in (oracle.encode, ace.encode):
        a = enc(d, min_match=8)
        assert_same(gpu_decode_all(a), d)


@pytest.mark.parametrize("cap", [0, 1, 2, 8, 30])
def test_level_caps(cap):
    d = synth.pe_fastq(3 << 20, ref_len=1_000_000)
    a = ace.encode(d, max_level=cap, min_match=12)
    assert_same(gpu_decode_all(a), d)


@pytest.mark.parametrize("log2_B", [14, 20])
def test_medium_fastq_block_sizes(log2_B):
    d = synth.pe_fastq(24 << 20, ref_len=5_000_000)
    a = ace.encode(d, log2_B=log2_B, min_match=16)
    assert_same(gpu_decode_all(a), d)
    b = oracle.encode(d[: 4 << 20], log2_B=log2_B)
    assert_same(gpu_decode_all(b), oracle.decode(b))


def test_fasta_with_distance_bound():
    d = synth.fasta(6_000_000, seed=11, n_chrom=4)
    a = ace.encode(d, dist_bound=1 << 20, min_match=12)
    assert_same(gpu_decode_all(a), d)


def test_repeat_decode_same_handle_and_streams():
    d = synth.tiny_fastq()
    a = ace.encode(d, min_match=16)
    with ace.Archive(a) as arc:
        s = torch.cuda.Stream()
        for i in range(4):
            out = torch.zeros(arc.size, dtype=torch.uint8, device="cuda")
            arc.decode_all(out, s if i % 2 else None)
            arc.check(s if i % 2 else None)
            assert_same(out.cpu().numpy(), d)


def test_cuda_graph_replay():
    d = synth.tiny_fastq()
    a = ace.encode(d, min_match=16)
    with ace.Archive(a) as arc:
        out = torch.zeros(arc.size, dtype=torch.uint8, device="cuda")
        s = torch.cuda.Stream()
        arc.decode_all(out, s)        # first call allocates scratch outside capture
        arc.check(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            arc.decode_all(out, s)
        for _ in range(3):
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            assert arc.last_error() == ace.OK
            assert_same(out.cpu().numpy(), d)


# ------------------------------------------------------------- range / lookup

def test_decode_range_random_ranges():
    d = synth.pe_fastq(8 << 20, ref_len=2_000_000)
    a = ace.encode(d, min_match=16)
    rng = np.random.default_rng(1)
    with ace.Archive(a) as arc:
        cases = [(0, 1), (0, d.size), (d.size - 1, d.size), (16383, 16385), (5, 5)]
        for _ in range(20):
            lo = int(rng.integers(0, d.size))
            hi = int(min(d.size, lo + rng.integers(1, 300_000)))
            cases.append((lo, hi))
        for lo, hi in cases:
            out = torch.zeros(max(hi - lo, 1), dtype=torch.uint8, device="cuda")
            arc.decode_range(lo, hi, out)
            arc.check()
            assert_same(out[: hi - lo].cpu().numpy(), d[lo:hi])


def test_read_lookup_then_decode():
    d = synth.tiny_fastq()
    reads = oracle.fastq_record_starts(d)
    a = ace.encode(d, reads=ace.fastq_index(d), min_match=16)
    text = d.tobytes()
    with ace.Archive(a) as arc:
        for r in [0, 1, 2, 777, 1998, 1999]:
            lo, hi = arc.read_lookup(r)
            assert lo == reads[r] and hi == (reads[r + 1] if r + 1 < len(reads) else d.size)
            out = torch.zeros(hi - lo, dtype=torch.uint8, device="cuda")
            arc.decode_range(lo, hi, out)
            arc.check()
            rec = out.cpu().numpy().tobytes()
            assert rec == text[lo:hi] and rec.startswith(b"@SIM:") and rec.count(b"\n") == 4
        with pytest.raises(ace.AceapexError):
            arc.read_lookup(2000)


def test_decode_region_by_coordinates():
    """chr:pos lookups through the coordinate index: the bases of (record,
    position, length) equal the record's sequence with its newlines removed,
    across line ends, segment ends and record ends."""
    f = synth.fasta(3_000_000, seed=13, n_chrom=3)
    idx, width = ace.fasta_index(f)
    a = ace.encode(f, min_match=12, dist_bound=1 << 20, reads=idx)
    text = f.tobytes()
    seqs = []
    for k in range(len(idx) // 2):
        end = int(idx[2 * k + 2]) if 2 * k + 2 < len(idx) else len(text)
        seqs.append(text[int(idx[2 * k + 1]):end].replace(b"\n", b""))
    rng = np.random.default_rng(4)
    with ace.Archive(a) as arc:
        cases = [(0, 0, 1), (0, 0, 60), (0, 59, 2), (1, 0, 12345), (2, len(seqs[2]) - 1, 1),
                 (1, len(seqs[1]) - 150, 150)]
        for _ in range(40):
            k = int(rng.integers(0, len(seqs)))
            n = int(rng.integers(1, 20_000))
            p = int(rng.integers(0, len(seqs[k]) - n))
            cases.append((k, p, n))
        for k, p, n in cases:
            lo, hi = arc.region_lookup(k, p, n, width)
            raw = text[lo:hi]
            assert raw.replace(b"\n", b"") == seqs[k][p:p + n]
            out = torch.zeros(n, dtype=torch.uint8, device="cuda")
            arc.decode_region(k, p, n, out, width)
            arc.check()
            assert out.cpu().numpy().tobytes() == seqs[k][p:p + n], (k, p, n)
        for bad in [(3, 0, 1), (0, len(seqs[0]), 1), (0, len(seqs[0]) - 5, 6)]:
            with pytest.raises(ace.AceapexError) as e:
                arc.region_lookup(*bad, width)
            assert e.value.code == ace.ERANGE


@pytest.mark.parametrize("cut", [0, 1, 77])
def test_fastq_stream_separation_round_trip(cut):
    """A FASTQ stored as four archives of its line streams decodes (a launch
    per part, a device newline index per stream, one warp per record) back to
    the original bytes, also when the file ends inside a record."""
    d = synth.pe_fastq(6 << 20, ref_len=1_000_000)
    d = d[: d.size - cut]
    streams, n_rec = ace.fastq_split(d)
    parts = [ace.Archive(ace.encode(x, min_match=16)) for x in streams]
    out = torch.zeros(d.size, dtype=torch.uint8, device="cuda")
    ace.decode_fastq_streams(parts, out)
    for p in parts:
        p.check()
    assert_same(out.cpu().numpy(), d)
    for p in parts:
        p.close()


@pytest.mark.parametrize("window", [0, 1, 16384 * 7, 1 << 22])
def test_decode_all_to_host_windows(window):
    """Decode straight to pinned host memory in windows copied out while the
    next ones decode: the bytes equal the source for any window size (a
    window below a segment is one segment), twice in a row on one handle."""
    d = synth.pe_fastq(8 << 20, ref_len=2_000_000)
    a = ace.encode(d, min_match=16)
    with ace.Archive(a) as arc:
        for _ in range(2):
            host = torch.zeros(d.size, dtype=torch.uint8).pin_memory()
            s = torch.cuda.Stream()
            arc.decode_all_to_host(host, window, s)
            s.synchronize()
            arc.check(s)
            assert_same(host.numpy(), d)


def test_decode_all_to_host_window_sizes_on_one_handle():
    """One handle decodes to host memory with window sizes that change from
    call to call (each change remakes the windows' work lists on the device),
    ragged last windows included; every output equals the source, and a
    whole-file decode on the device between them too."""
    d = synth.pe_fastq((8 << 20) + 12345, ref_len=2_000_000)
    a = ace.encode(d, min_match=12, max_level=5)
    with ace.Archive(a) as arc:
        s = torch.cuda.Stream()
        for window in (1 << 20, 16384 * 5, 1 << 20, 0, 16384):
            host = torch.zeros(d.size, dtype=torch.uint8).pin_memory()
            arc.decode_all_to_host(host, window, s)
            s.synchronize()
            arc.check(s)
            assert_same(host.numpy(), d)
            out = torch.zeros(d.size, dtype=torch.uint8, device="cuda")
            arc.decode_all(out, s)
            arc.check(s)
            assert_same(out.cpu().numpy(), d)


@pytest.mark.parametrize("window", [0, 1 << 20, 16384])
def test_decode_host_one_call(window):
    """aceapex_decode_host: host archive in, host output out, in one call,
    equal to the source; a short output buffer is ERANGE, a damaged header
    ECORRUPT (host validation) and a damaged payload ECORRUPT (the decode's
    own checks), each without a fault."""
    d = synth.pe_fastq(8 << 20, ref_len=2_000_000)
    a = ace.encode(d, min_match=16)
    host = torch.zeros(d.size, dtype=torch.uint8).pin_memory()
    ace.decode_host(torch.from_numpy(a).pin_memory(), host, window=window)
    assert_same(host.numpy(), d)
    with pytest.raises(ace.AceapexError) as e:
        ace.decode_host(a, torch.zeros(d.size - 1, dtype=torch.uint8))
    assert e.value.code == ace.ERANGE
    bad = a.copy()
    bad[0] ^= 1
    with pytest.raises(ace.AceapexError) as e:
        ace.decode_host(bad, host)
    assert e.value.code == ace.ECORRUPT
    bad = a.copy()
    off = oracle.sections(a)["off_payload"]
    bad[off:off + 4] = 0  # the first segment's first state below 2^16
    with pytest.raises(ace.AceapexError) as e:
        ace.decode_host(bad, host)
    assert e.value.code == ace.ECORRUPT
    ace.decode_host(ace.encode(np.zeros(0, np.uint8)), torch.zeros(0, dtype=torch.uint8))  # N = 0


def test_level_counts_match_directory():
    d = synth.pe_fastq(2 << 20, ref_len=500_000)
    a = ace.encode(d, min_match=12, max_level=5)
    lv = oracle.sections(a)["dir"]["level"]
    with ace.Archive(a) as arc:
        assert arc.level_counts() == np.bincount(lv, minlength=arc.stats()["max_level"] + 1).tolist()


# -------------------------------------------------------------- ring streaming

@pytest.mark.parametrize("log2_B,lo,cut", [(14, 0, 0), (14, 3 << 14, 0), (14, 0, 16384 - 515), (8, 0, 0),
                                            (8, 256 * 5, 37)])
def test_stream_range_crcs(log2_B, lo, cut):
    """Per-window CRC-32 of ring streaming equals zlib on the source bytes, for
    16 KiB segments (row-strided hashing), 256-byte segments (per-lane tails
    only) and ends that cut the last segment short."""
    d = synth.fasta(5_000_000, seed=12, n_chrom=3)
    D = 1 << 18
    a = ace.encode(d, log2_B=log2_B, dist_bound=D, min_match=12)
    window = 1 << 19
    ring = 1 << 21
    hi = d.size - cut
    with ace.Archive(a) as arc:
        nw = (hi - lo + window - 1) // window
        crc = torch.zeros(nw, dtype=torch.int32, device="cuda")
        arc.stream_range(lo, hi, ring, window, crc)
        arc.check()
        got = [int(c) & 0xFFFFFFFF for c in crc.cpu().tolist()]
    want = [zlib.crc32(d[b:min(hi, b + window)].tobytes()) for b in range(lo, hi, window)]
    assert got == want
    assert list(oracle.decode_stream_crcs(a, lo, hi, window)) == want


# ------------------------------------------------------------------- batching

def test_decode_batch():
    sizes = [16384, 1, 50_000, 16385, 300_000, 2_000_000]
    datas = [synth.random_bytes(9, i, s, b"ACGT") for i, s in enumerate(sizes)]
    datas.append(synth.tiny_fastq())
    arcs = [ace.Archive(ace.encode(x, min_match=6)) for x in datas]
    outs = [torch.zeros(max(x.size, 1), dtype=torch.uint8, device="cuda") for x in datas]
    ace.decode_batch(arcs, outs)
    arcs[0].check()
    for x, o in zip(datas, outs):
        assert_same(o[: x.size].cpu().numpy(), x)
    for a in arcs:
        a.close()


# -------------------------------------------------------------- failure paths

def test_timeout_is_reported_and_context_survives():
    d = synth.pe_fastq(2 << 20, ref_len=500_000)
    a = ace.encode(d, min_match=12)
    s = oracle.sections(a)
    dep_of = np.nonzero(np.diff(s["dep_ptr"]))[0]
    assert dep_of.size
    victim = int(s["deps"][s["dep_ptr"][dep_of[0]]])
    with ace.Archive(a) as arc:
        arc.set_wait_limit(20_000_000)  # 20 ms
        arc.debug_block_segments([victim])
        out = torch.zeros(arc.size, dtype=torch.uint8, device="cuda")
        arc.decode_all(out)
        assert arc.last_error() == ace.ETIMEOUT
        arc.debug_block_segments([])
        arc.set_wait_limit(0)
        arc.decode_all(out)
        arc.check()
        assert_same(out.cpu().numpy(), d)


def test_corrupt_payload_is_reported():
    d = synth.tiny_fastq()
    a = ace.encode(d, min_match=16)
    s = oracle.sections(a)
    b = a.copy()
    b[s["off_payload"]: s["off_payload"] + 4] = 0      # state below 2^16
    with ace.Archive(b) as arc:
        out = torch.zeros(arc.size, dtype=torch.uint8, device="cuda")
        arc.decode_all(out)
        assert arc.last_error() == ace.ECORRUPT
        arc.decode_all(out)  # still usable
        assert arc.last_error() == ace.ECORRUPT
    with ace.Archive(a) as arc:
        out = torch.zeros(arc.size, dtype=torch.uint8, device="cuda")
        arc.decode_all(out)
        arc.check()
        assert_same(out.cpu().numpy(), d)


def test_out_cap_checked():
    a = ace.encode(synth.tiny_fastq(), min_match=16)
    with ace.Archive(a) as arc:
        small = torch.zeros(100, dtype=torch.uint8, device="cuda")
        with pytest.raises(ace.AceapexError) as e:
            arc.decode_all(small)
        assert e.value.code == ace.ERANGE


# ------------------------------------------------------- launch knobs / tuner

def test_launch_knobs_same_output():
    """Every launch shape gives the same bytes, including a staging size that
    forces the global staging slot and a single working warp per CTA."""
    d = synth.pe_fastq(6 << 20, ref_len=2_000_000)
    a = ace.encode(d, min_match=12)
    with ace.Archive(a) as arc:
        lim = arc.get_launch()["max_ctas"]
        for ctas, warps, stage in [(0, 0, 0), (1, 1, 0), (lim // 2, 7, 64), (3, 32, 1024), (lim, 16, 3072)]:
            arc.set_launch(ctas, warps, stage)
            got = arc.get_launch()
            assert got["warps_per_cta"] == (warps or 32) and got["stage_bytes"] == (stage or 3072)
            out = torch.zeros(arc.size, dtype=torch.uint8, device="cuda")
            arc.decode_all(out)
            arc.check()
            assert_same(out.cpu().numpy(), d)
        with pytest.raises(ace.AceapexError):
            arc.set_launch(0, 33, 0)


def test_batch_graph_replay_and_autotune(tmp_path):
    from paper_2606_18900_gb300 import autotune
    sizes = synth.batch_sizes(24, seed=13, hi=1 << 21)
    datas = synth.batch_fastq(sizes, seed=13, ref_len=1_000_000)
    arcs = [ace.Archive(ace.encode(x, min_match=16, threads=1)) for x in datas]
    outs = [torch.zeros(x.size, dtype=torch.uint8, device="cuda") for x in datas]
    s = torch.cuda.Stream()
    run = lambda: ace.decode_batch(arcs, outs, s)
    cands = [(8, 32, 3072), (arcs[0].get_launch()["max_ctas"], 16, 1024)]
    cfg, table = autotune.tune(arcs[0], run, key="test", stream=s, reps=1, cands=cands,
                               cache_path=str(tmp_path / "tune.json"))
    assert len(table) == 2 and cfg in [dict(t[0], ms=t[1]) for t in table]
    cfg2, table2 = autotune.tune(arcs[0], run, key="test", stream=s, cache_path=str(tmp_path / "tune.json"))
    assert table2 == [] and cfg2 == cfg          # served from the cache
    run()
    arcs[0].check(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        run()
    for _ in range(3):
        for o in outs:
            o.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert arcs[0].last_error() == ace.OK
        for x, o in zip(datas, outs):
            assert_same(o.cpu().numpy(), x)
    for a in arcs:
        a.close()


def _closure_edges(sec, lo, hi):
    """Dependency entries a host walk of [lo, hi)'s closure visits."""
    dp, deps, lS = sec["dep_ptr"], sec["deps"], sec["log2_S"]
    seen = set(range(lo >> lS, ((hi - 1) >> lS) + 1))
    stack, edges = list(seen), 0
    while stack:
        s = stack.pop()
        edges += int(dp[s + 1] - dp[s])
        for d in deps[dp[s]:dp[s + 1]]:
            if int(d) not in seen:
                seen.add(int(d))
                stack.append(int(d))
    return edges, len(seen)


def test_range_decode_with_wide_closures():
    """Reads of a paired-end FASTQ whose segments each draw on about a hundred
    earlier segments: closures too wide for the host walk (more than 16,384
    dependency entries) are found on the device. Every read and range equals
    the source, and the closure query agrees with a walk in Python."""
    data = synth.pe_fastq(32 << 20, ref_len=5_000_000)
    arc = ace.encode(data, min_match=16, reads=ace.fastq_index(data))
    sec = oracle.sections(arc)
    wide = 0
    with ace.Archive(arc) as a:
        n_reads = a.stats()["n_reads"]
        buf = torch.empty(2 << 20, dtype=torch.uint8, device="cuda")
        ranges = [a.read_lookup(int(r)) for r in synth.uniform(9, 1, 16, n_reads)]
        starts = synth.uniform(9, 2, 6, data.size // 2)
        ranges += [(data.size // 2 + int(s), min(data.size, data.size // 2 + int(s) + (1 << 20))) for s in starts]
        ranges += [(data.size - (1 << 20), data.size), (data.size // 2, data.size // 2 + 3), (0, 100)]
        for lo, hi in ranges:
            edges, nseg = _closure_edges(sec, lo, hi)
            wide += edges > 16384
            assert a.range_closure(lo, hi)[0] == nseg
            buf.fill_(0)
            a.decode_range(lo, hi, buf)
            a.check()
            assert bytes(buf[: hi - lo].cpu().numpy()) == data[lo:hi].tobytes(), (lo, hi)
    assert wide >= 3
