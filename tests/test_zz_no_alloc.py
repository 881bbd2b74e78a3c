"""The allocation-free entry point (aceapex_decode_all_noalloc) serves callers
that may not allocate device memory while they decode, such as programs that
hand all device memory to their own pool at start-up. It must produce the
same bytes as aceapex_decode_all (bit-exact, like every decode test here) on
two calls in a row, and reject archives larger than its fixed scratch.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import paper_2606_18900_gb300 as ace
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def reference_decode(arc_bytes):
    with ace.Archive(arc_bytes) as a:
        out = torch.empty(a.size, dtype=torch.uint8, device="cuda")
        a.decode_all(out)
        a.check()
        return out.cpu().numpy()


@pytest.mark.parametrize("which", ["tiny_fastq", "pe_fastq_8m"])
def test_no_alloc_matches_decode_all(which):
    data = synth.tiny_fastq() if which == "tiny_fastq" else synth.pe_fastq(8 << 20, ref_len=2_000_000)
    arc = ace.encode(data, min_match=16)
    want = reference_decode(arc)
    assert np.array_equal(want, data)
    d_arc = torch.from_numpy(arc).to("cuda")        # caller-owned device copy of the archive
    out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for call in range(2):
        out.fill_(0)
        status.fill_(-1)
        rc = ace.decode_all_noalloc(d_arc, arc.size, out, status)
        assert rc == ace.OK, (call, rc)
        torch.cuda.synchronize()
        assert int(status.item()) == ace.OK, call
        assert np.array_equal(out.cpu().numpy(), want), call


def test_no_alloc_rejects_oversized_archive():
    data = synth.random_bytes(2, 2, 65537 * 16, b"ACGT")     # 16-byte segments: 65,537 of them
    arc = ace.encode(data, log2_B=4, min_match=4)
    d_arc = torch.from_numpy(arc).to("cuda")
    out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert ace.decode_all_noalloc(d_arc, arc.size, out, status) == ace.ERANGE
    small = torch.empty(10, dtype=torch.uint8, device="cuda")
    arc2 = ace.encode(synth.tiny_fastq(), min_match=16)
    assert ace.decode_all_noalloc(torch.from_numpy(arc2).to("cuda"), arc2.size, small, status) == ace.ERANGE


def _patched(arc, edits):
    a = arc.copy()
    for off, dtype, value in edits:
        a[off: off + np.dtype(dtype).itemsize] = np.frombuffer(np.array([value], dtype=dtype).tobytes(), np.uint8)
    return a


# Byte offsets of the archive layout: tables at 128 (four classes of 256 u16,
# the literal class last), the directory at 2176 (24 bytes per segment:
# payload offset u64, word count u32, command count u32, literal count u32,
# level u16).
_DIR = 2176


@pytest.mark.parametrize("what", ["table_sum", "symbol_count", "level", "payload_offset"])
def test_no_alloc_reports_corrupt_directory_on_the_device(what):
    """The directory and tables are not checked on the host by this entry
    point: the device rejects a bad record before touching memory through it,
    and the status word says ECORRUPT."""
    data = synth.pe_fastq(1 << 20, ref_len=200_000)
    arc = ace.encode(data, min_match=16)
    s = 5  # a segment in the middle
    rec = _DIR + 24 * s
    if what == "table_sum":
        lit = 128 + 3 * 512
        present = int(np.nonzero(arc[lit: lit + 512].view(np.uint16))[0][0])
        bad = _patched(arc, [(lit + 2 * present, np.uint16, int(arc[lit: lit + 512].view(np.uint16)[present]) + 1)])
    elif what == "symbol_count":
        bad = _patched(arc, [(rec + 12, np.uint32, 5000)])      # 5000 commands: more than 16,384 symbols
    elif what == "level":
        bad = _patched(arc, [(rec + 20, np.uint16, int(arc[30]) + 1)])  # above the archive's level cap
    else:
        payload_bytes = int(arc[112:120].view(np.uint64)[0])
        bad = _patched(arc, [(rec, np.uint64, payload_bytes - 64)])  # 16-byte aligned, but no room for the states
    d_arc = torch.from_numpy(bad).to("cuda")
    out = torch.empty(data.size, dtype=torch.uint8, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert ace.decode_all_noalloc(d_arc, bad.size, out, status) == ace.OK
    torch.cuda.synchronize()
    assert int(status.item()) == ace.ECORRUPT
    # the shared scratch is still good for the next call
    good = torch.from_numpy(arc).to("cuda")
    status.fill_(-1)
    assert ace.decode_all_noalloc(good, arc.size, out, status) == ace.OK
    torch.cuda.synchronize()
    assert int(status.item()) == ace.OK
    assert np.array_equal(out.cpu().numpy(), data)


def test_no_alloc_rejects_unpadded_payload_on_the_host():
    """A payload section whose length is not a multiple of 16 bytes would let
    the last 16-byte copy of a segment's words read past the archive: the
    header check rejects it before anything is queued."""
    arc = ace.encode(synth.tiny_fastq(), min_match=16)
    payload_bytes = int(arc[112:120].view(np.uint64)[0])
    total = int(arc[120:128].view(np.uint64)[0])
    bad = np.concatenate([_patched(arc, [(112, np.uint64, payload_bytes + 8), (120, np.uint64, total + 8)]),
                          np.zeros(8, np.uint8)])
    d_arc = torch.from_numpy(bad).to("cuda")
    out = torch.empty(arc.size * 8, dtype=torch.uint8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert ace.decode_all_noalloc(d_arc, bad.size, out, status) == ace.ECORRUPT
