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
