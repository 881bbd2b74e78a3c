"""Full-size parity on the 1 GiB paired-end FASTQ workload, in the launch
configuration bench.py times (16 KiB and 1 MiB blocks): the GPU output must
equal the generator's input byte for byte, and the oracle decoder's output on
sampled segments (the oracle decodes the whole archive sequentially once)."""
import numpy as np
import pytest

import oracle
import paper_2606_18900_gb300 as ace
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def fastq_1g():
    return synth.pe_fastq(1 << 30)


@pytest.mark.parametrize("log2_B", [14, 20])
def test_fullsize_fastq(fastq_1g, log2_B):
    d = fastq_1g
    a = ace.encode(d, log2_B=log2_B, min_match=16, reads=ace.fastq_index(d))
    with ace.Archive(a) as arc:
        out = torch.empty(arc.size, dtype=torch.uint8, device="cuda")
        for _ in range(2):
            out.fill_(0)
            arc.decode_all(out)
            arc.check()
        got = out.cpu().numpy()
    assert got.size == d.size
    assert np.array_equal(got, d)
    if log2_B == 14:
        # one call from the pinned host archive to pinned host output: the
        # payload (about 400 MB, 13 pieces) is uploaded while the windows
        # decode and are copied back
        h_arc = torch.from_numpy(a).pin_memory()
        host = torch.zeros(d.size, dtype=torch.uint8).pin_memory()
        ace.decode_host(h_arc, host)
        assert np.array_equal(host.numpy(), d)
        want = oracle.decode(a)
        rng = np.random.default_rng(0)
        S = 1 << 14
        for s in rng.integers(0, d.size // S, 64):
            assert np.array_equal(got[s * S:(s + 1) * S], want[s * S:(s + 1) * S])
