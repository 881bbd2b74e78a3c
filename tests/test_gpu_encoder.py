"""GPU encoder parity: for every input and parameter set, the GPU encoder's
archive must equal the host encoder's byte for byte, and the oracle must
decode it (validating every rule of the format on the way) back to the input.
The GPU decoder reads it back too. Inputs span the radix sort's tiles and
ragged tails, several parse batches (4-byte segments), sampled and full
hashing, a distance bound, small segments, min_match 1, and the degenerate
sizes."""
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
def enc():
    e = ace.GpuEncoder(0)
    yield e
    e.close()


def _inputs():
    tiny = synth.tiny_fastq()
    fa = synth.fasta(8_000_000, seed=41)
    pe = synth.pe_fastq(40_000_000, seed=42)
    rnd = synth.random_bytes(43, 1, 300_001)
    run = np.full(200_003, ord("A"), dtype=np.uint8)
    return {"tiny": tiny, "fasta": fa, "pe": pe, "random": rnd, "run": run}


_DATA = {}


def data(name):
    if not _DATA:
        _DATA.update(_inputs())
    return _DATA[name]


CASES = [
    ("tiny", dict(min_match=16), True),
    ("tiny", dict(), False),
    ("tiny", dict(log2_B=12, min_match=8, max_level=3), False),
    ("tiny", dict(min_match=40), False),
    ("tiny", dict(min_match=16, dist_bound=5000), False),
    ("tiny", dict(log2_B=10, min_match=6), False),
    ("tiny", dict(min_match=1), False),
    ("tiny", dict(log2_B=20, min_match=16, max_level=0), False),
    ("tiny", dict(log2_B=2, min_match=3), False),
    ("tiny", dict(log2_B=6, min_match=3, dist_bound=7), False),
    ("fasta", dict(min_match=32, dist_bound=1 << 20), False),
    ("fasta", dict(min_match=12), False),
    ("pe", dict(min_match=16), True),
    ("random", dict(), False),
    ("run", dict(), False),
]


def _check(enc, d, params, reads, decode_on_gpu=True):
    r = ace.fastq_index(d) if reads else None
    got = enc.encode(d, reads=r, **params)
    want = ace.encode(d, reads=r, **params)
    assert got.size == want.size
    assert got.tobytes() == want.tobytes()
    assert oracle.decode(got).tobytes() == np.asarray(d).tobytes()
    if decode_on_gpu and d.size:
        with ace.Archive(got) as a:
            out = torch.empty(a.size, dtype=torch.uint8, device="cuda")
            a.decode_all(out)
            a.check()
            assert np.array_equal(out.cpu().numpy(), d)
    return got


@pytest.mark.parametrize("name,params,reads", CASES, ids=[f"{c[0]}-{i}" for i, c in enumerate(CASES)])
def test_gpu_archive_equals_host_archive(enc, name, params, reads):
    _check(enc, data(name), params, reads)
    st = enc.last_stats
    assert st["input_bytes"] == data(name).size and st["ms_total"] > 0


@pytest.mark.parametrize("n", [0, 1, 7, 17, 16384, 16385])
def test_gpu_encoder_degenerate_sizes(enc, n):
    d = data("tiny")[:n].copy()
    _check(enc, d, dict(min_match=4), False, decode_on_gpu=n > 0)


def test_gpu_encoder_device_input_and_reuse(enc):
    d = data("pe")[:5_000_001]
    host = enc.encode(d, min_match=16)
    dev = enc.encode(torch.from_numpy(d.copy()).cuda(), min_match=16)
    assert host.tobytes() == dev.tobytes()
    # a smaller input after a larger one reuses the scratch
    small = data("tiny")
    assert enc.encode(small, min_match=16).tobytes() == ace.encode(small, min_match=16).tobytes()


def test_gpu_encoder_rejects_bad_arguments(enc):
    d = data("tiny")
    with pytest.raises(ace.AceapexError):
        enc.encode(d, log2_B=1)
    with pytest.raises(ace.AceapexError):
        enc.encode(d, min_match=300)
    with pytest.raises(ace.AceapexError):
        enc.encode(d, reads=np.array([5, 3], dtype=np.uint64))
    with pytest.raises(ace.AceapexError):
        enc.encode(d, dist_bound=1 << 31)
    # the encoder stays usable
    assert enc.encode(d, min_match=16).tobytes() == ace.encode(d, min_match=16).tobytes()


def test_gpu_encoder_two_windows():
    """Distance-bounded encode of more than one parse window (1 GiB each): the
    second window's chains start D bytes before it."""
    d = synth.fasta((1 << 30) + 5_000_000, seed=44)
    with ace.GpuEncoder(0) as e:
        got = e.encode(d, min_match=32, dist_bound=1 << 24)
        assert e.last_stats["windows"] == 2
    want = ace.encode(d, min_match=32, dist_bound=1 << 24)
    assert got.tobytes() == want.tobytes()
    with ace.Archive(got) as a:
        out = torch.empty(a.size, dtype=torch.uint8, device="cuda")
        a.decode_all(out)
        a.check()
        assert np.array_equal(out.cpu().numpy(), d)
