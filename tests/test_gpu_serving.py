"""Serving engine (continuous batching): every request's bytes must be the
same when served in a mix of concurrent requests as when decoded alone
(tolerance 0), and both must equal the source bytes; admission control
refuses requests that can never fit the budget and queues the rest."""
import numpy as np
import pytest

import paper_2606_18900_gb300 as ace
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def corpus():
    fq = synth.tiny_fastq()
    fa = synth.fasta(40_000_000, seed=21, n_chrom=4)
    a_fq = ace.Archive(ace.encode(fq, min_match=16, reads=ace.fastq_index(fq)))
    a_fa = ace.Archive(ace.encode(fa, min_match=32, dist_bound=1 << 20))
    yield fq, fa, a_fq, a_fa
    a_fq.close()
    a_fa.close()


def make_requests(fq, fa, a_fq, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n):
        if rng.random() < 0.9:
            lo, hi = a_fq.read_lookup(int(rng.integers(0, 2000)))
            reqs.append((0, lo, hi))
        else:
            length = int(np.exp(rng.uniform(np.log(1024), np.log(4 << 20))))
            lo = int(rng.integers(0, fa.size - length))
            reqs.append((1, lo, lo + length))
    return reqs


def test_mix_equals_solo_and_source(corpus):
    fq, fa, a_fq, a_fa = corpus
    src = [fq, fa]
    arcs = [a_fq, a_fa]
    reqs = make_requests(fq, fa, a_fq, 400, 1)
    outs = [torch.zeros(hi - lo, dtype=torch.uint8, device="cuda") for _, lo, hi in reqs]
    with ace.Server(arcs, mem_budget=512 << 20, slots=3) as srv:
        tickets = [srv.submit(a, lo, hi, o) for (a, lo, hi), o in zip(reqs, outs)]
        lats = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == st["submitted"] == len(reqs) and st["refused"] == 0
    assert st["batches"] >= 1 and all(l >= 0 for l in lats)
    torch.cuda.synchronize()
    for (a, lo, hi), o in zip(reqs, outs):
        got = o.cpu().numpy()
        assert np.array_equal(got, src[a][lo:hi])
    # solo: the same requests one at a time through the range decoder
    for (a, lo, hi), o in list(zip(reqs, outs))[:60]:
        solo = torch.zeros(hi - lo, dtype=torch.uint8, device="cuda")
        arcs[a].decode_range(lo, hi, solo)
        arcs[a].check()
        assert torch.equal(solo, o)


def test_continuous_batching_overlaps(corpus):
    """Requests submitted while earlier batches run are served in later
    batches; with several slots, batches overlap."""
    fq, fa, a_fq, a_fa = corpus
    reqs = make_requests(fq, fa, a_fq, 200, 2)
    outs = [torch.zeros(hi - lo, dtype=torch.uint8, device="cuda") for _, lo, hi in reqs]
    with ace.Server([a_fq, a_fa], mem_budget=256 << 20, slots=4) as srv:
        tickets, waited = [], set()
        for i, ((a, lo, hi), o) in enumerate(zip(reqs, outs)):
            tickets.append(srv.submit(a, lo, hi, o))
            if i % 20 == 19:                  # a completed ticket is released by its wait
                srv.wait(tickets[-20])
                waited.add(tickets[-20])
        for t in tickets:
            if t not in waited:
                srv.wait(t)
        st = srv.stats()
    assert st["batches"] > 1
    src = [fq, fa]
    for (a, lo, hi), o in zip(reqs, outs):
        assert np.array_equal(o.cpu().numpy(), src[a][lo:hi])


def test_replay_overlaps_batches_on_the_device(corpus):
    """Open-loop arrivals from the library's own submitting thread (Poisson
    gaps, 50 us mean): requests that arrive while earlier batches run are
    admitted into later batches on other slots, so at least two batches are
    on the device at once, and every result equals its source bytes."""
    fq, fa, a_fq, a_fa = corpus
    reqs = make_requests(fq, fa, a_fq, 600, 3)
    outs = [torch.zeros(hi - lo, dtype=torch.uint8, device="cuda") for _, lo, hi in reqs]
    gaps = synth.poisson_gaps_ns(3, 1, len(reqs), 20_000.0)
    with ace.Server([a_fq, a_fa], mem_budget=512 << 20, slots=4) as srv:
        tickets, status, secs = srv.replay(reqs, outs, gaps)
        assert all(s == ace.OK for s in status) and all(tickets)
        lats = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["max_inflight"] >= 2 and st["batches"] > 1
    # the submitting thread kept to the trace: the last request went out close
    # to its due time
    assert secs < 1.5 * float(np.sum(gaps)) * 1e-9 + 0.05
    assert all(l >= 0 for l in lats)
    torch.cuda.synchronize()
    src = [fq, fa]
    for (a, lo, hi), o in zip(reqs, outs):
        assert np.array_equal(o.cpu().numpy(), src[a][lo:hi])


def test_admission_refusal_and_queueing(corpus):
    fq, fa, a_fq, a_fa = corpus
    # arenas of 48 segments: a 2 MiB range (128 segments) can never fit; a read
    # of the 42-segment FASTQ always can
    # (per slot and segment: a 4-byte page-table entry and an 8-byte flag word)
    budget = 12 * (a_fq.stats()["n_segments"] + a_fa.stats()["n_segments"]) * 2 + 2 * 48 * 16384
    with ace.Server([a_fq, a_fa], mem_budget=budget, slots=2) as srv:
        big = torch.zeros(2 << 20, dtype=torch.uint8, device="cuda")
        with pytest.raises(ace.AceapexError) as e:
            srv.submit(1, 0, 2 << 20, big)
        assert e.value.code == ace.EBUSY
        # many small requests: admitted batch by batch as slots free up
        outs, tickets = [], []
        for r in range(0, 2000, 17):
            lo, hi = a_fq.read_lookup(r)
            o = torch.zeros(hi - lo, dtype=torch.uint8, device="cuda")
            outs.append((lo, hi, o))
            tickets.append(srv.submit(0, lo, hi, o))
        for t in tickets:
            srv.wait(t)
        st = srv.stats()
    assert st["refused"] == 1 and st["completed"] == len(tickets)
    for lo, hi, o in outs:
        assert o.cpu().numpy().tobytes() == fq[lo:hi].tobytes()
