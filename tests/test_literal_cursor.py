"""The literal-placement cursor of the decode kernel, restated step by step
on the CPU: in the literal phase the 32 lanes of a warp hold 32 consecutive
literals per step; after the parse each command's stage record holds the end
of its literal run (in literal numbering) and the match bytes of all commands
up to it; a warp-uniform cursor walks the run ends that fall inside the step,
and a lane at or after a run end takes that command's cumulative match length
as its offset (the lanes before it keep the offset of the previous run end);
four steps without a run end skip the walk. Every literal must land where the
command list puts it (positions from the oracle's commands of each
segment)."""
import numpy as np
import pytest

import oracle
import paper_2606_18900_gb300 as ace
import synth

INF = 0xFFFF  # the sentinel record after the last command: beyond every literal


def cursor_positions(ll, ml, n_sym, b3):
    """Output offset of every literal as the kernel's cursor places them."""
    nc = len(ll)
    nl = n_sym - b3
    ends = np.cumsum(ll)   # run ends (the parse's first field)
    cum = np.cumsum(ml)    # match bytes of commands 0..c (its second field)
    lanes = np.arange(32)
    got = np.full(nl, -1, dtype=np.int64)
    st = {"K0": ((b3 & ~31) - b3) if (b3 & 31) else 0, "cu": 0, "Sc": 0,
          "E": int(ends[0]) if nc else INF}
    out_k = st["K0"]       # output offset of literal K0 before any match byte

    def bound():
        sl = np.full(32, st["Sc"], dtype=np.int64)
        while st["E"] - st["K0"] < 32:
            st["Sc"] = int(cum[st["cu"]])
            sl[lanes >= st["E"] - st["K0"]] = st["Sc"]
            st["cu"] += 1
            st["E"] = int(ends[st["cu"]]) if st["cu"] < nc else INF
        return sl + lanes

    t0 = (b3 + 31) & ~31
    if b3 & 31:                                   # the step that crosses into the literals
        o = bound()
        for j in range(32):
            if j >= -st["K0"] and t0 - 32 + j < n_sym:
                got[st["K0"] + j] = out_k + o[j]
        out_k += 32
        st["K0"] += 32
    while t0 + 128 <= n_sym:                      # blocks of four steps
        if st["E"] - st["K0"] >= 128:
            for u in range(4):
                got[st["K0"] + 32 * u + lanes] = out_k + st["Sc"] + lanes + 32 * u
            st["K0"] += 128
        else:
            for u in range(4):
                o = bound()
                got[st["K0"] + lanes] = out_k + 32 * u + o
                st["K0"] += 32
        out_k += 128
        t0 += 128
    while t0 + 32 <= n_sym:
        o = bound()
        got[st["K0"] + lanes] = out_k + o
        out_k += 32
        st["K0"] += 32
        t0 += 32
    if t0 < n_sym:
        o = bound()
        for j in range(32):
            if t0 + j < n_sym:
                got[st["K0"] + j] = out_k + o[j]
    return got


def match_offsets(ll, ml):
    """The match phase's view of the same records: for each chunk of 32
    commands, a command's match length is its cumulative sum less the
    previous command's (the previous chunk's last sum for the first lane), and
    its output starts at its run end plus the match bytes before it."""
    ends, cum = np.cumsum(ll), np.cumsum(ml)
    lens, dsts, mbase = [], [], 0
    for c0 in range(0, len(ll), 32):
        c = np.arange(c0, min(c0 + 32, len(ll)))
        before = np.concatenate(([mbase], cum[c[:-1]]))
        lens.append(cum[c] - before)
        dsts.append(ends[c] + before)
        mbase = int(cum[c[-1]])
    return (np.concatenate(lens), np.concatenate(dsts)) if lens else (np.array([]), np.array([]))


@pytest.mark.parametrize("case", ["fastq_16k", "fastq_64b", "fastq_16b", "random", "abab", "tiny"])
def test_cursor_places_every_literal(case):
    if case.startswith("fastq"):
        data = synth.pe_fastq(1 << 20, ref_len=200_000)
        lb = {"fastq_16k": 14, "fastq_64b": 6, "fastq_16b": 4}[case]
        data = data if lb == 14 else data[:60_000]
        arc = ace.encode(data, log2_B=lb, min_match=16 if lb > 4 else 2)
    elif case == "random":
        arc = ace.encode(synth.random_bytes(1, 2, 100_000), log2_B=14, min_match=4)
    elif case == "abab":
        arc = ace.encode(np.frombuffer(b"ABAB" * 30_000, dtype=np.uint8), log2_B=14, min_match=2)
    else:
        arc = ace.encode(synth.tiny_fastq(), log2_B=14, min_match=8)
    sec = oracle.sections(arc)
    W = sec["W"]
    for s in range(sec["n_segments"]):
        rc, cmds, sym, _ = oracle.segment_info(arc, s)
        assert rc == oracle.OK
        ll = cmds["lit_len"].astype(np.int64)
        ml = cmds["mlen"].astype(np.int64)
        b3 = (4 + W) * len(cmds)
        nl = len(sym) - b3
        want = np.empty(nl, dtype=np.int64)
        k = pos = 0
        for a, b in zip(ll, ml):
            want[k:k + a] = np.arange(pos, pos + a)
            k += a
            pos += a + b
        want[k:] = np.arange(pos, pos + nl - k)
        assert np.array_equal(cursor_positions(ll, ml, len(sym), b3), want), s
        lens, dsts = match_offsets(ll, ml)
        assert np.array_equal(lens, ml), s
        assert np.array_equal(dsts, np.cumsum(ll + ml) - ml), s
