"""Brute-force pins of the oracle on tiny inputs (n <= 10, alphabets {a,b}
and {A,C,G,T}, block sizes 4 and 8, min_match 2).

* Every legal command list (the format's command rules: lengths, non-overlap, matches kept
  inside their segment) is enumerated, serialized and decoded; each must
  reproduce the input byte for byte. This exercises every way commands,
  literals, intra-segment chains and cross-segment sources can combine.
* The oracle encoder's own parse must be one of the enumerated legal parses,
  and its cost under a fixed cost model (literal 9 bits, match 9 + 8W bits)
  can be no better than the exhaustive optimum.
"""
import itertools
import random

import numpy as np
import pytest

import oracle


def segment_parses(x, b, e, min_match, allow_src):
    """All command lists of segment [b, e): list of (cmds, n_trail)."""
    out = []

    def rec(p, lit_start, cmds):
        if p == e:
            out.append((list(cmds), e - lit_start))
            return
        rec(p + 1, lit_start, cmds)                       # literal at p
        for L in range(min_match, e - p + 1):
            for src in range(0, p - L + 1):               # src + L <= dst
                if not allow_src(src, L):
                    continue
                if x[src:src + L] == x[p:p + L]:
                    cmds.append((p - lit_start, L, src))
                    rec(p + L, p + L, cmds)
                    cmds.pop()

    rec(b, b, [])
    return out


def cost(cmds, n_trail, W):
    return sum(9 * c[0] + 9 + 8 * W for c in cmds) + 9 * n_trail


def all_parses(x, S, min_match, intra_only=False):
    n = len(x)
    segs = []
    for b in range(0, n, S):
        e = min(n, b + S)
        allow = (lambda src, L, b=b: src >= b) if intra_only else (lambda src, L: True)
        segs.append(segment_parses(x, b, e, min_match, allow))
    return segs


def to_arrays(combo):
    cmds, ptr = [], [0]
    for seg_cmds, _ in combo:
        cmds.extend(seg_cmds)
        ptr.append(len(cmds))
    return np.array(cmds, dtype=oracle.CMD_DTYPE) if cmds else np.zeros(0, oracle.CMD_DTYPE), np.array(ptr)


def inputs():
    cases = [bytes(t) for n in (1, 2, 5, 6, 8) for t in itertools.product(b"ab", repeat=n)]
    rng = random.Random(7)
    for _ in range(12):
        n = rng.randint(7, 10)
        cases.append(bytes(rng.choice(b"ab") for _ in range(n)))
        cases.append(bytes(rng.choice(b"ACGT") for _ in range(n)))
    cases.append(b"aaaaaaaaaa")
    cases.append(b"abababab")
    return cases


@pytest.mark.parametrize("log2_B", [2, 3])
def test_every_legal_parse_decodes(log2_B):
    S = 1 << log2_B
    rng = random.Random(log2_B)
    checked = 0
    for x in inputs():
        segs = all_parses(x, S, 2)
        combos_total = int(np.prod([len(s) for s in segs]))
        if combos_total <= 300:
            combos = itertools.product(*segs)
        else:
            combos = (tuple(rng.choice(s) for s in segs) for _ in range(300))
        for combo in combos:
            cmds, ptr = to_arrays(combo)
            arc = oracle.serialize(x, cmds, ptr, log2_B=log2_B, min_match=2, max_level=255)
            out = oracle.decode(arc)
            assert out.tobytes() == x, (x, combo)
            checked += 1
    assert checked > 1500


@pytest.mark.parametrize("log2_B", [2, 3])
@pytest.mark.parametrize("cap", [0, 255])
def test_oracle_parse_is_legal_and_not_better_than_optimum(log2_B, cap):
    S = 1 << log2_B
    for x in inputs():
        W = 1
        segs = all_parses(x, S, 2, intra_only=(cap == 0))
        optimum = sum(min(cost(c, t, W) for c, t in s) for s in segs)
        cmds, ptr = oracle.parse(x, log2_B=log2_B, min_match=2, max_level=cap, chain=64)
        got = 0
        for si, s in enumerate(segs):
            mine = [tuple(int(v) for v in c) for c in cmds[ptr[si]:ptr[si + 1]]]
            b = si * S
            e = min(len(x), b + S)
            n_trail = (e - b) - sum(c[0] + c[1] for c in mine)
            assert (mine, n_trail) in s, (x, si, mine)
            got += cost(mine, n_trail, W)
        assert got >= optimum
        arc = oracle.encode(x, log2_B=log2_B, min_match=2, max_level=cap, chain=64)
        assert oracle.decode(arc).tobytes() == x


def test_illegal_commands_rejected():
    x = b"abababab"
    bad = [
        ([(2, 4, 0)], 2),     # src + len > dst (overlapping copy)
        ([(2, 1, 0)], 2),     # shorter than min_match
        ([(2, 8, 0)], 2),     # runs past the segment end
    ]
    for cmds, mm in bad:
        arr = np.array(cmds, dtype=oracle.CMD_DTYPE)
        with pytest.raises(oracle.OracleError):
            oracle.serialize(x, arr, np.array([0, len(cmds)]), log2_B=3, min_match=mm, max_level=255)
    # a level above the cap
    y = b"abcdabcdabcdabcd"
    arr = np.array([(0, 4, 0), (0, 4, 4)], dtype=oracle.CMD_DTYPE)  # seg1 <- seg0, seg2 <- seg1
    with pytest.raises(oracle.OracleError):
        oracle.serialize(y, arr, np.array([0, 0, 1, 2, 2]), log2_B=2, min_match=2, max_level=1)
    arc = oracle.serialize(y, arr, np.array([0, 0, 1, 2, 2]), log2_B=2, min_match=2, max_level=2)
    assert oracle.decode(arc).tobytes() == y
    assert list(oracle.sections(arc)["dir"]["level"]) == [0, 1, 2, 0]
