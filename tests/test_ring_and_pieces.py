"""CPU restatements of two pieces of the decode kernel's bookkeeping, checked
exhaustively or on random streams:

* the renormalisation-word ring: a 1 KiB ring of four 256-byte blocks filled
  by asynchronous 16-byte copies two blocks ahead of the reader, with the
  block of slot 0 also copied to the 256 bytes after the ring, read at
  unmasked addresses; every word a lane uses must be the right word of the
  stream, already copied and not yet overwritten, and no read may leave the
  1,280 bytes;
* the partial 16-byte output blocks of match copies: bytes [o, o + n) of a
  block written as naturally aligned pieces of 1, 2, 4 and 8 bytes, four
  pieces at most when one end is an end of the block, eight otherwise.

(The GPU tests check the kernel's output byte for byte; these tests check the
restated rules on every case, including ones no test archive reaches.)
"""
import random

import pytest

RING, MIRROR = 1024, 256


class Ring:
    """The ring with copy groups that complete at the waits."""

    def __init__(self, n_words):
        self.nw = n_words
        self.mem = [None] * (RING + MIRROR)  # (word index, group) per 2-byte word slot
        self.groups = []  # issued copy groups, oldest first: [writes, complete]

    def fetch(self, blk):
        writes = []
        for j in range(128):
            wi = blk * 128 + j
            if wi >= self.nw:
                continue
            # (the kernel copies 16-byte chunks that start before the last
            # word; a chunk's tail beyond it holds padding the decode never uses)
            writes.append(((blk & 3) * 256 + 2 * j, wi))
            if (blk & 3) == 0:
                writes.append((RING + 2 * j, wi))
        g = [writes, False]
        for off, _ in writes:
            self.mem[off // 2] = ("pending", g)
        self.groups.append(g)

    def wait(self, keep):
        for g in self.groups[: max(0, len(self.groups) - keep)]:
            if not g[1]:
                g[1] = True
                for off, wi in g[0]:
                    if self.mem[off // 2] == ("pending", g):
                        self.mem[off // 2] = wi

    def read(self, off):
        assert 0 <= off < RING + MIRROR, f"read at {off} leaves the ring"
        v = self.mem[off // 2]
        return v if isinstance(v, int) else None


def decode_stream(steps, groups, n_words):
    """Consumes `steps` (words taken by each step) in groups of at most four
    steps with an advance after each group but the last, as the command and
    literal loops do; returns the consumed byte count the kernel reports."""
    R = Ring(n_words)
    for b in range(4):
        R.fetch(b)
    R.wait(2)
    blk, wr, bnd = 0, 0, 256
    consumed = 0

    def advance():
        nonlocal blk, wr, bnd
        if wr >= bnd:
            blk += 1
            bnd += 256
            if bnd > RING:
                wr -= RING
                bnd -= RING
            R.fetch(blk + 3)
            R.wait(2)

    def step(k):
        nonlocal wr, consumed
        for r in range(32):  # every lane reads; lanes of rank < k use theirs
            off = wr + 2 * r
            got = R.read(off)
            if r < k:
                assert got == consumed + r, f"word {consumed + r} read as {got} at {off}"
        wr += 2 * k
        consumed += k

    i = 0
    for gi, g in enumerate(groups):
        assert 1 <= g <= 4
        for _ in range(g):
            step(steps[i])
            i += 1
        if gi + 1 < len(groups):
            advance()
    assert i == len(steps)
    return (blk & ~3) * 256 + wr, consumed


@pytest.mark.parametrize("seed", range(40))
def test_word_ring_reads_the_right_words(seed):
    rng = random.Random(seed)
    n_steps = rng.randrange(1, 600)
    style = seed % 4
    steps = []
    for _ in range(n_steps):
        if style == 0:
            steps.append(32)  # every lane every step: the fastest consumption
        elif style == 1:
            steps.append(rng.choice([0, 0, 1, 8, 31, 32]))
        else:
            steps.append(rng.randrange(0, 33))
    groups, left = [], n_steps
    while left:
        g = min(left, 4 if style < 2 else rng.randrange(1, 5))
        groups.append(g)
        left -= g
    total = sum(steps)
    wb, consumed = decode_stream(steps, groups, total)
    assert consumed == total
    assert wb == 2 * total  # the kernel's final check: bytes consumed == 2 * n_words


def pieces_one_sided(o, n):
    rise = o != 0
    out = []
    if n & 8:
        out.append((8 if rise else 0, 8))
    if n & 4:
        out.append((o + (n & 3) if rise else (n & 8), 4))
    if n & 2:
        out.append((o + (n & 1) if rise else (n & 12), 2))
    if n & 1:
        out.append((o if rise else (n & 14), 1))
    return out


def pieces_general(o, n):
    a, e, out = o, o + n, []
    if (a & 1) and a < e:
        out.append((a, 1)); a += 1
    if (a & 2) and a + 2 <= e:
        out.append((a, 2)); a += 2
    if (a & 4) and a + 4 <= e:
        out.append((a, 4)); a += 4
    if (a & 8) and a + 8 <= e:
        out.append((a, 8)); a += 8
    if a + 8 <= e:
        out.append((a, 8)); a += 8
    if a + 4 <= e:
        out.append((a, 4)); a += 4
    if a + 2 <= e:
        out.append((a, 2)); a += 2
    if a < e:
        out.append((a, 1)); a += 1
    return out


def test_partial_block_pieces_cover_exactly_and_are_aligned():
    for o in range(16):
        for n in range(1, 17 - o):
            if n == 16:
                continue  # a whole block: one 16-byte store
            one_sided = o == 0 or o + n == 16
            ps = pieces_one_sided(o, n) if one_sided else pieces_general(o, n)
            covered = sorted(b for a, s in ps for b in range(a, a + s))
            assert covered == list(range(o, o + n)), (o, n, ps)
            assert all(a % s == 0 for a, s in ps), (o, n, ps)
            assert len(ps) <= (4 if one_sided else 8)
            if one_sided:  # the general form gives the same bytes
                gen = sorted(b for a, s in pieces_general(o, n) for b in range(a, a + s))
                assert gen == covered
