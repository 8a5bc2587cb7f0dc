"""Index model of the ring form of the local solves' look-ahead sweep.

The ring form (Sec. 3.1 local solves A_j^-1, and the shift-invert solves of
Sec. 3.3.2, for subdomains whose local vector exceeds shared memory) keeps
tile row I of the vector in slot I mod rows of a ring of `rows` slots.  In
step q of a sweep (row I = q, or nt - 1 - q backward):

- the far warps read the rows at distance 2..dmax(I + 1) from the next row
  I + 1 and, after that, one of them fills the slot of row I + 1 with its
  right-hand side;
- the chain warps read row I (its right-hand side) and row I - 1 (the
  coupling; read even when the band has no off-diagonal tile, w = 0), then
  write the solved row I into its slot.

This model replays that schedule on slot tags and checks, for every tile
count and half-bandwidth up to 40, that every read finds the row it wants and
that no slot read in a step is refilled in the same step, with the ring size
the kernels use (max(w + 2, 3)).  The least size that works is max(w + 1, 3)
(the w rows a step reads plus the one it fills; three when the chain's
previous row and the refill would otherwise share a slot), and one slot fewer
than that must fail, so the model does detect a ring that is too small.  No
GPU needed.
"""
import pytest


def ring_rows(w):
    return max(w + 2, 3)


def replay(nt, w, backward, rows):
    """True when the schedule is race-free and every read is correct."""
    ring = [None] * rows

    def row(q):
        return nt - 1 - q if backward else q

    def dmax(i):
        return min(w, nt - 1 - i) if backward else min(w, i)

    def behind(i, d):
        return i + d if backward else i - d

    if nt > 0:
        ring[row(0) % rows] = ("b", row(0))
    for q in range(nt):
        i = row(q)
        read = set()
        if q + 1 < nt:
            nxt = row(q + 1)
            for d in range(2, dmax(nxt) + 1):
                j = behind(nxt, d)
                read.add(j % rows)
                if ring[j % rows] != ("y", j):
                    return False
        read.add(i % rows)
        if ring[i % rows] != ("b", i):
            return False
        if q > 0:
            j = behind(i, 1)
            read.add(j % rows)
            if ring[j % rows] != ("y", j):
                return False
        if q + 1 < nt:
            nxt = row(q + 1)
            if nxt % rows in read:
                return False
            ring[nxt % rows] = ("b", nxt)
        ring[i % rows] = ("y", i)
    return True


@pytest.mark.parametrize("backward", [False, True])
def test_ring_size_is_sufficient(backward):
    for nt in range(1, 41):
        for w in range(0, nt + 1):
            assert replay(nt, w, backward, ring_rows(w)), (nt, w)


@pytest.mark.parametrize("backward", [False, True])
def test_least_ring_size(backward):
    for w in range(0, 20):
        nt = w + 6
        least = max(w + 1, 3)
        assert ring_rows(w) >= least
        assert replay(nt, w, backward, least), w
        assert not replay(nt, w, backward, least - 1), w
