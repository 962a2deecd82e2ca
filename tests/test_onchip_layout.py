"""Host-side model of the on-chip schedule's data movement (no GPU): the
positions each thread of `k_onchip` reads and writes, restated from the
kernel's index rules, checked for the properties the kernel relies on --

* every line thread holds a distinct set of positions that together cover
  the line (forward input, spectral output, inverse input, spatial output);
* the swizzled line buffers are a bijection per line (within the padded
  stride);
* step A delivers to each CTA exactly one value per position of its k-space
  columns (so the byte count it waits for is R N values), step B one per
  position of its rows, and the positions read in steps B and C are exactly
  those written;

for every (n, rows per CTA) the library builds.  A change to the kernel's
index rules that breaks one of these would send a byte twice or never, and
its mbarrier wait would time out; this catches it on the CPU first."""

import itertools

import pytest


def split(n):
    log = n.bit_length() - 1
    n1 = 1 << ((log + 1) // 2)
    n2 = n // n1
    return n1, n2


def out_index(m, g, q):
    n1, n2 = split(m)
    return g + n2 * (q // n2) + n1 * (q % n2)


def in_index(m, g, q):
    n1, n2 = split(m)
    return n2 * q + g


class Line:
    """Line<N>: N = R M with a radix-R outer stage (R = 3 at 96 and 192)."""

    def __init__(self, n):
        self.r = 3 if n % 3 == 0 else (2 if n > 256 else 1)
        self.m = n // self.r
        self.gm = split(self.m)[1]
        self.g = self.r * self.gm
        self.nv = split(self.m)[0]

    def sp_in(self, l, q):
        return self.r * in_index(self.m, l % self.gm, q) + l // self.gm

    def sp_out(self, l, q):
        return self.r * out_index(self.m, l % self.gm, q) + l // self.gm

    def fr_out(self, l, q):
        return out_index(self.m, l % self.gm, q) + self.m * (l // self.gm)

    def fr_in(self, l, q):
        return in_index(self.m, l % self.gm, q) + self.m * (l // self.gm)


def swz(g_line, l, e):
    return e ^ (((l >> 1) * (16 // g_line)) & 7)


BUILDS = [(32, 16), (64, 16), (96, 16), (128, 16), (192, 16), (256, 16),
          (32, 8), (64, 8), (96, 8), (128, 8)]


@pytest.mark.parametrize("n, rows", BUILDS)
def test_line_positions_partition_the_line(n, rows):
    L = Line(n)
    assert L.g * L.nv == n
    for f in (L.sp_in, L.sp_out, L.fr_out, L.fr_in):
        pos = [f(l, q) for l in range(L.g) for q in range(L.nv)]
        assert sorted(pos) == list(range(n)), f.__name__
    # a thread's spectral output set equals its spectral input set (the
    # forward -> multiply -> inverse chain stays in registers)
    for l in range(L.g):
        assert {L.fr_out(l, q) for q in range(L.nv)} == {L.fr_in(l, q) for q in range(L.nv)}


@pytest.mark.parametrize("n, rows", BUILDS)
def test_swizzle_is_a_bijection_per_line(n, rows):
    L = Line(n)
    for l in range(rows):
        assert sorted(swz(L.g, l, e) for e in range(n)) == list(range(n))


@pytest.mark.parametrize("n, rows", BUILDS)
def test_hand_offs_deliver_each_position_once(n, rows):
    """Step A: thread (row j, line thread l) of CTA c sends its spectral
    output kx to CTA kx // rows, column kx % rows, position row0 + j.  Step
    B: thread (column kk, l) of CTA c sends its spatial output jy to CTA
    jy // rows, row jy % rows, position c rows + kk."""
    L = Line(n)
    ctas = n // rows
    assert 2 <= ctas <= 16 and (rows * L.g) % 32 == 0
    cb = {}   # (dest CTA, column, swizzled position) -> sender
    rb = {}
    for c, j, l in itertools.product(range(ctas), range(rows), range(L.g)):
        for q in range(L.nv):
            kx = L.fr_out(l, q)
            key = (kx // rows, kx % rows, swz(L.g, kx % rows, c * rows + j))
            assert key not in cb
            cb[key] = (c, j, l, q)
            jy = L.sp_out(l, q)
            key = (jy // rows, jy % rows, swz(L.g, jy % rows, c * rows + j))
            assert key not in rb
            rb[key] = (c, j, l, q)
    for d in range(ctas):
        assert sum(1 for k in cb if k[0] == d) == rows * n   # LINE_BYTES / 8 per round
        assert sum(1 for k in rb if k[0] == d) == rows * n
    # the positions steps B and C read are exactly the ones delivered
    for c, kk, l in itertools.product(range(ctas), range(rows), range(L.g)):
        for q in range(L.nv):
            assert (c, kk, swz(L.g, kk, L.sp_in(l, q))) in cb      # step B loads its column
            assert (c, kk, swz(L.g, kk, L.fr_in(l, q))) in rb      # step C loads its row
