"""Host check of the index maps of the TMEM exchange between the last two
passes of the segment FFT (ols_fft_passes.cuh, tx9/tx10/tx11/tx12 and the
relabelled shared exchanges).

The lane/column layouts of the tcgen05 shapes below are the ones measured on
GB300 by storing lane*100 + column through the 32x32b shape and reading every
register back through each shape.  Each test restates the kernel's register
assignment, pushes every (position, re/im) value of one warp through the
round trips and checks that each thread ends with the pass-2 layout: thread
t holds positions 16 t + k in register k.  The shared-memory exchange of
passes 0 and 1 (relabelled pass 1) is checked for being a bijection with 16
distinct 8-byte bank pairs per half warp in both layouts.
"""
import itertools

import pytest


def bits(v, n):
    return [(v >> i) & 1 for i in range(n)]


# thread T, register i -> (lane, column); lane base lb (0 or 16), column base c0
def L32(T, i, lb=0, c0=0):
    return (lb + T, c0 + i)


def L256(T, i, lb=0, c0=0):
    rep, j, e = i // 4, (i >> 1) & 1, i & 1
    return (lb + 8 * j + (T >> 2), c0 + 8 * rep + 2 * (T & 3) + e)


def L128(T, i, lb=0, c0=0):
    rep, j = i // 2, i & 1
    return (lb + 8 * j + (T >> 2), c0 + 4 * rep + (T & 3))


def L64(T, i, lb=0, c0=0):
    return (lb + 8 * (T & 1) + (T >> 2), c0 + 2 * i + ((T >> 1) & 1))


def L32x2(T, i, lb=0, c0=0, off=0):
    return (lb + (T & 15), c0 + i + off * (T >> 4))


def pos(lane_pos, reg_pos, T, k):
    """Position (within a warp) of register k of lane T, given which position
    bit each lane bit and each register bit carries."""
    t, kb = bits(T, 5), bits(k, 4)
    p = 0
    for b, pb in zip(t, lane_pos):
        p |= b << pb
    for b, pb in zip(kb, reg_pos):
        p |= b << pb
    return p


class Tmem:
    def __init__(self):
        self.cells = {}

    def st(self, layout, T, regs, **kw):
        for i, v in enumerate(regs):
            a = layout(T, i, **kw)
            assert a not in self.cells, "two values stored to one cell"
            self.cells[a] = v

    def ld(self, layout, T, n, **kw):
        return [self.cells[layout(T, i, **kw)] for i in range(n)]


def final_check(x):
    for T in range(32):
        for k in range(16):
            for e in range(2):
                assert x[T][k][e] == (16 * T + k, e)


def test_layout_probe_facts():
    """The shape layouts restate the probe: 16x256b thread 5 reads lane 1,
    columns 2..3 and lane 9 likewise; 16x64b thread 1 reads lane 8, column 0;
    16x32bx2 (offset 16) thread 16 reads lane 0, column 16."""
    assert [L256(5, i) for i in range(4)] == [(1, 2), (1, 3), (9, 2), (9, 3)]
    assert L64(1, 0) == (8, 0) and L64(2, 0) == (0, 1) and L64(4, 1) == (1, 2)
    assert L128(3, 0) == (0, 3) and L128(3, 1) == (8, 3)
    assert L32x2(16, 0, off=16) == (0, 16) and L32x2(15, 1, off=16) == (15, 1)


def test_n1024_one_round_trip():
    lanes, regs = (6, 7, 8, 0, 1), (2, 3, 4, 5)      # relabelled pass 1
    m = Tmem()
    for T in range(32):
        v = [None] * 32
        for mm in range(32):
            e, p4, p5, p2, p3 = bits(mm, 5)
            v[mm] = (pos(lanes, regs, T, p2 + 2 * p3 + 4 * p4 + 8 * p5), e)
        m.st(L32, T, v)
    x = [[[None, None] for _ in range(16)] for _ in range(32)]
    for T in range(32):
        w = [m.ld(L256, T, 16, lb=16 * p1) for p1 in range(2)]
        for k in range(16):
            p0, p1, p23 = k & 1, (k >> 1) & 1, k >> 2
            x[T][k] = [w[p1][4 * p23 + 2 * p0], w[p1][4 * p23 + 2 * p0 + 1]]
    final_check(x)


def test_n2048_two_round_trips():
    lanes, regs = (8, 0, 1, 2, 7), (3, 4, 5, 6)      # relabelled pass 1
    m = Tmem()
    for T in range(32):
        for k in range(8):
            a, b, c = k & 1, (k >> 1) & 1, k >> 2
            p = [(pos(lanes, regs, T, k), 0), (pos(lanes, regs, T, k), 1),
                 (pos(lanes, regs, T, k + 8), 0), (pos(lanes, regs, T, k + 8), 1)]
            m.st(L32x2, T, p, lb=16 * a, c0=8 * b + 16 * c, off=4)
    z = [[m.ld(L256, T, 16, lb=16 * h) for h in range(2)] for T in range(32)]
    m = Tmem()
    for T in range(32):
        v = [None] * 32
        for mm in range(32):
            e, p2, p3, p4, p5 = bits(mm, 5)
            v[2 * (p4 + 2 * p5 + 4 * p2 + 8 * p3) + e] = z[T][p3][4 * (p4 + 2 * p5) + 2 * p2 + e]
        m.st(L32, T, v)
    x = [[[None, None] for _ in range(16)] for _ in range(32)]
    for T in range(32):
        w = [m.ld(L256, T, 16, lb=16 * h) for h in range(2)]
        for k in range(16):
            p0, p1, p2, p3 = bits(k, 4)
            x[T][k] = [w[p1][4 * (p2 + 2 * p3) + 2 * p0], w[p1][4 * (p2 + 2 * p3) + 2 * p0 + 1]]
    final_check(x)


def test_n4096_two_round_trips():
    lanes, regs = (0, 1, 8, 2, 3), (4, 5, 6, 7)      # relabelled pass 1
    m = Tmem()
    for T in range(32):
        for p4 in range(2):
            v = [None] * 16
            for i in range(16):
                p7, p6, e, p5 = bits(i, 4)
                v[i] = (pos(lanes, regs, T, p4 + 2 * p5 + 4 * p6 + 8 * p7), e)
            m.st(L256, T, v, lb=16 * p4)
    z = [[m.ld(L64, T, 16, lb=16 * p4) for p4 in range(2)] for T in range(32)]
    m = Tmem()
    for T in range(32):
        v = [None] * 32
        for mm in range(32):
            e, p4, p5, p0, p1 = bits(mm, 5)
            v[mm] = z[T][p4][p0 + 2 * p1 + 4 * e + 8 * p5]
        m.st(L32, T, v)
    x = [[[None, None] for _ in range(16)] for _ in range(32)]
    for T in range(32):
        w = [m.ld(L256, T, 16, lb=16 * p3) for p3 in range(2)]
        for k in range(16):
            p01, p2, p3 = k & 3, (k >> 2) & 1, k >> 3
            x[T][k] = [w[p3][4 * p01 + 2 * p2], w[p3][4 * p01 + 2 * p2 + 1]]
    final_check(x)


def test_n512_one_round_trip():
    lanes, regs = (5, 0, 6, 7, 8), (1, 2, 3, 4)      # relabelled pass 1
    m = Tmem()
    for T in range(32):
        for p2 in range(2):
            v = [None] * 16
            for i in range(16):
                p4, p1, e, p3 = bits(i, 4)
                v[i] = (pos(lanes, regs, T, p1 + 2 * p2 + 4 * p3 + 8 * p4), e)
            m.st(L256, T, v, lb=16 * p2)
    x = [[[None, None] for _ in range(16)] for _ in range(32)]
    for T in range(32):
        w = [m.ld(L128, T, 16, lb=16 * p2) for p2 in range(2)]
        for k in range(16):
            p0, p1, p2, p3 = bits(k, 4)
            x[T][k] = [w[p2][2 * (p0 + 4 * p3) + p1], w[p2][2 * (p0 + 2 + 4 * p3) + p1]]
    final_check(x)


# shared-memory exchange of passes 0 and 1 with pass 1 relabelled:
# (log2N, threads per segment, pass-1 lane bits, pass-1 register bits, address map)
SHARED = [
    (10, 64, (6, 7, 8, 0, 1), (2, 3, 4, 5), lambda q: q + 2 * (q >> 6)),
    (11, 128, (8, 0, 1, 2, 7), (3, 4, 5, 6), lambda q: q ^ (((q >> 8) & 1) << 3)),
    (12, 256, (0, 1, 8, 2, 3), (4, 5, 6, 7), lambda q: q + 8 * (q >> 8)),
    (9, 32, (5, 0, 6, 7, 8), (1, 2, 3, 4), lambda q: q + 2 * (q >> 5)),
]


@pytest.mark.parametrize("log2n,T,lanes,regs,A", SHARED)
def test_relabelled_shared_exchange(log2n, T, lanes, regs, A):
    N = 1 << log2n
    pad = N + N // 16                    # the buffer of one segment
    assert sorted({A(q) for q in range(N)}) == sorted(A(q) for q in range(N))
    assert len({A(q) for q in range(N)}) == N and max(A(q) for q in range(N)) < pad

    def pos1(t, k):
        return pos(lanes, regs, t & 31, k) | ((t >> 5) << 9)

    def pos0(t, k):
        return t + T * k
    for w in range(T // 32):
        for k in range(16):
            for h in range(2):
                ts = range(32 * w + 16 * h, 32 * w + 16 * h + 16)
                assert len({A(pos1(t, k)) % 16 for t in ts}) == 16
                assert len({A(pos0(t, k)) % 16 for t in ts}) == 16
    # the kernels' own address formulas
    for t in range(T):
        for k in range(16):
            if log2n == 10:
                a0 = t + 66 * k
                a1 = ((t >> 3) & 3) + 66 * ((t & 7) + 8 * (t >> 5)) + 4 * k
            elif log2n == 11:
                a0 = ((t ^ 8) if (k & 2) else t) + 128 * k
                base = ((t >> 1) & 7) + 128 * ((t >> 4) & 1) + 256 * (t & 1) + 512 * (t >> 5)
                a1 = base + 8 * ((k & 1) ^ (t & 1)) + 16 * (k >> 1)
            elif log2n == 12:
                a0 = t + 264 * k
                a1 = ((t & 3) + 4 * ((t >> 3) & 1) + 8 * ((t >> 4) & 1) + 264 * ((t >> 2) & 1) + 528 * (t >> 5)
                      + 16 * k)
            else:
                a0 = t + 34 * k
                a1 = ((t >> 1) & 1) + 34 * ((t & 1) + 2 * ((t >> 2) & 1) + 4 * ((t >> 3) & 1)
                                            + 8 * ((t >> 4) & 1)) + 2 * k
            assert a0 == A(pos0(t, k)) and a1 == A(pos1(t, k))
    # the pass-1 twiddle index: position mod the pass's stride, from the relabelled lanes
    s = {10: 4, 11: 8, 12: 16, 9: 2}[log2n]
    for t in range(T):
        if log2n == 10:
            n1 = (t >> 3) & 3
        elif log2n == 11:
            n1 = (t >> 1) & 7
        elif log2n == 12:
            n1 = (t & 3) + 4 * ((t >> 3) & 1) + 8 * ((t >> 4) & 1)
        else:
            n1 = (t >> 1) & 1
        assert n1 == pos1(t, 0) % s
