"""Host check of the staged column pass's geometry (ce_col_bulk_kernel in field.cu).

The kernel numbers the lines of a launch l = sample * ncols + x, copies G =
2048 / P consecutive lines (one 16 KB chunk) per stage with one bulk copy, and
lets a persistent grid of 128-thread blocks take chunks blockIdx.x, blockIdx.x
+ gridDim.x, ...  This test restates its index predicates, thread by thread,
and checks that every bulk copy is aligned, sized in 16-byte units, inside the
stage and inside the intermediate; that every shared-memory read and write
stays in the stage; and that every output of the fine field, the coarse field
and the plain coarse field is written exactly once.
"""
import numpy as np
import pytest

THREADS = 128
ELEMS = THREADS * 16


def pitch(P):
    return P + (P >> 4)


def pad(i):
    return i + (i >> 4)


def run(P, m, ncols, count, coarse, plain, grid):
    G = ELEMS // P
    tpf = P // 16
    SL = G * pitch(P)
    nlines = count * ncols
    nchunks = (nlines + G - 1) // G
    mc = m // 2
    nout = mc + 1 if coarse else m + 1
    side = mc + 1 if coarse else m + 1
    kout = np.zeros((count, side, side), int)
    kcp = np.zeros((count, mc + 1, mc + 1), int)
    assert SL * 8 % 16 == 0 and 2 * SL * 8 + 16 <= 48 * 1024   # stages, then the barriers
    tid = np.arange(THREADS)
    g, t = tid // tpf, tid % tpf
    for r in range(16):   # first-pass reads of the copied lines
        idx = g * P + t + r * tpf
        assert idx.max() < SL and idx.min() >= 0
    # padded line buffers of the in-place transform
    assert (G - 1) * pitch(P) + pad(P - 1) < SL
    gq = tid & (G - 1)
    ystep = THREADS // G
    jmax = (nout + ystep - 1) // ystep + 1
    th0 = np.repeat(tid, jmax)
    y0 = th0 // G + np.tile(np.arange(jmax), THREADS) * ystep
    q0 = gq[th0]
    for b in range(grid):
        for c in range(b, nchunks, grid):
            l0, nl = c * G, min(G, nlines - c * G)
            nbytes = nl * P * 8
            assert nbytes % 16 == 0 and (l0 * P * 8) % 16 == 0
            assert nbytes <= SL * 8 and (l0 + nl) * P <= nlines * P
            keep = (q0 < nl) & (y0 < nout)
            y, q = y0[keep], q0[keep]
            line = l0 + q
            sl, x = line // ncols, line % ncols
            src = q * pitch(P) + pad(2 * y if coarse else y)
            assert src.max(initial=0) < SL
            np.add.at(kout, (sl, y, x), 1)
            if plain and not coarse:
                e = ((x | y) & 1) == 0
                np.add.at(kcp, (sl[e], y[e] >> 1, x[e] >> 1), 1)
    return kout, kcp


@pytest.mark.parametrize("P,m,count", [(16, 4, 37), (32, 8, 37), (64, 16, 37), (128, 32, 37),
                                       (256, 64, 9), (512, 128, 3), (1024, 256, 3), (2048, 512, 2),
                                       (128, 64, 5), (2048, 1024, 1), (64, 16, 1), (512, 256, 1)])
def test_every_output_written_once(P, m, count):
    for coarse, plain in ((False, True), (False, False), (True, False)):
        ncols = m // 2 + 1 if coarse else m + 1
        G = ELEMS // P
        nchunks = (count * ncols + G - 1) // G
        for grid in sorted({1, min(nchunks, 5), nchunks}):
            kout, kcp = run(P, m, ncols, count, coarse, plain, grid)
            assert np.all(kout == 1), (P, m, count, coarse, grid)
            if plain:
                assert np.all(kcp == 1)
