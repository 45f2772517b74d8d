"""Host check of the tiled multigrid kernels' geometry (mg_tiles.cuh).

The down and up tile kernels each write only the fine (and, for the down
kernel, coarse) vertices they own.  Their window origins and owned extents
follow from the number of Gauss-Seidel sweeps per side (nu): mg_down's window
starts 2 nu + 2 fine vertices before its owned region, mg_up's 2 nu; a tile
owns CW = 32 - 2 nu - 1 coarse columns and CH = SH / 2 - 2 nu - 1 coarse rows
of a window SH rows high.  This test restates those predicates, lane by lane
and warp by warp as the kernels evaluate them, and checks that every fine
vertex of the grid and every coarse vertex of the next level is written by
exactly one tile, for both cycles and every window height the tuner can pick,
and that mg_up's reads of its coarse window stay inside the buffer it loads.
"""
import numpy as np
import pytest

SW = 64          # window width: 32 lanes x 2 columns
CCW = SW // 2 + 1


def geometry(nu, sh):
    od, ou = 2 * nu + 2, 2 * nu
    cw, ch = SW // 2 - 2 * nu - 1, sh // 2 - 2 * nu - 1
    return od, ou, cw, ch


def writes(n, sh, nu):
    od, ou, cw, ch = geometry(nu, sh)
    nw = sh // 4
    nc = n // 2
    tiles_x = (nc + 1 + cw - 1) // cw
    tiles_y = (nc + 1 + ch - 1) // ch
    fine_down = np.zeros((n + 1, n + 1), int)
    fine_up = np.zeros((n + 1, n + 1), int)
    coarse = np.zeros((nc + 1, nc + 1), int)
    lane = np.arange(32)
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            i0, j0 = tx * cw, ty * ch
            for warp in range(nw):
                for r in range(4):
                    lj = 4 * warp + r
                    for c in range(2):
                        li = 2 * lane + c
                        for org, acc in ((od, fine_down), (ou, fine_up)):
                            gi = 2 * i0 - org + li
                            gj = 2 * j0 - org + lj
                            own = ((li >= org) & (li < org + 2 * cw) & (lj >= org) &
                                   (lj < org + 2 * ch) & (gi <= n) & (gj <= n))
                            if own.any():
                                assert gj >= 0 and np.all(gi[own] >= 0)
                                np.add.at(acc[gj], gi[own], 1)
                for k in range(2):
                    ci = i0 - od // 2 + lane
                    cj = j0 - od // 2 + 2 * warp + k
                    own = ((ci - i0 >= 0) & (ci - i0 < cw) & (cj - j0 >= 0) & (cj - j0 < ch) &
                           (ci <= nc) & (cj <= nc))
                    if own.any():
                        np.add.at(coarse[cj], ci[own], 1)
    return fine_down, fine_up, coarse


@pytest.mark.parametrize("nu", [1, 2, 3])
@pytest.mark.parametrize("sh", [16, 24, 32, 48, 64])
@pytest.mark.parametrize("n", [128, 256])
def test_every_vertex_written_once(nu, sh, n):
    fine_down, fine_up, coarse = writes(n, sh, nu)
    assert np.all(fine_down == 1)
    assert np.all(fine_up == 1)
    assert np.all(coarse == 1)


@pytest.mark.parametrize("nu", [1, 2, 3])
@pytest.mark.parametrize("sh", [16, 24, 32, 48, 64])
def test_coarse_window_reads_stay_in_the_buffer(nu, sh):
    """mg_up loads SH/2 coarse rows of CCW entries plus a zero row; lane x of
    warp w reads rows 2w .. 2w + 2, columns x and x + 1."""
    cch = sh // 2
    allocated = (cch + 1) * CCW + 1
    nw = sh // 4
    top = (2 * (nw - 1) + 2) * CCW + 31 + 1
    assert top < allocated
    # and the owned vertices need only the loaded rows and columns: the
    # highest owned fine row / column maps to coarse row / column < loaded
    od, ou, cw, ch = geometry(nu, sh)
    assert (ou + 2 * ch - 1 + 1) // 2 < cch
    assert (ou + 2 * cw - 1 + 1) // 2 < CCW - 1


@pytest.mark.parametrize("nu", [1, 2, 3])
@pytest.mark.parametrize("sh", [16, 24, 32, 48, 64])
def test_owned_region_inside_the_valid_part_of_the_window(nu, sh):
    """Ring bookkeeping of a window with last index E (63 across, SH - 1 up).
    mg_down: the first red update from z = 0 is exact except at index 0 (no
    west / south conductance there); each of the 2 nu - 1 half-sweeps after it
    invalidates one more ring at both edges, and the residual another, so the
    residual is valid on (2 nu, E - 2 nu]; a coarse vertex needs the residuals
    of its diagonal neighbours, and the owned z the swept values.  mg_up: after
    the prolongation only index 0 (1/diag) and, across rows, the top row (the
    zero spare coarse row) are invalid; each of the 2 nu half-sweeps adds a
    ring."""
    od, ou, cw, ch = geometry(nu, sh)
    for e, owned, top_invalid_after_prolongation in ((SW - 1, cw, False), (sh - 1, ch, True)):
        # mg_down
        res_lo, res_hi = 2 * nu, e - 2 * nu          # valid: res_lo < x <= res_hi
        z_lo, z_hi = 2 * nu - 1, e - 2 * nu + 1      # swept z valid: z_lo < x <= z_hi
        first, last = od, od + 2 * (owned - 1)       # owned coarse vertices (even x)
        assert first - 1 > res_lo and last + 1 <= res_hi
        assert od > z_lo and od + 2 * owned - 1 <= z_hi
        # mg_up
        up_lo = 2 * nu - 1
        up_hi = e - 2 * nu - (1 if top_invalid_after_prolongation else 0)
        assert ou > up_lo and ou + 2 * owned - 1 <= up_hi
