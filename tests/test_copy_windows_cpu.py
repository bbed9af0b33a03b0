"""CPU check of the bulk copies the pipelined kernels issue: every
cp.async.bulk must start on a 16-byte boundary in global and shared memory,
move a multiple of 16 bytes, stay inside its source row's allocation (the
pitch) and inside its shared-memory slot.  The copy lists are re-derived here
from the producers' rules (tile windows with a 16-byte halo, wrap copies at
periodic row ends, the Scheme II Phi rows, the batched kernel's side slots for
unaligned periodic rows) and checked over many extents, tile widths and
periodicities.  The stores staged in shared memory are checked the same way:
the store warp's shared-to-global bulk copies, and the in-place odd step's
aligned chunks, which together with its single elements must write every
destination slot exactly once.  Nothing here runs on a GPU."""
import itertools

import numpy as np
import pytest


def _pitch(nx, esize):
    per = 16 // esize
    return (nx + per - 1) // per * per


def _check(copies, esize, pitch, slot_elems):
    for src0, n, dst0 in copies:
        assert (src0 * esize) % 16 == 0, ("source", src0)
        assert (n * esize) % 16 == 0 and n > 0, ("size", n)
        assert (dst0 * esize) % 16 == 0, ("destination", dst0)
        assert 0 <= src0 and src0 + n <= pitch, ("row", src0, n, pitch)
        assert 0 <= dst0 and dst0 + n <= slot_elems, ("slot", dst0, n, slot_elems)


def _row_copies(nx, X, esize, periodic, nx_round=None):
    """Per tile of one row: (source start, elements, slot offset) of the main
    window [x0 - H, x0 + X + H) clipped to the row, and of the wrap halos of a
    periodic row (the single-lattice kernel's rule; the batched kernel rounds
    the window end into the pitch, nx_round)."""
    H = 16 // esize
    end = nx if nx_round is None else nx_round
    out = []
    for x0 in range(0, nx, X):
        xe = min(x0 + X, nx)
        lo, hi = max(x0 - H, 0), min(xe + H, end)
        c = [(lo, hi - lo, lo - (x0 - H))]
        aligned = nx % H == 0
        if periodic and aligned and x0 == 0:
            c.append((nx - H, H, 0))
        if periodic and aligned and xe == nx:
            c.append((0, H, H + (nx - x0)))
        out.append((x0, xe, c))
    return out


@pytest.mark.parametrize("esize,widths", [(4, (256, 384, 512)), (2, (256, 384, 512)),
                                          (8, (128, 192, 256))])
def test_single_lattice_windows(esize, widths):
    """k_step_tma / k_step_aa_tma: extents the variant list admits (nx a whole
    number of 16-byte units, nx >= 2 units)."""
    H = 16 // esize
    rng = np.random.default_rng(3)
    sizes = sorted({2 * H, 3 * H, H * 64, 511 * H // H * H} |
                   {int(v) * H for v in rng.integers(2, 400, 60)})
    for nx, X, per in itertools.product(sizes, widths, (0, 1)):
        slot = X + 2 * H
        for _, _, copies in _row_copies(nx, X, esize, per):
            _check(copies, esize, _pitch(nx, esize), slot)


@pytest.mark.parametrize("esize,widths", [(4, (256, 384, 512)), (8, (128, 192, 256))])
def test_scheme2_phi_rows(esize, widths):
    """MODE 2 of k_step_tma: Phi (arithmetic precision R, 4 or 8 bytes) is
    dense ([D][nx ny nz]), so its rows have no padding; the own x row is copied
    with an HR halo and wraps, the y / z rows over the tile only."""
    rsize = 8 if esize == 8 else 4
    HR = 16 // rsize
    H = 16 // esize
    rng = np.random.default_rng(4)
    for nx in sorted({int(v) * H for v in rng.integers(2, 300, 50)}):
        for X, per in itertools.product(widths, (0, 1)):
            slot = X + 2 * HR
            for x0 in range(0, nx, X):
                xe = min(x0 + X, nx)
                lo, hi = max(x0 - HR, 0), min(xe + HR, nx)
                copies = [(lo, hi - lo, lo - (x0 - HR)), (x0, xe - x0, HR)]
                if per and x0 == 0:
                    copies.append((nx - HR, HR, 0))
                if per and xe == nx:
                    copies.append((0, HR, HR + (nx - x0)))
                # Phi rows start at multiples of nx (dense), so the row length
                # itself must be a whole number of 16-byte units
                assert (nx * rsize) % 16 == 0
                _check(copies, rsize, nx, slot)


@pytest.mark.parametrize("esize", [4, 2])
def test_batched_windows_and_side_slots(esize):
    """k_batch_tma: any nx; the window end is rounded into the pitch, and an
    unaligned periodic row gets the aligned chunks around x = nx - 1 and x = 0
    in two side slots of H elements each."""
    H = 16 // esize
    for nx in range(1, 700):
        pitch = _pitch(nx, esize)
        nxr = (nx + H - 1) // H * H
        for X, per in itertools.product((128, 256), (0, 1)):
            for x0, xe, copies in _row_copies(nx, X, esize, per, nx_round=nxr):
                _check(copies, esize, pitch, X + 2 * H)
                if per and nx % H != 0:
                    side = []
                    if x0 == 0:
                        a = (nx - 1) // H * H
                        side.append((a, H, 0))
                        assert a <= nx - 1 < a + H  # the chunk holds x = nx - 1
                    if xe == nx:
                        side.append((0, H, H))
                    _check(side, esize, pitch, 2 * H)


@pytest.mark.parametrize("esize,widths", [(4, (256, 384, 512)), (2, (256, 384, 512))])
def test_staged_bulk_store_rows(esize, widths):
    """MODE 3 of k_step_tma: the store warp copies each staging row (plane i of
    the tile) to [x0, x0 + wdt) of its destination row: one bulk copy of the
    16-byte multiple of the row segment (16-byte aligned in global and shared
    memory), then the remaining elements one by one; together they write the
    segment exactly once, inside the row and inside the staging row."""
    H = 16 // esize
    rng = np.random.default_rng(5)
    for nx in sorted({2 * H, 3 * H} | {int(v) * H for v in rng.integers(2, 400, 60)}):
        pitch = _pitch(nx, esize)
        for X in widths:
            for x0 in range(0, nx, X):
                wdt = min(X, nx - x0)
                nb = (wdt * esize) // 16 * 16 // esize
                if nb:
                    _check([(x0, nb, 0)], esize, pitch, X)
                written = list(range(x0, x0 + nb)) + list(range(x0 + nb, x0 + wdt))
                assert written == list(range(x0, x0 + wdt))
                assert x0 + wdt <= nx <= pitch


def _aa_odd_writes(nx, X, esize, per, ex, rw):
    """Destinations written for one plane of one row by the staged AA odd step:
    the store warp's bulk copy of the 16-byte aligned interior of the tile's
    window [lo, hi) (as (start, elements, staging-row offset)) and its single
    elements at either end, and the direct stores of the tile-end threads
    (wraps, x walls as ("opp", x))."""
    VE = 16 // esize
    HT = VE
    sh = 0 if rw else ex
    vec, single = [], []
    for x0 in range(0, nx, X):
        wdt = min(X, nx - x0)
        lo, hi = max(x0 + sh, x0), min(x0 + wdt + sh, nx, x0 + X)
        ca = min(hi, (lo + VE - 1) // VE * VE)
        cb = max(ca, hi // VE * VE)
        if cb > ca:
            vec.append((ca, cb - ca, HT + ca - x0))
        single += list(range(lo, ca)) + list(range(cb, hi))
        if ex != 0 and not rw:
            for j in {0, wdt - 1}:
                x = x0 + j
                xd = x + ex
                if x0 <= xd < min(x0 + X, nx):
                    continue
                if 0 <= xd < nx:
                    single.append(xd)
                elif per:
                    single.append(xd % nx)
                else:
                    single.append(("opp", x))
    return vec, single


@pytest.mark.parametrize("esize,widths", [(4, (256, 384, 512)), (2, (256, 384, 512)),
                                          (8, (128, 192, 256))])
def test_aa_odd_staged_stores_cover_each_slot_once(esize, widths):
    """k_step_aa_tma, odd step: node x writes f*_i to x + e_ix of the
    destination row (wrapped across a periodic x axis, bounced to its own
    opposite slot at an x wall; a plane whose destination row lies beyond a y /
    z wall goes to the node's own row unshifted).  The store warp's copy (the
    aligned interior of the tile's window [lo, hi) by one bulk copy, single
    elements at its ends) and the tile-end threads' direct stores must write
    every destination exactly once; the bulk copy must be 16-byte aligned in
    the row and in the staging row and stay inside both."""
    VE = 16 // esize
    rng = np.random.default_rng(6)
    for nx in sorted({2 * VE, 3 * VE} | {int(v) * VE for v in rng.integers(2, 300, 40)}):
        pitch = _pitch(nx, esize)
        for X, per, ex, rw in itertools.product(widths, (0, 1), (-1, 0, 1), (False, True)):
            vec, single = _aa_odd_writes(nx, X, esize, per, ex, rw)
            _check(vec, esize, pitch, X + 2 * VE)
            written = [x for c, n, _ in vec for x in range(c, c + n)] + single
            sh = 0 if rw else ex
            want = []
            for x in range(nx):
                xd = x + sh
                want.append(xd if 0 <= xd < nx else (xd % nx if per else ("opp", x)))
            key = lambda v: (1, v[1]) if isinstance(v, tuple) else (0, v)
            assert sorted(written, key=key) == sorted(want, key=key), (nx, X, per, ex, rw)
