"""Host check of the aligned x-pairs sweep's row geometry (no GPU).

The sweep gives a block 64 x-adjacent sites x0 .. x0 + 63 of one x row.  For
velocity i each of the two warps (sub = 0, 1) copies value x0 + 32 sub + lane
of the velocity's source row to position H + 32 sub + lane + v_x of the
velocity's row in shared memory (64 + 2H values, H = the lattice's reach),
and lanes < H copy the halo on the side v_x needs: for v_x > 0, sub 0 copies
x0 - H + lane (wrapped at the row's start) to position lane + v_x; for
v_x < 0, sub 1 copies x0 + 64 + lane (wrapped at the row's end) to position
H + 64 + lane + v_x.  Site x0 + p then reads position H + p.

This restates those positions and checks, for every velocity of every set
the sweep serves and every pair position of rows of 64, 128 and 192 sites:
every write lands inside the row, no two writes put different values in one
position, and position H + p holds f_i(x0 + p - v_x) (periodic in x), i.e.
the pull g_i(x) = f_i(x - v_i) of the streaming step.  The velocity tables
are the library's own (pkr_lattice_info, host only).
"""
import ctypes

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on the path)


@pytest.fixture(scope="module")
def pk():
    from paper_1504_05869_gb300 import build
    build.build()
    import paper_1504_05869_gb300 as pkg
    pkg._pkr.load()
    return pkg


def _velocities(pk, lattice, order):
    lib = pk._pkr.load()
    q = ctypes.c_int32()
    dim = ctypes.c_int32()
    vel = (ctypes.c_int32 * (3 * 256))()
    rc = lib.pkr_lattice_info(pk.LATTICES[lattice], order, ctypes.byref(q), ctypes.byref(dim),
                              vel, None, None, None, None)
    assert rc == 0
    return [tuple(vel[3 * k:3 * k + 3]) for k in range(q.value)]


def _row(vx, x0, nx, H):
    """Positions written for one velocity of one pair: {position: source x}."""
    rl = 64 + 2 * H
    row = {}

    def put(pos, x):
        assert 0 <= pos < rl, ("outside the row", vx, x0, pos)
        assert row.get(pos, x) == x, ("two values in one position", vx, x0, pos)
        row[pos] = x

    for sub in (0, 1):
        for lane in range(32):
            put(H + 32 * sub + lane + vx, x0 + 32 * sub + lane)
    for lane in range(H):
        if vx > 0:
            xl = (x0 - H if x0 >= H else x0 - H + nx) + lane
            put(lane + vx, xl)
        elif vx < 0:
            xr = (x0 + 64 if x0 + 64 < nx else 0) + lane
            assert xr < nx
            put(H + 64 + lane + vx, xr)
    return row


@pytest.mark.parametrize("lattice,order", [("D3Q111", 5), ("D2Q81", 5), ("D2Q169", 7)])
def test_pair_rows_hold_the_pull(pk, lattice, order):
    vel = _velocities(pk, lattice, order)
    assert len(vel) > 64                      # the sets the x-pairs sweep serves
    H = max(abs(c) for v in vel for c in v)   # halo = the reach
    for nx in (64, 128, 192):
        for x0 in range(0, nx, 64):
            for vx in sorted({v[0] for v in vel}):
                row = _row(vx, x0, nx, H)
                for p in range(64):
                    assert row.get(H + p) == (x0 + p - vx) % nx, (lattice, nx, x0, vx, p)


def test_pair_rows_fit_the_shared_split(pk):
    """Three D3Q111 blocks of 8-byte rows (64 + 2 x 3 values per velocity)
    plus their exchange rows (2.1 KB fixed point, 2.6 KB binary64) and the
    1 KB the SM reserves per block fit the 196 KB shared split (200,704 B),
    so 60 KB of the SM's 256 KB stay L1; a halo of 4 would not fit."""
    vel = _velocities(pk, "D3Q111", 5)
    H = max(abs(c) for v in vel for c in v)
    assert H == 3
    for static in (2112, 2624):
        per_block = len(vel) * (64 + 2 * H) * 8 + static + 1024
        assert 3 * per_block <= 200704, per_block
        per_block4 = len(vel) * (64 + 2 * 4) * 8 + static + 1024
        assert 3 * per_block4 > 200704
