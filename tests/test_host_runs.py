"""Host-side tables of the run kernels and the cell-resident sweep, read
back from the library without a GPU (hhg_run_lists, hhg_slab_planes) and
checked against the definitions they implement.

Run lists (Sec. 3.4: the surrogate is evaluated along the lines (j, k) of a
macro cell): per colour (i + 2j + 3k) mod 4 every interior point of the cell
is in exactly one run; a run is 1..8 points i0, i0 + 4, .. (stride 1 for the
all-points segment) of one line, all deep-interior (every neighbour
interior) or all next to the cell boundary, as its flag says; deep runs come
first and each part is in plane order; the per-plane index table points at
the first run of each part on a plane >= k.  Every memory access of the run
kernels and of the resident sweep is derived from these items, so a wrong
item would read outside a cell.

Slabs: the cell-resident sweep splits a cell's interior planes 1 .. N - 3
into `cluster` contiguous, non-empty slabs of near-equal point counts."""
import pytest

import paper_1608_06473_gb300 as hhg


def interior(N):
    return [(i, j, k) for k in range(1, N) for j in range(1, N - k) for i in range(1, N - j - k)]


def is_deep(i, j, k, N):
    return i >= 2 and j >= 2 and k >= 2 and i + j + k <= N - 2


def plane_points(N, k):
    m = N - 2 - k
    return m * (m + 1) // 2 if m > 0 else 0


@pytest.mark.parametrize("N", [4, 8, 16, 32, 64])
def test_run_lists_partition_the_interior(N):
    items, off, kidx = hhg.hhg_run_lists(N)
    assert off[5] == len(items)
    pts = interior(N)
    for g in range(5):
        seg = items[off[g]:off[g + 1]]
        h = 4 if g < 4 else 1
        seen = []
        flags = []
        for x, y in seg:
            i0, j, k = int(x & 1023), int((x >> 10) & 1023), int(x >> 20)
            cnt, deep = int(y & 0xFF), bool(y & 0x100)
            assert 1 <= cnt <= 8
            flags.append((deep, k))
            for s in range(cnt):
                p = (i0 + h * s, j, k)
                assert 1 <= p[0] and p[0] + j + k <= N - 1 and j >= 1 and k >= 1, p
                assert is_deep(*p, N) == deep, p
                if g < 4:
                    assert (p[0] + 2 * j + 3 * k) % 4 == g
                seen.append(p)
        want = [p for p in pts if g == 4 or (p[0] + 2 * p[1] + 3 * p[2]) % 4 == g]
        assert len(seen) == len(set(seen)) == len(want)
        assert set(seen) == set(want)
        # deep runs first, each part in plane order
        n_deep = sum(d for d, _ in flags)
        assert all(d for d, _ in flags[:n_deep]) and not any(d for d, _ in flags[n_deep:])
        for part in (flags[:n_deep], flags[n_deep:]):
            ks = [k for _, k in part]
            assert ks == sorted(ks)
        if g < 4:
            for part, (lo, hi) in enumerate(((0, n_deep), (n_deep, len(flags)))):
                for k in range(N + 1):
                    first = next((e for e in range(lo, hi) if flags[e][1] >= k), hi)
                    assert kidx[g, k, part] == first, (g, k, part)


def test_run_lengths_balance_long_lines():
    """A line's deep points of one colour split into runs whose lengths
    differ by at most one."""
    items, off, _ = hhg.hhg_run_lists(128)
    seg = items[off[0]:off[1]]
    lines = {}
    for x, y in seg:
        if y & 0x100:
            lines.setdefault((int((x >> 10) & 1023), int(x >> 20)), []).append(int(y & 0xFF))
    assert max(len(v) for v in lines.values()) >= 2
    for cnts in lines.values():
        assert max(cnts) - min(cnts) <= 1


@pytest.mark.parametrize("N", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_slab_planes_split_the_cell(N, cluster):
    kb = hhg.hhg_slab_planes(N, cluster)
    assert kb[0] == 1 and kb[-1] == N - 2
    assert all(a <= b for a, b in zip(kb, kb[1:]))
    if N >= 32:
        # every slab holds at least one plane, and its points are within one
        # plane's worth of an equal share
        n_int = (N - 1) * (N - 2) * (N - 3) // 6
        big = plane_points(N, 1)
        for r in range(cluster):
            assert kb[r + 1] > kb[r]
            n = sum(plane_points(N, k) for k in range(kb[r], kb[r + 1]))
            assert abs(n - n_int / cluster) <= big


def test_rejects_bad_arguments():
    with pytest.raises(hhg.HHGError):
        hhg.hhg_run_lists(2)
    with pytest.raises(hhg.HHGError):
        hhg.hhg_slab_planes(64, 16)
    assert hhg.hhg_last_error() != ""
    hhg.hhg_slab_planes(64, 2)   # a successful call clears the message
    assert hhg.hhg_last_error() == ""


# Direction offsets (i, j, k) of the 14 neighbours (the order of the stencil
# weights: me mw mn ms mnw mse tc tw ts tse bc be bn bnw).
DIRS = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (-1, 1, 0), (1, -1, 0), (0, 0, 1), (-1, 0, 1), (0, -1, 1),
        (1, -1, 1), (0, 0, -1), (1, 0, -1), (0, 1, -1), (-1, 1, -1)]


def lin_interior(i, j, k, N):
    """Position of interior point (i, j, k) in its cell's block (i fastest,
    then j, then k)."""
    tet = lambda n: (n + 1) * (n + 2) * (n + 3) // 6
    M, a, b, c = N - 4, i - 1, j - 1, k - 1
    m = M - c
    return tet(M) - tet(M - c) + b * (m + 1) - b * (b - 1) // 2 + a


@pytest.mark.parametrize("N,cluster", [(16, 1), (16, 4), (32, 2), (32, 8), (64, 8)])
def test_resident_sweep_reads_stay_in_the_owning_slab(N, cluster):
    """The cell-resident sweep keeps slab r (planes [k_r, k_{r+1})) of a cell
    in CTA r's shared memory and reads a neighbour on plane k - 1 (k + 1)
    from CTA r - 1 (r + 1) only when k is the slab's first (last) plane.
    Every interior neighbour of every run point of the slab must then lie in
    the slab chosen for it, and every point's update lands in its own slab;
    boundary neighbours come from the halo."""
    items, off, kidx = hhg.hhg_run_lists(N)
    kb = hhg.hhg_slab_planes(N, cluster)
    start = [lin_interior(1, 1, k, N) for k in range(1, N - 1)] + [lin_interior(1, 1, N - 2, N)]
    pos0 = lambda k: start[k - 1]   # first position of plane k (plane N - 2 starts at n_int)
    for r in range(cluster):
        k0, k1 = int(kb[r]), int(kb[r + 1])
        for g in range(4):
            seg = items[off[g]:off[g + 1]]
            d0, d1, n0, n1 = kidx[g, k0, 0], kidx[g, k1, 0], kidx[g, k0, 1], kidx[g, k1, 1]
            for x, y in list(seg[d0:d1]) + list(seg[n0:n1]):
                i0, j, k = int(x & 1023), int((x >> 10) & 1023), int(x >> 20)
                assert k0 <= k < k1
                lo = r - 1 if k == k0 else r
                hi = r + 1 if k + 1 == k1 else r
                for s in range(int(y & 0xFF)):
                    i = i0 + 4 * s
                    assert pos0(k0) <= lin_interior(i, j, k, N) < pos0(k1)
                    for di, dj, dk in DIRS:
                        i2, j2, k2 = i + di, j + dj, k + dk
                        if not (i2 >= 1 and j2 >= 1 and k2 >= 1 and i2 + j2 + k2 <= N - 1):
                            assert not (y & 0x100)   # deep points have interior neighbours only
                            continue
                        owner = lo if dk < 0 else (hi if dk > 0 else r)
                        assert 0 <= owner < cluster
                        p = lin_interior(i2, j2, k2, N)
                        assert pos0(int(kb[owner])) <= p < pos0(int(kb[owner + 1])), (r, owner, (i2, j2, k2))
