"""The union rule of the coarse labelling kernel, as an algorithm.

The coarse carve starts every run of consecutive occupied voxels within a
32-voxel word as one union-find tree rooted at its first voxel, and the
union kernel then joins runs: the first voxel of a word with the last voxel
of the word before it in the same row, and, for each of the four earlier
neighbour rows (y-1, z) and (y-1..y+1, z-1), a run's first voxel with the
run holding the leftmost occupied of the neighbour row's voxels l-1, l, and
any voxel l with the run starting at l+1 when l is empty there.  This test
runs that rule sequentially on bit rows and checks that it yields exactly
the 26-connected components scipy finds, on random grids of several
densities and on diagonal chains across word boundaries.  (The kernel
itself is checked against the oracle by the GPU parity tests.)"""
import numpy as np
import pytest
from scipy import ndimage


def _words(occ):
    nz, ny, nx = occ.shape
    nxw = (nx + 31) // 32
    w = np.zeros((nz, ny, nxw), np.uint64)
    for x in range(nx):
        w[:, :, x // 32] |= occ[:, :, x].astype(np.uint64) << np.uint64(x % 32)
    return w.astype(np.uint32), nxw


def _run_start(word, lane):
    starts = word & ~(word << 1) & 0xFFFFFFFF
    return max(b for b in range(lane + 1) if (starts >> b) & 1)


def _labels_by_rule(occ):
    nz, ny, nx = occ.shape
    W, nxw = _words(occ)
    parent = {}

    def find(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    def unite(a, b):
        a, b = find(a), find(b)
        if a != b:
            if a < b:
                a, b = b, a
            parent[a] = b

    def word(y, z, wx):
        if y < 0 or z < 0 or y >= ny or z >= nz or wx < 0 or wx >= nxw:
            return 0
        return int(W[z, y, wx])

    # the coarse carve: each run of a word is one tree rooted at its first voxel
    for z in range(nz):
        for y in range(ny):
            for wx in range(nxw):
                w = int(W[z, y, wx])
                base = (z * ny + y) * nx + wx * 32
                for lane in range(32):
                    if (w >> lane) & 1:
                        parent[base + lane] = base + _run_start(w, lane)
    # the union kernel: join runs
    for z in range(nz):
        for y in range(ny):
            for wx in range(nxw):
                w = int(W[z, y, wx])
                starts = w & ~(w << 1) & 0xFFFFFFFF
                base = (z * ny + y) * nx + wx * 32
                for lane in range(32):
                    if not (w >> lane) & 1:
                        continue
                    run0 = base + _run_start(w, lane)
                    if lane == 0 and (word(y, z, wx - 1) >> 31) & 1:
                        unite(run0, run0 - 1)
                    for dy, dz in ((-1, 0), (-1, -1), (0, -1), (1, -1)):
                        n, n_prev, n_next = (word(y + dy, z + dz, wx + d) for d in (0, -1, 1))
                        left = (n >> (lane - 1)) & 1 if lane > 0 else (n_prev >> 31) & 1
                        mid = (n >> lane) & 1
                        right = (n >> (lane + 1)) & 1 if lane < 31 else n_next & 1
                        nrow = ((z + dz) * ny + (y + dy)) * nx + wx * 32
                        if (starts >> lane) & 1 and (left or mid):
                            unite(run0, nrow + (lane - 1 if left else lane))
                        if not mid and right:
                            unite(run0, nrow + lane + 1)
    lab = np.zeros(occ.shape, np.int64)
    for v in parent:
        z, rem = divmod(v, ny * nx)
        y, x = divmod(rem, nx)
        lab[z, y, x] = find(v) + 1
    return lab


def _same_components(a, b):
    assert np.array_equal(a > 0, b > 0)
    pairs = set(zip(a[a > 0].tolist(), b[b > 0].tolist()))
    return len(pairs) == len(np.unique(a[a > 0])) == len(np.unique(b[b > 0]))


@pytest.mark.parametrize("density", [0.05, 0.2, 0.4, 0.6, 0.8])
def test_run_rule_gives_26_connected_components(density):
    rng = np.random.default_rng(int(density * 100))
    for _ in range(8):
        shape = (int(rng.integers(1, 6)), int(rng.integers(1, 7)), int(rng.integers(1, 100)))
        occ = rng.random(shape) < density
        ref, _ = ndimage.label(occ, structure=np.ones((3, 3, 3), int))
        assert _same_components(_labels_by_rule(occ), ref)


def test_run_rule_across_word_boundaries():
    occ = np.zeros((3, 3, 70), bool)
    for x in range(70):
        occ[x % 3, (x // 3) % 3, x] = True          # a diagonal chain through every word edge
    ref, n = ndimage.label(occ, structure=np.ones((3, 3, 3), int))
    assert _same_components(_labels_by_rule(occ), ref)
    occ = np.zeros((2, 2, 66), bool)
    occ[0, 0, 31] = occ[1, 1, 32] = occ[0, 1, 63] = occ[1, 0, 64] = True   # two corner contacts, at x = 31|32 and 63|64
    ref, n = ndimage.label(occ, structure=np.ones((3, 3, 3), int))
    assert n == 2 and _same_components(_labels_by_rule(occ), ref)
