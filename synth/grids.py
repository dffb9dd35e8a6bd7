"""Seeded coarse occupancy grids for the labelling tests.

Silhouettes of ellipsoid players only ever give a few compact blobs, so the
26-connected labelling (Sec. II-B-2) is also fed grids that no camera rig
produces: i.i.d. random occupancy at densities around the 26-neighbour site
percolation threshold (about 0.097), and structured shapes whose components
are long and thin (a serpentine chain that visits every row of the grid,
staircases that cross a 32-voxel word boundary at every step, square spirals
stacked over the planes), which make deep union-find trees.

Grids are uint8 arrays indexed (z, y, x), 1 = occupied.  Nothing here holds
any of the method's arithmetic; the oracle and the CUDA path both read these
arrays (the CUDA path after packing them into 32-voxel words).
"""
from __future__ import annotations

import numpy as np

from .scenes import SEED_BASE


def random_grid(dims, density: float, seed: int) -> np.ndarray:
    """(nz, ny, nx) grid with each voxel occupied with probability `density`."""
    nx, ny, nz = dims
    rng = np.random.default_rng([SEED_BASE, 7, int(seed), int(round(density * 1e6))])
    return (rng.random((nz, ny, nx)) < density).astype(np.uint8)


def serpentine_grid(dims) -> np.ndarray:
    """One chain through the whole grid: in every plane z the even rows y are
    full lines along x, joined at alternating ends by one voxel in the odd row
    between them; consecutive planes are joined at one corner.  A single
    26-connected component of about nx*ny*nz/2 voxels."""
    nx, ny, nz = dims
    occ = np.zeros((nz, ny, nx), np.uint8)
    for z in range(0, nz, 2):
        rows = list(range(0, ny, 2))
        for k, y in enumerate(rows):
            occ[z, y, :] = 1
            if k + 1 < len(rows):
                occ[z, y + 1, nx - 1 if k % 2 == 0 else 0] = 1
        if z + 2 < nz:
            last = rows[-1]
            occ[z + 1, last, nx - 1 if (len(rows) - 1) % 2 == 0 else 0] = 1
            # the next plane starts its first row from that corner, reversed
            occ[z + 2, last, :] = 1
    return occ


def staircase_grid(dims, period: int = 3) -> np.ndarray:
    """Diagonal staircases: in plane z, row y holds single voxels at every x
    with (x - s) % (2*period) == 0, where s = y in even planes and ny-1-y in
    odd ones.  Each voxel is a run of its own that touches the row before it
    only through an edge contact (x-1 or x+1), many of the steps cross a
    32-voxel word boundary, and the stairs of neighbouring planes run the
    other way, so they merge through the planes into long components."""
    nx, ny, nz = dims
    occ = np.zeros((nz, ny, nx), np.uint8)
    x = np.arange(nx)
    for z in range(nz):
        for y in range(ny):
            s = y if z % 2 == 0 else ny - 1 - y
            occ[z, y, :] = ((x - s) % (2 * period) == 0).astype(np.uint8)
    return occ


def _spiral_plane(nx, ny) -> np.ndarray:
    """A square spiral path of width 1 walked inward from the corner (0, 0):
    the walker steps on while the voxel ahead is inside the plane and empty
    and the one after it is not part of the path, else turns clockwise; it
    stops when it cannot step after a turn.  Neighbouring arms keep one empty
    voxel between them."""
    p = np.zeros((ny, nx), np.uint8)
    dirs = ((1, 0), (0, 1), (-1, 0), (0, -1))

    def inside(x, y):
        return 0 <= x < nx and 0 <= y < ny

    def can_step(x, y, d):
        dx, dy = dirs[d]
        x1, y1, x2, y2 = x + dx, y + dy, x + 2 * dx, y + 2 * dy
        return inside(x1, y1) and not p[y1, x1] and not (inside(x2, y2) and p[y2, x2])

    x, y, d = 0, 0, 0
    p[y, x] = 1
    while True:
        if not can_step(x, y, d):
            d = (d + 1) % 4
            if not can_step(x, y, d):
                break
        x, y = x + dirs[d][0], y + dirs[d][1]
        p[y, x] = 1
    return p


def spiral_grid(dims) -> np.ndarray:
    """Square spirals (width 1, gaps of 1) in the even planes, each joined to
    the next through the voxel above the spiral's start, so that the grid
    holds one long component whose union paths wind around."""
    nx, ny, nz = dims
    occ = np.zeros((nz, ny, nx), np.uint8)
    plane = _spiral_plane(nx, ny)
    for z in range(0, nz, 2):
        occ[z] = plane
        if z + 1 < nz:
            occ[z + 1, 0, 0] = 1
    return occ


def corner_contacts_grid(dims) -> np.ndarray:
    """Single voxels on a lattice of spacing 2 in every axis: each touches its
    neighbours only through corners (the 26-connectivity a 6- or
    18-connected labelling would miss), so the grid is one component; plus
    the eight grid corners, which are occupied."""
    nx, ny, nz = dims
    occ = np.zeros((nz, ny, nx), np.uint8)
    occ[::2, ::2, ::2] = 1
    occ[1::2, 1::2, 1::2] = 1
    for z in (0, nz - 1):
        for y in (0, ny - 1):
            for x in (0, nx - 1):
                occ[z, y, x] = 1
    return occ


def pack_words(occ: np.ndarray) -> np.ndarray:
    """(nz, ny, nx) uint8 -> (nz*ny*ceil(nx/32),) uint32: bit x%32 of word x/32
    of each row (the layout of the library's coarse grid)."""
    nz, ny, nx = occ.shape
    nxw = (nx + 31) // 32
    pad = np.zeros((nz, ny, nxw * 32), np.uint8)
    pad[:, :, :nx] = occ != 0
    return np.packbits(pad, axis=-1, bitorder="little").view(np.uint32).reshape(-1).copy()
