"""Values the paper prints, checked against the oracle's grid definition."""
import os

import numpy as np

from oracle import Oracle
from tests.helpers import affine_rig

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_grid_counts.txt")


def test_paper_coarse_voxel_count():
    """Sec. II-B-1 / III-A: an 18x18x9 m volume at 50 mm has 2.3e7 voxels."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    for x, y, z, s, printed, digits in rows:
        x, y, z, s = float(x), float(y), float(z), float(s)
        rig = affine_rig([[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1]]], 8, 8,
                         (-x / 2, -y / 2, 0.0), (x / 2, y / 2, z), s)
        dims = Oracle(rig).grid_dims()
        n = int(np.prod(dims))
        assert float(f"{n:.{int(digits) - 1}e}") == float(printed)
        assert dims == (360, 360, 180)
