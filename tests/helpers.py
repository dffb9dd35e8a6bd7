"""Small rigs and checks shared by the tests (no arithmetic of the method)."""
import math

import numpy as np

from synth import Rig


def affine_rig(views, W, H, vol_min, vol_max, coarse, fine=None, steps=0, centres=None, **kw):
    """A rig of affine cameras (last row of P = 0 0 0 1) given as 3x4 matrices."""
    P = np.asarray(views, np.float64).reshape(-1, 3, 4)
    n = len(P)
    if centres is None:
        centres = np.zeros((n, 3))
    return Rig(name="affine", P=P.astype(np.float32), centre=np.asarray(centres, np.float32),
               width=np.full(n, W, np.int32), height=np.full(n, H, np.int32),
               vol_min=tuple(vol_min), vol_max=tuple(vol_max), coarse_m=coarse,
               fine_m=fine if fine is not None else coarse, bisect_steps=steps, P64=P,
               C64=np.asarray(centres, np.float64), **kw)


def canonical_labels(lab):
    """Renumber labels 1..C in order of each component's smallest linear index."""
    flat = lab.ravel()
    ids = np.unique(flat[flat > 0])
    first = np.array([np.flatnonzero(flat == i)[0] for i in ids]) if len(ids) else np.zeros(0, int)
    order = ids[np.argsort(first)]
    remap = np.zeros(int(flat.max()) + 1 if flat.size else 1, np.int32)
    remap[order] = np.arange(1, len(order) + 1)
    return remap[lab]


def edge_use(tris):
    """Map undirected edge -> (uses in one direction, uses in the other)."""
    t = np.asarray(tris, np.int64)
    a = np.concatenate([t[:, 0], t[:, 1], t[:, 2]])
    b = np.concatenate([t[:, 1], t[:, 2], t[:, 0]])
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    fwd = (a < b).astype(np.int64)
    key = lo * (int(t.max()) + 1 if t.size else 1) + hi
    order = np.argsort(key, kind="stable")
    key, fwd = key[order], fwd[order]
    uniq, start, counts = np.unique(key, return_index=True, return_counts=True)
    nf = np.add.reduceat(fwd, start) if len(start) else np.zeros(0, np.int64)
    return uniq, counts, nf


def closed_oriented(tris) -> bool:
    """Every undirected edge used by exactly two triangles, once each way."""
    if len(tris) == 0:
        return True
    _, counts, nf = edge_use(tris)
    return bool(np.all(counts == 2) and np.all(nf == 1))


def euler_characteristic(tris):
    t = np.asarray(tris, np.int64)
    V = len(np.unique(t))
    uniq, _, _ = edge_use(t)
    return V - len(uniq) + len(t)


def signed_volume(verts, tris):
    v = np.asarray(verts, np.float64)
    t = np.asarray(tris, np.int64)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def mesh_shells(n_verts, tris):
    """Connected components of the mesh graph (union-find over triangle edges)."""
    par = np.arange(n_verts)

    def find(x):
        while par[x] != x:
            par[x] = par[par[x]]
            x = par[x]
        return x
    for i, j, k in np.asarray(tris, np.int64):
        for p, q in ((i, j), (j, k)):
            rp, rq = find(p), find(q)
            if rp != rq:
                par[max(rp, rq)] = min(rp, rq)
    used = np.unique(np.asarray(tris, np.int64))
    return len({find(int(u)) for u in used})


def sphere_rig(n=12, r=6.0, h=2.0, W=640, H=480, f=700.0, vol=1.0, coarse=0.05, fine=0.01, steps=8):
    """A ring of cameras around a sphere at the origin-centred volume."""
    from synth.scenes import _make_rig, _gen
    cs = [(r * math.cos(2 * math.pi * k / n), r * math.sin(2 * math.pi * k / n), h + (k % 3) * 1.5 - 1.5)
          for k in range(n)]
    return _make_rig("sphere", cs, [(0, 0, 1.0)] * n, f, W, H, _gen("sphere/rig"),
                     (-vol, -vol, 1.0 - vol), (vol, vol, 1.0 + vol), coarse, fine, steps, jitter_deg=0.0)


def fma32(a, b, c):
    """Correctly rounded binary32 fused multiply-add a*b + c of binary32
    arrays, in numpy.  The product is exact in binary64 (24 + 24 significant
    bits); the binary64 sum s and its exact error e (Knuth's TwoSum) give the
    exact value s + e.  Rounding s to binary32 is correct unless s lies
    exactly halfway between two binary32 numbers while e != 0; the exact value
    then lies on e's side of s."""
    a, b, c = (np.asarray(x, np.float32).astype(np.float64) for x in (a, b, c))
    p = a * b
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    r = s.astype(np.float32)
    r64 = r.astype(np.float64)
    nb = np.nextafter(r, np.where(s > r64, np.float32(np.inf), np.float32(-np.inf)).astype(np.float32))
    tie = (s != r64) & (np.abs(s - r64) == np.abs(nb.astype(np.float64) - s))
    return np.where(tie & (e != 0) & ((e > 0) == (s > r64)), nb, r)


def project32(P, X, Y, Z):
    """(x', y', w') of binary32 points through a 3x4 matrix, each row
    ((p3 + p2 Z) + p1 Y) + p0 X in three fused multiply-adds (binary32)."""
    P = np.asarray(P, np.float32)
    X, Y, Z = (np.asarray(v, np.float32) for v in (X, Y, Z))
    return [fma32(P[r, 0], X, fma32(P[r, 1], Y, fma32(P[r, 2], Z, P[r, 3]))) for r in range(3)]
