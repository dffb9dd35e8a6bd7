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


# ---- exact binary32 arithmetic on rationals (an emulation independent of numpy
# and of the C library: every operation is done exactly in Fractions and then
# rounded once, to nearest with ties to even, as IEEE binary32 prescribes)

def round32(q):
    """The binary32 number nearest to the rational q (ties to even), as a
    Fraction; normal and subnormal ranges (no overflow handling)."""
    from fractions import Fraction
    q = Fraction(q)
    if q == 0:
        return Fraction(0)
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    # now 2^e <= a < 2^(e+1)
    e = max(e, -126)
    quantum = Fraction(2) ** (e - 23)
    m = a / quantum
    n = m.numerator // m.denominator
    r = m - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    out = n * quantum
    return out if q > 0 else -out


def fma_exact32(a, b, c):
    """Correctly rounded binary32 fused multiply-add a*b + c of rationals."""
    return round32(a * b + c)


def cover_binary32_exact(P, X, Y, Z, px, py):
    """The depth-image coverage reading, evaluated exactly as written with
    Fractions: is the centre of pixel (px, py) covered by the triangle with
    binary32 vertices (X[j], Y[j], Z[j]) in the view of the binary32 3x4
    matrix P?  Homogeneous points: each row ((p3 + p2 Z) + p1 Y) + p0 X in
    three fused multiply-adds; a vertex with w <= 0 or a zero determinant
    skips the triangle; the centre p must lie in the closed box of the
    projections (signs of p_x w_j - x_j and p_y w_j - y_j, one fused rounding
    each) and on the same side of the three edge functions
    (p_x a - p_y b) + c, with a = y_i w_j - w_i y_j, b = x_i w_j - w_i x_j,
    c = x_i y_j - y_i x_j for edges (0,1), (1,2), (2,0), every product and
    difference rounded on its own; all >= 0 or all <= 0 counts."""
    from fractions import Fraction as F
    p = [[F(float(v)) for v in row] for row in np.asarray(P, np.float32).reshape(3, 4)]
    r, m = round32, round32
    h = []
    for j in range(3):
        xj, yj, zj = F(float(X[j])), F(float(Y[j])), F(float(Z[j]))
        h.append([fma_exact32(p[k][0], xj, fma_exact32(p[k][1], yj, fma_exact32(p[k][2], zj, p[k][3])))
                  for k in range(3)])
    if any(hj[2] <= 0 for hj in h):
        return False
    ea, eb, ec = [], [], []
    for i, j in ((0, 1), (1, 2), (2, 0)):
        xi, yi, wi = h[i]
        xj, yj, wj = h[j]
        ea.append(r(m(yi * wj) - m(wi * yj)))
        eb.append(r(m(xi * wj) - m(wi * xj)))
        ec.append(r(m(xi * yj) - m(yi * xj)))
    det = r(r(m(h[0][0] * ea[1]) - m(h[0][1] * eb[1])) + m(h[0][2] * ec[1]))
    if det == 0:
        return False
    pcx, pcy = F(int(px)) + F(1, 2), F(int(py)) + F(1, 2)
    for c, k in ((pcx, 0), (pcy, 1)):
        s = [fma_exact32(c, h[j][2], -h[j][k]) for j in range(3)]
        if not (any(v >= 0 for v in s) and any(v <= 0 for v in s)):
            return False
    e = [r(r(m(pcx * ea[k]) - m(pcy * eb[k])) + ec[k]) for k in range(3)]
    return all(v >= 0 for v in e) or all(v <= 0 for v in e)
