"""Python front end of the CPU oracle (oracle/fvv_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark call it; the product path never does.  The C file is built
here with gcc (-O2 -ffp-contract=off) into two libraries: binary32 (the parity
target) and binary64 (for the count of voxels whose occupancy flips).

Every function follows a section of the paper, named in its docstring; the
C file states the readings taken where the paper is silent or garbled.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fvv_oracle.c")
BUILD = os.path.join(HERE, "_build")
_lock = threading.Lock()
_libs: dict = {}


def build(force: bool = False) -> dict:
    """Compile the binary32 and binary64 oracles; return their paths."""
    os.makedirs(BUILD, exist_ok=True)
    out = {}
    for prec, real in (("f32", "float"), ("f64", "double")):
        so = os.path.join(BUILD, f"liboracle_{prec}.so")
        if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(SRC):
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                                   "-fPIC", "-shared", f"-DORC_REAL={real}", "-o", tmp, SRC, "-lm"])
            os.replace(tmp, so)
        out[prec] = so
    return out


class OrcRig(C.Structure):
    _fields_ = [("n_cams", C.c_int), ("P", C.POINTER(C.c_float)), ("centre", C.POINTER(C.c_float)),
                ("width", C.POINTER(C.c_int)), ("height", C.POINTER(C.c_int)),
                ("vol_min", C.c_float * 3), ("vol_max", C.c_float * 3),
                ("coarse_m", C.c_float), ("fine_m", C.c_float), ("bisect_steps", C.c_int),
                ("t_np", C.c_int), ("t_nb", C.c_int), ("t_v", C.c_float), ("oob_policy", C.c_int),
                ("surface_rule", C.c_int)]


class OrcRoi(C.Structure):
    _fields_ = [("cmin", C.c_int * 3), ("cmax", C.c_int * 3), ("gmin", C.c_int * 3), ("gmax", C.c_int * 3),
                ("fdim", C.c_int * 3), ("forigin", C.c_double * 3), ("count", C.c_longlong)]


class OrcFrame(C.Structure):
    _fields_ = [("dims", C.c_int * 3), ("coarse", C.POINTER(C.c_uint8)), ("labels", C.POINTER(C.c_int32)),
                ("n_components", C.c_int), ("n_rois", C.c_int), ("rois", C.POINTER(OrcRoi)),
                ("fine_offset", C.POINTER(C.c_longlong)), ("fine", C.POINTER(C.c_uint8)),
                ("n_verts", C.c_longlong), ("n_tris", C.c_longlong),
                ("roi_vert_offset", C.POINTER(C.c_longlong)), ("roi_tri_offset", C.POINTER(C.c_longlong)),
                ("verts", C.POINTER(C.c_double)), ("vert_key", C.POINTER(C.c_uint64)),
                ("vert_a", C.POINTER(C.c_double)), ("vert_b", C.POINTER(C.c_double)),
                ("tris", C.POINTER(C.c_uint32)),
                ("tests_coarse", C.c_longlong), ("tests_fine", C.c_longlong), ("tests_bisect", C.c_longlong)]


def _lib(prec: str):
    with _lock:
        if prec not in _libs:
            paths = build()
            lib = C.CDLL(paths[prec])
            lib.orc_reconstruct.restype = C.c_int
            lib.orc_frame_free.restype = None
            lib.orc_mc_cell.restype = C.c_int
            lib.orc_real_bytes.restype = C.c_int
            _libs[prec] = lib
        return _libs[prec]


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


@dataclass
class Roi:
    cmin: tuple
    cmax: tuple
    gmin: tuple
    gmax: tuple
    fdim: tuple
    forigin: np.ndarray
    count: int


@dataclass
class FrameResult:
    dims: tuple
    coarse: np.ndarray        # (nz,ny,nx) uint8
    labels: np.ndarray        # (nz,ny,nx) int32 canonical labels
    n_components: int
    rois: list
    fine: list                # per ROI (fz,fy,fx) uint8
    verts: np.ndarray         # (V,3) float64 holding values of the oracle's type
    vert_key: np.ndarray      # (V,) uint64
    vert_a: np.ndarray        # (V,3) final ON end of each bisection
    vert_b: np.ndarray        # (V,3) final OFF end of each bisection
    roi_vert_offset: np.ndarray
    roi_tri_offset: np.ndarray
    tris: np.ndarray          # (T,3) uint32
    tests_coarse: int
    tests_fine: int
    tests_bisect: int

    @property
    def tests(self) -> int:
        return self.tests_coarse + self.tests_fine + self.tests_bisect


class Oracle:
    """The oracle for one rig (cameras + parameters) in one precision."""

    def __init__(self, rig, precision: str = "f32"):
        assert precision in ("f32", "f64")
        self.prec = precision
        self.real = np.float32 if precision == "f32" else np.float64
        self.lib = _lib(precision)
        self.rig = rig
        self._P = np.ascontiguousarray(rig.P.reshape(-1, 12), np.float32)
        self._centre = np.ascontiguousarray(rig.centre, np.float32)
        self._w = np.ascontiguousarray(rig.width, np.int32)
        self._h = np.ascontiguousarray(rig.height, np.int32)
        r = OrcRig()
        r.n_cams = rig.n_cams
        r.P = _p(self._P, C.c_float)
        r.centre = _p(self._centre, C.c_float)
        r.width = _p(self._w, C.c_int)
        r.height = _p(self._h, C.c_int)
        r.vol_min = (C.c_float * 3)(*rig.vol_min)
        r.vol_max = (C.c_float * 3)(*rig.vol_max)
        r.coarse_m = rig.coarse_m
        r.fine_m = rig.fine_m
        r.bisect_steps = rig.bisect_steps
        r.t_np = rig.t_np
        r.t_nb = rig.t_nb
        r.t_v = rig.t_v
        r.oob_policy = rig.oob_policy
        r.surface_rule = getattr(rig, "surface_rule", 0)
        self._rig = r

    # -- helpers
    def _images(self, imgs):
        arrs = [np.ascontiguousarray(np.asarray(m), dtype=np.uint8) for m in imgs]
        ptrs = (C.POINTER(C.c_uint8) * len(arrs))(*[_p(a, C.c_uint8) for a in arrs])
        return arrs, ptrs

    # -- Sec. II-B-1
    def points_on(self, masks, pts):
        """Occupancy of world points (M,3): ON iff every camera sees it in its silhouette."""
        arrs, ptrs = self._images(masks)
        pts = np.ascontiguousarray(np.asarray(pts, np.float64))
        out = np.zeros(len(pts), np.uint8)
        tests = C.c_longlong(0)
        self.lib.orc_points_on(C.byref(self._rig), ptrs, C.c_longlong(len(pts)), _p(pts, C.c_double),
                               _p(out, C.c_uint8), C.byref(tests))
        return out, tests.value

    # -- Sec. II-C, Eqs. (2)-(3)
    def edge_lambda(self, masks, a, b):
        """The paper's isovalue of grid edges from ON ends a (M,3) to OFF ends
        b (M,3): per camera the Bresenham walk ratio of Eq. (2), and their
        minimum, Eq. (3).  Returns (lambda (M,), per camera (M,N), pixels read)."""
        arrs, ptrs = self._images(masks)
        a = np.ascontiguousarray(np.asarray(a, np.float64).reshape(-1, 3))
        b = np.ascontiguousarray(np.asarray(b, np.float64).reshape(-1, 3))
        lam = np.zeros(len(a), np.float64)
        lam_n = np.zeros((len(a), self.rig.n_cams), np.float64)
        t = C.c_longlong(0)
        rc = self.lib.orc_edge_lambda(C.byref(self._rig), ptrs, C.c_longlong(len(a)), _p(a, C.c_double),
                                      _p(b, C.c_double), _p(lam, C.c_double), _p(lam_n, C.c_double), C.byref(t))
        assert rc == 0
        return lam.astype(self.real), lam_n.astype(self.real), int(t.value)

    def grid_dims(self):
        d = (C.c_int * 3)()
        if self.lib.orc_grid_dims(C.byref(self._rig), d):
            raise ValueError("empty grid")
        return tuple(d)

    def coarse(self, masks):
        """Sec. II-B-1: coarse occupancy (nz,ny,nx) and the camera-test count."""
        nx, ny, nz = self.grid_dims()
        arrs, ptrs = self._images(masks)
        occ = np.zeros((nz, ny, nx), np.uint8)
        tests = C.c_longlong(0)
        self.lib.orc_coarse(C.byref(self._rig), ptrs, _p(occ, C.c_uint8), C.byref(tests))
        return occ, tests.value

    # -- Sec. II-B-2
    def ccl_bfs(self, occ):
        """26-connected components by flood fill, numbered by smallest index."""
        occ = np.ascontiguousarray(occ, np.uint8)
        nz, ny, nx = occ.shape
        lab = np.zeros(occ.shape, np.int32)
        c = self.lib.orc_ccl_bfs(nx, ny, nz, _p(occ, C.c_uint8), _p(lab, C.c_int32))
        return lab, c

    def ccl_uf(self, occ):
        """The oracle's second labelling (sequential union-find), same numbering."""
        occ = np.ascontiguousarray(occ, np.uint8)
        nz, ny, nx = occ.shape
        lab = np.zeros(occ.shape, np.int32)
        c = self.lib.orc_ccl_uf(nx, ny, nz, _p(occ, C.c_uint8), _p(lab, C.c_int32))
        return lab, c

    def filter(self, raw, n_comp, max_rois=4096):
        """Eq. (1) (prose reading) and the grown 3D ROI of each kept component."""
        raw = np.ascontiguousarray(raw, np.int32)
        nz, ny, nx = raw.shape
        lab = np.zeros(raw.shape, np.int32)
        rois = (OrcRoi * max(max_rois, 1))()
        k = self.lib.orc_filter(C.byref(self._rig), nx, ny, nz, _p(raw, C.c_int32), n_comp,
                                _p(lab, C.c_int32), rois, max_rois)
        if k < 0:
            raise MemoryError("oracle filter failed")
        return lab, [self._roi(rois[i]) for i in range(min(k, max_rois))]

    @staticmethod
    def _roi(r):
        return Roi(tuple(r.cmin), tuple(r.cmax), tuple(r.gmin), tuple(r.gmax), tuple(r.fdim),
                   np.array(list(r.forigin)), int(r.count))

    # -- Sec. II-C
    @staticmethod
    def mc_cell(case: int, prec: str = "f32"):
        """Triangles (as cube-edge triples) of one MC cell from the face rule."""
        lib = _lib(prec)
        buf = (C.c_int * 36)()
        n = lib.orc_mc_cell(int(case), buf)
        if n < 0:
            raise ValueError(f"face segments of case {case} do not close")
        return [tuple(buf[3 * i:3 * i + 3]) for i in range(n)]

    # -- Sec. II-B and II-C for a whole frame
    def reconstruct(self, masks, max_rois=4096) -> FrameResult:
        arrs, ptrs = self._images(masks)
        f = OrcFrame()
        rc = self.lib.orc_reconstruct(C.byref(self._rig), ptrs, max_rois, C.byref(f))
        if rc == -2:
            raise OverflowError("more ROIs than max_rois")
        if rc != 0:
            raise RuntimeError(f"oracle reconstruct failed ({rc})")
        try:
            nx, ny, nz = tuple(f.dims)
            n = nx * ny * nz
            coarse = np.ctypeslib.as_array(f.coarse, (n,)).copy().reshape(nz, ny, nx)
            labels = np.ctypeslib.as_array(f.labels, (n,)).copy().reshape(nz, ny, nx)
            K = f.n_rois
            rois = [self._roi(f.rois[i]) for i in range(K)]
            foff = np.ctypeslib.as_array(f.fine_offset, (K + 1,)).copy()
            fine = []
            if K:
                fb = np.ctypeslib.as_array(f.fine, (int(foff[K]),)).copy() if foff[K] else np.zeros(0, np.uint8)
                for i, r in enumerate(rois):
                    fine.append(fb[foff[i]:foff[i + 1]].reshape(r.fdim[2], r.fdim[1], r.fdim[0]))
            verts, keys, va, vb, tris = self._mesh_arrays(f)
            rvo = np.ctypeslib.as_array(f.roi_vert_offset, (K + 1,)).copy()
            rto = np.ctypeslib.as_array(f.roi_tri_offset, (K + 1,)).copy()
            return FrameResult((nx, ny, nz), coarse, labels, f.n_components, rois, fine, verts, keys, va, vb,
                               rvo, rto, tris, f.tests_coarse, f.tests_fine, f.tests_bisect)
        finally:
            self.lib.orc_frame_free(C.byref(f))

    @staticmethod
    def _mesh_arrays(f):
        V, T = f.n_verts, f.n_tris

        def take(ptr, n, shape, dtype):
            return np.ctypeslib.as_array(ptr, (n,)).copy().reshape(shape) if n else np.zeros(shape, dtype)
        verts = take(f.verts, V * 3, (V, 3), np.float64)
        keys = take(f.vert_key, V, (V,), np.uint64)
        va = take(f.vert_a, V * 3, (V, 3), np.float64)
        vb = take(f.vert_b, V * 3, (V, 3), np.float64)
        tris = take(f.tris, T * 3, (T, 3), np.uint32)
        return verts, keys, va, vb, tris

    def mesh_one(self, masks, roi: Roi, occ):
        """Sec. II-C for one ROI with the fine occupancy given as (fz,fy,fx):
        returns (verts, keys, a, b, tris, bisection tests)."""
        arrs, ptrs = self._images(masks)
        r = OrcRoi()
        r.cmin = (C.c_int * 3)(*roi.cmin); r.cmax = (C.c_int * 3)(*roi.cmax)
        r.gmin = (C.c_int * 3)(*roi.gmin); r.gmax = (C.c_int * 3)(*roi.gmax)
        r.fdim = (C.c_int * 3)(*roi.fdim); r.forigin = (C.c_double * 3)(*[float(x) for x in roi.forigin])
        r.count = roi.count
        occ = np.ascontiguousarray(occ, np.uint8)
        assert occ.shape == (roi.fdim[2], roi.fdim[1], roi.fdim[0])
        f = OrcFrame()
        if self.lib.orc_mesh_one(C.byref(self._rig), ptrs, C.byref(r), _p(occ, C.c_uint8), C.byref(f)):
            raise RuntimeError("oracle mesh failed")
        try:
            return self._mesh_arrays(f) + (f.tests_bisect,)
        finally:
            self.lib.orc_frame_free(C.byref(f))

    # -- Sec. II-D-1
    def depth(self, verts, tris):
        """Depth image of every camera (Eq. (4)): list of (H,W) arrays, +inf where empty."""
        verts = np.ascontiguousarray(np.asarray(verts, np.float64))
        tris = np.ascontiguousarray(np.asarray(tris, np.uint32))
        sizes = [(int(h), int(w)) for h, w in zip(self.rig.height, self.rig.width)]
        total = sum(h * w for h, w in sizes)
        buf = np.empty(total, self.real)
        ctype = C.c_float if self.prec == "f32" else C.c_double
        rc = self.lib.orc_depth(C.byref(self._rig), C.c_longlong(len(verts)), _p(verts, C.c_double),
                                C.c_longlong(len(tris)), _p(tris, C.c_uint32), _p(buf, ctype))
        if rc:
            raise ValueError("triangle index out of range")
        out, o = [], 0
        for h, w in sizes:
            out.append(buf[o:o + h * w].reshape(h, w))
            o += h * w
        return out

    # -- Sec. II-D-2 and II-E
    def colour(self, rgb, viewpoint, depth, verts):
        """Per-vertex colour from the nearest camera that sees it unoccluded."""
        arrs, ptrs = self._images(rgb)
        verts = np.ascontiguousarray(np.asarray(verts, np.float64))
        dep = np.ascontiguousarray(np.concatenate([np.asarray(d, self.real).ravel() for d in depth]))
        vp = np.ascontiguousarray(np.asarray(viewpoint, np.float32))
        out = np.zeros((len(verts), 3), np.uint8)
        cam = np.zeros(len(verts), np.int32)
        ctype = C.c_float if self.prec == "f32" else C.c_double
        self.lib.orc_colour(C.byref(self._rig), ptrs, _p(vp, C.c_float), _p(dep, ctype),
                            C.c_longlong(len(verts)), _p(verts, C.c_double), _p(out, C.c_uint8),
                            _p(cam, C.c_int32))
        return out, cam

    # -- Sec. II-E, step E: a novel view
    def render_view(self, rgb, depth, verts, tris, P, centre, width, height):
        """The coloured mesh seen from a virtual camera (3x4 matrix P, centre,
        image width x height): per pixel the nearest covering triangle (by
        squared centroid distance, ties to the lower index) and the colour of
        its centroid from the nearest capture camera that sees it unoccluded.
        Returns (triangle index (H,W) int64, -1 = none; squared distance
        (H,W), +inf = none; RGB (H,W,3) uint8; capture camera (H,W) int32)."""
        arrs, ptrs = self._images(rgb)
        verts = np.ascontiguousarray(np.asarray(verts, np.float64))
        tris = np.ascontiguousarray(np.asarray(tris, np.uint32))
        dep = np.ascontiguousarray(np.concatenate([np.asarray(d, self.real).ravel() for d in depth]))
        Pv = np.ascontiguousarray(np.asarray(P, np.float32).reshape(12))
        Cv = np.ascontiguousarray(np.asarray(centre, np.float32).reshape(3))
        tri = np.empty((height, width), np.int64)
        d2 = np.empty((height, width), self.real)
        out = np.empty((height, width, 3), np.uint8)
        cam = np.empty((height, width), np.int32)
        ctype = C.c_float if self.prec == "f32" else C.c_double
        rc = self.lib.orc_render_view(C.byref(self._rig), ptrs, _p(dep, ctype), C.c_longlong(len(verts)),
                                      _p(verts, C.c_double), C.c_longlong(len(tris)), _p(tris, C.c_uint32),
                                      _p(Pv, C.c_float), _p(Cv, C.c_float), C.c_int(width), C.c_int(height),
                                      _p(tri, C.c_int64), _p(d2, ctype), _p(out, C.c_uint8), _p(cam, C.c_int32))
        if rc:
            raise ValueError("triangle index out of range")
        return tri, d2, out, cam
