"""Thin Python binding of libfvv (include/fvv.h).

Argument marshalling only: every step of the reconstruction runs in the
library's sm_103a kernels.  PyTorch provides the device memory (the rig's
arena is a torch tensor unless the library is asked to allocate it) and the
stream (torch's current stream).  There is no fallback: if libfvv.so is
missing, importing this module raises.

The module-level functions carry the C names (fvv_create_rig, ...); `Rig`
wraps them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfvv.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1903_11785_gb300.build.build() "
                      "(or __graft_entry__.build()); there is no CPU fallback")
_lib = C.CDLL(LIB_PATH)

FVV_OK, FVV_ERR_INVALID_ARG, FVV_ERR_OUT_OF_MEMORY, FVV_ERR_CAPACITY, FVV_ERR_NOT_READY, FVV_ERR_TIMEOUT, \
    FVV_ERR_CUDA = range(7)
FVV_OOB_STRICT, FVV_OOB_ABSTAIN = 0, 1
FVV_SURFACE_BISECT, FVV_SURFACE_LAMBDA = 0, 1
FVV_MAPPED_HOST = 2
FVV_RGB_MAPPED_HOST = FVV_MAPPED_HOST
FVV_MAX_CAMS, FVV_MAX_BATCH = 64, 256
FVV_DEBUG_SIL_BITS, FVV_DEBUG_COARSE_BITS, FVV_DEBUG_LABELS, FVV_DEBUG_FINE_BITS, FVV_DEBUG_DEPTH = range(5)
FLAG_NAMES = {1: "ROOTS", 2: "ROIS", 4: "FINE", 8: "VERTS", 16: "TRIS", 32: "LOOP"}
STAGES = ("pack", "coarse", "ccl", "fine", "mc", "bisect", "depth", "colour")
TUNE_KNOBS = ("coarse", "fine", "bisect", "zbuffer", "triangles")
N_TUNE = len(TUNE_KNOBS)
FINE_TILES = ((4, 4, 8), (4, 4, 4), (4, 8, 8))   # FVV_TILE_*: fine-hull tile (x, y, z) samples
ZBUFFER_CAMS = (1, 2, 4)                          # cameras one z-buffer block serves
TUNE_INTS = 2 * N_TUNE + 2


def tuning_dict(cfg):
    """{kernel: (threads per block, blocks per SM)}, the fine-hull tile
    shape ("fine_tile": (x, y, z)) and the cameras per z-buffer block
    ("zbuffer_cams") from the flat C layout."""
    d = {k: (cfg[i], cfg[N_TUNE + i]) for i, k in enumerate(TUNE_KNOBS)}
    d["fine_tile"] = FINE_TILES[cfg[2 * N_TUNE]]
    d["zbuffer_cams"] = cfg[2 * N_TUNE + 1]
    return d


class RigDesc(C.Structure):
    _fields_ = [("n_cams", C.c_int), ("P", C.POINTER(C.c_float)), ("centre", C.POINTER(C.c_float)),
                ("width", C.POINTER(C.c_int)), ("height", C.POINTER(C.c_int)), ("max_slots", C.c_int),
                ("host_staging", C.c_int)]


class ReconParams(C.Structure):
    _fields_ = [("vol_min", C.c_float * 3), ("vol_max", C.c_float * 3), ("coarse_m", C.c_float),
                ("fine_m", C.c_float), ("bisect_steps", C.c_int), ("t_np", C.c_int), ("t_nb", C.c_int),
                ("t_v", C.c_float), ("oob_policy", C.c_int), ("max_components", C.c_int), ("max_rois", C.c_int),
                ("max_fine_words", C.c_longlong), ("max_verts", C.c_longlong), ("max_tris", C.c_longlong),
                ("surface_rule", C.c_int)]


class Roi(C.Structure):
    _fields_ = [("cmin", C.c_int * 3), ("cmax", C.c_int * 3), ("gmin", C.c_int * 3), ("gmax", C.c_int * 3),
                ("fdim", C.c_int * 3), ("forigin", C.c_float * 3), ("count", C.c_int), ("label", C.c_int),
                ("vert_offset", C.c_longlong), ("n_verts", C.c_longlong), ("tri_offset", C.c_longlong),
                ("n_tris", C.c_longlong)]


class Counts(C.Structure):
    _fields_ = [("flags", C.c_uint), ("n_components", C.c_int), ("n_rois", C.c_int), ("pad_", C.c_int),
                ("n_coarse_on", C.c_longlong), ("n_fine_words", C.c_longlong), ("n_verts", C.c_longlong),
                ("n_tris", C.c_longlong), ("tests_coarse", C.c_longlong), ("tests_fine", C.c_longlong),
                ("tests_bisect", C.c_longlong), ("lookups_fine", C.c_longlong), ("lookups_bisect", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class ResultsDst(C.Structure):
    _fields_ = [("counts", Counts), ("rois", C.c_void_p), ("verts", C.c_void_p), ("tris", C.c_void_p),
                ("rgb", C.c_void_p), ("cam", C.c_void_p)]


_vp = C.c_void_p
_sigs = {
    "fvv_query_arena": ([C.POINTER(RigDesc), C.POINTER(ReconParams), C.POINTER(C.c_size_t)], C.c_int),
    "fvv_create_rig": ([C.POINTER(RigDesc), C.POINTER(ReconParams), _vp, C.c_size_t, C.POINTER(_vp)], C.c_int),
    "fvv_destroy_rig": ([_vp], C.c_int),
    "fvv_upload_silhouettes": ([_vp, C.c_int, C.POINTER(_vp), C.c_int, _vp], C.c_int),
    "fvv_upload_silhouettes_batch": ([_vp, C.POINTER(C.c_int), C.c_int, C.POINTER(_vp), C.c_int, _vp], C.c_int),
    "fvv_reconstruct": ([_vp, C.POINTER(C.c_int), C.c_int, _vp], C.c_int),
    "fvv_colour": ([_vp, C.POINTER(C.c_int), C.c_int, C.POINTER(_vp), C.c_int, C.POINTER(C.c_float), _vp], C.c_int),
    "fvv_get_counts": ([_vp, C.c_int, C.POINTER(Counts), _vp], C.c_int),
    "fvv_get_results": ([_vp, C.c_int, _vp, _vp, _vp, _vp, _vp, C.c_int, _vp], C.c_int),
    "fvv_get_results_batch": ([_vp, C.POINTER(C.c_int), C.c_int, C.POINTER(ResultsDst), C.c_int, _vp], C.c_int),
    "fvv_debug_bytes": ([_vp, C.c_int, C.c_int, C.POINTER(C.c_size_t)], C.c_int),
    "fvv_get_debug": ([_vp, C.c_int, C.c_int, _vp, C.c_size_t, _vp], C.c_int),
    "fvv_mc_table": ([_vp, _vp], C.c_int),
    "fvv_debug_pixels": ([_vp, C.c_int, C.c_longlong, _vp, _vp, _vp, _vp], C.c_int),
    "fvv_debug_label_coarse": ([_vp, C.c_int, _vp, _vp], C.c_int),
    "fvv_label_components_noalloc": ([_vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _vp, _vp, _vp], C.c_int),
    "fvv_set_timing": ([_vp, C.c_int], C.c_int),
    "fvv_autotune": ([_vp, C.POINTER(C.c_int), C.c_int, _vp, C.POINTER(C.c_int)], C.c_int),
    "fvv_get_tuning": ([_vp, C.POINTER(C.c_int)], C.c_int),
    "fvv_set_tuning": ([_vp, C.POINTER(C.c_int)], C.c_int),
    "fvv_set_graphs": ([_vp, C.c_int], C.c_int),
    "fvv_get_timing": ([_vp, C.POINTER(C.c_float), C.POINTER(C.c_int)], C.c_int),
    "fvv_render_view": ([_vp, C.c_int, C.POINTER(_vp), C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int,
                         C.c_int, _vp, _vp, _vp, _vp], C.c_int),
    "fvv_probe_l2": ([C.c_int, _vp, C.c_size_t, C.c_int, _vp, C.c_int, C.c_int, _vp], C.c_int),
    "fvv_probe_fma": ([C.c_int, C.c_float, C.c_float, _vp, C.c_int, C.c_int, _vp], C.c_int),
    "fvv_last_error": ([_vp], C.c_char_p),
    "fvv_status_string": ([C.c_int], C.c_char_p),
    "fvv_version": ([], C.c_int),
}
for _name, (_args, _res) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res
EXPORTED = tuple(_sigs)


class FvvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.fvv_status_string(status).decode()}: {msg}")
        self.status = status


def _check(status, rig_ptr=None):
    if status != FVV_OK:
        raise FvvError(status, (_lib.fvv_last_error(rig_ptr) or b"").decode())


def _stream(stream=None):
    if stream is None:
        stream = torch.cuda.current_stream()
    return _vp(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr_array(ptrs):
    return (_vp * len(ptrs))(*[_vp(int(p)) for p in ptrs])


# ------------------------------------------------------------ C-named calls

def fvv_version() -> int:
    return _lib.fvv_version()


def fvv_mc_table():
    ntri = np.zeros(256, np.uint8)
    edges = np.zeros(256 * 12 * 3, np.uint8)
    _check(_lib.fvv_mc_table(ntri.ctypes.data, edges.ctypes.data))
    return ntri, edges.reshape(256, 12, 3)


def make_desc(rig, max_slots=1, host_staging=1):
    keep = dict(P=np.ascontiguousarray(np.asarray(rig.P, np.float32).reshape(-1, 12)),
                centre=np.ascontiguousarray(np.asarray(rig.centre, np.float32)),
                width=np.ascontiguousarray(np.asarray(rig.width, np.int32)),
                height=np.ascontiguousarray(np.asarray(rig.height, np.int32)))
    d = RigDesc()
    d.n_cams = int(keep["P"].shape[0])
    d.P = keep["P"].ctypes.data_as(C.POINTER(C.c_float))
    d.centre = keep["centre"].ctypes.data_as(C.POINTER(C.c_float))
    d.width = keep["width"].ctypes.data_as(C.POINTER(C.c_int))
    d.height = keep["height"].ctypes.data_as(C.POINTER(C.c_int))
    d.max_slots = max_slots
    d.host_staging = host_staging
    d._keep = keep
    return d


def make_params(rig, **caps):
    p = ReconParams()
    p.vol_min = (C.c_float * 3)(*rig.vol_min)
    p.vol_max = (C.c_float * 3)(*rig.vol_max)
    p.coarse_m = rig.coarse_m
    p.fine_m = rig.fine_m
    p.bisect_steps = rig.bisect_steps
    p.t_np = rig.t_np
    p.t_nb = rig.t_nb
    p.t_v = rig.t_v
    p.oob_policy = rig.oob_policy
    p.surface_rule = getattr(rig, "surface_rule", FVV_SURFACE_BISECT)
    for k, v in caps.items():
        setattr(p, k, v)
    return p


def fvv_query_arena(desc, params) -> int:
    n = C.c_size_t(0)
    _check(_lib.fvv_query_arena(C.byref(desc), C.byref(params), C.byref(n)))
    return n.value


def fvv_create_rig(desc, params, arena=None):
    """arena: a CUDA uint8 tensor of >= fvv_query_arena bytes, or None for a
    library-allocated arena."""
    out = _vp()
    ptr = _vp(arena.data_ptr()) if arena is not None else None
    nbytes = arena.numel() if arena is not None else 0
    _check(_lib.fvv_create_rig(C.byref(desc), C.byref(params), ptr, nbytes, C.byref(out)))
    return out


def fvv_destroy_rig(rig_ptr):
    _check(_lib.fvv_destroy_rig(rig_ptr))


def fvv_upload_silhouettes(rig_ptr, slot, masks, stream=None, in_place=False):
    """masks: list of per-camera uint8 tensors (H,W) (or one (N,H,W) tensor),
    all on the GPU or all in host memory; in_place: pinned host tensors are
    read in place by the packing kernel (FVV_MAPPED_HOST)."""
    ms = list(masks) if not torch.is_tensor(masks) else list(masks.unbind(0))
    on_dev = _rgb_mode(int(ms[0].is_cuda), ms, in_place)
    for m in ms:
        assert m.dtype == torch.uint8 and m.is_contiguous() and m.is_cuda == ms[0].is_cuda
    _check(_lib.fvv_upload_silhouettes(rig_ptr, slot, _ptr_array([m.data_ptr() for m in ms]), on_dev,
                                       _stream(stream)), rig_ptr)


def fvv_upload_silhouettes_batch(rig_ptr, slots, masks, stream=None, in_place=False):
    """masks: per slot, a list of per-camera uint8 tensors (H,W) (or one
    (N,H,W) tensor, or an (F,N,H,W) tensor for all slots); memory kinds as
    for fvv_upload_silhouettes."""
    ptrs, ms = [], []
    for per_slot in masks:
        imgs = list(per_slot) if not torch.is_tensor(per_slot) else list(per_slot.unbind(0))
        for m in imgs:
            assert m.dtype == torch.uint8 and m.is_contiguous()
            ptrs.append(m.data_ptr())
            ms.append(m)
    assert ms and all(m.is_cuda == ms[0].is_cuda for m in ms)
    on_dev = _rgb_mode(int(ms[0].is_cuda), ms, in_place)
    arr = (C.c_int * len(slots))(*slots)
    _check(_lib.fvv_upload_silhouettes_batch(rig_ptr, arr, len(slots), _ptr_array(ptrs), on_dev,
                                             _stream(stream)), rig_ptr)


def fvv_reconstruct(rig_ptr, slots, stream=None):
    arr = (C.c_int * len(slots))(*slots)
    _check(_lib.fvv_reconstruct(rig_ptr, arr, len(slots), _stream(stream)), rig_ptr)


def _rgb_mode(on_dev, imgs, in_place):
    if on_dev or not in_place:
        return on_dev
    assert all(t.is_pinned() for t in imgs), "reading in place needs pinned host tensors"
    return FVV_MAPPED_HOST


def fvv_colour(rig_ptr, slots, rgb, viewpoints, stream=None, in_place=False):
    """rgb: per slot, a list of per-camera (H,W,3) uint8 tensors (or an
    (N,H,W,3) tensor); viewpoints: (n_slots,3).  in_place: pinned host
    tensors are read in place by the kernel (FVV_RGB_MAPPED_HOST) instead of
    being copied to the device."""
    ptrs, on_dev, all_imgs = [], None, []
    for per_slot in rgb:
        imgs = list(per_slot) if not torch.is_tensor(per_slot) else list(per_slot.unbind(0))
        for t in imgs:
            assert t.dtype == torch.uint8 and t.is_contiguous()
            on_dev = int(t.is_cuda) if on_dev is None else on_dev
            assert int(t.is_cuda) == on_dev
            ptrs.append(t.data_ptr())
            all_imgs.append(t)
    on_dev = _rgb_mode(on_dev, all_imgs, in_place)
    vp = np.ascontiguousarray(np.asarray(viewpoints, np.float32).reshape(len(slots), 3))
    arr = (C.c_int * len(slots))(*slots)
    _check(_lib.fvv_colour(rig_ptr, arr, len(slots), _ptr_array(ptrs), on_dev,
                           vp.ctypes.data_as(C.POINTER(C.c_float)), _stream(stream)), rig_ptr)


def fvv_render_view(rig_ptr, slot, rgb, P, centre, width, height, stream=None, with_cam=True, in_place=False):
    """Step E: a novel view of a reconstructed slot from a virtual camera.
    rgb: per-camera (H,W,3) uint8 tensors (or an (N,H,W,3) tensor), all on
    the device or all in host memory.  Returns device tensors (key (H,W)
    int64 = squared-distance bits << 32 | triangle, -1 where empty; rgb
    (H,W,3) uint8; capture camera (H,W) int32 or None)."""
    imgs = list(rgb) if not torch.is_tensor(rgb) else list(rgb.unbind(0))
    on_dev = None
    for t in imgs:
        assert t.dtype == torch.uint8 and t.is_contiguous()
        on_dev = int(t.is_cuda) if on_dev is None else on_dev
        assert int(t.is_cuda) == on_dev
    on_dev = _rgb_mode(on_dev, imgs, in_place)
    Pm = np.ascontiguousarray(np.asarray(P, np.float32).reshape(12))
    Cm = np.ascontiguousarray(np.asarray(centre, np.float32).reshape(3))
    key = torch.empty((height, width), dtype=torch.int64, device="cuda")
    out = torch.empty((height, width, 3), dtype=torch.uint8, device="cuda")
    cam = torch.empty((height, width), dtype=torch.int32, device="cuda") if with_cam else None
    _check(_lib.fvv_render_view(rig_ptr, slot, _ptr_array([t.data_ptr() for t in imgs]), on_dev,
                                Pm.ctypes.data_as(C.POINTER(C.c_float)), Cm.ctypes.data_as(C.POINTER(C.c_float)),
                                width, height, _vp(key.data_ptr()), _vp(out.data_ptr()),
                                _vp(cam.data_ptr()) if cam is not None else None, _stream(stream)), rig_ptr)
    return key, out, cam


def fvv_get_counts(rig_ptr, slot, stream=None, allow_capacity=False) -> dict:
    c = Counts()
    st = _lib.fvv_get_counts(rig_ptr, slot, C.byref(c), _stream(stream))
    if not (allow_capacity and st == FVV_ERR_CAPACITY):
        _check(st, rig_ptr)
    return c.as_dict()


def fvv_get_results(rig_ptr, slot, device="cuda", stream=None) -> dict:
    """Mesh of a slot: rois (list of dicts), verts (V,3) float32, tris (T,3)
    int32 (uint32 values), rgb (V,3) uint8, cam (V,) int32."""
    c = fvv_get_counts(rig_ptr, slot, stream)
    V, T, K = c["n_verts"], c["n_tris"], c["n_rois"]
    dev = torch.device(device)
    verts = torch.empty((V, 3), dtype=torch.float32, device=dev)
    tris = torch.empty((T, 3), dtype=torch.int32, device=dev)
    rgb = torch.empty((V, 3), dtype=torch.uint8, device=dev)
    cam = torch.empty((V,), dtype=torch.int32, device=dev)
    rois = (Roi * max(K, 1))()
    _check(_lib.fvv_get_results(rig_ptr, slot, C.cast(rois, _vp), _vp(verts.data_ptr()), _vp(tris.data_ptr()),
                                _vp(rgb.data_ptr()), _vp(cam.data_ptr()), int(dev.type == "cuda"),
                                _stream(stream)), rig_ptr)
    if dev.type == "cuda":
        torch.cuda.current_stream().synchronize()
    out_rois = [{f: (tuple(getattr(r, f)) if isinstance(getattr(r, f), C.Array) else getattr(r, f))
                 for f, _ in Roi._fields_} for r in rois[:K]]
    return dict(counts=c, rois=out_rois, verts=verts, tris=tris, rgb=rgb, cam=cam)


def fvv_get_results_batch(rig_ptr, slots, outs, stream=None):
    """Results of several slots with one wait.  outs[i]: dict of tensors
    "verts", "tris", "rgb", "cam" (any may be missing), all in host memory
    (pinned, for asynchronous copies) or all on the device, large enough for
    slot slots[i].  Returns each slot's counts; the copies are enqueued on
    the stream."""
    n = len(slots)
    dst = (ResultsDst * n)()
    on_dev = None
    for d, o in zip(dst, outs):
        for k in ("verts", "tris", "rgb", "cam"):
            t = o.get(k)
            if t is not None:
                on_dev = t.is_cuda if on_dev is None else on_dev
                assert t.is_cuda == on_dev and t.is_contiguous()
                setattr(d, k, t.data_ptr())
    arr = (C.c_int * n)(*slots)
    _check(_lib.fvv_get_results_batch(rig_ptr, arr, n, dst, int(bool(on_dev)), _stream(stream)), rig_ptr)
    return [d.counts.as_dict() for d in dst]


def fvv_set_timing(rig_ptr, enable: bool):
    _check(_lib.fvv_set_timing(rig_ptr, int(enable)), rig_ptr)


def fvv_get_timing(rig_ptr):
    """{stage: (summed ms, intervals)} since the previous call."""
    ms = (C.c_float * len(STAGES))()
    calls = (C.c_int * len(STAGES))()
    _check(_lib.fvv_get_timing(rig_ptr, ms, calls), rig_ptr)
    return {name: (ms[i], calls[i]) for i, name in enumerate(STAGES)}


def fvv_probe_l2(mode: int, buf: torch.Tensor, reps: int, out: torch.Tensor, blocks: int, threads: int,
                 stream=None):
    """L2 micro-benchmark: mode 0 reads `buf` coalesced `reps` times, mode 1
    does `reps` random 32-bit gathers per thread from it; `out` (int32 or
    uint32, blocks*threads elements) receives each thread's XOR."""
    if buf.device.type != "cuda" or out.device.type != "cuda" or out.numel() < blocks * threads:
        raise ValueError("fvv_probe_l2: device buffers, out of blocks*threads words")
    nbytes = buf.numel() * buf.element_size()
    _check(_lib.fvv_probe_l2(mode, buf.data_ptr(), nbytes, reps, out.data_ptr(), blocks, threads, _stream(stream)))


def fvv_debug_label_coarse(rig_ptr, slot, coarse_bits: torch.Tensor, stream=None):
    """Label a given coarse grid (device int32/uint32 words in the
    FVV_DEBUG_COARSE_BITS layout) in `slot` with the library's CCL kernels."""
    assert coarse_bits.is_cuda and coarse_bits.is_contiguous() and coarse_bits.element_size() == 4
    _check(_lib.fvv_debug_label_coarse(rig_ptr, slot, _vp(coarse_bits.data_ptr()), _stream(stream)), rig_ptr)


def fvv_probe_fma(reps: int, a: float, b: float, out: torch.Tensor, blocks: int, threads: int, stream=None):
    """FP32 micro-benchmark: blocks*threads threads, 16 chains x = fma(x, a, b)
    of `reps` steps each; out (float32, blocks*threads elements) receives each
    thread's sum of its chains."""
    if out.device.type != "cuda" or out.dtype != torch.float32 or out.numel() < blocks * threads:
        raise ValueError("fvv_probe_fma: a float32 device buffer of blocks*threads elements")
    _check(_lib.fvv_probe_fma(reps, a, b, out.data_ptr(), blocks, threads, _stream(stream)))


def fvv_get_debug(rig_ptr, slot, what, stream=None) -> torch.Tensor:
    n = C.c_size_t(0)
    _check(_lib.fvv_debug_bytes(rig_ptr, slot, what, C.byref(n)), rig_ptr)
    dtype = {FVV_DEBUG_LABELS: torch.int32, FVV_DEBUG_DEPTH: torch.float32}.get(what, torch.int32)
    buf = torch.empty(max(n.value // 4, 1), dtype=dtype, device="cuda")
    _check(_lib.fvv_get_debug(rig_ptr, slot, what, _vp(buf.data_ptr()), n.value, _stream(stream)), rig_ptr)
    return buf[: n.value // 4]


# ------------------------------------------------------------ convenience

class Rig:
    """One camera rig on the current CUDA device, with max_slots frame slots."""

    def __init__(self, rig, max_slots=1, host_staging=1, torch_arena=True, **caps):
        self.scene_rig = rig
        self.desc = make_desc(rig, max_slots, host_staging)
        self.params = make_params(rig, **caps)
        self.arena_bytes = fvv_query_arena(self.desc, self.params)
        self.arena = torch.empty(self.arena_bytes, dtype=torch.uint8, device="cuda") if torch_arena else None
        self.ptr = fvv_create_rig(self.desc, self.params, self.arena)
        self.n_cams = rig.n_cams
        self.max_slots = max_slots

    def close(self):
        if self.ptr:
            fvv_destroy_rig(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload_silhouettes(self, slot, masks, stream=None, in_place=False):
        fvv_upload_silhouettes(self.ptr, slot, masks, stream, in_place)

    def upload_silhouettes_batch(self, slots, masks, stream=None, in_place=False):
        fvv_upload_silhouettes_batch(self.ptr, list(slots), masks, stream, in_place)

    def reconstruct(self, slots, stream=None):
        fvv_reconstruct(self.ptr, list(slots), stream)

    def colour(self, slots, rgb, viewpoints, stream=None, in_place=False):
        fvv_colour(self.ptr, list(slots), rgb, viewpoints, stream, in_place)

    def render_view(self, slot, rgb, P, centre, width, height, stream=None, with_cam=True, in_place=False):
        return fvv_render_view(self.ptr, slot, rgb, P, centre, width, height, stream, with_cam, in_place)

    def counts(self, slot, stream=None, allow_capacity=False):
        return fvv_get_counts(self.ptr, slot, stream, allow_capacity)

    def results(self, slot, device="cuda", stream=None):
        return fvv_get_results(self.ptr, slot, device, stream)

    def debug(self, slot, what, stream=None):
        return fvv_get_debug(self.ptr, slot, what, stream)

    def debug_label_coarse(self, slot, coarse_bits, stream=None):
        fvv_debug_label_coarse(self.ptr, slot, coarse_bits, stream)

    def set_timing(self, enable=True):
        fvv_set_timing(self.ptr, enable)

    def timing(self):
        return fvv_get_timing(self.ptr)

    def autotune(self, slots, stream=None):
        """Pick the fastest launch shapes on reconstructed slots; returns them."""
        arr = (C.c_int * len(slots))(*slots)
        cfg = (C.c_int * TUNE_INTS)()
        _check(_lib.fvv_autotune(self.ptr, arr, len(slots), _stream(stream), cfg), self.ptr)
        return tuning_dict(list(cfg))

    def get_tuning(self):
        cfg = (C.c_int * TUNE_INTS)()
        _check(_lib.fvv_get_tuning(self.ptr, cfg), self.ptr)
        return tuning_dict(list(cfg))

    def set_tuning(self, tuning):
        """tuning: as get_tuning returns it; "fine_tile" may be left out
        (4 x 4 x 8) and may be given as an (x, y, z) shape or an FVV_TILE_*
        index; "zbuffer_cams" may be left out (4, the default)."""
        tile = tuning.get("fine_tile", FINE_TILES[0])
        tile = FINE_TILES.index(tuple(tile)) if not isinstance(tile, int) else tile
        cfg = [tuning[k][0] for k in TUNE_KNOBS] + [tuning[k][1] for k in TUNE_KNOBS] + [tile]
        cfg.append(int(tuning.get("zbuffer_cams", 4)))
        _check(_lib.fvv_set_tuning(self.ptr, (C.c_int * len(cfg))(*cfg)), self.ptr)

    def set_graphs(self, enable=True):
        _check(_lib.fvv_set_graphs(self.ptr, int(enable)), self.ptr)
