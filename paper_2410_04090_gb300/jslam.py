"""Thin Python binding of libjslam's C ABI (``include/jslam.h``).

Argument marshalling only: every step of the frontend runs in the library's
CUDA kernels.  Device images are passed as CUDA tensors (uint8, 2-D, rows
may be strided) and read in place; host images are passed as numpy arrays
and copied by the library.  PyTorch provides device memory and streams.

The binding never falls back to another implementation: if the compiled
library is missing it raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjslam.so")

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_CAPACITY, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
MEM_DEVICE, MEM_HOST = 0, 1
CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy


class JslamError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)} ({status})")
        self.status = status


class Config(C.Structure):
    _fields_ = [("device", C.c_int32), ("cuda_stream", C.c_void_p),
                ("max_width", C.c_int32), ("max_height", C.c_int32), ("max_levels", C.c_int32),
                ("max_feats", C.c_int32), ("max_pairs", C.c_int32), ("fast_thresh_lo", C.c_int32),
                ("p_min", C.c_int32), ("p_max", C.c_int32), ("k_per_cell", C.c_int32),
                ("nms_q", C.c_int32), ("border", C.c_int32), ("max_disp", C.c_int32),
                ("row_band_px", C.c_int32), ("match_max_dist", C.c_int32), ("pfa_rule", C.c_int32),
                ("response_mode", C.c_int32), ("pyramid_mode", C.c_int32)]


class Image(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("pitch", C.c_int32),
                ("memory", C.c_int32), ("data", C.c_void_p)]


class StereoJob(C.Structure):
    _fields_ = [("left", Image), ("right", Image), ("levels", C.c_int32), ("scale", C.c_float),
                ("fast_thresh", C.c_int32), ("cell", C.c_int32), ("max_feats", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("tile_w_px", C.c_int32), ("tile_h_px", C.c_int32), ("nms_kernel", C.c_int32),
                ("detect_ctas_per_sm", C.c_int32), ("tile_order", C.c_int32)]

    def as_tuple(self) -> tuple:
        return self.tile_w_px, self.tile_h_px, self.nms_kernel, self.detect_ctas_per_sm, self.tile_order


class SkipView(C.Structure):
    _fields_ = [("w8", C.c_int32), ("h8", C.c_int32), ("cells_x", C.c_int32), ("cells_y", C.c_int32),
                ("logits", C.c_void_p), ("skip", C.c_void_p)]


class Keypoints(C.Structure):
    _fields_ = [("count", C.c_int32), ("capacity", C.c_int32),
                ("x", C.c_void_p), ("y", C.c_void_p), ("X", C.c_void_p), ("Y", C.c_void_p),
                ("level", C.c_void_p), ("angle_bin", C.c_void_p), ("response", C.c_void_p),
                ("k_levels", C.c_void_p), ("k_resp", C.c_void_p), ("angle", C.c_void_p),
                ("desc", C.c_void_p)]


class Matches(C.Structure):
    _fields_ = [("count", C.c_int32), ("right_idx", C.c_void_p), ("disparity", C.c_void_p),
                ("dist", C.c_void_p)]


class Refined(C.Structure):
    _fields_ = [("count", C.c_int32), ("disparity", C.c_void_p), ("depth", C.c_void_p), ("sad", C.c_void_p)]


REFINED_FIELDS = (("disparity", np.float32), ("depth", np.float32), ("sad", np.uint32))


class LevelView(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("raw_pitch", C.c_int32),
                ("blurred_pitch", C.c_int32), ("raw", C.c_void_p), ("blurred", C.c_void_p)]


# (field, numpy dtype, words per keypoint)
KP_FIELDS = (("x", np.uint16, 1), ("y", np.uint16, 1), ("X", np.uint16, 1), ("Y", np.uint16, 1),
             ("level", np.uint8, 1), ("angle_bin", np.uint8, 1), ("response", np.uint16, 1),
             ("k_levels", np.uint8, 1), ("k_resp", np.uint32, 1), ("angle", np.float32, 1),
             ("desc", np.uint32, 8))
MATCH_FIELDS = (("right_idx", np.int32), ("disparity", np.int16), ("dist", np.uint16))

# The C-ABI symbols declared in include/jslam.h.
SYMBOLS = ("jslam_default_config", "jslam_create", "jslam_extract", "jslam_extract_batch", "jslam_match",
           "jslam_sync", "jslam_get_keypoints", "jslam_get_matches", "jslam_get_level", "jslam_result_bytes",
           "jslam_download", "jslam_result_view", "jslam_destroy", "jslam_status_str", "jslam_pattern_table",
           "jslam_level_geometry", "jslam_project", "jslam_match_band", "jslam_enable_stage_timing",
           "jslam_stage_times", "jslam_pfa_scores_static", "jslam_corner_table", "jslam_set_tuning",
           "jslam_autotune", "jslam_autotune_cached", "jslam_tune_key", "jslam_tune_cache_get",
           "jslam_tune_cache_put", "jslam_graph_capture", "jslam_graph_launch", "jslam_graph_launch_jobs",
           "jslam_set_skip_model",
           "jslam_get_skip_view", "jslam_result_range", "jslam_download_range", "jslam_refine_matches",
           "jslam_get_refined", "jslam_result_refined_view", "jslam_track", "jslam_fc_ablation",
           "jslam_fc_ablation_view", "jslam_fc_ablation_times", "jslam_crf_view", "jslam_selftest_wait")
STAGES = ("pyramid", "skip", "detect", "pfa_nms", "pfa_final", "orb", "match", "refine")

_lib = None


def lib():
    """Load libjslam.so (built by ``paper_2410_04090_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2410_04090_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        st = C.c_int
        L.jslam_default_config.argtypes = [C.POINTER(Config)]
        L.jslam_default_config.restype = None
        L.jslam_create.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Config)]
        L.jslam_create.restype = st
        L.jslam_extract.argtypes = [C.c_void_p, Image, Image, C.c_int32, C.c_float, C.c_int32, C.c_int32, C.c_int32]
        L.jslam_extract.restype = st
        L.jslam_extract_batch.argtypes = [C.c_void_p, C.POINTER(StereoJob), C.c_int32]
        L.jslam_extract_batch.restype = st
        L.jslam_match.argtypes = [C.c_void_p]
        L.jslam_match.restype = st
        L.jslam_sync.argtypes = [C.c_void_p]
        L.jslam_sync.restype = st
        L.jslam_get_keypoints.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(Keypoints)]
        L.jslam_get_keypoints.restype = st
        L.jslam_get_matches.argtypes = [C.c_void_p, C.c_int32, C.POINTER(Matches)]
        L.jslam_get_matches.restype = st
        L.jslam_get_level.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.POINTER(LevelView)]
        L.jslam_get_level.restype = st
        L.jslam_track.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_int32, C.c_float, C.c_int32, C.c_void_p, C.c_void_p]
        L.jslam_track.restype = st
        L.jslam_fc_ablation.argtypes = [C.c_void_p, C.c_int32]
        L.jslam_fc_ablation.restype = st
        L.jslam_fc_ablation_view.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p),
                                             C.POINTER(C.c_void_p), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.jslam_fc_ablation_view.restype = st
        L.jslam_fc_ablation_times.argtypes = [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)]
        L.jslam_fc_ablation_times.restype = st
        L.jslam_crf_view.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.jslam_crf_view.restype = st
        L.jslam_selftest_wait.argtypes = [C.c_void_p]
        L.jslam_selftest_wait.restype = st
        L.jslam_refine_matches.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_float]
        L.jslam_refine_matches.restype = st
        L.jslam_get_refined.argtypes = [C.c_void_p, C.c_int32, C.POINTER(Refined)]
        L.jslam_get_refined.restype = st
        L.jslam_result_refined_view.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(Refined)]
        L.jslam_result_refined_view.restype = st
        L.jslam_result_bytes.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_size_t)]
        L.jslam_result_bytes.restype = st
        L.jslam_download.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_size_t]
        L.jslam_download.restype = st
        L.jslam_result_range.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_size_t),
                                         C.POINTER(C.c_size_t)]
        L.jslam_result_range.restype = st
        L.jslam_download_range.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_size_t]
        L.jslam_download_range.restype = st
        L.jslam_result_view.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.POINTER(Keypoints),
                                        C.POINTER(Matches)]
        L.jslam_result_view.restype = st
        L.jslam_destroy.argtypes = [C.c_void_p]
        L.jslam_destroy.restype = None
        L.jslam_status_str.argtypes = [C.c_int]
        L.jslam_status_str.restype = C.c_char_p
        L.jslam_pattern_table.argtypes = [C.c_void_p]
        L.jslam_pattern_table.restype = None
        L.jslam_level_geometry.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_int32,
                                           C.c_void_p, C.c_void_p, C.c_void_p]
        L.jslam_level_geometry.restype = st
        L.jslam_project.argtypes = [C.c_int32, C.c_int32, C.c_float, C.c_int32]
        L.jslam_project.restype = C.c_int32
        L.jslam_match_band.argtypes = [C.c_int32, C.c_float, C.c_int32]
        L.jslam_match_band.restype = C.c_int32
        L.jslam_set_skip_model.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_float]
        L.jslam_set_skip_model.restype = st
        L.jslam_get_skip_view.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(SkipView)]
        L.jslam_get_skip_view.restype = st
        L.jslam_set_tuning.argtypes = [C.c_void_p, C.POINTER(Tuning)]
        L.jslam_set_tuning.restype = st
        L.jslam_autotune.argtypes = [C.c_void_p, C.POINTER(StereoJob), C.c_int32, C.POINTER(Tuning)]
        L.jslam_autotune.restype = st
        L.jslam_autotune_cached.argtypes = [C.c_void_p, C.POINTER(StereoJob), C.c_int32, C.c_char_p,
                                            C.POINTER(Tuning), C.POINTER(C.c_int32)]
        L.jslam_autotune_cached.restype = st
        L.jslam_tune_key.argtypes = [C.c_char_p, C.c_int32, C.POINTER(Config), C.POINTER(StereoJob), C.c_int32,
                                     C.c_char_p, C.c_size_t]
        L.jslam_tune_key.restype = st
        L.jslam_tune_cache_get.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(Tuning), C.POINTER(C.c_int32)]
        L.jslam_tune_cache_get.restype = st
        L.jslam_tune_cache_put.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(Tuning), C.c_float]
        L.jslam_tune_cache_put.restype = st
        L.jslam_graph_capture.argtypes = [C.c_void_p, C.POINTER(StereoJob), C.c_int32]
        L.jslam_graph_capture.restype = st
        L.jslam_graph_launch.argtypes = [C.c_void_p]
        L.jslam_graph_launch.restype = st
        L.jslam_graph_launch_jobs.argtypes = [C.c_void_p, C.POINTER(StereoJob), C.c_int32]
        L.jslam_graph_launch_jobs.restype = st
        L.jslam_corner_table.argtypes = [C.c_int32, C.c_int32, C.c_void_p]
        L.jslam_corner_table.restype = st
        L.jslam_enable_stage_timing.argtypes = [C.c_void_p, C.c_int32]
        L.jslam_enable_stage_timing.restype = st
        L.jslam_stage_times.argtypes = [C.c_void_p, C.c_void_p]
        L.jslam_stage_times.restype = st
        vp = C.c_void_p
        L.jslam_pfa_scores_static.argtypes = [vp, vp, vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                              C.c_float, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, C.c_int32, vp]
        L.jslam_pfa_scores_static.restype = st
        _lib = L
    return _lib


def status_str(s: int) -> str:
    return lib().jslam_status_str(s).decode()


def _check(s: int, what: str):
    if s != OK:
        raise JslamError(s, what)


# ------------------------------------------------------------ host tables

def pattern_table() -> np.ndarray:
    out = np.zeros(30 * 256 * 4, np.int8)
    lib().jslam_pattern_table(out.ctypes.data)
    return out.reshape(30, 256, 4)


def level_geometry(width: int, height: int, levels: int, scale: float, cell: int):
    w = np.zeros(levels, np.int32); h = np.zeros(levels, np.int32); c = np.zeros(levels, np.int32)
    _check(lib().jslam_level_geometry(width, height, levels, scale, cell, w.ctypes.data, h.ctypes.data,
                                      c.ctypes.data), "jslam_level_geometry")
    return w, h, c


def project(v: int, level: int, scale: float, extent: int) -> int:
    return lib().jslam_project(v, level, scale, extent)


def corner_table(p_min: int = 9, p_max: int = 13) -> np.ndarray:
    out = np.zeros(2048, np.uint32)
    _check(lib().jslam_corner_table(p_min, p_max, out.ctypes.data), "jslam_corner_table")
    return out


def match_band(level: int, scale: float, row_band_px: int) -> int:
    return lib().jslam_match_band(level, scale, row_band_px)


# ------------------------------------------------------------ tuning cache (host only)

def tune_key(gpu_name: str, sm_count: int, config: dict, jobs) -> str:
    """Key of a batch in the tuning cache (jslam_tune_key; no device work).
    `config` holds jslam_config fields (defaults for the rest); `jobs` are
    Job objects whose images may be numpy arrays."""
    cfg = Config()
    lib().jslam_default_config(C.byref(cfg))
    for k, v in config.items():
        setattr(cfg, k, v)
    pb = PreparedBatch(jobs)
    buf = C.create_string_buffer(1 << 16)
    _check(lib().jslam_tune_key(gpu_name.encode(), sm_count, C.byref(cfg), pb.array, pb.n, buf, len(buf)),
           "jslam_tune_key")
    return buf.value.decode()


def tune_cache_get(path: str, key: str):
    """The cached pick (tile_w_px, tile_h_px, nms_kernel, detect_ctas_per_sm,
    tile_order) or None."""
    t, found = Tuning(), C.c_int32(0)
    _check(lib().jslam_tune_cache_get(os.fsencode(path), key.encode(), C.byref(t), C.byref(found)),
           "jslam_tune_cache_get")
    return t.as_tuple() if found.value else None


def tune_cache_put(path: str, key: str, tuning, stage_ms: float = 0.0) -> None:
    t = Tuning(*tuning)
    _check(lib().jslam_tune_cache_put(os.fsencode(path), key.encode(), C.byref(t), stage_ms), "jslam_tune_cache_put")


# ------------------------------------------------------------ no-allocation PFA scores

def pfa_scores_static(level, x, y, response, width0: int, height0: int, levels: int, scale: float = 1.2,
                      nms_q: int = 3, pfa_rule: int = 0, stream=None) -> dict:
    """PFA scores of culled corners (CUDA tensors: level u8, x/y/response
    u16) through jslam_pfa_scores_static, which allocates no device memory.
    The output tensors are allocated here, by the caller side.  The four
    inputs must be contiguous 1-D tensors of equal length on one CUDA device
    (the kernel reads n entries of each by raw pointer)."""
    import torch
    ins = {"level": (level, torch.uint8), "x": (x, torch.uint16), "y": (y, torch.uint16),
           "response": (response, torch.uint16)}
    n = int(level.numel()) if isinstance(level, torch.Tensor) else -1
    for name, (t, dt) in ins.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if t.dtype != dt or t.dim() != 1 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous 1-D {dt} tensor")
        if t.numel() != n or t.device != level.device:
            raise ValueError(f"{name} must have the length and device of level")
    dev = level.device
    out = {"X": torch.empty(n, dtype=torch.uint16, device=dev), "Y": torch.empty(n, dtype=torch.uint16, device=dev),
           "k_levels": torch.empty(n, dtype=torch.uint8, device=dev),
           "k_resp": torch.empty(n, dtype=torch.uint32, device=dev),
           "alive": torch.empty(n, dtype=torch.uint8, device=dev)}
    handle = (stream if isinstance(stream, int) else stream.cuda_stream) if stream is not None else \
        torch.cuda.current_stream(dev).cuda_stream
    _check(lib().jslam_pfa_scores_static(level.data_ptr(), x.data_ptr(), y.data_ptr(), response.data_ptr(), n,
                                         width0, height0, levels, scale, nms_q, pfa_rule, out["X"].data_ptr(),
                                         out["Y"].data_ptr(), out["k_levels"].data_ptr(), out["k_resp"].data_ptr(),
                                         out["alive"].data_ptr(), dev.index, handle), "jslam_pfa_scores_static")
    return out


# ------------------------------------------------------------ images

def _image(img) -> Image:
    """jslam_image of a CUDA tensor (device) or a numpy array (host)."""
    if isinstance(img, np.ndarray):
        if img.dtype != np.uint8 or img.ndim != 2 or img.strides[1] != 1:
            raise ValueError("host image must be a 2-D uint8 array with contiguous rows")
        return Image(img.shape[1], img.shape[0], img.strides[0], MEM_HOST, img.ctypes.data)
    import torch
    if not isinstance(img, torch.Tensor) or img.dtype != torch.uint8 or img.dim() != 2 or img.stride(1) != 1:
        raise ValueError("device image must be a 2-D uint8 CUDA tensor with contiguous rows")
    if not img.is_cuda:
        raise ValueError("tensor images must live on the GPU; pass numpy arrays for host memory")
    return Image(img.shape[1], img.shape[0], img.stride(0), MEM_DEVICE, img.data_ptr())


class _CudaView:
    """Minimal __cuda_array_interface__ over library-owned device memory."""

    def __init__(self, ptr: int, shape, dtype):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": np.dtype(dtype).str,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _device_view(ptr: int, shape, dtype, device: int):
    import torch
    n = int(np.prod(shape))
    if n == 0 or not ptr:
        return torch.zeros(shape, dtype=getattr(torch, np.dtype(dtype).name), device=f"cuda:{device}")
    return torch.as_tensor(_CudaView(ptr, shape, dtype), device=f"cuda:{device}")


@dataclass
class Job:
    left: object
    right: object
    levels: int = 8
    scale: float = 1.2
    fast_thresh: int = 20
    cell: int = 32
    max_feats: int = 2000


class PreparedBatch:
    """A marshalled jslam_stereo_job array (keeps its images alive)."""

    def __init__(self, jobs):
        self.jobs = tuple(jobs)
        self.n = len(self.jobs)
        self.array = (StereoJob * self.n)()
        for i, j in enumerate(self.jobs):
            self.array[i] = StereoJob(_image(j.left), _image(j.right), j.levels, j.scale, j.fast_thresh, j.cell,
                                      j.max_feats)


class Frontend:
    """One libjslam context (one device, one stream)."""

    def __init__(self, device: int = 0, stream=None, **config):
        cfg = Config()
        lib().jslam_default_config(C.byref(cfg))
        cfg.device = device
        if stream is not None:
            handle = stream if isinstance(stream, int) else stream.cuda_stream
            # handle 0 is the legacy default stream; NULL in the config means
            # "create a stream", so name the legacy stream explicitly
            cfg.cuda_stream = handle if handle else CUDA_STREAM_LEGACY
        for k, v in config.items():
            if k not in {f[0] for f in Config._fields_}:
                raise TypeError(f"unknown config field {k!r}")
            setattr(cfg, k, v)
        self.cfg = cfg
        self.device = device
        h = C.c_void_p()
        _check(lib().jslam_create(C.byref(h), C.byref(cfg)), "jslam_create")
        self._h = h
        self._keep = ()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().jslam_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- enqueue
    def extract(self, left, right, levels=8, scale=1.2, fast_thresh=20, cell=32, max_feats=2000):
        li, ri = _image(left), _image(right)
        self._keep = (left, right)
        _check(lib().jslam_extract(self._h, li, ri, levels, scale, fast_thresh, cell, max_feats), "jslam_extract")

    def prepare_batch(self, jobs) -> "PreparedBatch":
        """Marshal a list of Job once, for repeated extract_batch calls on the
        same buffers (the tensors must stay alive and in place)."""
        return PreparedBatch(jobs)

    def extract_batch(self, jobs):
        pb = jobs if isinstance(jobs, PreparedBatch) else PreparedBatch(jobs)
        self._keep = pb
        _check(lib().jslam_extract_batch(self._h, pb.array, pb.n), "jslam_extract_batch")

    def match(self):
        _check(lib().jslam_match(self._h), "jslam_match")

    def refine_matches(self, half_window: int = 5, search: int = 5, bf: float = 0.0):
        """Enqueue the correlation minimisation of the last match (sub-pixel
        disparity and depth of every accepted match)."""
        _check(lib().jslam_refine_matches(self._h, half_window, search, bf), "jslam_refine_matches")

    def track(self, pair: int, side: int, u, v, level, desc, radius: float, max_dist: int = 100):
        """Enqueue tracking of caller-projected queries (CUDA tensors: u, v
        float32 [n], level uint8 [n], desc int32/uint32 [n, 8]) against the
        keypoints of (pair, side); returns (idx int32 [n], dist uint16-as-int32
        [n]) CUDA tensors, valid after sync()."""
        import torch
        n = int(u.numel())
        for t, dt in ((u, torch.float32), (v, torch.float32), (level, torch.uint8)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous() and t.numel() == n):
                raise ValueError("u, v: float32 and level: uint8 contiguous CUDA tensors of the same length")
        if not (desc.is_cuda and desc.dtype in (torch.int32, torch.uint32) and desc.is_contiguous()
                and desc.numel() == 8 * n):
            raise ValueError("desc: contiguous int32 CUDA tensor of shape [n, 8]")
        idx = torch.empty(n, dtype=torch.int32, device=u.device)
        dist = torch.empty(n, dtype=torch.int16, device=u.device)
        _check(lib().jslam_track(self._h, pair, side, u.data_ptr(), v.data_ptr(), level.data_ptr(), desc.data_ptr(),
                                 n, radius, max_dist, idx.data_ptr(), dist.data_ptr()), "jslam_track")
        self._keep_track = (u, v, level, desc, idx, dist)
        return idx, dist

    def fc_ablation(self, n_max: int = 8):
        """Enqueue the paper-style feature culling (CRF-matrix + MLPT/TEWA) of
        the last extraction (an ablation baseline)."""
        _check(lib().jslam_fc_ablation(self._h, n_max), "jslam_fc_ablation")

    def fc_ablation_keys(self, pair: int, side: int, level: int):
        """(ablation keys, fused-kernel keys) of one level as [cells_y, cells_x] CUDA tensors."""
        a, f = C.c_void_p(), C.c_void_p()
        cx, cy = C.c_int32(), C.c_int32()
        _check(lib().jslam_fc_ablation_view(self._h, pair, side, level, C.byref(a), C.byref(f), C.byref(cx),
                                            C.byref(cy)), "jslam_fc_ablation_view")
        shape = (cy.value, cx.value)
        return _device_view(a.value, shape, np.uint32, self.device), _device_view(f.value, shape, np.uint32, self.device)

    def crf(self, pair: int, side: int, level: int = 0):
        """CRF-matrix of one level from the last fc_ablation(): [H, W] uint16 CUDA view
        (corner response, 0 for non-corners)."""
        p = C.c_void_p()
        w, h = C.c_int32(), C.c_int32()
        _check(lib().jslam_crf_view(self._h, pair, side, level, C.byref(p), C.byref(w), C.byref(h)), "jslam_crf_view")
        return _device_view(p.value, (h.value, w.value), np.uint16, self.device)

    def selftest_wait(self):
        """Enqueue the failure-detection self-test: the next sync() raises with
        JSLAM_ERR_TIMEOUT after about a second."""
        _check(lib().jslam_selftest_wait(self._h), "jslam_selftest_wait")

    def fc_ablation_times(self):
        a, b = C.c_float(), C.c_float()
        _check(lib().jslam_fc_ablation_times(self._h, C.byref(a), C.byref(b)), "jslam_fc_ablation_times")
        return {"crf_ms": a.value, "fc_ms": b.value}

    def refined(self, pair: int = 0) -> dict:
        r = Refined()
        _check(lib().jslam_get_refined(self._h, pair, C.byref(r)), "jslam_get_refined")
        n = max(r.count, 0)
        out = {"count": r.count}
        for name, dt in REFINED_FIELDS:
            out[name] = _device_view(getattr(r, name), (n,), dt, self.device)
        return out

    def result_refined_view(self, pair: int, block) -> dict:
        """Host arrays (copies) of the refinement inside a downloaded result block."""
        base = block.ctypes.data if isinstance(block, np.ndarray) else block.data_ptr()
        r = Refined()
        _check(lib().jslam_result_refined_view(self._h, pair, base, C.byref(r)), "jslam_result_refined_view")
        n = max(r.count, 0)
        out = {"count": r.count}
        for name, dt in REFINED_FIELDS:
            buf = (C.c_char * (n * np.dtype(dt).itemsize)).from_address(getattr(r, name)) if n else b""
            out[name] = np.frombuffer(buf, dtype=dt).copy() if n else np.zeros(0, dt)
        return out

    def set_skip_model(self, blob, thresh: float = 0.0):
        """Enable the learned cell-skip proposal (blob: bytes of a model) or
        return to the exact path (blob None)."""
        if blob is None:
            _check(lib().jslam_set_skip_model(self._h, None, 0, 0.0), "jslam_set_skip_model")
            return
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _check(lib().jslam_set_skip_model(self._h, buf, len(blob), thresh), "jslam_set_skip_model")

    def skip_view(self, pair: int = 0, side: int = 0) -> dict:
        v = SkipView()
        _check(lib().jslam_get_skip_view(self._h, pair, side, C.byref(v)), "jslam_get_skip_view")
        return {"logits": _device_view(v.logits, (v.h8, v.w8), np.float32, self.device),
                "skip": _device_view(v.skip, (v.cells_y, v.cells_x), np.uint8, self.device)}

    def set_tuning(self, tile_w_px: int, tile_h_px: int, nms_kernel: int = 0, detect_ctas_per_sm: int = 0,
                   tile_order: int = 0):
        t = Tuning(tile_w_px, tile_h_px, nms_kernel, detect_ctas_per_sm, tile_order)
        _check(lib().jslam_set_tuning(self._h, C.byref(t)), "jslam_set_tuning")

    def autotune(self, jobs, cache: str | None = None) -> tuple:
        """Tune the launch shapes on `jobs`; returns (tile_w_px, tile_h_px,
        nms_kernel, detect_ctas_per_sm, tile_order).  With `cache` (a JSON file path) a
        stored pick for this GPU and batch is applied without tuning, and a new
        pick is stored; `last_tune_hit` tells which happened."""
        pb = jobs if isinstance(jobs, PreparedBatch) else PreparedBatch(jobs)
        self._keep = pb
        t = Tuning()
        if cache is None:
            _check(lib().jslam_autotune(self._h, pb.array, pb.n, C.byref(t)), "jslam_autotune")
            self.last_tune_hit = None
        else:
            hit = C.c_int32(0)
            _check(lib().jslam_autotune_cached(self._h, pb.array, pb.n, os.fsencode(cache), C.byref(t),
                                               C.byref(hit)), "jslam_autotune_cached")
            self.last_tune_hit = bool(hit.value)
        return t.as_tuple()

    def graph_capture(self, jobs):
        pb = jobs if isinstance(jobs, PreparedBatch) else PreparedBatch(jobs)
        self._graph_keep = pb
        _check(lib().jslam_graph_capture(self._h, pb.array, pb.n), "jslam_graph_capture")

    def graph_launch(self, jobs=None):
        """Replay the captured graph; with `jobs` (the captured batch shape,
        device images), on those frames instead of the captured ones."""
        if jobs is None:
            _check(lib().jslam_graph_launch(self._h), "jslam_graph_launch")
            return
        pb = jobs if isinstance(jobs, PreparedBatch) else PreparedBatch(jobs)
        self._keep = pb
        _check(lib().jslam_graph_launch_jobs(self._h, pb.array, pb.n), "jslam_graph_launch_jobs")

    def sync(self):
        _check(lib().jslam_sync(self._h), "jslam_sync")

    def enable_stage_timing(self, on: bool = True):
        _check(lib().jslam_enable_stage_timing(self._h, int(on)), "jslam_enable_stage_timing")

    def stage_times(self) -> dict:
        """Milliseconds per stage of the last extraction (+ match), after sync."""
        ms = np.zeros(len(STAGES), np.float32)
        _check(lib().jslam_stage_times(self._h, ms.ctypes.data), "jslam_stage_times")
        return dict(zip(STAGES, ms.tolist()))

    # -- device views
    def keypoints(self, pair: int = 0, side: int = 0) -> dict:
        kp = Keypoints()
        _check(lib().jslam_get_keypoints(self._h, pair, side, C.byref(kp)), "jslam_get_keypoints")
        n = max(kp.count, 0)
        out = {"count": kp.count}
        for name, dt, words in KP_FIELDS:
            shape = (n, words) if words > 1 else (n,)
            out[name] = _device_view(getattr(kp, name), shape, dt, self.device)
        return out

    def matches(self, pair: int = 0) -> dict:
        m = Matches()
        _check(lib().jslam_get_matches(self._h, pair, C.byref(m)), "jslam_get_matches")
        n = max(m.count, 0)
        out = {"count": m.count}
        for name, dt in MATCH_FIELDS:
            out[name] = _device_view(getattr(m, name), (n,), dt, self.device)
        return out

    def level(self, pair: int, side: int, level: int) -> dict:
        v = LevelView()
        _check(lib().jslam_get_level(self._h, pair, side, level, C.byref(v)), "jslam_get_level")
        raw = _device_view(v.raw, (v.height, v.raw_pitch), np.uint8, self.device)[:, : v.width]
        blur = _device_view(v.blurred, (v.height, v.blurred_pitch), np.uint8, self.device)[:, : v.width]
        return {"raw": raw, "blurred": blur}

    # -- host results
    def result_bytes(self, pair: int = 0) -> int:
        n = C.c_size_t()
        _check(lib().jslam_result_bytes(self._h, pair, C.byref(n)), "jslam_result_bytes")
        return n.value

    def download(self, pair: int, dst) -> None:
        """Enqueue the copy of pair `pair`'s result block into `dst` (a pinned
        CPU tensor or a numpy array of at least result_bytes bytes)."""
        if isinstance(dst, np.ndarray):
            ptr, size = dst.ctypes.data, dst.nbytes
        else:
            ptr, size = dst.data_ptr(), dst.numel() * dst.element_size()
        _check(lib().jslam_download(self._h, pair, ptr, size), "jslam_download")

    def result_range(self, first: int, count: int):
        """(total bytes, per-pair offsets) of the result blocks of pairs
        [first, first + count), which lie back to back."""
        n = C.c_size_t()
        offs = (C.c_size_t * count)()
        _check(lib().jslam_result_range(self._h, first, count, C.byref(n), offs), "jslam_result_range")
        return n.value, list(offs)

    def download_range(self, first: int, count: int, dst) -> None:
        """Enqueue one copy of the result blocks of pairs [first, first +
        count) into `dst` (pinned CPU tensor or numpy array)."""
        if isinstance(dst, np.ndarray):
            ptr, size = dst.ctypes.data, dst.nbytes
        else:
            ptr, size = dst.data_ptr(), dst.numel() * dst.element_size()
        _check(lib().jslam_download_range(self._h, first, count, ptr, size), "jslam_download_range")

    def result_view(self, pair: int, block, side: int) -> dict:
        """Host arrays (copies) of one side of a downloaded result block."""
        if isinstance(block, np.ndarray):
            base = block.ctypes.data
        else:
            base = block.data_ptr()
        kp = Keypoints(); m = Matches()
        _check(lib().jslam_result_view(self._h, pair, base, side, C.byref(kp), C.byref(m)), "jslam_result_view")
        n = max(kp.count, 0)
        out = {"count": kp.count}
        for name, dt, words in KP_FIELDS:
            buf = (C.c_char * (n * words * np.dtype(dt).itemsize)).from_address(getattr(kp, name)) if n else b""
            a = np.frombuffer(buf, dtype=dt).copy() if n else np.zeros(0, dt)
            out[name] = a.reshape(n, words) if words > 1 else a
        if side == 0 and m.count >= 0:
            for name, dt in MATCH_FIELDS:
                buf = (C.c_char * (n * np.dtype(dt).itemsize)).from_address(getattr(m, name)) if n else b""
                out["match_" + name] = np.frombuffer(buf, dtype=dt).copy() if n else np.zeros(0, dt)
        return out


def to_numpy(d: dict) -> dict:
    """Copy a dict of device views to host numpy arrays."""
    out = {}
    for k, v in d.items():
        out[k] = v.cpu().numpy() if hasattr(v, "cpu") else v
    return out
