"""ctypes wrapper around the plain-C CPU oracle (``jslam_oracle.c``).

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this module.  The
product path (``paper_2410_04090_gb300``) never imports it.

The oracle is a plain single-threaded C implementation of the stereo frontend
hot path of Jetson-SLAM (arXiv 2410.04090): pyramid (Sec. III), FAST with
Bounded Rectification (Sec. II-A, Eq. 1-3), Feature Culling (Sec. II-C-1),
Pyramidal Feature Aggregation (Sec. II-C-2), ORB orientation and steered
BRIEF (Sec. III) and stereo row matching (Sec. III, middle-end).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jslam_oracle.c")
_LIB = os.path.join(_HERE, "libjslam_oracle.so")

NBINS = 30
NPAIRS = 256


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so that double
    roundings are the IEEE ones the definitions state)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("levels", C.c_int32), ("scale", C.c_float), ("fast_thresh", C.c_int32),
        ("fast_thresh_lo", C.c_int32), ("p_min", C.c_int32), ("p_max", C.c_int32),
        ("cell", C.c_int32), ("k_per_cell", C.c_int32), ("nms_q", C.c_int32),
        ("border", C.c_int32), ("max_feats", C.c_int32), ("pfa_rule", C.c_int32),
        ("max_disp", C.c_int32), ("row_band_px", C.c_int32), ("match_max_dist", C.c_int32),
        ("response_mode", C.c_int32), ("pyramid_mode", C.c_int32),
    ]


class _Keypoints(C.Structure):
    _fields_ = [
        ("capacity", C.c_int32), ("count", C.c_int32),
        ("x", C.c_void_p), ("y", C.c_void_p), ("X", C.c_void_p), ("Y", C.c_void_p),
        ("level", C.c_void_p), ("response", C.c_void_p), ("k_levels", C.c_void_p),
        ("k_resp", C.c_void_p), ("angle", C.c_void_p), ("angle_bin", C.c_void_p),
        ("desc", C.c_void_p), ("m10", C.c_void_p), ("m01", C.c_void_p),
    ]


@dataclass
class FrontendParams:
    """Parameters of one extraction (defaults: the paper's values where it
    gives them -- eps = 20, P_min = 9, P_max = 13, q = 3, zeta = 1.2, 32x32
    cells -- and the stated readings elsewhere)."""
    levels: int = 8
    scale: float = 1.2
    fast_thresh: int = 20
    fast_thresh_lo: int = 0
    p_min: int = 9
    p_max: int = 13
    cell: int = 32
    k_per_cell: int = 1
    nms_q: int = 3
    border: int = 19
    max_feats: int = 2000
    pfa_rule: int = 0
    max_disp: int = 128
    row_band_px: int = 2
    match_max_dist: int = 100
    response_mode: int = 0   # 1: arc response (reading O3's alternative)
    pyramid_mode: int = 0    # 1: cascaded pyramid (reading O1's alternative)

    def to_c(self) -> Params:
        return Params(**asdict(self))


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        i8p = np.ctypeslib.ndpointer(np.int8, flags="C")
        u16p = np.ctypeslib.ndpointer(np.uint16, flags="C")
        i16p = np.ctypeslib.ndpointer(np.int16, flags="C")
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
        i32 = C.c_int32
        L.or_level_scale.restype = C.c_double
        L.or_level_scale.argtypes = [C.c_float, i32]
        L.or_level_geometry.argtypes = [i32, i32, i32, C.c_float, i32, i32p, i32p, i32p]
        L.or_pyramid_level.argtypes = [u8p, i32, i32, i32, C.c_float, i32, u8p, i32, i32, i32]
        L.or_blur_weights.argtypes = [i32p]
        L.or_blur.argtypes = [u8p, i32, i32, i32, u8p, i32]
        L.or_ring.argtypes = [i32p, i32p]
        L.or_longest_run.restype = i32
        L.or_longest_run.argtypes = [C.c_uint32]
        L.or_corner_from_masks.restype = i32
        L.or_corner_from_masks.argtypes = [C.c_uint32, C.c_uint32, i32, i32]
        L.or_fast.argtypes = [u8p, i32, i32, i32, i32, i32, i32, i32, u8p, u16p]
        L.or_fast_arc.argtypes = [u8p, i32, i32, i32, i32, i32, i32, i32, u8p, u16p]
        L.or_arc_positions.restype = C.c_uint32
        L.or_arc_positions.argtypes = [C.c_uint32]
        L.or_arc_response.restype = i32
        L.or_arc_response.argtypes = [i32p, C.c_uint32, C.c_uint32, i32, i32, i32]
        L.or_cull_level.restype = i32
        L.or_cull_level.argtypes = [u8p, C.c_void_p, u16p, i32, i32, i32, i32, i32p, i32p, i32p, i32]
        L.or_project.restype = i32
        L.or_project.argtypes = [i32, i32, C.c_float, i32]
        L.or_pfa_core.argtypes = [i32, i32p, i32p, i32p, i32p, i32, i32, i32, i32, i32, i32p, i32p, u8p]
        L.or_bin_tables.argtypes = [f64p, f64p]
        L.or_orient.argtypes = [u8p, i32, i32, i32, C.POINTER(i32), C.POINTER(i32),
                                C.POINTER(C.c_double), C.POINTER(i32)]
        L.or_splitmix64_next.restype = C.c_uint64
        L.or_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
        L.or_std_normal.restype = C.c_double
        L.or_std_normal.argtypes = [C.POINTER(C.c_uint64)]
        L.or_pattern_base.argtypes = [i8p]
        L.or_pattern_rotated.argtypes = [i8p]
        L.or_describe.argtypes = [u8p, i32, i32, i32, i8p, u32p]
        L.or_check_params.restype = i32
        L.or_check_params.argtypes = [i32, i32, C.POINTER(Params)]
        L.or_extract_image.restype = i32
        L.or_extract_image.argtypes = [u8p, i32, i32, i32, C.POINTER(Params), C.POINTER(_Keypoints)]
        L.or_match_band.restype = i32
        L.or_match_band.argtypes = [i32, C.c_float, i32]
        L.or_match.argtypes = [C.POINTER(_Keypoints), C.POINTER(_Keypoints), C.POINTER(Params),
                               i32p, i16p, u16p]
        f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
        L.or_track.argtypes = [C.POINTER(_Keypoints), C.c_float, f32p, f32p, u8p, u32p, i32, C.c_float, i32,
                               i32p, u16p]
        L.or_subpixel.argtypes = [u8p, u8p, i32, i32, i32, C.POINTER(_Keypoints), C.POINTER(_Keypoints), i32p,
                                  C.POINTER(Params), i32, i32, C.c_double, f32p, f32p, u32p]
        _lib = L
    return _lib


# ---------------------------------------------------------------- stages

def level_scale(scale: float, n: int) -> float:
    return lib().or_level_scale(scale, n)


def level_geometry(W0: int, H0: int, levels: int, scale: float, cell: int):
    W = np.zeros(levels, np.int32); H = np.zeros(levels, np.int32); c = np.zeros(levels, np.int32)
    lib().or_level_geometry(W0, H0, levels, scale, cell, W, H, c)
    return W, H, c


def pyramid_level(L0: np.ndarray, scale: float, n: int) -> np.ndarray:
    L0 = np.ascontiguousarray(L0, np.uint8)
    H0, W0 = L0.shape
    W, H, _ = level_geometry(W0, H0, n + 1, scale, 32)
    out = np.zeros((int(H[n]), int(W[n])), np.uint8)
    lib().or_pyramid_level(L0, W0, H0, W0, scale, n, out, int(W[n]), int(H[n]), int(W[n]))
    return out


def pyramid_level_sized(L0: np.ndarray, scale: float, n: int, Wn: int, Hn: int) -> np.ndarray:
    L0 = np.ascontiguousarray(L0, np.uint8)
    H0, W0 = L0.shape
    out = np.zeros((Hn, Wn), np.uint8)
    lib().or_pyramid_level(L0, W0, H0, W0, scale, n, out, Wn, Hn, Wn)
    return out


def blur_weights() -> np.ndarray:
    w = np.zeros(7, np.int32)
    lib().or_blur_weights(w)
    return w


def blur(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    out = np.zeros_like(img)
    lib().or_blur(img, W, H, W, out, W)
    return out


def ring():
    dx = np.zeros(16, np.int32); dy = np.zeros(16, np.int32)
    lib().or_ring(dx, dy)
    return dx, dy


def longest_run(mask: int) -> int:
    return lib().or_longest_run(mask)


def corner_from_masks(Bb: int, Bd: int, p_min: int, p_max: int) -> bool:
    return bool(lib().or_corner_from_masks(Bb, Bd, p_min, p_max))


def fast(img: np.ndarray, eps: int, p_min: int = 9, p_max: int = 13, border: int = 3):
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    corner = np.zeros((H, W), np.uint8); resp = np.zeros((H, W), np.uint16)
    lib().or_fast(img, W, H, W, eps, p_min, p_max, border, corner, resp)
    return corner, resp


def fast_arc(img: np.ndarray, eps: int, p_min: int = 9, p_max: int = 13, border: int = 3):
    """CRF-matrix with the arc response (the alternative reading of the
    response): corners as fast(), response = sum of (|d| - eps) over the
    qualifying arc."""
    img = np.ascontiguousarray(img, np.uint8)
    H, W = img.shape
    corner = np.zeros((H, W), np.uint8); resp = np.zeros((H, W), np.uint16)
    lib().or_fast_arc(img, W, H, W, eps, p_min, p_max, border, corner, resp)
    return corner, resp


def arc_positions(mask: int) -> int:
    return lib().or_arc_positions(mask)


def arc_response(d, Bb: int, Bd: int, eps: int, p_min: int = 9, p_max: int = 13) -> int:
    return lib().or_arc_response(np.ascontiguousarray(d, np.int32), Bb, Bd, eps, p_min, p_max)


def cull_level(corner_hi, corner_lo, resp, c: int, k: int):
    corner_hi = np.ascontiguousarray(corner_hi, np.uint8)
    resp = np.ascontiguousarray(resp, np.uint16)
    H, W = corner_hi.shape
    cap = ((W + c - 1) // c) * ((H + c - 1) // c) * k
    xs = np.zeros(cap + 1, np.int32); ys = np.zeros(cap + 1, np.int32); rs = np.zeros(cap + 1, np.int32)
    lo_ptr = None
    if corner_lo is not None:
        corner_lo = np.ascontiguousarray(corner_lo, np.uint8)
        lo_ptr = corner_lo.ctypes.data
    m = lib().or_cull_level(corner_hi, lo_ptr, resp, W, H, c, k, xs, ys, rs, cap)
    return xs[:m].copy(), ys[:m].copy(), rs[:m].copy()


def project(x: int, n: int, scale: float, W0: int) -> int:
    return lib().or_project(x, n, scale, W0)


def pfa_core(lev, X, Y, r, W0: int, H0: int, Ns: int, q: int = 3, rule: int = 0):
    lev = np.ascontiguousarray(lev, np.int32); X = np.ascontiguousarray(X, np.int32)
    Y = np.ascontiguousarray(Y, np.int32); r = np.ascontiguousarray(r, np.int32)
    n = len(lev)
    Kl = np.zeros(n + 1, np.int32); Kr = np.zeros(n + 1, np.int32); alive = np.zeros(n + 1, np.uint8)
    lib().or_pfa_core(n, lev, X, Y, r, W0, H0, Ns, q, rule, Kl, Kr, alive)
    return Kl[:n], Kr[:n], alive[:n].astype(bool)


def bin_tables():
    cb = np.zeros(NBINS, np.float64); sb = np.zeros(NBINS, np.float64)
    lib().or_bin_tables(cb, sb)
    return cb, sb


def orient(img: np.ndarray, x: int, y: int):
    img = np.ascontiguousarray(img, np.uint8)
    m10 = C.c_int32(); m01 = C.c_int32(); th = C.c_double(); b = C.c_int32()
    lib().or_orient(img, img.shape[1], x, y, C.byref(m10), C.byref(m01), C.byref(th), C.byref(b))
    return m10.value, m01.value, th.value, b.value


def splitmix64(seed: int, n: int):
    st = C.c_uint64(seed)
    return [lib().or_splitmix64_next(C.byref(st)) for _ in range(n)]


def std_normals(seed: int, n: int) -> np.ndarray:
    st = C.c_uint64(seed)
    return np.array([lib().or_std_normal(C.byref(st)) for _ in range(n)])


def pattern_base() -> np.ndarray:
    out = np.zeros(NPAIRS * 4, np.int8)
    lib().or_pattern_base(out)
    return out.reshape(NPAIRS, 4)


def pattern_rotated() -> np.ndarray:
    out = np.zeros(NBINS * NPAIRS * 4, np.int8)
    lib().or_pattern_rotated(out)
    return out.reshape(NBINS, NPAIRS, 4)


def describe(blurred: np.ndarray, x: int, y: int, rot_bin: np.ndarray) -> np.ndarray:
    blurred = np.ascontiguousarray(blurred, np.uint8)
    d = np.zeros(8, np.uint32)
    lib().or_describe(blurred, blurred.shape[1], x, y, np.ascontiguousarray(rot_bin, np.int8).reshape(-1), d)
    return d


def match_band(n: int, scale: float, row_band_px: int) -> int:
    return lib().or_match_band(n, scale, row_band_px)


def check_params(W0: int, H0: int, p: FrontendParams) -> bool:
    cp = p.to_c()
    return lib().or_check_params(W0, H0, C.byref(cp)) == 0


# ---------------------------------------------------------------- pipeline

KP_FIELDS = (("x", np.uint16), ("y", np.uint16), ("X", np.uint16), ("Y", np.uint16),
             ("level", np.uint8), ("response", np.uint16), ("k_levels", np.uint8),
             ("k_resp", np.uint32), ("angle", np.float32), ("angle_bin", np.uint8))


def _kp_struct(arrs: dict, cap: int, count: int = 0) -> _Keypoints:
    s = _Keypoints()
    s.capacity = cap
    s.count = count
    for name, _ in KP_FIELDS:
        setattr(s, name, arrs[name].ctypes.data)
    s.desc = arrs["desc"].ctypes.data
    s.m10 = arrs["m10"].ctypes.data
    s.m01 = arrs["m01"].ctypes.data
    return s


def extract_image(img: np.ndarray, p: FrontendParams) -> dict:
    """Keypoints of one image in canonical order (level, y, x)."""
    img = np.ascontiguousarray(img, np.uint8)
    H0, W0 = img.shape
    cap = p.max_feats
    arrs = {name: np.zeros(cap + 1, dt) for name, dt in KP_FIELDS}
    arrs["desc"] = np.zeros((cap + 1) * 8, np.uint32)
    arrs["m10"] = np.zeros(cap + 1, np.int32)
    arrs["m01"] = np.zeros(cap + 1, np.int32)
    s = _kp_struct(arrs, cap)
    cp = p.to_c()
    rc = lib().or_extract_image(img, W0, H0, W0, C.byref(cp), C.byref(s))
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    n = s.count
    out = {name: arrs[name][:n].copy() for name, _ in KP_FIELDS}
    out["desc"] = arrs["desc"][: n * 8].reshape(n, 8).copy()
    out["m10"] = arrs["m10"][:n].copy()
    out["m01"] = arrs["m01"][:n].copy()
    out["count"] = n
    return out


def _as_struct(kp: dict):
    n = kp["count"]
    arrs = {name: np.ascontiguousarray(kp[name], dt) for name, dt in KP_FIELDS}
    arrs["desc"] = np.ascontiguousarray(kp["desc"], np.uint32).reshape(-1)
    arrs["m10"] = np.zeros(max(n, 1), np.int32)
    arrs["m01"] = np.zeros(max(n, 1), np.int32)
    for name, dt in KP_FIELDS:
        if arrs[name].size == 0:
            arrs[name] = np.zeros(1, dt)
    if arrs["desc"].size == 0:
        arrs["desc"] = np.zeros(8, np.uint32)
    return _kp_struct(arrs, n, n), arrs


def match(kl: dict, kr: dict, p: FrontendParams):
    """Stereo row matching of left keypoints against right keypoints."""
    sl, keep_l = _as_struct(kl)
    sr, keep_r = _as_struct(kr)
    n = kl["count"]
    idx = np.zeros(n + 1, np.int32); disp = np.zeros(n + 1, np.int16); dist = np.zeros(n + 1, np.uint16)
    cp = p.to_c()
    lib().or_match(C.byref(sl), C.byref(sr), C.byref(cp), idx, disp, dist)
    del keep_l, keep_r
    return idx[:n].copy(), disp[:n].copy(), dist[:n].copy()


def subpixel(left: np.ndarray, right: np.ndarray, kl: dict, kr: dict, right_idx: np.ndarray,
             p: FrontendParams, half_window: int = 5, search: int = 5, bf: float = 0.0):
    """Correlation minimisation of the accepted matches (Sec. III middle-end):
    per left keypoint the sub-pixel disparity (-1 rejected), depth (0
    rejected) and best SAD (0xFFFFFFFF when none was computed)."""
    left = np.ascontiguousarray(left, np.uint8)
    right = np.ascontiguousarray(right, np.uint8)
    assert left.shape == right.shape and 1 <= search <= 7 and half_window >= 1
    sl, keep_l = _as_struct(kl)
    sr, keep_r = _as_struct(kr)
    n = kl["count"]
    ridx = np.ascontiguousarray(np.concatenate([np.asarray(right_idx, np.int32)[:n], [-1]]), np.int32)
    disp = np.zeros(n + 1, np.float32); depth = np.zeros(n + 1, np.float32); sad = np.zeros(n + 1, np.uint32)
    cp = p.to_c()
    H, W = left.shape
    lib().or_subpixel(left, right, W, H, W, C.byref(sl), C.byref(sr), ridx, C.byref(cp), half_window, search,
                      float(bf), disp, depth, sad)
    del keep_l, keep_r
    return {"disparity": disp[:n].copy(), "depth": depth[:n].copy(), "sad": sad[:n].copy()}


def track(kf: dict, scale: float, u, v, level, desc, radius: float, max_dist: int = 100):
    """Feature tracking by projection (Sec. III middle-end): per query the
    index of the matched keypoint of `kf` (-1 none/rejected) and the best
    Hamming distance (0xFFFF: no candidate)."""
    sk, keep = _as_struct(kf)
    n = len(u)
    u = np.ascontiguousarray(np.concatenate([np.asarray(u, np.float32), [0]]), np.float32)
    v = np.ascontiguousarray(np.concatenate([np.asarray(v, np.float32), [0]]), np.float32)
    lv = np.ascontiguousarray(np.concatenate([np.asarray(level, np.uint8), [0]]), np.uint8)
    ds = np.ascontiguousarray(np.concatenate([np.asarray(desc, np.uint32).reshape(-1), np.zeros(8, np.uint32)]),
                              np.uint32)
    idx = np.zeros(n + 1, np.int32); dist = np.zeros(n + 1, np.uint16)
    lib().or_track(C.byref(sk), scale, u, v, lv, ds, n, radius, max_dist, idx, dist)
    del keep
    return idx[:n].copy(), dist[:n].copy()


def extract_pair(left: np.ndarray, right: np.ndarray, p: FrontendParams):
    kl = extract_image(left, p)
    kr = extract_image(right, p)
    m = match(kl, kr, p)
    return kl, kr, m
