"""FP64 CPU oracle for the DDHF per-pixel frequency-analysis path.

Test infrastructure: only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library and
its Python binding never import it, and the two share no code.

The arithmetic lives in ``ddhf_oracle.c`` (plain single-threaded C, FP64,
compiled with FMA contraction off); this module compiles it with the system C
compiler and wraps each function with numpy arguments. Every function cites
the passage of arXiv 2603.08386 it restates:

  bin_events      Sec. 3.5 "Event processing" (sort by pixel, n_min)
  ndft            Sec. 3.3 Eq. 6 and P_k = |F_k|^2
  ndft_f32        the same in FP32 (the benchmark's FP32 CPU baseline)
  ndft_at         Eq. 6 at arbitrary frequencies plus dF/df (soft comb)
  log_sf          Sec. 3.4 Eq. 7
  comb, comb_f32  Sec. 3.4 Eq. 8-11
  ccl8            Sec. 3.5 "Segmentation mask processing"
  boxes           Sec. 3.5 and Eq. 12
  box_frequencies Eq. 11 (dominant frequency of rotor pixels) per detection
  classify        Sec. 3.5 per-pixel pipeline (Eq. 6-11)
  softcomb        soft comb score and its gradients (differentiation pattern)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddhf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libddhf_oracle.so")
_lib = None
_lock = threading.Lock()

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libddhf_oracle.so`` (no-op if fresh)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cc = os.environ.get("CC", "cc")
    subprocess.check_call([cc, *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i16p = np.ctypeslib.ndpointer(np.int16, flags="C")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
            i8p = np.ctypeslib.ndpointer(np.int8, flags="C")
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            f32p = np.ctypeslib.ndpointer(np.float32, flags="C")
            c_i32, c_i64, c_f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            vp = ctypes.c_void_p

            lib.oracle_bin_events.restype = c_i64
            lib.oracle_bin_events.argtypes = [c_i32, c_i32, c_i64, i16p, i16p, i64p, i8p,
                                              c_i64, c_i64, c_i32, i64p, i64p, i64p, i8p,
                                              ctypes.POINTER(c_i64)]
            lib.oracle_ndft.restype = None
            lib.oracle_ndft.argtypes = [c_i64, i64p, i8p, c_i64, c_i64, c_i64, c_i32, f64p, vp]
            lib.oracle_ndft_f32.restype = None
            lib.oracle_ndft_f32.argtypes = [c_i64, i64p, i8p, c_i64, c_i64, c_i64, c_i32, f32p]
            lib.oracle_ndft_at.restype = None
            lib.oracle_ndft_at.argtypes = [c_i64, i64p, i8p, c_f64, c_i32, f64p, f64p, vp]
            lib.oracle_log_sf.restype = c_f64
            lib.oracle_log_sf.argtypes = [c_i32, f64p]
            lib.oracle_comb.restype = c_f64
            lib.oracle_comb.argtypes = [c_i32, f64p, c_i32, c_i32, c_i32,
                                        ctypes.POINTER(c_i32)]
            lib.oracle_comb_f32.restype = ctypes.c_float
            lib.oracle_comb_f32.argtypes = [c_i32, f32p, c_i32, c_i32, c_i32,
                                            ctypes.POINTER(c_i32)]
            lib.oracle_ccl8.restype = c_i32
            lib.oracle_ccl8.argtypes = [c_i32, c_i32, u8p, i32p]
            lib.oracle_boxes.restype = c_i32
            lib.oracle_boxes.argtypes = [c_i32, c_i32, i32p, c_i32, c_f64, c_i32, i32p]
            lib.oracle_softcomb.restype = c_f64
            lib.oracle_softcomb.argtypes = [c_i64, i64p, i8p, c_f64, c_f64, c_i32, f64p, f64p,
                                            c_f64, c_i32, c_f64, vp, vp, vp, vp]
            lib.oracle_classify.restype = c_i64
            lib.oracle_classify.argtypes = [c_i32, c_i32, i64p, i64p, i8p, c_i64, c_i64, c_i64,
                                            c_i32, c_f64, c_f64, c_i32, c_i32, c_i32, c_i32,
                                            c_i64, vp, vp, vp, vp, vp, vp]
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# Table 2 (final column): tau_sf, tau_comb, M, Delta k (= d), h_min, n_min, A_min, alpha.
TABLE2 = dict(tau_sf=0.89, tau_comb=1.5, M=4, d=3, h_min=4, n_min=6, A_min=147, alpha=19.05)


def bin_events(W, H, x, y, t, p, t0, window_us, polarity_01=False):
    """Window, validate and stably bin events by pixel key y*W+x (Sec. 3.5).

    Returns dict(counts[W*H], offsets[W*H+1], tau[n_valid], pol[n_valid],
    n_valid, n_dropped), all int64 except pol (int8, +-1)."""
    lib = _load()
    x, y = _c(x, np.int16), _c(y, np.int16)
    t, p = _c(t, np.int64), _c(p, np.int8)
    n = int(x.shape[0])
    npx = int(W) * int(H)
    counts = np.zeros(npx, np.int64)
    offsets = np.zeros(npx + 1, np.int64)
    tau = np.zeros(max(n, 1), np.int64)
    pol = np.zeros(max(n, 1), np.int8)
    nd = ctypes.c_int64(0)
    nv = lib.oracle_bin_events(int(W), int(H), n, x, y, t, p, int(t0), int(window_us),
                               int(bool(polarity_01)), counts, offsets, tau, pol,
                               ctypes.byref(nd))
    return dict(counts=counts, offsets=offsets, tau=tau[:nv].copy(), pol=pol[:nv].copy(),
                n_valid=int(nv), n_dropped=int(nd.value))


def ndft(tau, pol, a0, da, denom, n_bins, return_f=False):
    """Eq. 6 power spectrum P_j = |sum_k p_k exp(-2 pi i a_j tau_k / denom)|^2 (FP64)."""
    lib = _load()
    tau, pol = _c(tau, np.int64), _c(pol, np.int8)
    P = np.zeros(int(n_bins), np.float64)
    F = np.zeros(2 * int(n_bins), np.float64) if return_f else None
    lib.oracle_ndft(int(tau.shape[0]), tau, pol, int(a0), int(da), int(denom), int(n_bins),
                    P, _ptr(F))
    if return_f:
        return P, F[0::2] + 1j * F[1::2]
    return P


def ndft_f32(tau, pol, a0, da, denom, n_bins):
    """The same power spectrum in single precision (the FP32 CPU baseline of
    the benchmark; parity is always checked against the FP64 ndft)."""
    lib = _load()
    tau, pol = _c(tau, np.int64), _c(pol, np.int8)
    P = np.zeros(int(n_bins), np.float32)
    lib.oracle_ndft_f32(int(tau.shape[0]), tau, pol, int(a0), int(da), int(denom), int(n_bins), P)
    return P


def ndft_at(tau, pol, f_hz, tau_c=0.0):
    """F(f) and dF/df at arbitrary frequencies (Hz), tau in microseconds,
    referenced to tau_c. Returns (F, D) complex128 arrays."""
    lib = _load()
    tau, pol = _c(tau, np.int64), _c(pol, np.int8)
    f = _c(np.atleast_1d(f_hz), np.float64)
    F = np.zeros(2 * f.shape[0], np.float64)
    D = np.zeros(2 * f.shape[0], np.float64)
    lib.oracle_ndft_at(int(tau.shape[0]), tau, pol, float(tau_c), int(f.shape[0]), f, F,
                       _ptr(D))
    return F[0::2] + 1j * F[1::2], D[0::2] + 1j * D[1::2]


def log_sf(P):
    """ln of the spectral flatness of Eq. 7."""
    return float(_load().oracle_log_sf(int(len(P)), _c(P, np.float64)))


def comb(P, M=4, d=3, h_min=4):
    """Eq. 8-11 in FP64: returns (best SNR, dominant bin or -1)."""
    w = ctypes.c_int32(-1)
    s = _load().oracle_comb(int(len(P)), _c(P, np.float64), int(M), int(d), int(h_min),
                            ctypes.byref(w))
    return float(s), int(w.value)


def comb_f32(P, M=4, d=3, h_min=4):
    """Eq. 8-11 in FP32 with the fixed operation order (see the C source)."""
    w = ctypes.c_int32(-1)
    s = _load().oracle_comb_f32(int(len(P)), _c(P, np.float32), int(M), int(d), int(h_min),
                                ctypes.byref(w))
    return np.float32(s), int(w.value)


def ccl8(mask, W, H):
    """8-connected labels, label = smallest linear index of the component, -1 else."""
    mask = _c(mask, np.uint8).reshape(-1)
    labels = np.zeros(int(W) * int(H), np.int32)
    n = _load().oracle_ccl8(int(W), int(H), mask, labels)
    return labels, int(n)


def boxes(labels, W, H, A_min=147, alpha=19.05, cap=4096):
    """Boxes, area filter and Eq. 12 merge; returns int32 array [n, 5]
    (x0, y0, x1, y1, n_px) sorted by (y0, x0, y1, x1, n_px)."""
    labels = _c(labels, np.int32).reshape(-1)
    out = np.zeros(5 * int(cap), np.int32)
    n = _load().oracle_boxes(int(W), int(H), labels, int(A_min), float(alpha), int(cap), out)
    return out[: 5 * min(n, cap)].reshape(-1, 5).copy()


def classify(W, H, binned, grid, params=None, pixels=None):
    """Per-pixel Eq. 6-11 over a binned window. ``grid`` = (a0, da, denom, n_bins).
    ``pixels`` restricts the work to those pixel keys (active ones are kept).
    Returns dict(active, log_sf, snr, w, mask)."""
    prm = dict(TABLE2)
    if params:
        prm.update(params)
    lib = _load()
    offsets = _c(binned["offsets"], np.int64)
    tau = _c(binned["tau"] if binned["tau"].size else np.zeros(1, np.int64), np.int64)
    pol = _c(binned["pol"] if binned["pol"].size else np.zeros(1, np.int8), np.int8)
    npx = int(W) * int(H)
    if pixels is None:
        n_list, plist, cap = -1, None, npx
    else:
        plist = _c(pixels, np.int64)
        n_list, cap = int(plist.shape[0]), max(int(plist.shape[0]), 1)
    active = np.zeros(cap, np.int64)
    lsf = np.zeros(cap, np.float64)
    snr = np.zeros(cap, np.float64)
    w = np.zeros(cap, np.int32)
    mask = np.zeros(npx, np.uint8)
    a0, da, denom, nb = grid
    na = lib.oracle_classify(int(W), int(H), offsets, tau, pol, int(a0), int(da), int(denom),
                             int(nb), float(prm["tau_sf"]), float(prm["tau_comb"]),
                             int(prm["M"]), int(prm["d"]), int(prm["h_min"]), int(prm["n_min"]),
                             n_list, _ptr(plist), _ptr(active), _ptr(lsf), _ptr(snr), _ptr(w),
                             _ptr(mask))
    return dict(active=active[:na].copy(), log_sf=lsf[:na].copy(), snr=snr[:na].copy(),
                w=w[:na].copy(), mask=mask)


def detect(W, H, ev, t0, window_us, grid, params=None):
    """Whole window: bin, classify, label, boxes (Sec. 3.5). ``ev`` = dict(x, y, t, p)."""
    prm = dict(TABLE2)
    if params:
        prm.update(params)
    b = bin_events(W, H, ev["x"], ev["y"], ev["t"], ev["p"], t0, window_us)
    c = classify(W, H, b, grid, prm)
    labels, ncomp = ccl8(c["mask"], W, H)
    bx = boxes(labels, W, H, prm["A_min"], prm["alpha"])
    return dict(binned=b, classified=c, labels=labels, n_components=ncomp, boxes=bx)


def softcomb(tau, pol, f0, w, sigma, delta, Q, B, tau_c=0.0):
    """Soft comb score S and its gradients (see the C source for the formulas).

    Returns dict(S, dS_df0, dS_dw[n_h], dS_dsigma[n_h], dS_df[n_h, 2Q+1])."""
    lib = _load()
    tau, pol = _c(tau, np.int64), _c(pol, np.int8)
    w, sigma = _c(w, np.float64), _c(sigma, np.float64)
    nh = int(w.shape[0])
    g0 = np.zeros(1, np.float64)
    gw = np.zeros(nh, np.float64)
    gs = np.zeros(nh, np.float64)
    gf = np.zeros(nh * (2 * int(Q) + 1), np.float64)
    S = lib.oracle_softcomb(int(tau.shape[0]), tau, pol, float(tau_c), float(f0), nh, w, sigma,
                            float(delta), int(Q), float(B), _ptr(g0), _ptr(gw), _ptr(gs),
                            _ptr(gf))
    return dict(S=float(S), dS_df0=float(g0[0]), dS_dw=gw, dS_dsigma=gs,
                dS_df=gf.reshape(nh, 2 * int(Q) + 1))


def box_median_hz(boxes, active, mask, f0_bin, W, grid):
    """Per box: the lower median (the element of rank floor((n-1)/2) of the n
    sorted values) of the dominant bins of the rotor pixels inside it, as Hz
    ((a0 + j da) 1e6 / denom for grid (a0, da, denom, n)); 0.0 without any."""
    active = np.asarray(active, np.int64)
    ys, xs = active // W, active % W
    rot = np.asarray(mask, bool)[active]
    a0, da, denom = (int(v) for v in grid[:3])
    out = []
    for b in np.asarray(boxes).reshape(-1, np.asarray(boxes).shape[-1]):
        x0, y0, x1, y1 = (int(v) for v in b[:4])
        sel = rot & (xs >= x0) & (xs <= x1) & (ys >= y0) & (ys <= y1)
        v = np.sort(np.asarray(f0_bin)[sel])
        out.append(0.0 if v.size == 0 else (a0 + int(v[(v.size - 1) // 2]) * da) * 1e6 / denom)
    return np.array(out, np.float32)


def box_frequencies(boxes, active, mask, snr, f0_bin, W):
    """Eq. 11 returns a dominant frequency per rotor pixel; a detection box
    takes that of its strongest rotor pixel: for each box (x0, y0, x1, y1,
    inclusive bounds), among the active pixels (keys y*W + x, ascending, with
    snr and f0_bin in active order) whose mask entry is set and whose (x, y)
    lies in the box, the largest SNR, ties to the smallest key. Returns
    (f0_bin, snr) per box, (-1, 0.0) for a box without rotor pixels."""
    active = np.asarray(active, np.int64)
    ys, xs = active // W, active % W
    rot = np.asarray(mask, bool)[active]
    out_f, out_s = [], []
    for b in np.asarray(boxes).reshape(-1, np.asarray(boxes).shape[-1]):
        x0, y0, x1, y1 = (int(v) for v in b[:4])
        best = -1
        for i in range(active.size):
            if rot[i] and x0 <= xs[i] <= x1 and y0 <= ys[i] <= y1:
                if best < 0 or snr[i] > snr[best]:  # first index wins ties
                    best = i
        out_f.append(int(f0_bin[best]) if best >= 0 else -1)
        out_s.append(float(snr[best]) if best >= 0 else 0.0)
    return np.array(out_f, np.int32), np.array(out_s, np.float32)
