"""Python binding of libddhf (include/ddhf.h), argument marshalling only.

Every function named ``ddhf_*`` here calls the C entry point of the same name
with device pointers taken from torch CUDA tensors and the current torch
stream; all computation happens in the library's CUDA kernels. A missing or
unloadable library raises ``DDHFLibraryError``: there is no fallback path.

``Context`` wraps one ``ddhf_ctx`` with tensor-returning helpers.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# DDHF_LIB names another build of the library (e.g. the debug build,
# libddhf_debug.so); the default is the in-tree release build.
LIB_PATH = os.environ.get("DDHF_LIB") or os.path.join(_HERE, "libddhf.so")

DDHF_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "CAPACITY", 4: "TIMEOUT", 5: "UNSUPPORTED",
          6: "STATE"}
FORM = dict(sincos=0, recur=1, blocked=2, naive32=3, kahan=4, f64=5, hybrid=6)
FLAG_CAPACITY, FLAG_TIMEOUT = 1, 2


class DDHFLibraryError(RuntimeError):
    pass


class DDHFError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"ddhf status {status} ({STATUS.get(status, '?')}): {msg}")


class ddhf_grid(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_int64), ("da", ctypes.c_int64), ("denom", ctypes.c_int64),
                ("n_bins", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ddhf_params(ctypes.Structure):
    _fields_ = [("tau_sf", ctypes.c_float), ("tau_comb", ctypes.c_float), ("M", ctypes.c_int32),
                ("d", ctypes.c_int32), ("h_min", ctypes.c_int32), ("n_min", ctypes.c_int32),
                ("A_min", ctypes.c_int32), ("polarity_01", ctypes.c_int32),
                ("alpha", ctypes.c_double)]


class ddhf_window(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("t_us", ctypes.c_void_p),
                ("p", ctypes.c_void_p), ("n", ctypes.c_int64), ("t0_us", ctypes.c_int64),
                ("window_us", ctypes.c_int64)]


class ddhf_stats(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int64), ("n_valid", ctypes.c_int64),
                ("n_dropped", ctypes.c_int64), ("n_active", ctypes.c_int64),
                ("n_rotor", ctypes.c_int64), ("n_boxes", ctypes.c_int64),
                ("terms", ctypes.c_int64), ("graph_kernels", ctypes.c_int64),
                ("device_flags", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class ddhf_tuning(ctypes.Structure):
    _fields_ = [("heavy_min", ctypes.c_int32), ("warps_per_block", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("rows_per_lane", ctypes.c_int32),
                ("fuse", ctypes.c_int32), ("overlap", ctypes.c_int32),
                ("hybrid_min", ctypes.c_int32)]


class ddhf_component(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("label", "x0", "y0", "x1", "y1", "n_px")]


class ddhf_box(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("x0", "y0", "x1", "y1", "n_px")]


class ddhf_pipe_peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int32), ("sm_clock_max_mhz", ctypes.c_int32),
                ("ffma_per_s", ctypes.c_double), ("ffma2_lane_per_s", ctypes.c_double),
                ("sin_approx_per_s", ctypes.c_double), ("lg2_approx_per_s", ctypes.c_double),
                ("elapsed_ms", ctypes.c_float * 4)]


class ddhf_slide_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "t_end_us", "pushes", "rebuilds", "n_added", "n_dropped", "n_expired", "n_window",
        "last_delta", "last_pixels", "ring_used")]


# exported symbol -> (restype, argtypes)
_VP, _I32, _I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "ddhf_status_string": (ctypes.c_char_p, [_I32]),
    "ddhf_default_params": (_I32, [ctypes.POINTER(ddhf_params)]),
    "ddhf_create": (_I32, [_I32, _I32, ctypes.POINTER(ddhf_grid), ctypes.POINTER(ddhf_params),
                           _I64, _I32, ctypes.POINTER(_VP)]),
    "ddhf_destroy": (_I32, [_VP]),
    "ddhf_set_tuning": (_I32, [_VP, ctypes.POINTER(ddhf_tuning)]),
    "ddhf_set_params": (_I32, [_VP, ctypes.POINTER(ddhf_params)]),
    "ddhf_set_loop_limit": (_I32, [_VP, _I32]),
    "ddhf_hybrid_geometry": (_I32, [ctypes.POINTER(ddhf_grid), _I64, _I32, _VP, _VP, _VP, _VP]),
    "ddhf_get_tuning": (_I32, [_VP, ctypes.POINTER(ddhf_tuning)]),
    "ddhf_bin_events": (_I32, [_VP, _VP, _VP, _VP, _VP, _I64, _I64, _I64, _VP]),
    "ddhf_export_csr": (_I32, [_VP, _VP, _VP, _I64, _VP, _VP, _VP]),
    "ddhf_power_spectrum": (_I32, [_VP, _I32, _VP, _I64, _VP]),
    "ddhf_comb_score": (_I32, [_VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP]),
    "ddhf_label": (_I32, [_VP, _VP, _VP, _VP]),
    "ddhf_boxes": (_I32, [_VP, _VP, _VP, _I32, _VP, _VP]),
    "ddhf_detect": (_I32, [_VP, _VP, _VP, _VP, _VP, _I64, _I64, _I64, _VP, _I32, _VP, _VP, _VP]),
    "ddhf_detect_batch": (_I32, [_VP, ctypes.POINTER(ddhf_window), _I32, _VP, _I32, _VP, _VP,
                                 _I32, _VP]),
    "ddhf_export_scores": (_I32, [_VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ddhf_get_stats": (_I32, [_VP, ctypes.POINTER(ddhf_stats)]),
    "ddhf_enable_stage_timing": (_I32, [_VP, _I32]),
    "ddhf_stage_times": (_I32, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "ddhf_last_error": (ctypes.c_char_p, [_VP]),
    "ddhf_softcomb": (_I32, [_VP, _I64, _VP, _VP, _I32, _I32, ctypes.c_double, ctypes.c_double,
                             _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "ddhf_spectrum_median": (_I32, [_VP, _VP, _I64, _VP, _VP]),
    "ddhf_power_spectrum_noalloc": (_I32, [ctypes.POINTER(ddhf_grid), _VP, _VP, _I64, _VP, _I64,
                                           _VP, _I64, _VP, _VP]),
    "ddhf_detect_batch_host": (_I32, [_VP, ctypes.POINTER(ddhf_window), _I32, _VP, _I32, _VP,
                                      _VP, _VP]),
    "ddhf_set_row_offset": (_I32, [_VP, _I32]),
    "ddhf_components": (_I32, [_VP, _VP, _I32, _VP, _I32, _VP, _VP]),
    "ddhf_merge_bands": (_I32, [_I32, _I32, _I32, _VP, _VP, _VP, _VP, ctypes.POINTER(ddhf_params),
                                _VP, _I32, _VP]),
    "ddhf_slide_begin": (_I32, [_VP, _I64, _I64, _I64, _I32]),
    "ddhf_slide_end": (_I32, [_VP]),
    "ddhf_slide_push": (_I32, [_VP, _VP, _VP, _VP, _VP, _I64, _I64, _VP]),
    "ddhf_slide_spectra": (_I32, [_VP, _VP, _I64, _VP]),
    "ddhf_slide_detect": (_I32, [_VP, _VP, _I32, _VP, _VP, _VP]),
    "ddhf_slide_get_stats": (_I32, [_VP, ctypes.POINTER(ddhf_slide_stats)]),
    "ddhf_measure_pipes": (_I32, [ctypes.POINTER(ddhf_pipe_peaks), _I32, _VP]),
    "ddhf_export_labels": (_I32, [_VP, _I32, _VP, _VP]),
    "ddhf_box_frequencies": (_I32, [_VP, _I32, _VP, _VP, _I32, _VP, _VP, _VP, _VP]),
    "ddhf_debug_fail_alloc_after": (_I32, [_I32]),
    "ddhf_debug_corrupt_guard": (_I32, [_VP, _I32]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libddhf.so (built by ``build.build()``); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise DDHFLibraryError(f"{path} not found: build it with "
                                   "paper_2603_08386_gb300.build.build()")
        try:
            lib = ctypes.CDLL(path)
        except OSError as e:
            raise DDHFLibraryError(f"cannot load {path}: {e}") from e
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream if hasattr(s, "cuda_stream") else int(s)


def _check(st, ctx=None):
    if st != DDHF_OK:
        msg = ""
        if ctx:
            raw = load().ddhf_last_error(ctx)
            msg = raw.decode() if raw else ""
        raise DDHFError(st, msg)


def make_grid(a0, da, denom, n_bins) -> ddhf_grid:
    return ddhf_grid(int(a0), int(da), int(denom), int(n_bins), 0)


def default_params(**over) -> ddhf_params:
    p = ddhf_params()
    _check(load().ddhf_default_params(ctypes.byref(p)))
    for k, v in over.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- same names

def ddhf_create(W, H, grid, params, max_events, max_windows=1):
    h = ctypes.c_void_p()
    _check(load().ddhf_create(int(W), int(H), ctypes.byref(grid), ctypes.byref(params),
                              int(max_events), int(max_windows), ctypes.byref(h)))
    return h.value


def ddhf_destroy(ctx):
    _check(load().ddhf_destroy(ctx))


def ddhf_set_tuning(ctx, heavy_min=1024, warps_per_block=4, blocks_per_sm=0, rows_per_lane=0,
                    fuse=0, overlap=0, hybrid_min=0):
    t = ddhf_tuning(int(heavy_min), int(warps_per_block), int(blocks_per_sm), int(rows_per_lane),
                    int(fuse), int(overlap), int(hybrid_min))
    _check(load().ddhf_set_tuning(ctx, ctypes.byref(t)), ctx)


def ddhf_set_params(ctx, params):
    _check(load().ddhf_set_params(ctx, ctypes.byref(params)), ctx)


def ddhf_hybrid_geometry(grid, window_us, hybrid_min):
    """Host-only: (status, s_us, rows, threshold, dec[n_bins] numpy float32)
    of the hybrid route for a window on this grid (no device needed)."""
    import numpy as np
    g = grid if isinstance(grid, ddhf_grid) else make_grid(*grid)
    s = ctypes.c_int64()
    rows, thr = ctypes.c_int32(), ctypes.c_int32()
    dec = np.zeros(g.n_bins, np.float32)
    st = load().ddhf_hybrid_geometry(ctypes.byref(g), int(window_us), int(hybrid_min),
                                     ctypes.byref(s), ctypes.byref(rows), ctypes.byref(thr),
                                     dec.ctypes.data_as(ctypes.c_void_p))
    return st, s.value, rows.value, thr.value, dec


def ddhf_set_loop_limit(ctx, limit):
    _check(load().ddhf_set_loop_limit(ctx, int(limit)), ctx)


def ddhf_get_tuning(ctx):
    t = ddhf_tuning()
    _check(load().ddhf_get_tuning(ctx, ctypes.byref(t)), ctx)
    return dict(heavy_min=t.heavy_min, warps_per_block=t.warps_per_block,
                blocks_per_sm=t.blocks_per_sm, rows_per_lane=t.rows_per_lane, fuse=t.fuse,
                overlap=t.overlap, hybrid_min=t.hybrid_min)


def ddhf_bin_events(ctx, x, y, t, p, n, t0, window_us, stream=None):
    _check(load().ddhf_bin_events(ctx, _ptr(x), _ptr(y), _ptr(t), _ptr(p), int(n), int(t0),
                                  int(window_us), _stream(stream)), ctx)


def ddhf_export_csr(ctx, offsets, ev, cap_ev, active, counts, stream=None):
    _check(load().ddhf_export_csr(ctx, _ptr(offsets), _ptr(ev), int(cap_ev), _ptr(active),
                                  _ptr(counts), _stream(stream)), ctx)


def ddhf_power_spectrum(ctx, form, P, cap_px, stream=None):
    _check(load().ddhf_power_spectrum(ctx, int(form), _ptr(P), int(cap_px), _stream(stream)), ctx)


def ddhf_comb_score(ctx, P, cap_px, log_sf, snr, f0_bin, mask, stream=None):
    _check(load().ddhf_comb_score(ctx, _ptr(P), int(cap_px), _ptr(log_sf), _ptr(snr),
                                  _ptr(f0_bin), _ptr(mask), _stream(stream)), ctx)


def ddhf_label(ctx, mask, labels, stream=None):
    _check(load().ddhf_label(ctx, _ptr(mask), _ptr(labels), _stream(stream)), ctx)


def ddhf_boxes(ctx, labels, boxes, cap, n_boxes, stream=None):
    _check(load().ddhf_boxes(ctx, _ptr(labels), _ptr(boxes), int(cap), _ptr(n_boxes),
                             _stream(stream)), ctx)


def _hptr(t):
    if t is None:
        return None
    if t.is_cuda:
        raise ValueError("expected a host tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def ddhf_detect_batch_host(ctx, windows, boxes_host, cap, n_boxes_host, masks_host=None,
                           stream=None):
    """windows: list of (x, y, t, p, n, t0, window_us) with HOST tensors
    (pin_memory() for overlap); outputs are host tensors, complete after the
    stream finishes."""
    arr = (ddhf_window * len(windows))()
    for i, (x, y, t, p, n, t0, win) in enumerate(windows):
        arr[i] = ddhf_window(_hptr(x), _hptr(y), _hptr(t), _hptr(p), int(n), int(t0), int(win))
    _check(load().ddhf_detect_batch_host(ctx, arr, len(windows), _hptr(boxes_host), int(cap),
                                         _hptr(n_boxes_host), _hptr(masks_host),
                                         _stream(stream)), ctx)


def ddhf_set_row_offset(ctx, row0):
    _check(load().ddhf_set_row_offset(ctx, int(row0)), ctx)


def ddhf_components(ctx, labels, row0, comps, cap, n_dev, stream=None):
    """comps: int32 CUDA tensor [cap, 6] (label, x0, y0, x1, y1, n_px)."""
    _check(load().ddhf_components(ctx, _ptr(labels), int(row0), _ptr(comps), int(cap),
                                  _ptr(n_dev), _stream(stream)), ctx)


def ddhf_merge_bands(W, H, band_row0, edge_labels, comps, comp_off, params, cap):
    """Host call. band_row0 int32 [n+1], edge_labels int32 [n, 2, W] (band-local
    labels), comps int32 [total, 6], comp_off int64 [n+1] (numpy arrays).
    Returns (boxes int32 [min(total, cap), 5], total)."""
    import numpy as np
    n = len(band_row0) - 1
    br = np.ascontiguousarray(band_row0, dtype=np.int32)
    el = np.ascontiguousarray(edge_labels, dtype=np.int32)
    cp = np.ascontiguousarray(comps, dtype=np.int32).reshape(-1, 6)
    co = np.ascontiguousarray(comp_off, dtype=np.int64)
    out = np.zeros((max(int(cap), 1), 5), dtype=np.int32)
    nb = ctypes.c_int32(0)
    st = load().ddhf_merge_bands(int(W), int(H), n, br.ctypes.data, el.ctypes.data,
                                 cp.ctypes.data if cp.size else None, co.ctypes.data,
                                 ctypes.byref(params), out.ctypes.data, int(cap),
                                 ctypes.byref(nb))
    if st not in (DDHF_OK, 3):  # CAPACITY: the first cap boxes are valid
        _check(st)
    return out[: min(nb.value, int(cap))].copy(), nb.value


def ddhf_detect(ctx, x, y, t, p, n, t0, window_us, boxes, cap, n_boxes, mask_out=None,
                stream=None):
    _check(load().ddhf_detect(ctx, _ptr(x), _ptr(y), _ptr(t), _ptr(p), int(n), int(t0),
                              int(window_us), _ptr(boxes), int(cap), _ptr(n_boxes),
                              _ptr(mask_out), _stream(stream)), ctx)


def ddhf_detect_batch(ctx, windows, boxes, cap, n_boxes, masks_out=None, use_graph=False,
                      stream=None):
    """windows: list of (x, y, t, p, n, t0, window_us) with device tensors."""
    arr = (ddhf_window * len(windows))()
    for i, (x, y, t, p, n, t0, win) in enumerate(windows):
        arr[i] = ddhf_window(_ptr(x), _ptr(y), _ptr(t), _ptr(p), int(n), int(t0), int(win))
    _check(load().ddhf_detect_batch(ctx, arr, len(windows), _ptr(boxes), int(cap), _ptr(n_boxes),
                                    _ptr(masks_out), int(bool(use_graph)), _stream(stream)), ctx)


def ddhf_export_scores(ctx, slot, active, log_sf, snr, f0_bin, counts, stream=None):
    _check(load().ddhf_export_scores(ctx, int(slot), _ptr(active), _ptr(log_sf), _ptr(snr),
                                     _ptr(f0_bin), _ptr(counts), _stream(stream)), ctx)


def ddhf_debug_fail_alloc_after(n):
    _check(load().ddhf_debug_fail_alloc_after(int(n)))


def ddhf_export_labels(ctx, slot, labels, stream=None):
    _check(load().ddhf_export_labels(ctx, int(slot), _ptr(labels), _stream(stream)), ctx)


def ddhf_box_frequencies(ctx, slot, boxes, n_boxes, cap, f0_bin, snr=None, f0_hz_median=None,
                         stream=None):
    """Per detected box: the dominant bin and SNR of its strongest rotor pixel
    and the lower median (Hz) of its rotor pixels' dominant frequencies."""
    _check(load().ddhf_box_frequencies(ctx, int(slot), _ptr(boxes), _ptr(n_boxes), int(cap),
                                       _ptr(f0_bin), _ptr(snr), _ptr(f0_hz_median),
                                       _stream(stream)), ctx)


def ddhf_debug_corrupt_guard(ctx, index):
    """Test hook: overwrite one guard byte after workspace buffer `index`."""
    _check(load().ddhf_debug_corrupt_guard(ctx, int(index)), ctx)


def ddhf_enable_stage_timing(ctx, enable=True):
    _check(load().ddhf_enable_stage_timing(ctx, int(bool(enable))), ctx)


def ddhf_stage_times(ctx):
    """Device milliseconds of {binning, classification, labels + boxes,
    spectrum kernels, comb kernels} of the last timed detection call (the last
    two are 0 on the fused path)."""
    out = (ctypes.c_float * 5)()
    _check(load().ddhf_stage_times(ctx, out), ctx)
    return [float(v) for v in out]


def ddhf_power_spectrum_noalloc(grid, offsets, ev, n_events, active, n_active, P, cap_px,
                                flags=None, stream=None):
    """Blocked-form spectra from a caller-owned per-pixel list; the library
    allocates nothing (see include/ddhf.h for who needs this and its limits).
    flags: optional device int32 tensor of one element that receives the
    DDHF_FLAG_* bits the call raised."""
    _check(load().ddhf_power_spectrum_noalloc(ctypes.byref(grid), _ptr(offsets), _ptr(ev),
                                              int(n_events), _ptr(active), int(n_active),
                                              _ptr(P), int(cap_px), _ptr(flags), _stream(stream)))


def ddhf_softcomb(ctx, pixels, f0, n_h, Q, delta_hz, tau_c_us, w, sigma, B, S=None,
                  grad_S=None, grad_f0=None, grad_w=None, grad_sigma=None, grad_f=None,
                  stream=None):
    _check(load().ddhf_softcomb(ctx, int(pixels.numel()), _ptr(pixels), _ptr(f0), int(n_h), int(Q),
                                float(delta_hz), float(tau_c_us), _ptr(w), _ptr(sigma), _ptr(B),
                                _ptr(S), _ptr(grad_S), _ptr(grad_f0), _ptr(grad_w),
                                _ptr(grad_sigma), _ptr(grad_f), _stream(stream)), ctx)


def ddhf_spectrum_median(ctx, P, rows, median, stream=None):
    _check(load().ddhf_spectrum_median(ctx, _ptr(P), int(rows), _ptr(median), _stream(stream)), ctx)


class SoftComb(torch.autograd.Function):
    """Soft comb score S per pixel as a differentiable function of the
    per-pixel fundamentals f0 and the shared harmonic weights w and widths
    sigma; forward and backward both run in the library's kernels
    (ddhf_softcomb). B (background) is held constant."""

    @staticmethod
    def forward(ctx_, f0, w, sigma, handle, pixels, B, Q, delta_hz, tau_c_us):
        f0c, wc, sc = f0.contiguous(), w.contiguous(), sigma.contiguous()
        S = torch.empty_like(f0c)
        ddhf_softcomb(handle, pixels, f0c, wc.numel(), Q, delta_hz, tau_c_us, wc, sc, B, S=S)
        ctx_.save_for_backward(f0c, wc, sc)
        ctx_.extra = (handle, pixels, B, Q, delta_hz, tau_c_us)
        return S

    @staticmethod
    def backward(ctx_, gS):
        f0c, wc, sc = ctx_.saved_tensors
        handle, pixels, B, Q, delta_hz, tau_c_us = ctx_.extra
        g_f0 = torch.empty_like(f0c)
        g_w = torch.empty_like(wc)
        g_s = torch.empty_like(sc)
        ddhf_softcomb(handle, pixels, f0c, wc.numel(), Q, delta_hz, tau_c_us, wc, sc, B,
                      grad_S=gS.contiguous(), grad_f0=g_f0, grad_w=g_w, grad_sigma=g_s)
        return g_f0, g_w, g_s, None, None, None, None, None, None


def ddhf_measure_pipes(iters=1 << 16, stream=None):
    """Pipe throughput of the current device (dict of the struct's fields)."""
    out = ddhf_pipe_peaks()
    _check(load().ddhf_measure_pipes(ctypes.byref(out), int(iters), _stream(stream)))
    d = {k: getattr(out, k) for k, _ in ddhf_pipe_peaks._fields_ if k != "elapsed_ms"}
    d["elapsed_ms"] = list(out.elapsed_ms)
    return d


def ddhf_get_stats(ctx, raise_on_flags=True):
    s = ddhf_stats()
    st = load().ddhf_get_stats(ctx, ctypes.byref(s))
    out = {k: getattr(s, k) for k, _ in ddhf_stats._fields_ if k != "reserved"}
    out["status"] = st
    if raise_on_flags:
        _check(st, ctx)
    return out


def ddhf_slide_begin(ctx, window_us, t_begin_us, capacity, rebuild_every=64):
    _check(load().ddhf_slide_begin(ctx, int(window_us), int(t_begin_us), int(capacity),
                                   int(rebuild_every)), ctx)


def ddhf_slide_end(ctx):
    _check(load().ddhf_slide_end(ctx), ctx)


def ddhf_slide_push(ctx, x, y, t, p, n, t_end_us, stream=None):
    _check(load().ddhf_slide_push(ctx, _ptr(x), _ptr(y), _ptr(t), _ptr(p), int(n),
                                  int(t_end_us), _stream(stream)), ctx)


def ddhf_slide_spectra(ctx, P, cap_px, stream=None):
    _check(load().ddhf_slide_spectra(ctx, _ptr(P), int(cap_px), _stream(stream)), ctx)


def ddhf_slide_detect(ctx, boxes, cap, n_boxes, mask_out=None, stream=None):
    _check(load().ddhf_slide_detect(ctx, _ptr(boxes), int(cap), _ptr(n_boxes), _ptr(mask_out),
                                    _stream(stream)), ctx)


def ddhf_slide_get_stats(ctx):
    s = ddhf_slide_stats()
    _check(load().ddhf_slide_get_stats(ctx, ctypes.byref(s)), ctx)
    return {k: getattr(s, k) for k, _ in ddhf_slide_stats._fields_}


# ---------------------------------------------------------------- convenience

class Context:
    """One ddhf context bound to the current CUDA device."""

    def __init__(self, W, H, grid, params=None, max_events=1 << 20, max_windows=1):
        if isinstance(grid, tuple):
            grid = make_grid(*grid)
        self.W, self.H, self.npx = int(W), int(H), int(W) * int(H)
        self.grid = grid
        self.n_bins = grid.n_bins
        self.params = params if params is not None else default_params()
        self.max_events = int(max_events)
        self.max_windows = int(max_windows)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.h = ddhf_create(W, H, grid, self.params, max_events, max_windows)

    def close(self):
        if self.h:
            ddhf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        ddhf_set_params(self.h, params)
        self.params = params

    def set_tuning(self, **kw):
        cur = ddhf_get_tuning(self.h)
        cur.update(kw)
        ddhf_set_tuning(self.h, **cur)

    def bin_events(self, x, y, t, p, t0, window_us):
        ddhf_bin_events(self.h, x, y, t, p, x.numel(), t0, window_us)

    def csr(self, cap_ev=None):
        cap_ev = self.max_events if cap_ev is None else cap_ev
        off = torch.empty(self.npx + 1, dtype=torch.int32, device=self.dev)
        ev = torch.empty(max(cap_ev, 1), dtype=torch.int32, device=self.dev)
        act = torch.empty(self.npx, dtype=torch.int32, device=self.dev)
        cnt = torch.zeros(4, dtype=torch.int64, device=self.dev)
        ddhf_export_csr(self.h, off, ev, cap_ev, act, cnt)
        c = cnt.cpu().tolist()
        return dict(offsets=off, ev=ev[: c[0]], active=act[: c[2]], n_valid=c[0],
                    n_dropped=c[1], n_active=c[2], n_in=c[3])

    def n_active(self):
        cnt = torch.zeros(4, dtype=torch.int64, device=self.dev)
        ddhf_export_csr(self.h, None, None, 0, None, cnt)
        return int(cnt[2].item())

    def power_spectrum(self, form="blocked", cap_px=None):
        f = FORM[form] if isinstance(form, str) else int(form)
        na = self.n_active() if cap_px is None else cap_px
        P = torch.empty((max(na, 1), self.n_bins), dtype=torch.float32, device=self.dev)
        ddhf_power_spectrum(self.h, f, P, na)
        return P[:na]

    def comb_score(self, P):
        na = P.shape[0]
        lsf = torch.empty(max(na, 1), dtype=torch.float32, device=self.dev)
        snr = torch.empty_like(lsf)
        f0 = torch.empty(max(na, 1), dtype=torch.int32, device=self.dev)
        mask = torch.empty(self.npx, dtype=torch.uint8, device=self.dev)
        ddhf_comb_score(self.h, P.contiguous() if na else lsf, na, lsf, snr, f0, mask)
        return dict(log_sf=lsf[:na], snr=snr[:na], f0_bin=f0[:na], mask=mask)

    def label(self, mask):
        lab = torch.empty(self.npx, dtype=torch.int32, device=self.dev)
        ddhf_label(self.h, mask.contiguous(), lab)
        return lab

    def boxes(self, labels, cap=4096):
        bx = torch.empty((max(cap, 1), 5), dtype=torch.int32, device=self.dev)
        nb = torch.zeros(1, dtype=torch.int32, device=self.dev)
        ddhf_boxes(self.h, labels, bx, cap, nb)
        n = int(nb.item())
        return bx[: min(n, cap)], n

    def detect(self, x, y, t, p, t0, window_us, cap=4096, want_mask=False):
        bx = torch.empty((max(cap, 1), 5), dtype=torch.int32, device=self.dev)
        nb = torch.zeros(1, dtype=torch.int32, device=self.dev)
        mask = torch.empty(self.npx, dtype=torch.uint8, device=self.dev) if want_mask else None
        ddhf_detect(self.h, x, y, t, p, x.numel(), t0, window_us, bx, cap, nb, mask)
        return bx, nb, mask

    def scores(self, slot=0):
        act = torch.empty(self.npx, dtype=torch.int32, device=self.dev)
        lsf = torch.empty(self.npx, dtype=torch.float32, device=self.dev)
        snr = torch.empty_like(lsf)
        f0 = torch.empty(self.npx, dtype=torch.int32, device=self.dev)
        cnt = torch.zeros(4, dtype=torch.int64, device=self.dev)
        ddhf_export_scores(self.h, slot, act, lsf, snr, f0, cnt)
        na = int(cnt[2].item())
        return dict(active=act[:na], log_sf=lsf[:na], snr=snr[:na], f0_bin=f0[:na], n_active=na)

    def stats(self, raise_on_flags=True):
        return ddhf_get_stats(self.h, raise_on_flags)

    # sliding window (Sec. 3.3: terms of the events entering and leaving)
    def slide_begin(self, window_us, t_begin_us, capacity=None, rebuild_every=64):
        cap = self.max_events if capacity is None else capacity
        ddhf_slide_begin(self.h, window_us, t_begin_us, cap, rebuild_every)

    def slide_push(self, x, y, t, p, t_end_us):
        ddhf_slide_push(self.h, x, y, t, p, x.numel(), t_end_us)

    def slide_spectra(self):
        """(active keys, P [n_active, n_bins]) of the current window."""
        ddhf_slide_spectra(self.h, None, 0)
        act = self.scores()["active"]
        na = act.numel()
        P = torch.empty((max(na, 1), self.n_bins), dtype=torch.float32, device=self.dev)
        ddhf_slide_spectra(self.h, P, na)
        return act, P[:na]

    def slide_detect(self, cap=4096, want_mask=False):
        bx = torch.empty((max(cap, 1), 5), dtype=torch.int32, device=self.dev)
        nb = torch.zeros(1, dtype=torch.int32, device=self.dev)
        mask = torch.empty(self.npx, dtype=torch.uint8, device=self.dev) if want_mask else None
        ddhf_slide_detect(self.h, bx, cap, nb, mask)
        return bx, nb, mask

    def slide_stats(self):
        return ddhf_slide_get_stats(self.h)

    def slide_end(self):
        ddhf_slide_end(self.h)


def events_to_device(scene, device="cuda"):
    """Upload a synthetic Scene's event arrays to device tensors."""
    return (torch.from_numpy(scene.x).to(device), torch.from_numpy(scene.y).to(device),
            torch.from_numpy(scene.t).to(device), torch.from_numpy(scene.p).to(device))


def stack_windows(windows, H):
    """Lay several windows of one H-row sensor out as one window of a sensor
    len(windows) times as tall, so that one binning and one call (for
    instance one ddhf_softcomb over the whole batch) cover them all.

    windows: sequence of (x, y, t, p, t0) numpy arrays / ints, all of the same
    window length. Window b's rows go to y + b H and its times to t - t0_b, so
    every event keeps its offset tau = t - t0 in the stacked window (t0 = 0);
    a pixel's events, their order and their tau are those of its own window,
    so per-pixel results equal the per-window ones bit for bit. Returns
    (x, y, t, p) numpy arrays; the stacked sensor is W x (len(windows) H) and
    pixel key y*W + x of window b is key_b + b*H*W."""
    import numpy as np
    if len(windows) * H > 32767:
        raise ValueError("stacked sensor taller than int16 rows allow")
    xs, ys, ts, ps = [], [], [], []
    for b, (x, y, t, p, t0) in enumerate(windows):
        xs.append(np.asarray(x, np.int16))
        ys.append((np.asarray(y, np.int32) + b * H).astype(np.int16))
        ts.append(np.asarray(t, np.int64) - np.int64(t0))
        ps.append(np.asarray(p, np.int8))
    return np.concatenate(xs), np.concatenate(ys), np.concatenate(ts), np.concatenate(ps)
