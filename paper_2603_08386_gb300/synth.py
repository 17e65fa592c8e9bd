"""Seeded synthetic event streams shaped like the scenes of arXiv 2603.08386.

The paper's EVK4-HD recordings (Sec. 4.1) are not available, so every input of
the library, its tests and its benchmark comes from these generators. They hold
none of the detection method's arithmetic: they only draw events
(x, y, t_us, p) for a window, with the shapes, rates and count distributions
stated per configuration below, plus the ground-truth rotor pixels.

Event model (Sec. 3.1, Sec. 3.2): a rotor pixel sees a periodic occlusion at the
blade-pass frequency f0 with duty cycle tau; each occlusion start emits a short
burst of -1 events (the background darkens) and each end a burst of +1 events,
with Gaussian timing jitter. Background pixels emit uniformly timed events with
random polarity. Timestamps are integer microseconds (continuous times rounded
to the nearest microsecond) and the stream is ordered by time at a granularity
of window/65535 (as a sensor delivers it; order inside a granule is arbitrary).

Configurations (seed = 1000 + configuration number; window w of stream s of a
batched configuration uses seed*1000 + 32*s + w):

  C1  128x128, one 20 ms window, Poisson 5 Hz/pixel background, one 4-rotor
      drone (~300 px, 150 Hz), uniform fill events up to 200k events in total;
      grid 0..990 Hz step 10 Hz (100 bins).
  C2  640x480, 50 ms, Poisson 10 Hz/pixel plus a translating edge texture with
      lognormal per-pixel counts (median 8, sigma 1.16, cap 2000) in bursts at
      edge-crossing instants, two drones at 120 Hz and 210 Hz; 1 Hz grid, 2000 bins.
  C3  1280x720, 8 consecutive 30 ms windows x 4 independent streams, per-pixel
      counts floor(x_m U^(-1/1.5)) capped at 20000 (Pareto alpha = 1.5, about
      20M events per window), uniform times with burst clustering, three drones
      at 100/200/300 Hz covering 10/300/2000 px; grid 0..1498 Hz step 2 Hz (750 bins).
  C4  640x480, 40 ms windows, batch 16, density as C2; grid 0..1498 Hz step 2 Hz.
  C5  1280x720, one 200 ms window, about 60M events (C3 shape, x_m scaled),
      t0 = 2^40 - 2e5 us so timestamps reach 2^40 us; grid 0..4999.5 Hz step 0.5 Hz.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

HZ_DENOM = 1_000_000_000  # grid in mHz, time in us: cycles = a*tau / 1e9


@dataclass
class Scene:
    W: int
    H: int
    t0: int
    window_us: int
    x: np.ndarray  # int16
    y: np.ndarray  # int16
    t: np.ndarray  # int64, absolute microseconds
    p: np.ndarray  # int8, +-1
    grid: tuple  # (a0, da, denom, n_bins)
    drones: list = field(default_factory=list)  # dict(f0_hz, keys, box)
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def events(self) -> dict:
        return dict(x=self.x, y=self.y, t=self.t, p=self.p)


def hz_grid(f_lo_hz: float, step_hz: float, n_bins: int) -> tuple:
    """(a0, da, denom, n_bins) of a frequency grid in integer mHz."""
    a0 = int(round(f_lo_hz * 1000))
    da = int(round(step_hz * 1000))
    return (a0, da, HZ_DENOM, int(n_bins))


def mode_grid(window_us: int, n_modes: int) -> tuple:
    """Integer modes k = 0..K-1 over the window (Sec. 3.5): f_k = k / window."""
    return (0, 1, int(window_us), int(n_modes))


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------

def _disc_keys(W, H, cx, cy, n_px):
    """Pixel keys of a disc of about n_px pixels centred at (cx, cy)."""
    r = max(np.sqrt(n_px / np.pi), 0.5)
    R = int(np.ceil(r)) + 1
    xs, ys = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1))
    d2 = xs.astype(np.float64) ** 2 + ys.astype(np.float64) ** 2
    order = np.argsort(d2.ravel(), kind="stable")[: max(int(n_px), 1)]
    px = (cx + xs.ravel()[order]).astype(np.int64)
    py = (cy + ys.ravel()[order]).astype(np.int64)
    ok = (px >= 0) & (px < W) & (py >= 0) & (py < H)
    return np.unique(py[ok] * W + px[ok])


def drone_keys(W, H, cx, cy, n_px):
    """Four rotor discs on a square around (cx, cy), about n_px pixels in total."""
    per = max(n_px / 4.0, 1.0)
    r = np.sqrt(per / np.pi)
    arm = max(int(np.ceil(1.6 * r)) + 1, 2)
    keys = [_disc_keys(W, H, cx + sx * arm, cy + sy * arm, per)
            for sx, sy in ((-1, -1), (1, -1), (-1, 1), (1, 1))]
    return [k for k in keys if k.size]


def rotor_events(rng, keys, f0_hz, t_lo, t_hi, per_edge=3, spacing_us=15.0,
                 jitter_us=50.0, duty=(0.15, 0.4)):
    """Occlusion-edge bursts of one rotor over [t_lo, t_hi) (continuous us).

    Each pixel gets its own duty cycle and phase; each period emits `per_edge`
    events of polarity -1 at occlusion start and `per_edge` of +1 at its end."""
    keys = np.asarray(keys, np.int64)
    if keys.size == 0:
        return np.zeros(0, np.int64), np.zeros(0, np.float64), np.zeros(0, np.int8)
    T = 1e6 / f0_hz
    n_per = int(np.ceil((t_hi - t_lo) / T)) + 2
    tau = rng.uniform(duty[0], duty[1], keys.size)
    ph = rng.uniform(0.0, T, keys.size)
    k = np.arange(-1, n_per - 1, dtype=np.float64)
    start = t_lo + ph[:, None] + k[None, :] * T  # [px, periods]
    end = start + tau[:, None] * T
    j = np.arange(per_edge, dtype=np.float64) * spacing_us
    ts = np.concatenate([(start[:, :, None] + j).reshape(keys.size, -1),
                         (end[:, :, None] + j).reshape(keys.size, -1)], axis=1)
    pol = np.concatenate([np.full((keys.size, n_per * per_edge), -1, np.int8),
                          np.full((keys.size, n_per * per_edge), 1, np.int8)], axis=1)
    ts = ts + rng.normal(0.0, jitter_us, ts.shape)
    kk = np.repeat(keys, ts.shape[1])
    ts, pol = ts.ravel(), pol.ravel()
    ok = (ts >= t_lo) & (ts < t_hi)
    return kk[ok], ts[ok], pol[ok]


def _uniform(rng, keys, counts, t_lo, t_hi):
    kk = np.repeat(np.asarray(keys, np.int32), counts)
    ts = rng.integers(int(np.ceil(t_lo)), int(np.ceil(t_hi)), kk.size, dtype=np.int32)
    pol = (rng.integers(0, 2, kk.size, dtype=np.int8) * 2 - 1).astype(np.int8)
    return kk, ts, pol


def _bursty(rng, keys, counts, t_lo, t_hi, frac=0.3, spread_us=300.0):
    """Uniform times, a fraction `frac` clustered around one instant per pixel."""
    kk, ts, pol = _uniform(rng, keys, counts, t_lo, t_hi)
    centre = rng.uniform(t_lo, t_hi, len(keys))
    b = np.flatnonzero(rng.random(kk.size, dtype=np.float32) < frac)
    tb = np.rint(centre[kk[b]] + rng.normal(0.0, spread_us, b.size))
    np.clip(tb, np.ceil(t_lo), np.ceil(t_hi) - 1, out=tb)
    ts[b] = tb.astype(np.int32)
    return kk, ts, pol


def _edge_texture(rng, W, H, t_lo, t_hi, mu=np.log(8.0), sigma=1.16, cap=2000):
    """Ego-motion edges: lognormal counts, bursts at 1-3 crossing instants."""
    npx = W * H
    counts = np.minimum(np.floor(rng.lognormal(mu, sigma, npx)), cap).astype(np.int64)
    keys = np.arange(npx, dtype=np.int64)
    ncross = 1 + rng.integers(0, 3, npx)
    kk = np.repeat(keys, counts)
    # crossing index per event, crossing instants per pixel
    which = (rng.random(kk.size) * np.repeat(ncross, counts)).astype(np.int64)
    inst = rng.uniform(t_lo, t_hi, (npx, 3))
    base = inst[kk, which]
    ts = base + rng.exponential(250.0, kk.size) * rng.choice([-1.0, 1.0], kk.size)
    pol_c = (rng.integers(0, 2, (npx, 3), dtype=np.int8) * 2 - 1).astype(np.int8)
    pol = pol_c[kk, which]
    flip = rng.random(kk.size) < 0.1
    pol[flip] = -pol[flip]
    ok = (ts >= t_lo) & (ts < t_hi)
    return kk[ok], ts[ok], pol[ok]


def _pareto_counts(rng, npx, x_m, alpha=1.5, cap=20000):
    u = rng.random(npx)
    u = np.maximum(u, 1e-300)
    return np.minimum(np.floor(x_m * u ** (-1.0 / alpha)), cap).astype(np.int64)


def pareto_x_m(mean, alpha=1.5, cap=20000):
    """x_m such that E[min(floor(x_m U^(-1/alpha)), cap)] = mean."""
    c = np.arange(1, cap + 1, dtype=np.float64)

    def expect(xm):
        return float(np.minimum(1.0, (xm / c) ** alpha).sum())

    lo, hi = 0.5, mean
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if expect(mid) < mean else (lo, mid)
    return 0.5 * (lo + hi)


def _as_int_times(ts):
    if np.issubdtype(np.asarray(ts).dtype, np.integer):
        return np.asarray(ts, np.int64)
    return np.rint(ts).astype(np.int64)


def _assemble(W, H, t0, window_us, parts, grid, rng, drones, meta):
    if parts:
        kk = np.concatenate([np.asarray(p[0], np.int32) for p in parts])
        ti = np.concatenate([_as_int_times(p[1]) for p in parts])
        pol = np.concatenate([np.asarray(p[2], np.int8) for p in parts])
    else:
        kk, ti, pol = np.zeros(0, np.int32), np.zeros(0, np.int64), np.zeros(0, np.int8)
    np.clip(ti, 0, window_us - 1, out=ti)
    if window_us <= 65536:
        gran = ti.astype(np.uint16)
    else:
        gran = ((ti * 65535) // window_us).astype(np.uint16)
    order = np.argsort(gran, kind="stable")
    kk, ti, pol = kk[order], ti[order], pol[order]
    y32, x32 = np.divmod(kk, np.int32(W))
    return Scene(W=W, H=H, t0=int(t0), window_us=int(window_us), x=x32.astype(np.int16),
                 y=y32.astype(np.int16), t=ti + np.int64(t0), p=pol, grid=grid,
                 drones=drones, meta=meta)


def _drones(rng, W, H, specs, t_lo, t_hi, per_edge=3):
    """specs: list of (cx, cy, n_px, f0_hz). Returns parts, drone info, keys."""
    parts, info, allkeys = [], [], []
    for cx, cy, n_px, f0 in specs:
        rotors = drone_keys(W, H, cx, cy, n_px)
        keys = np.unique(np.concatenate(rotors)) if rotors else np.zeros(0, np.int64)
        for rk in rotors:
            parts.append(rotor_events(rng, rk, f0 * rng.uniform(0.995, 1.005), t_lo, t_hi,
                                      per_edge=per_edge))
        if keys.size:
            xs, ys = keys % W, keys // W
            box = (int(xs.min()), int(ys.min()), int(xs.max()), int(ys.max()))
        else:
            box = None
        info.append(dict(f0_hz=float(f0), keys=keys, box=box, center=(cx, cy)))
        allkeys.append(keys)
    ak = np.unique(np.concatenate(allkeys)) if allkeys else np.zeros(0, np.int64)
    return parts, info, ak


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

def config1(seed: int = 1001, total: int = 200_000) -> Scene:
    W, H, win = 128, 128, 20_000
    rng = np.random.default_rng(seed)
    parts, info, dk = _drones(rng, W, H, [(64, 64, 300, 150.0)], 0.0, win, per_edge=3)
    npx = W * H
    bg = rng.poisson(5.0 * win * 1e-6, npx)
    parts.append(_uniform(rng, np.arange(npx), bg, 0.0, win))
    n_now = sum(p[0].size for p in parts)
    fill = max(total - n_now, 0)
    fk = rng.integers(0, npx, fill + fill // 20 + 64)
    fk = fk[~np.isin(fk, dk)][:fill]
    parts.append((fk.astype(np.int64), rng.uniform(0.0, win, fk.size),
                  (rng.integers(0, 2, fk.size, dtype=np.int8) * 2 - 1).astype(np.int8)))
    meta = dict(config="C1", n_literal=n_now, n_fill=int(fk.size))
    return _assemble(W, H, 0, win, parts, hz_grid(0, 10, 100), rng, info, meta)


def config2(seed: int = 1002, W: int = 640, H: int = 480, window_us: int = 50_000,
            grid=None) -> Scene:
    rng = np.random.default_rng(seed)
    specs = [(W // 3, H // 2, 450, 120.0), (2 * W // 3, H // 3, 450, 210.0)]
    parts, info, dk = _drones(rng, W, H, specs, 0.0, window_us, per_edge=4)
    npx = W * H
    kk, ts, pol = _edge_texture(rng, W, H, 0.0, window_us)
    keep = ~np.isin(kk, dk)
    parts.append((kk[keep], ts[keep], pol[keep]))
    bg = rng.poisson(10.0 * window_us * 1e-6, npx)
    parts.append(_uniform(rng, np.arange(npx), bg, 0.0, window_us))
    meta = dict(config="C2")
    g = grid if grid is not None else hz_grid(0, 1, 2000)
    return _assemble(W, H, 0, window_us, parts, g, rng, info, meta)


def config3_window(stream: int = 0, window: int = 0, seed: int = 1003,
                   W: int = 1280, H: int = 720, window_us: int = 30_000,
                   mean_per_px: float = 21.7, grid=None) -> Scene:
    """One window of one stream of C3 (consecutive windows share the drones)."""
    rng = np.random.default_rng(seed * 1000 + 32 * stream + window)
    srng = np.random.default_rng(seed * 1000 + 977 + stream)  # per-stream layout
    npx = W * H
    sizes, freqs = (10, 300, 2000), (100.0, 200.0, 300.0)
    specs = []
    for n_px, f0 in zip(sizes, freqs):
        cx = int(srng.integers(W // 8, 7 * W // 8)) + 3 * window
        cy = int(srng.integers(H // 8, 7 * H // 8))
        specs.append((min(cx, W - 1), cy, n_px, f0))
    t_lo = 0.0
    parts, info, dk = _drones(rng, W, H, specs, t_lo, window_us, per_edge=4)
    x_m = pareto_x_m(mean_per_px)
    counts = _pareto_counts(rng, npx, x_m)
    counts[dk] = rng.poisson(10.0 * window_us * 1e-6, dk.size)
    parts.append(_bursty(rng, np.arange(npx), counts, 0.0, window_us))
    t0 = window * window_us
    meta = dict(config="C3", stream=stream, window=window, x_m=x_m)
    g = grid if grid is not None else hz_grid(0, 2, 750)
    return _assemble(W, H, t0, window_us, parts, g, rng, info, meta)


def config3_batch(n_streams: int = 4, n_windows: int = 8, seed: int = 1003, **kw) -> list:
    return [config3_window(s, w, seed, **kw) for s in range(n_streams) for w in range(n_windows)]


def config4_batch(batch: int = 16, seed: int = 1004, W: int = 640, H: int = 480,
                  window_us: int = 40_000) -> list:
    return [config2(seed * 1000 + b, W=W, H=H, window_us=window_us, grid=hz_grid(0, 2, 750))
            for b in range(batch)]


def config5(seed: int = 1005, W: int = 1280, H: int = 720, window_us: int = 200_000,
            mean_per_px: float = 65.0) -> Scene:
    s = config3_window(0, 0, seed, W=W, H=H, window_us=window_us, mean_per_px=mean_per_px,
                       grid=hz_grid(0, 0.5, 10_000))
    t0 = (1 << 40) - 200_000
    s.t = s.t - np.int64(s.t0) + np.int64(t0)
    s.t0 = t0
    s.meta["config"] = "C5"
    return s


def small_scene(seed: int, W: int = 48, H: int = 40, window_us: int = 20_000,
                n_noise: int = 20_000, drone_px: int = 120, f0_hz: float = 150.0,
                grid=None, extra_invalid: int = 0) -> Scene:
    """A small seeded scene for parity tests: heavy-tailed noise counts, one
    drone, optional out-of-range events (bad x/y/t/p) mixed into the stream."""
    rng = np.random.default_rng(seed)
    npx = W * H
    parts, info, dk = _drones(rng, W, H, [(W // 2, H // 2, drone_px, f0_hz)], 0.0,
                              window_us, per_edge=3)
    x_m = max(n_noise / npx / 3.0, 0.3)
    counts = _pareto_counts(rng, npx, x_m, cap=max(n_noise // 4, 8))
    counts[dk] = 0
    parts.append(_bursty(rng, np.arange(npx), counts, 0.0, window_us))
    g = grid if grid is not None else hz_grid(0, 10, 100)
    s = _assemble(W, H, 0, window_us, parts, g, rng, info, dict(config="small"))
    if extra_invalid:
        m = int(extra_invalid)
        bx = rng.integers(-3, W + 3, m).astype(np.int16)
        by = rng.integers(-3, H + 3, m).astype(np.int16)
        bt = rng.integers(-window_us // 4, window_us + window_us // 4, m).astype(np.int64)
        bp = rng.choice(np.array([-1, 1, 0, 2], np.int8), m)
        at = rng.integers(0, s.n + 1, m)
        s.x = np.insert(s.x, at, bx)
        s.y = np.insert(s.y, at, by)
        s.t = np.insert(s.t, at, bt + s.t0)
        s.p = np.insert(s.p, at, bp)
    return s


def slide_stream(seed: int, W: int = 48, H: int = 40, duration_us: int = 80_000,
                 n_noise: int = 60_000, drone_px: int = 150, f0_hz: float = 150.0,
                 n_hot: int = 3, hot_events: int = 6000, t_base: int = 0, grid=None,
                 extra_invalid: int = 0) -> Scene:
    """A seeded event stream over [t_base, t_base + duration_us) for the
    sliding-window tests: one drone, heavy-tailed bursty noise and n_hot
    pixels with hot_events uniform events each (many per hop), in time order
    up to the generator's granularity; optional invalid events (bad x/y/p)."""
    rng = np.random.default_rng(seed)
    npx = W * H
    parts, info, dk = _drones(rng, W, H, [(W // 2, H // 2, drone_px, f0_hz)], 0.0,
                              duration_us, per_edge=3)
    x_m = max(n_noise / npx / 3.0, 0.3)
    counts = _pareto_counts(rng, npx, x_m, cap=max(n_noise // 8, 8))
    counts[dk] = 0
    parts.append(_bursty(rng, np.arange(npx), counts, 0.0, duration_us))
    if n_hot:
        hot = rng.choice(np.setdiff1d(np.arange(npx), dk), n_hot, replace=False)
        parts.append(_uniform(rng, hot, np.full(n_hot, hot_events), 0.0, duration_us))
    g = grid if grid is not None else hz_grid(0, 10, 100)
    s = _assemble(W, H, t_base, duration_us, parts, g, rng, info, dict(config="stream"))
    if extra_invalid:
        m = int(extra_invalid)
        bx = rng.integers(-3, W + 3, m).astype(np.int16)
        by = rng.integers(-3, H + 3, m).astype(np.int16)
        bp = rng.choice(np.array([-1, 1, 0, 2], np.int8), m)
        bt = rng.integers(0, duration_us, m).astype(np.int64) + t_base
        at = np.searchsorted(s.t, bt)
        s.x = np.insert(s.x, at, bx)
        s.y = np.insert(s.y, at, by)
        s.t = np.insert(s.t, at, bt)
        s.p = np.insert(s.p, at, bp)
    return s


def labelled_scene(seed: int, W: int = 320, H: int = 240, window_us: int = 30_000,
                   mean_per_px: float = 21.7, grid=None, max_drones: int = 3,
                   min_sep: int = 140) -> Scene:
    """A labelled window for detection-quality tests: the C3 noise recipe
    (bursty, Pareto(1.5) per-pixel counts of mean `mean_per_px`) with 1 to
    `max_drones` drones of 60-600 rotor pixels at 100-300 Hz blade-pass,
    centres at least `min_sep` pixels apart. Each drone's ground-truth box
    (``drones[i]["box"]``) circumscribes its rotor pixels."""
    rng = np.random.default_rng(seed)
    npx = W * H
    n_dr = int(rng.integers(1, max_drones + 1))
    specs, centres = [], []
    for _ in range(50 * n_dr):
        if len(specs) == n_dr:
            break
        cx = int(rng.integers(W // 8, W - W // 8))
        cy = int(rng.integers(H // 8, H - H // 8))
        if all((cx - a) ** 2 + (cy - b) ** 2 >= min_sep ** 2 for a, b in centres):
            centres.append((cx, cy))
            specs.append((cx, cy, int(rng.choice([60, 150, 300, 600])),
                          float(rng.uniform(100.0, 300.0))))
    parts, info, dk = _drones(rng, W, H, specs, 0.0, window_us, per_edge=4)
    counts = _pareto_counts(rng, npx, pareto_x_m(mean_per_px))
    counts[dk] = rng.poisson(10.0 * window_us * 1e-6, dk.size)
    parts.append(_bursty(rng, np.arange(npx), counts, 0.0, window_us))
    g = grid if grid is not None else hz_grid(0, 2, 750)
    return _assemble(W, H, 0, window_us, parts, g, rng, info, dict(config="labelled"))


def synthetic_spectra(n_px: int, N: int, seed: int) -> np.ndarray:
    """Seeded FP32 power spectra [n_px, N] for scoring tests: exponential noise
    rows, rows with harmonic combs (one or two fundamentals, peaks spread over
    +-1 bin), rows with repeated values, zero bins and constant rows."""
    rng = np.random.default_rng(seed)
    P = rng.exponential(1.0, (n_px, N)).astype(np.float32)
    kind = rng.integers(0, 6, n_px)
    for i in range(n_px):
        k = kind[i]
        if k in (1, 2):
            for _ in range(k):
                w = int(rng.integers(3, max(4, N // 5)))
                amp = float(rng.uniform(2.0, 40.0))
                for m in range(1, 7):
                    c = m * w + int(rng.integers(-1, 2))
                    if 0 <= c < N:
                        P[i, c] += np.float32(amp * rng.uniform(0.5, 1.0))
        elif k == 3:
            P[i] = np.round(P[i] * 4.0) / 4.0  # many exact ties
        elif k == 4:
            P[i, rng.random(N) < 0.3] = 0.0
        elif k == 5 and rng.random() < 0.3:
            P[i] = np.float32(rng.uniform(0.5, 2.0))  # constant row
    return P


def clustered_spectra(n_px: int, N: int, seed: int) -> np.ndarray:
    """Seeded FP32 spectra [n_px, N] whose middle order statistics are crowded:
    row kinds cycle through (0) zeros below the middle, 40 values spread
    geometrically over two decades across the middle ranks and large values
    above (a middle band spanning many binades), (1) values quantised to a coarse step so that hundreds tie, (2) a
    cluster of 8 distinct values within a few ulps of each other straddling
    the middle rank, (3) 40 values within 1e-4 relative of the median."""
    rng = np.random.default_rng(seed)
    P = rng.exponential(1.0, (n_px, N)).astype(np.float32)
    for i in range(n_px):
        k = i % 4
        row = P[i]
        if k == 0:
            perm = rng.permutation(N)
            n0 = N // 2 - 20
            big = rng.uniform(50.0, 60.0, N - n0 - 40)
            mean = big.sum() / N
            row[perm[:n0]] = 0.0
            row[perm[n0:n0 + 40]] = (mean * np.geomspace(0.005, 0.5, 40)
                                     * rng.uniform(0.99, 1.01, 40)).astype(np.float32)
            row[perm[n0 + 40:]] = big.astype(np.float32)
        elif k == 1:
            row[:] = np.round(row * 2.0) / 2.0
        else:
            order = np.argsort(row, kind="stable")
            mid = N // 2 - int(rng.integers(0, 12))
            m = float(row[order[mid]])
            width = 8 if k == 2 else 40
            idx = order[max(0, mid - width // 2):mid + width // 2]
            rel = 1e-6 if k == 2 else 1e-4
            row[idx] = (m * (1.0 + rel * rng.random(idx.size))).astype(np.float32)
    return P

