"""Sliding-window spectra (Sec. 3.3: each event's terms added as it arrives,
subtracted as it leaves) against the FP64 oracle evaluated from scratch on
the events of each window.

The reference window is bookkeeping only: the events a push keeps are those
with max(t_prev, t_end - T) <= t < t_end on the sensor with a valid
polarity, and the window at t_end holds the kept events with t >= t_end - T.
Spectra must match the oracle within 1e-4 of each pixel's peak power after
every push, whatever the rebuild period; detection is compared as for
ddhf_detect (rotor decisions outside the score margins, boxes when no pixel
is within a margin)."""
import numpy as np
import pytest
import torch

import oracle
import oracle_margins
from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu

TOL_SPEC = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_08386_gb300 import build
    build.build()
    oracle.build()
    ddhf.load()
    assert torch.cuda.is_available()
    yield


def kept(x, y, t, p, W, H, t_lo, t_end, pol01=False):
    okp = (p == 0) | (p == 1) if pol01 else (p == 1) | (p == -1)
    return okp & (x >= 0) & (x < W) & (y >= 0) & (y < H) & (t >= t_lo) & (t < t_end)


class Pushes:
    """Pushes of a stream scene with hop `hop`: push i carries the events of
    [t_prev - late_us, t_end) (the late part was in the previous push and must
    be dropped), optionally shuffled."""

    def __init__(self, s, T, hop, late_us=300, shuffle_seed=None):
        self.s, self.T, self.hop, self.late = s, T, hop, late_us
        self.rng = np.random.default_rng(shuffle_seed) if shuffle_seed is not None else None
        self.t_end = s.t0
        self.acc = [np.zeros(0, a.dtype) for a in (s.x, s.y, s.t, s.p)]

    def next(self, t_end=None, empty=False):
        s = self.s
        t_prev = self.t_end
        t_end = t_prev + self.hop if t_end is None else t_end
        sel = np.flatnonzero((s.t >= t_prev - self.late) & (s.t < t_end))
        if empty:
            sel = sel[:0]
        if self.rng is not None:
            sel = self.rng.permutation(sel)
        ev = [a[sel] for a in (s.x, s.y, s.t, s.p)]
        k = kept(*ev, s.W, s.H, max(t_prev, t_end - self.T), t_end)
        self.acc = [np.concatenate([a, e[k]]) for a, e in zip(self.acc, ev)]
        self.t_end = t_end
        return ev, t_end, int(k.sum()), int(len(sel) - k.sum())

    def window(self):
        x, y, t, p = self.acc
        w = t >= self.t_end - self.T
        return x[w], y[w], t[w], p[w]


def push(c, ev, t_end):
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in ev]
    c.slide_push(d[0], d[1], d[2], d[3], t_end)


def check_spectra(c, pu, params):
    s = pu.s
    act, P = c.slide_spectra()
    act, P = act.cpu().numpy(), P.cpu().numpy()
    x, y, t, p = pu.window()
    o = oracle.bin_events(s.W, s.H, x, y, t, p, pu.t_end - pu.T, pu.T)
    want = np.flatnonzero(o["counts"] >= params.n_min)
    np.testing.assert_array_equal(act, want)
    worst = 0.0
    for a, k in enumerate(act):
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        ref = oracle.ndft(o["tau"][o0:o1], o["pol"][o0:o1], *s.grid)
        worst = max(worst, np.abs(P[a].astype(np.float64) - ref).max() / max(ref.max(), 1e-30))
    assert worst <= TOL_SPEC, worst
    st = c.slide_stats()
    assert st["n_window"] == len(t)
    return len(act)


@pytest.mark.parametrize("rebuild_every", [0, 1, 3])
@pytest.mark.parametrize("nb,step", [(100, 10), (750, 2), (2000, 1)])
def test_slide_spectra_every_push(rebuild_every, nb, step):
    T, hop = 20_000, 5_000
    s = synth.slide_stream(41 + nb, duration_us=70_000, t_base=(1 << 40) - 30_000,
                           grid=synth.hz_grid(0, step, nb), extra_invalid=400)
    params = ddhf.default_params()
    c = ddhf.Context(s.W, s.H, s.grid, params, max_events=s.n)
    c.slide_begin(T, s.t0, capacity=s.n, rebuild_every=rebuild_every)
    pu = Pushes(s, T, hop)
    added = dropped = 0
    n_push = 70_000 // hop
    for i in range(n_push):
        ev, t_end, k, d = pu.next()
        push(c, ev, t_end)
        added += k
        dropped += d
        if i % 3 == 2 or i == n_push - 1:
            assert check_spectra(c, pu, params) > 100
    st = c.slide_stats()
    assert st["n_added"] == added and st["n_dropped"] == dropped
    assert st["pushes"] == n_push
    assert st["rebuilds"] == (n_push // rebuild_every if rebuild_every else 0)
    assert st["n_expired"] == added - st["n_window"]
    c.stats()
    c.close()


def test_slide_heavy_pixels_take_the_block_path():
    # 3 pixels with 12000 events over 60 ms: ~1000 events enter and ~1000
    # leave per 5 ms hop, far above the whole-block threshold
    T, hop = 20_000, 5_000
    s = synth.slide_stream(77, duration_us=60_000, n_hot=3, hot_events=12_000,
                           grid=synth.hz_grid(0, 2, 750))
    params = ddhf.default_params()
    c = ddhf.Context(s.W, s.H, s.grid, params, max_events=s.n)
    c.slide_begin(T, s.t0, capacity=s.n, rebuild_every=0)
    pu = Pushes(s, T, hop)
    for _ in range(60_000 // hop):
        ev, t_end, _, _ = pu.next()
        push(c, ev, t_end)
        assert c.slide_stats()["last_delta"] > 0
    check_spectra(c, pu, params)
    c.close()


def test_slide_unordered_pushes_empty_pushes_and_long_hops():
    T = 20_000
    s = synth.slide_stream(5, duration_us=120_000, t_base=123_456, extra_invalid=200)
    params = ddhf.default_params()
    c = ddhf.Context(s.W, s.H, s.grid, params, max_events=s.n)
    c.slide_begin(T, s.t0, capacity=s.n, rebuild_every=0)
    pu = Pushes(s, T, 4_000, shuffle_seed=9)
    for _ in range(6):
        push(c, *pu.next()[:2])
    check_spectra(c, pu, params)
    # empty pushes: events only leave
    for _ in range(2):
        ev, t_end, k, _ = pu.next(empty=True)
        assert k == 0
        push(c, ev, t_end)
    check_spectra(c, pu, params)
    # a hop longer than the window: everything leaves, only the newest stay
    push(c, *pu.next(t_end=pu.t_end + 2 * T + 700)[:2])
    check_spectra(c, pu, params)
    st = c.slide_stats()
    assert st["n_window"] == len(pu.window()[2])
    # a push with t_end equal to the previous end keeps the window
    push(c, *pu.next(t_end=pu.t_end)[:2])
    check_spectra(c, pu, params)
    for _ in range(5):
        push(c, *pu.next()[:2])
    check_spectra(c, pu, params)
    c.close()


def test_slide_equals_itself_bitwise_and_restarts():
    T = 20_000
    s = synth.slide_stream(13, duration_us=50_000, grid=synth.hz_grid(0, 2, 750))
    out = []
    for _ in range(2):
        c = ddhf.Context(s.W, s.H, s.grid, None, max_events=s.n)
        c.slide_begin(T, s.t0, capacity=s.n, rebuild_every=4)
        pu = Pushes(s, T, 5_000)
        for _ in range(10):
            push(c, *pu.next()[:2])
        out.append(c.slide_spectra()[1].cpu().numpy())
        # begin again on the same context: a fresh, zero state
        c.slide_begin(T, s.t0, capacity=s.n, rebuild_every=0)
        pu = Pushes(s, T, 5_000)
        for _ in range(3):
            push(c, *pu.next()[:2])
        check_spectra(c, pu, ddhf.default_params())
        c.slide_end()
        c.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_slide_capacity_and_state_errors():
    T = 20_000
    s = synth.slide_stream(17, duration_us=40_000)
    params = ddhf.default_params()
    c = ddhf.Context(s.W, s.H, s.grid, params, max_events=s.n)
    with pytest.raises(ddhf.DDHFError) as e:
        push(c, [a[:0] for a in (s.x, s.y, s.t, s.p)], s.t0 + 10)
    assert e.value.status == 6
    with pytest.raises(ddhf.DDHFError) as e:
        c.slide_begin(T, s.t0, capacity=s.n + 1)
    assert e.value.status == 1
    pu = Pushes(s, T, 5_000)
    first = pu.next()
    cap = len(first[0][0]) + 10
    c.slide_begin(T, s.t0, capacity=cap, rebuild_every=0)
    push(c, *first[:2])
    # the next push does not fit: nothing happens, the window stays
    nxt = pu.next()
    with pytest.raises(ddhf.DDHFError) as e:
        push(c, *nxt[:2])
    assert e.value.status == 3
    st = c.slide_stats()
    assert st["pushes"] == 1 and st["t_end_us"] == first[1]
    with pytest.raises(ddhf.DDHFError) as e:
        push(c, nxt[0], first[1] - 1)
    assert e.value.status == 1
    c.slide_end()
    with pytest.raises(ddhf.DDHFError) as e:
        c.slide_stats()
    assert e.value.status == 6
    c.close()


def test_slide_detect_matches_oracle():
    T, hop = 20_000, 2_500
    s = synth.slide_stream(23, duration_us=60_000, drone_px=200, n_noise=50_000,
                           grid=synth.hz_grid(0, 10, 100))
    params = ddhf.default_params()
    c = ddhf.Context(s.W, s.H, s.grid, params, max_events=s.n)
    c.slide_begin(T, s.t0, capacity=s.n, rebuild_every=16)
    pu = Pushes(s, T, hop)
    for i in range(60_000 // hop):
        push(c, *pu.next()[:2])
        if i % 6 != 5:
            continue
        bx, nb, mask = c.slide_detect(cap=256, want_mask=True)
        sc = c.scores()
        x, y, t, p = pu.window()
        prm = dict(tau_sf=0.89, tau_comb=1.5, M=4, d=3, h_min=4)
        b = oracle.bin_events(s.W, s.H, x, y, t, p, pu.t_end - T, T)
        act = sc["active"].cpu().numpy().astype(np.int64)
        np.testing.assert_array_equal(act, np.flatnonzero(b["counts"] >= 6))
        P32 = c.slide_spectra()[1].cpu().numpy()  # |F|^2 of the state the comb scored
        rot, close = oracle_margins.decisions(b, act, P32, s.grid, prm)
        assert close.mean() < 0.01
        gm = mask.cpu().numpy()
        np.testing.assert_array_equal(gm[act[~close]], rot[~close].astype(np.uint8))
        n = int(nb.item())
        np.testing.assert_array_equal(bx[:n].cpu().numpy(),
                                      oracle_margins.segment(gm, s.W, s.H, 147, 19.05, cap=256))
        if not close.any():
            om = np.zeros(s.W * s.H, np.uint8)
            om[act[rot]] = 1
            np.testing.assert_array_equal(
                bx[:n].cpu().numpy(), oracle_margins.segment(om, s.W, s.H, 147, 19.05, cap=256))
    c.stats()
    c.close()


def test_slide_full_size_c3_stream_sampled():
    # one C3 stream (1280x720, Pareto(1.5) counts, ~20M events per 30 ms):
    # the window slides by 3.75 ms over 4 consecutive windows; after the last
    # push a seeded sample of pixels is checked against the oracle
    T, hop = 30_000, 3_750
    wins = [synth.config3_window(stream=0, window=w) for w in range(4)]
    W, H, grid = wins[0].W, wins[0].H, wins[0].grid
    x = np.concatenate([w.x for w in wins])
    y = np.concatenate([w.y for w in wins])
    t = np.concatenate([w.t for w in wins])
    p = np.concatenate([w.p for w in wins])
    t0 = wins[0].t0
    order = np.argsort(t, kind="stable")
    x, y, t, p = x[order], y[order], t[order], p[order]
    n_push = (4 * T - T // 2) // hop
    fill = T // hop
    bounds = np.searchsorted(t, t0 + hop * np.arange(n_push + 1))
    cap = int(max(bounds[min(i + fill + 1, n_push)] - bounds[i] for i in range(n_push)) * 1.05)
    params = ddhf.default_params()
    c = ddhf.Context(W, H, grid, params, max_events=cap)
    c.slide_begin(T, t0, capacity=cap, rebuild_every=64)
    dx, dy, dt, dp = (torch.from_numpy(a).cuda() for a in (x, y, t, p))
    for i in range(n_push):
        lo, hi = int(bounds[i]), int(bounds[i + 1])
        c.slide_push(dx[lo:hi], dy[lo:hi], dt[lo:hi], dp[lo:hi], t0 + hop * (i + 1))
    t_end = t0 + hop * n_push
    act, P = c.slide_spectra()
    st = c.slide_stats()
    w = (t >= t_end - T) & (t < t_end)
    assert st["n_window"] == int(w.sum())
    o = oracle.bin_events(W, H, x[w], y[w], t[w], p[w], t_end - T, T)
    want = np.flatnonzero(o["counts"] >= params.n_min)
    act = act.cpu().numpy()
    np.testing.assert_array_equal(act, want)
    rng = np.random.default_rng(3)
    heavy = np.argsort(o["counts"][act])[-8:]
    rows = np.concatenate([rng.choice(len(act), 56, replace=False), heavy])
    Ph = P[torch.from_numpy(rows).cuda()].cpu().numpy()
    for r, a in enumerate(rows):
        k = act[a]
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        ref = oracle.ndft(o["tau"][o0:o1], o["pol"][o0:o1], *grid)
        err = np.abs(Ph[r].astype(np.float64) - ref).max() / max(ref.max(), 1e-30)
        assert err <= TOL_SPEC, (k, o1 - o0, err)
    c.close()
