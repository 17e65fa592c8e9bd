"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars: binning, labels and boxes bit-exact; spectra within 1e-4 of each
pixel's peak power; comb scores bit-exact against the oracle's FP32
restatement on the same (generator-made) spectra; rotor decisions equal to
the FP64 oracle's outside a stated margin.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import oracle_margins
from paper_2603_08386_gb300 import ddhf, synth

pytestmark = pytest.mark.gpu

TOL_SPEC = 1e-4      # max_j |P_gpu - P_oracle| <= TOL_SPEC * max_j P_oracle, per pixel
# the SF decision on a given FP32 spectrum is compared with the FP64 oracle's
# on the same spectrum wherever |ln SF - ln tau_sf| exceeds this (the FP32
# arithmetic of Eq. 7); against the oracle's own FP64 spectrum the margins
# also take the spectrum's difference into account (oracle_margins)
SF_MARGIN = 1e-5
D9 = synth.HZ_DENOM


@pytest.fixture(scope="session", autouse=True)
def built():
    from paper_2603_08386_gb300 import build
    build.build()
    oracle.build()
    ddhf.load()
    assert torch.cuda.is_available()
    yield


def ctx_for(scene, params=None, max_events=None, max_windows=1, **tuning):
    c = ddhf.Context(scene.W, scene.H, scene.grid, params,
                     max_events=max(max_events or scene.n, 1), max_windows=max_windows)
    if tuning:
        c.set_tuning(**tuning)
    return c


def decode(ev):
    u = ev.cpu().numpy().view(np.uint32)
    return (u & 0x7FFFFFFF).astype(np.int64), np.where(u >> 31, -1, 1).astype(np.int8)


def oracle_bin(scene, polarity_01=False):
    return oracle.bin_events(scene.W, scene.H, scene.x, scene.y, scene.t, scene.p, scene.t0,
                             scene.window_us, polarity_01)


def check_binning(scene, params=None):
    c = ctx_for(scene, params)
    x, y, t, p = ddhf.events_to_device(scene)
    c.bin_events(x, y, t, p, scene.t0, scene.window_us)
    g = c.csr()
    o = oracle_bin(scene, bool(params.polarity_01) if params is not None else False)
    n_min = params.n_min if params is not None else 6
    assert g["n_valid"] == o["n_valid"] and g["n_dropped"] == o["n_dropped"]
    assert g["n_in"] == scene.n
    np.testing.assert_array_equal(g["offsets"].cpu().numpy().astype(np.int64), o["offsets"])
    tau, pol = decode(g["ev"])
    np.testing.assert_array_equal(tau, o["tau"])
    np.testing.assert_array_equal(pol, o["pol"])
    act = np.flatnonzero(o["counts"] >= n_min)
    np.testing.assert_array_equal(g["active"].cpu().numpy().astype(np.int64), act)
    st = c.stats()
    assert st["terms"] == int(o["counts"][act].sum()) * scene.grid[3]
    c.close()
    return o


# ------------------------------------------------------------------ binning

@pytest.mark.parametrize("W,H,seed", [(40, 30, 1), (128, 128, 2), (97, 61, 3), (3000, 2000, 4)])
def test_binning_bit_exact(W, H, seed):
    # 1, 2 and 3 radix passes (key widths 11, 14, 13 and 23 bits), ragged chunks,
    # invalid events (bad x, y, t, p) mixed into the stream
    s = synth.small_scene(seed, W=W, H=H, n_noise=60_000, drone_px=80, extra_invalid=3000)
    check_binning(s)


def test_binning_empty_and_single_pixel():
    s = synth.small_scene(5, W=33, H=17, n_noise=100)
    e = synth.Scene(W=33, H=17, t0=0, window_us=1000, x=s.x[:0], y=s.y[:0], t=s.t[:0],
                    p=s.p[:0], grid=s.grid)
    check_binning(e)
    n = 20_000  # all events on one pixel, duplicate timestamps, window edges
    rng = np.random.default_rng(6)
    t = rng.integers(0, 1000, n).astype(np.int64)
    t[:3] = [0, 999, 1000]  # 1000 = t0 + W is outside
    one = synth.Scene(W=33, H=17, t0=0, window_us=1000, x=np.full(n, 7, np.int16),
                      y=np.full(n, 9, np.int16), t=t, p=rng.choice(np.array([-1, 1], np.int8), n),
                      grid=s.grid)
    o = check_binning(one)
    assert o["n_dropped"] == 1


def test_binning_polarity_01():
    s = synth.small_scene(7, W=50, H=40, n_noise=20_000)
    s.p = ((s.p + 1) // 2).astype(np.int8)  # {-1, 1} -> {0, 1}
    check_binning(s, ddhf.default_params(polarity_01=1))


# ------------------------------------------------------------------ spectra

def spectra_case(scene, form, pixels=None, **tuning):
    c = ctx_for(scene, **tuning)
    x, y, t, p = ddhf.events_to_device(scene)
    c.bin_events(x, y, t, p, scene.t0, scene.window_us)
    P = c.power_spectrum(form).cpu().numpy()
    act = c.csr()["active"].cpu().numpy()
    c.stats()
    c.close()
    o = oracle_bin(scene)
    rows = range(len(act)) if pixels is None else pixels
    worst = 0.0
    for a in rows:
        k = act[a]
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        ref = oracle.ndft(o["tau"][o0:o1], o["pol"][o0:o1], *scene.grid)
        err = np.abs(P[a].astype(np.float64) - ref).max() / max(ref.max(), 1e-30)
        worst = max(worst, err)
    return worst, P, act


@pytest.mark.parametrize("form", ["sincos", "recur", "kahan", "blocked", "f64"])
@pytest.mark.parametrize("nb", [100, 37, 333])
def test_spectrum_forms_small(form, nb):
    s = synth.small_scene(11 + nb, W=24, H=20, n_noise=9_000, drone_px=60,
                          grid=synth.hz_grid(0, 10, nb))
    worst, _, act = spectra_case(s, form)
    assert len(act) > 50
    assert worst <= (1e-6 if form == "f64" else TOL_SPEC), worst  # f64 stored as FP32


@pytest.mark.parametrize("nb,step", [(750, 2), (2000, 1)])
def test_spectrum_blocked_passes_and_heavy_path(nb, step):
    # 2000 bins: two row passes per pixel; heavy_min=32 sends pixels with at
    # least 32 events through the whole-block path (events split over warps)
    s = synth.small_scene(23, W=30, H=20, n_noise=30_000, drone_px=60,
                          grid=synth.hz_grid(0, step, nb))
    worst, _, act = spectra_case(s, "blocked", heavy_min=32)
    assert worst <= TOL_SPEC, worst
    worst2, _, _ = spectra_case(s, "recur")
    assert worst2 <= TOL_SPEC, worst2


def test_spectrum_mode_grid():
    s = synth.small_scene(29, W=20, H=20, n_noise=6000, window_us=33_333)
    s.grid = synth.mode_grid(33_333, 120)
    for form in ("blocked", "sincos"):
        worst, _, _ = spectra_case(s, form)
        assert worst <= TOL_SPEC, (form, worst)


def test_spectrum_capacity_flag():
    s = synth.small_scene(31, W=20, H=20, n_noise=5000)
    c = ctx_for(s)
    x, y, t, p = ddhf.events_to_device(s)
    c.bin_events(x, y, t, p, s.t0, s.window_us)
    na = c.n_active()
    P = torch.empty((na, s.grid[3]), dtype=torch.float32, device="cuda")
    ddhf.ddhf_power_spectrum(c.h, ddhf.FORM["blocked"], P, na // 2)
    st = c.stats(raise_on_flags=False)
    assert st["status"] == 3 and st["device_flags"] & ddhf.FLAG_CAPACITY
    c.close()


# ------------------------------------------------------------------ comb

@pytest.mark.parametrize("N,M,d,h_min,kind", [(750, 4, 3, 4, "mixed"), (100, 4, 3, 4, "mixed"),
                                              (333, 6, 2, 3, "mixed"), (200, 16, 4, 8, "mixed"),
                                              (64, 2, 0, 1, "mixed"), (1024, 4, 3, 4, "mixed"),
                                              (1025, 4, 3, 4, "mixed"),
                                              (750, 4, 3, 4, "clustered"),
                                              (1024, 4, 3, 4, "clustered"),
                                              (331, 6, 2, 3, "clustered")])
def test_comb_bit_exact_on_generated_spectra(N, M, d, h_min, kind):
    # the comb's input spectra come from the seeded generators; GPU and the
    # oracle's FP32 restatement must agree bit for bit. "clustered" rows crowd
    # the middle order statistics (ties, near-equal values, a median among
    # zeros and tiny values), the cases the fast selection hands to its exact
    # radix fallback.
    n_px = 600
    W, H = 40, 15  # 600 pixels, one event each -> every pixel active (n_min = 1)
    params = ddhf.default_params(M=M, d=d, h_min=h_min, n_min=1)
    s = synth.Scene(W=W, H=H, t0=0, window_us=100, x=(np.arange(n_px) % W).astype(np.int16),
                    y=(np.arange(n_px) // W).astype(np.int16), t=np.zeros(n_px, np.int64),
                    p=np.ones(n_px, np.int8), grid=synth.hz_grid(0, 1, N))
    c = ctx_for(s, params)
    x, y, t, p = ddhf.events_to_device(s)
    c.bin_events(x, y, t, p, 0, 100)
    assert c.n_active() == n_px
    gen = synth.synthetic_spectra if kind == "mixed" else synth.clustered_spectra
    Pn = gen(n_px, N, seed=N + M)
    out = c.comb_score(torch.from_numpy(Pn).cuda())
    lsf = out["log_sf"].cpu().numpy()
    snr = out["snr"].cpu().numpy()
    f0 = out["f0_bin"].cpu().numpy()
    mask = out["mask"].cpu().numpy()
    c.close()
    ln_tau = math.log(0.89)
    checked = 0
    for a in range(n_px):
        lo = oracle.log_sf(Pn[a].astype(np.float64))
        assert abs(lsf[a] - lo) <= 1e-4 * max(1.0, abs(lo)), (a, lsf[a], lo)
        gpu_pass = f0[a] >= 0 or snr[a] != 0
        if abs(lo - ln_tau) > SF_MARGIN:
            assert (lsf[a] <= np.float32(ln_tau)) == (lo <= ln_tau), a
        if lsf[a] <= np.float32(ln_tau):
            s32, w32 = oracle.comb_f32(Pn[a], M=M, d=d, h_min=h_min)
            assert w32 == f0[a], (a, w32, f0[a])
            assert np.float32(s32).view(np.uint32) == np.float32(snr[a]).view(np.uint32), \
                (a, s32, snr[a])
            assert mask[a] == (1 if (w32 >= 0 and s32 >= np.float32(1.5)) else 0)
            checked += 1
        else:
            assert not gpu_pass and mask[a] == 0
    assert checked > n_px // 3


# ------------------------------------------------------------------ labels and boxes

@pytest.mark.parametrize("seed,density", [(1, 0.05), (2, 0.3), (3, 0.55), (4, 0.75)])
def test_label_and_boxes_bit_exact(seed, density):
    rng = np.random.default_rng(seed)
    W, H = 301, 157
    blob = rng.random((H // 4 + 1, W // 4 + 1)) < density
    mask = np.kron(blob, np.ones((4, 4), bool))[:H, :W] & (rng.random((H, W)) < 0.9)
    mask = mask.astype(np.uint8)
    s = synth.Scene(W=W, H=H, t0=0, window_us=10, x=np.zeros(0, np.int16),
                    y=np.zeros(0, np.int16), t=np.zeros(0, np.int64), p=np.zeros(0, np.int8),
                    grid=synth.hz_grid(0, 10, 10))
    for A_min, alpha in ((1, 0.5), (16, 2.0), (147, 19.05)):
        c = ctx_for(s, ddhf.default_params(A_min=A_min, alpha=alpha))
        lab = c.label(torch.from_numpy(mask.ravel()).cuda())
        ref, _ = oracle.ccl8(mask.ravel(), W, H)
        np.testing.assert_array_equal(lab.cpu().numpy(), ref)
        bx, n = c.boxes(lab, cap=8192)
        rb = oracle.boxes(ref, W, H, A_min=A_min, alpha=alpha, cap=8192)
        assert n == rb.shape[0]
        np.testing.assert_array_equal(bx.cpu().numpy(), rb)
        c.stats()
        c.close()


def _structured_masks(W, H, rng):
    yy, xx = np.mgrid[0:H, 0:W]
    out = {
        "full": np.ones((H, W), bool),
        "checkerboard": (xx + yy) % 2 == 0,      # connected through diagonals only
        "anti-diagonals": (xx + yy) % 3 == 0,    # separate diagonal lines
        "diagonals": (xx - yy) % 4 == 0,
        "rows": yy % 2 == 0,
        "columns": xx % 2 == 0,
        "staircase": (xx // 2) == (yy % (W // 2)),
        "single pixels": (xx % 2 == 0) & (yy % 2 == 0),
        "dense noise": rng.random((H, W)) < 0.6,
        "sparse noise": rng.random((H, W)) < 0.3,
    }
    # a ring with a gap closed only by one diagonal step, and an X
    ring = np.zeros((H, W), bool)
    ring[5, 5:40] = ring[30, 5:40] = ring[5:31, 5] = ring[5:31, 39] = True
    ring[30, 20] = False
    ring[31, 20] = True
    x_shape = (np.abs(xx - yy) == 0) | (np.abs(xx + yy - (H - 1)) == 0)
    out["ring with a diagonal bridge"] = ring
    out["cross of diagonals"] = x_shape & (xx < H)
    return out


def test_label_structured_masks_bit_exact():
    # diagonal-only connections and every left / up / up-left / up-right
    # neighbour pattern, against the oracle's breadth-first labelling
    W, H = 97, 61
    rng = np.random.default_rng(11)
    s = synth.Scene(W=W, H=H, t0=0, window_us=10, x=np.zeros(0, np.int16),
                    y=np.zeros(0, np.int16), t=np.zeros(0, np.int64), p=np.zeros(0, np.int8),
                    grid=synth.hz_grid(0, 10, 10))
    c = ctx_for(s)
    for name, m in _structured_masks(W, H, rng).items():
        mask = m.astype(np.uint8).ravel()
        lab = c.label(torch.from_numpy(mask).cuda())
        ref, _ = oracle.ccl8(mask, W, H)
        np.testing.assert_array_equal(lab.cpu().numpy(), ref, err_msg=name)
    c.stats()
    c.close()


def test_boxes_cap_and_hand_cases():
    W, H = 80, 10
    m = np.zeros((H, W), np.uint8)
    m[0:3, 0:3] = 1
    m[0:3, 30:33] = 1
    m[7:9, 60:62] = 1
    s = synth.Scene(W=W, H=H, t0=0, window_us=10, x=np.zeros(0, np.int16),
                    y=np.zeros(0, np.int16), t=np.zeros(0, np.int64), p=np.zeros(0, np.int8),
                    grid=synth.hz_grid(0, 10, 10))
    for alpha in (10.0, 10.0 + 1e-9, 3.0):
        c = ctx_for(s, ddhf.default_params(A_min=1, alpha=alpha))
        lab = c.label(torch.from_numpy(m.ravel()).cuda())
        bx, n = c.boxes(lab, cap=1)
        rb = oracle.boxes(oracle.ccl8(m.ravel(), W, H)[0], W, H, A_min=1, alpha=alpha)
        assert n == rb.shape[0]
        np.testing.assert_array_equal(bx.cpu().numpy(), rb[:1])
        st = c.stats(raise_on_flags=False)
        assert (st["status"] == 3) == (n > 1)
        c.close()


# ------------------------------------------------------------------ whole window

def test_detect_c1_matches_oracle():
    # C1 with Table 2's values: the FP64 oracle's rotor bit of every active
    # pixel outside its margins, the boxes always against the oracle's
    # segmentation of the GPU mask, and against the oracle's own boxes when
    # no pixel is inside a margin
    s = synth.config1()
    prm = dict(tau_sf=0.89, tau_comb=1.5, M=4, d=3, h_min=4, A_min=147, alpha=19.05)
    c = ctx_for(s)
    x, y, t, p = ddhf.events_to_device(s)
    bx, nb, mask = c.detect(x, y, t, p, s.t0, s.window_us, cap=256, want_mask=True)
    sc = c.scores()
    P32 = c.power_spectrum("blocked").cpu().numpy()
    c.stats()
    c.close()
    b = oracle_bin(s)
    act = sc["active"].cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(act, np.flatnonzero(b["counts"] >= 6))
    gm = mask.cpu().numpy()
    n = int(nb.item())
    np.testing.assert_array_equal(bx[:n].cpu().numpy(),
                                  oracle_margins.segment(gm, s.W, s.H, 147, 19.05, cap=256))
    rot, close = oracle_margins.decisions(b, act, P32, s.grid, prm)
    assert close.mean() < 0.01
    np.testing.assert_array_equal(gm[act[~close]], rot[~close].astype(np.uint8))
    if not close.any():
        om = np.zeros(s.W * s.H, np.uint8)
        om[act[rot]] = 1
        np.testing.assert_array_equal(bx[:n].cpu().numpy(),
                                      oracle_margins.segment(om, s.W, s.H, 147, 19.05, cap=256))


@pytest.mark.parametrize("nb,step", [(750, 2), (2000, 1)])
def test_fused_equals_unfused_bitwise(nb, step):
    # 750 bins: the fast comb; 2000 bins: the generic comb (fused kernel and
    # separate comb kernel alike)
    s = synth.small_scene(41, W=64, H=48, n_noise=60_000, drone_px=150,
                          grid=synth.hz_grid(0, step, nb))
    for heavy_min in (32, 1024):
        c = ctx_for(s, heavy_min=heavy_min, fuse=1)
        x, y, t, p = ddhf.events_to_device(s)
        bx, nb, mask = c.detect(x, y, t, p, s.t0, s.window_us, want_mask=True)
        sc = c.scores()
        P = c.power_spectrum("blocked")
        out = c.comb_score(P)
        c.stats()
        c.close()
        assert torch.equal(out["mask"], mask)
        assert torch.equal(out["f0_bin"], sc["f0_bin"])
        assert torch.equal(out["snr"].view(torch.int32), sc["snr"].view(torch.int32))
        assert torch.equal(out["log_sf"].view(torch.int32), sc["log_sf"].view(torch.int32))
        # the unfused detection path (spectrum kernel + comb kernel per window)
        c2 = ctx_for(s, heavy_min=heavy_min, fuse=0)
        bx2, nb2, mask2 = c2.detect(x, y, t, p, s.t0, s.window_us, want_mask=True)
        sc2 = c2.scores()
        c2.stats()
        c2.close()
        assert torch.equal(mask2, mask) and torch.equal(sc2["f0_bin"], sc["f0_bin"])
        assert torch.equal(sc2["snr"].view(torch.int32), sc["snr"].view(torch.int32))
        assert int(nb2.item()) == int(nb.item())
        assert torch.equal(bx2[: int(nb.item())], bx[: int(nb.item())])


def test_batch_graph_equals_single_windows():
    scenes = [synth.small_scene(50 + i, W=48, H=40, n_noise=20_000 + 3000 * i, drone_px=120,
                                grid=synth.hz_grid(0, 2, 750)) for i in range(5)]
    W, H = 48, 40
    maxev = max(sc.n for sc in scenes)
    cap = 64
    single = []
    c1 = ddhf.Context(W, H, scenes[0].grid, max_events=maxev)
    for sc in scenes:
        bx, nb, m = c1.detect(*ddhf.events_to_device(sc), sc.t0, sc.window_us, cap=cap,
                              want_mask=True)
        single.append((bx[: int(nb.item())].clone(), m.clone()))
    c1.stats()
    c1.close()
    cb = ddhf.Context(W, H, scenes[0].grid, max_events=maxev, max_windows=len(scenes))
    dev = [ddhf.events_to_device(sc) for sc in scenes]
    wins = [(d[0], d[1], d[2], d[3], sc.n, sc.t0, sc.window_us) for d, sc in zip(dev, scenes)]
    boxes = torch.empty((len(scenes) * cap, 5), dtype=torch.int32, device="cuda")
    nbx = torch.zeros(len(scenes), dtype=torch.int32, device="cuda")
    masks = torch.empty((len(scenes), W * H), dtype=torch.uint8, device="cuda")
    ddhf.ddhf_enable_stage_timing(cb.h, True)
    for fuse, overlap, use_graph in ((1, 0, False), (1, 0, True), (1, 0, True), (0, 0, False),
                                     (0, 0, True), (0, 0, True), (0, 1, False), (0, 1, True),
                                     (0, 1, True)):
        cb.set_tuning(fuse=fuse, overlap=overlap)
        boxes.fill_(-7)
        masks.fill_(3)
        ddhf.ddhf_detect_batch(cb.h, wins, boxes, cap, nbx, masks, use_graph=use_graph)
        times = ddhf.ddhf_stage_times(cb.h)
        assert all(t > 0 for t in times[:3])
        if fuse:
            assert times[3] == times[4] == 0.0
        else:
            assert times[3] > 0 and times[4] > 0
        torch.cuda.synchronize()
        for i, (bref, mref) in enumerate(single):
            n = int(nbx[i].item())
            assert torch.equal(boxes[i * cap: i * cap + n], bref)
            assert torch.equal(masks[i], mref)
    st = cb.stats()
    assert st["graph_kernels"] > 3 * len(scenes)
    cb.close()


def test_detect_empty_window():
    s = synth.small_scene(60, W=32, H=32, n_noise=100)
    c = ctx_for(s)
    x, y, t, p = ddhf.events_to_device(s)
    bx, nb, mask = c.detect(x[:0], y[:0], t[:0], p[:0], 0, 1000, want_mask=True)
    st = c.stats()
    assert int(nb.item()) == 0 and int(mask.sum().item()) == 0
    assert st["n_active"] == 0 and st["n_valid"] == 0
    c.close()


def test_invalid_arguments_raise():
    s = synth.small_scene(61, W=32, H=32, n_noise=1000)
    c = ctx_for(s)
    x, y, t, p = ddhf.events_to_device(s)
    with pytest.raises(ddhf.DDHFError) as e:
        ddhf.ddhf_bin_events(c.h, x, y, t, p, s.n + 10**9, 0, 1000)
    assert e.value.status == 1
    with pytest.raises(ddhf.DDHFError) as e:
        ddhf.ddhf_bin_events(c.h, x, y, t, p, s.n, 0, 0)
    assert e.value.status == 1
    c.close()


# ------------------------------------------------------------------ full size (1280x720)

def test_c3_window_full_size_sampled():
    s = synth.config3_window(stream=1, window=3)
    o = oracle_bin(s)
    c = ctx_for(s, max_windows=1)
    x, y, t, p = ddhf.events_to_device(s)
    c.bin_events(x, y, t, p, s.t0, s.window_us)
    g = c.csr()
    np.testing.assert_array_equal(g["offsets"].cpu().numpy().astype(np.int64), o["offsets"])
    tau, pol = decode(g["ev"])
    np.testing.assert_array_equal(tau, o["tau"])
    np.testing.assert_array_equal(pol, o["pol"])
    act = g["active"].cpu().numpy()
    counts = o["counts"][act]
    rng = np.random.default_rng(3)
    sample = np.unique(np.concatenate([np.argsort(-counts, kind="stable")[:12],
                                       rng.choice(len(act), 150, replace=False),
                                       np.flatnonzero(np.isin(act, s.drones[2]["keys"]))[:40]]))
    P = c.power_spectrum("blocked").cpu().numpy()
    for a in sample:
        k = act[a]
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        ref = oracle.ndft(o["tau"][o0:o1], o["pol"][o0:o1], *s.grid)
        err = np.abs(P[a].astype(np.float64) - ref).max() / ref.max()
        assert err <= TOL_SPEC, (a, counts[a], err)
    c.stats()
    c.close()


# ------------------------------------------------------------------ large grids

@pytest.mark.parametrize("N,n_px", [(10_000, 8), (16_384, 3)])
def test_comb_large_grid_bit_exact(N, n_px):
    # the generic comb on the largest grids the header allows (C5's 10,000
    # bins: spectrum and scratch in shared memory, one warp per block; 16,384:
    # the row is scored where it is in global memory), against the oracle's
    # FP32 restatement; rows with harmonic combs, noise, ties and zeros
    params = ddhf.default_params(n_min=1)
    s = synth.Scene(W=n_px, H=1, t0=0, window_us=100, x=np.arange(n_px).astype(np.int16),
                    y=np.zeros(n_px, np.int16), t=np.zeros(n_px, np.int64),
                    p=np.ones(n_px, np.int8), grid=synth.hz_grid(0, 1, N))
    c = ctx_for(s, params)
    x, y, t, p = ddhf.events_to_device(s)
    c.bin_events(x, y, t, p, 0, 100)
    Pn = synth.synthetic_spectra(n_px, N, seed=N)
    out = c.comb_score(torch.from_numpy(Pn).cuda())
    c.stats()
    c.close()
    lsf = out["log_sf"].cpu().numpy()
    snr = out["snr"].cpu().numpy()
    f0 = out["f0_bin"].cpu().numpy()
    ln_tau = np.float32(math.log(0.89))
    scored = 0
    for a in range(n_px):
        lo = oracle.log_sf(Pn[a].astype(np.float64))
        assert abs(lsf[a] - lo) <= 1e-4 * max(1.0, abs(lo)), (a, lsf[a], lo)
        if lsf[a] <= ln_tau:
            s32, w32 = oracle.comb_f32(Pn[a])
            assert w32 == f0[a], (a, w32, f0[a])
            assert np.float32(s32).view(np.uint32) == np.float32(snr[a]).view(np.uint32)
            scored += 1
        else:
            assert f0[a] == -1 and snr[a] == 0
    assert scored >= 1


def test_detect_large_grid():
    # detection on C5's grid (0.5 Hz steps, 10,000 bins): the unfused path
    # equals the spectrum + comb calls bit for bit, spectra match the FP64
    # oracle and sampled scores match the oracle's FP32 comb on them
    s = synth.small_scene(81, W=12, H=10, n_noise=6_000, drone_px=30, f0_hz=150.0,
                          grid=synth.hz_grid(0, 0.5, 10_000))
    c = ctx_for(s)
    x, y, t, p = ddhf.events_to_device(s)
    bx, nb, mask = c.detect(x, y, t, p, s.t0, s.window_us, want_mask=True)
    sc = c.scores()
    P = c.power_spectrum("blocked")
    out = c.comb_score(P)
    st = c.stats()
    c.close()
    assert st["n_active"] > 20
    assert torch.equal(out["mask"], mask)
    assert torch.equal(out["f0_bin"], sc["f0_bin"])
    assert torch.equal(out["snr"].view(torch.int32), sc["snr"].view(torch.int32))
    o = oracle_bin(s)
    act = sc["active"].cpu().numpy()
    Ph = P.cpu().numpy()
    lsf = sc["log_sf"].cpu().numpy()
    snr = sc["snr"].cpu().numpy()
    f0 = sc["f0_bin"].cpu().numpy()
    ln_tau = np.float32(math.log(0.89))
    for a in np.linspace(0, len(act) - 1, 3).astype(int):
        k = act[a]
        o0, o1 = o["offsets"][k], o["offsets"][k + 1]
        ref = oracle.ndft(o["tau"][o0:o1], o["pol"][o0:o1], *s.grid)
        assert np.abs(Ph[a].astype(np.float64) - ref).max() <= TOL_SPEC * ref.max()
        if lsf[a] <= ln_tau:
            s32, w32 = oracle.comb_f32(Ph[a])
            assert w32 == f0[a]
            assert np.float32(s32).view(np.uint32) == np.float32(snr[a]).view(np.uint32)


def test_c3_window_full_size_comb_bits():
    # the benchmarked path on a full 1280x720 C3 window: ddhf_detect with the
    # bench's tuning (hybrid spectra from 128 events), scores exported, and the
    # rows it scored (ddhf_power_spectrum HYBRID, the same kernels) given to the
    # oracle's FP32 comb: SNR bits and dominant bin of ~300 sampled pixels
    # (the heaviest, random ones, drone pixels) must be equal
    s = synth.config3_window(stream=2, window=5)
    c = ctx_for(s, heavy_min=1024, warps_per_block=8, overlap=1, hybrid_min=128)
    x, y, t, p = ddhf.events_to_device(s)
    bx, nb, mask = c.detect(x, y, t, p, s.t0, s.window_us, cap=256, want_mask=True)
    sc = c.scores()
    P = c.power_spectrum("hybrid")
    c.stats()
    c.close()
    act = sc["active"].cpu().numpy()
    o = oracle_bin(s)
    counts = o["counts"][act]
    rng = np.random.default_rng(11)
    drone = np.flatnonzero(np.isin(act, np.concatenate([d["keys"] for d in s.drones])))
    sample = np.unique(np.concatenate([np.argsort(-counts, kind="stable")[:60],
                                       rng.choice(len(act), 200, replace=False),
                                       rng.choice(drone, min(60, drone.size), replace=False)]))
    rows = P[torch.from_numpy(sample).cuda()].cpu().numpy()
    lsf = sc["log_sf"].cpu().numpy()[sample]
    snr = sc["snr"].cpu().numpy()[sample]
    f0 = sc["f0_bin"].cpu().numpy()[sample]
    ln_tau = np.float32(math.log(0.89))
    scored = 0
    for i in range(sample.size):
        lo = oracle.log_sf(rows[i].astype(np.float64))
        assert abs(lsf[i] - lo) <= 1e-4 * max(1.0, abs(lo))
        if abs(lo - math.log(0.89)) > SF_MARGIN:
            assert (lsf[i] <= ln_tau) == (lo <= math.log(0.89))
        if lsf[i] <= ln_tau:
            s32, w32 = oracle.comb_f32(rows[i])
            assert w32 == f0[i], (sample[i], w32, f0[i])
            assert np.float32(s32).view(np.uint32) == np.float32(snr[i]).view(np.uint32)
            scored += 1
    assert scored > 0.9 * sample.size
