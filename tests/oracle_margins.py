"""Rotor decisions of the FP64 oracle with the margins inside which a CUDA
decision may differ from it (shared by the detection parity tests).

For an active pixel the oracle evaluates Eq. 6 in FP64 and Eq. 7-11 on that
spectrum. The CUDA detector scores its own FP32 spectrum P32 in FP32. Two
things separate the two decisions, and each gives a margin around the
thresholds, outside which the decisions must be equal:
  * the arithmetic of SF and of the comb: REL (absolute on ln SF, relative to
    tau_comb on SNR);
  * the spectrum: ln SF of P32 minus ln SF of P64 (both in FP64, exact); for
    SNR, eps (1 + SNR) / (T - eps), where eps = max_j |P32_j - P64_j|, and T
    is P64's value at the first rank of the median band (every complement
    median is at least T; window maxima, and medians, move by at most eps).
The work is spread over spawned worker processes (one oracle call each).
"""
import math
import multiprocessing as mp
import os

import numpy as np

REL = 1e-5


def _rows(args):
    import oracle
    tau, pol, offs, P32, grid, prm = args
    N = grid[3]
    hmax = prm["M"] * (2 * prm["d"] + 1)
    lo_r = max((N - hmax - 1) // 2, 0)
    ln_tsf = math.log(prm["tau_sf"])
    out = []
    for i in range(P32.shape[0]):
        t, p = tau[offs[i]:offs[i + 1]], pol[offs[i]:offs[i + 1]]
        P64 = oracle.ndft(t, p, *grid)
        p32 = P32[i].astype(np.float64)
        lsf64 = oracle.log_sf(P64)
        m_sf = REL + abs(oracle.log_sf(p32) - lsf64)
        snr64, m_snr = 0.0, 0.0
        if lsf64 <= ln_tsf + m_sf:
            snr64, _ = oracle.comb(P64, M=prm["M"], d=prm["d"], h_min=prm["h_min"])
            eps = float(np.abs(p32 - P64).max())
            T = float(np.sort(P64)[lo_r])
            m_snr = REL * prm["tau_comb"] + (eps * (1.0 + max(snr64, prm["tau_comb"])) /
                                             (T - eps) if T > eps else math.inf)
        rot = lsf64 <= ln_tsf and snr64 >= prm["tau_comb"]
        close = abs(lsf64 - ln_tsf) <= m_sf or (
            lsf64 <= ln_tsf and abs(snr64 - prm["tau_comb"]) <= m_snr)
        out.append((rot, close))
    return out


def decisions(binned, act, P32, grid, prm):
    """(rotor, close) per active pixel act[i] (rows P32[i]). binned: the
    oracle's binning of the window; prm: tau_sf, tau_comb, M, d, h_min."""
    procs = max(1, min(16, os.cpu_count() or 1))
    jobs = []
    for part in np.array_split(np.arange(act.size), 4 * procs):
        if not part.size:
            continue
        keys = act[part]
        cnt = binned["counts"][keys]
        offs = np.zeros(keys.size + 1, np.int64)
        offs[1:] = np.cumsum(cnt)
        sel = np.concatenate([np.arange(binned["offsets"][k], binned["offsets"][k + 1])
                              for k in keys])
        jobs.append((binned["tau"][sel], binned["pol"][sel], offs, P32[part], tuple(grid),
                     dict(prm)))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_rows, jobs, chunksize=1)
    flat = [r for chunk in res for r in chunk]
    return np.array([r[0] for r in flat], bool), np.array([r[1] for r in flat], bool)


def segment(mask, W, H, A_min, alpha, cap=4096):
    """The oracle's labelling, area filter and Eq. 12 merging of a mask."""
    import oracle
    lab, _ = oracle.ccl8(np.ascontiguousarray(mask, np.uint8), W, H)
    return oracle.boxes(lab, W, H, A_min=A_min, alpha=alpha, cap=cap)
