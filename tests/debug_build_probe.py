"""Helper run as a child process by tests/test_gpu_debug_build.py (not a test
module): one small detection, its spectra and scores through whichever build
of the library DDHF_LIB names; prints a JSON digest and the device flags."""
import hashlib
import json
import sys

import numpy as np
import torch

from paper_2603_08386_gb300 import ddhf, synth


def digest(t):
    return hashlib.sha256(np.ascontiguousarray(t.cpu().numpy()).tobytes()).hexdigest()


def main():
    out = {}
    for seed, (W, H) in ((11, (64, 48)), (12, (97, 61))):
        s = synth.small_scene(seed, W=W, H=H, n_noise=30_000, drone_px=150)
        c = ddhf.Context(s.W, s.H, s.grid, max_events=s.n, max_windows=2)
        x, y, t, p = ddhf.events_to_device(s)
        bx, nb, mask = c.detect(x, y, t, p, s.t0, s.window_us, cap=64, want_mask=True)
        sc = c.scores()
        P = c.power_spectrum("blocked")
        st = c.stats(raise_on_flags=False)
        c.close()
        out[str(seed)] = dict(boxes=bx[: int(nb.item())].cpu().numpy().tolist(),
                              mask=digest(mask), snr=digest(sc["snr"]),
                              f0=digest(sc["f0_bin"]), P=digest(P),
                              flags=int(st["device_flags"]), status=int(st["status"]))
    print(json.dumps(out))


if __name__ == "__main__":
    sys.exit(main())
