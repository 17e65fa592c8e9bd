"""Row-band sharding of one window over ranks, one GPU per rank.

Binning and Eq. 6-11 are per pixel, so each rank takes the rows
[row0, row0 + h) of the sensor (its own context with a row offset: events of
other rows are dropped by the binning kernel) and produces its rotor mask,
labels and per-component boxes on its GPU. Only the segmentation of Sec. 3.5
couples the bands; the one exchange step is an all-gather of every band's
boundary-row labels and component list (a few KB), after which each rank
joins components across the boundaries and runs the area filter and the
Eq. 12 merge on the host (``ddhf_merge_bands``). The boxes equal those of the
whole sensor on one device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ddhf


def band_rows(H: int, n_bands: int) -> list:
    """Row starts of n_bands near-equal bands of H rows (n_bands + 1 entries)."""
    if not 1 <= n_bands <= H:
        raise ValueError("need 1 <= n_bands <= H")
    return [H * b // n_bands for b in range(n_bands + 1)]


def exchange_and_merge(part, rows, W, H, params, cap=4096, group=None):
    """All-gather the bands' parts and merge them into the sensor's boxes.

    part: (edge_labels int32 [2, W] band-local, comps int32 [k, 6] in sensor
    coordinates) of this rank's band; rows: band_rows(H, world). Without an
    initialised process group, ``part`` must be the list of all bands' parts.
    Returns (boxes int32 [n, 5], total)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        parts = [None] * dist.get_world_size(group)
        dist.all_gather_object(parts, part, group=group)
    else:
        parts = part
    if len(parts) != len(rows) - 1:
        raise ValueError("one part per band expected")
    edges = np.stack([np.asarray(e, np.int32).reshape(2, W) for e, _ in parts])
    comps = [np.asarray(c, np.int32).reshape(-1, 6) for _, c in parts]
    off = np.zeros(len(comps) + 1, np.int64)
    off[1:] = np.cumsum([c.shape[0] for c in comps])
    allc = np.concatenate(comps) if off[-1] else np.zeros((0, 6), np.int32)
    return ddhf.ddhf_merge_bands(W, H, rows, edges, allc, off, params, cap)


class BandDetector:
    """This rank's row band of a W x H sensor."""

    def __init__(self, W, H, grid, band, n_bands, params=None, max_events=1 << 24,
                 comp_cap=1 << 16):
        self.W, self.H = int(W), int(H)
        self.rows = band_rows(self.H, n_bands)
        self.row0 = self.rows[band]
        self.h = self.rows[band + 1] - self.row0
        self.params = params if params is not None else ddhf.default_params()
        self.ctx = ddhf.Context(self.W, self.h, grid, self.params, max_events=max_events)
        ddhf.ddhf_set_row_offset(self.ctx.h, self.row0)
        dev = self.ctx.dev
        self.mask = torch.empty(self.W * self.h, dtype=torch.uint8, device=dev)
        self.labels = torch.empty(self.W * self.h, dtype=torch.int32, device=dev)
        self.comp_cap = int(comp_cap)
        self.comps = torch.empty((self.comp_cap, 6), dtype=torch.int32, device=dev)
        self.ncomp = torch.zeros(1, dtype=torch.int32, device=dev)
        self.bx = torch.empty((4096, 5), dtype=torch.int32, device=dev)  # band-local boxes
        self.nbx = torch.zeros(1, dtype=torch.int32, device=dev)

    def part(self, x, y, t, p, t0, window_us):
        """This band's mask, labels and components for one window (device
        tensors of the whole sensor's events); returns host (edge_labels
        [2, W], comps [k, 6])."""
        ddhf.ddhf_detect(self.ctx.h, x, y, t, p, x.numel(), t0, window_us, self.bx,
                         self.bx.shape[0], self.nbx, self.mask)
        ddhf.ddhf_export_labels(self.ctx.h, 0, self.labels)  # the detection's own labels
        ddhf.ddhf_components(self.ctx.h, self.labels, self.row0, self.comps, self.comp_cap,
                             self.ncomp)
        lab = self.labels.view(self.h, self.W)
        edge = torch.stack([lab[0], lab[self.h - 1]]).cpu().numpy()
        n = int(self.ncomp.item())
        if n > self.comp_cap:
            raise ddhf.DDHFError(3, f"{n} components > comp_cap {self.comp_cap}")
        self.ctx.stats()
        return edge, self.comps[:n].cpu().numpy()

    def detect(self, x, y, t, p, t0, window_us, cap=4096, group=None):
        """Boxes of the whole sensor: this band's part, then the exchange."""
        return exchange_and_merge(self.part(x, y, t, p, t0, window_us), self.rows, self.W,
                                  self.H, self.params, cap, group)

    def close(self):
        self.ctx.close()
