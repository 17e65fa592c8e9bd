"""GB300-native DDHF hot path (arXiv 2603.08386): per-pixel NDFT power spectra
of event-camera windows, spectral flatness, median-normalised harmonic comb,
and rotor-mask boxes, as hand-written sm_103a CUDA kernels behind the C ABI in
include/ddhf.h.

Modules:
  build   compiles csrc/*.cu into libddhf.so (nvcc, sm_103a)
  ddhf    ctypes binding of the C ABI (same function names) and ``Context``
  synth   seeded synthetic event streams shaped like the paper's scenes
"""
