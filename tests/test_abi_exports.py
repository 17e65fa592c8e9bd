"""The C ABI library loads on a machine without a GPU and exports every entry
point that include/ddhf.h declares (no compute calls are made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ddhf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ddhf_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ddhf_create", "ddhf_destroy", "ddhf_bin_events", "ddhf_power_spectrum",
                     "ddhf_comb_score", "ddhf_detect", "ddhf_label", "ddhf_boxes"):
        assert required in names


def test_library_exports_every_declared_symbol():
    if not os.environ.get("DDHF_SKIP_BUILD"):
        from paper_2603_08386_gb300 import build
        try:
            build.build()
        except (RuntimeError, FileNotFoundError) as e:  # no nvcc on this machine
            pytest.skip(f"cannot build libddhf: {e}")
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2603_08386_gb300", "libddhf.so"))
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_header():
    from paper_2603_08386_gb300 import ddhf
    assert set(declared_functions()) <= set(ddhf.SIGNATURES)


def test_default_params_are_table2_without_gpu():
    from paper_2603_08386_gb300 import ddhf
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "table2.json")))
    p = ddhf.default_params()
    assert p.tau_sf == pytest.approx(g["tau_sf"]["final"])
    assert p.tau_comb == pytest.approx(g["tau_comb"]["final"])
    assert (p.M, p.d, p.h_min, p.n_min, p.A_min) == tuple(
        g[k]["final"] for k in ("M", "d", "h_min", "n_min", "A_min"))
    assert p.alpha == g["alpha"]["final"]


def test_bad_arguments_rejected_without_gpu():
    # ddhf_create validates its arguments before touching the device
    from paper_2603_08386_gb300 import ddhf
    lib = ddhf.load()
    h = ctypes.c_void_p()
    p = ddhf.default_params()
    g = ddhf.make_grid(0, 10_000, 10**9, 100)
    assert lib.ddhf_create(0, 10, ctypes.byref(g), ctypes.byref(p), 10, 1, ctypes.byref(h)) == 1
    bad = ddhf.make_grid(0, 0, 10**9, 100)
    assert lib.ddhf_create(10, 10, ctypes.byref(bad), ctypes.byref(p), 10, 1, ctypes.byref(h)) == 1
    p.M = 40
    assert lib.ddhf_create(10, 10, ctypes.byref(g), ctypes.byref(p), 10, 1, ctypes.byref(h)) == 5
    assert lib.ddhf_bin_events(None, None, None, None, None, 0, 0, 1, None) == 1
    assert lib.ddhf_status_string(3) == b"capacity exceeded"


def test_binding_forms_and_tuning_match_header():
    # the DDHF_FORM_* numbers and the ddhf_tuning fields of the header are
    # the ones the binding marshals
    import ctypes as ct
    from paper_2603_08386_gb300 import ddhf
    src = open(os.path.join(ROOT, "include", "ddhf.h")).read()
    forms = {m.group(1).lower(): int(m.group(2))
             for m in re.finditer(r"#define DDHF_FORM_(\w+) (\d+)", src)}
    assert forms == ddhf.FORM
    body = re.search(r"typedef struct \{([^}]*)\} ddhf_tuning;", src).group(1)
    fields = re.findall(r"int32_t (\w+);", body)
    assert fields == [f for f, _ in ddhf.ddhf_tuning._fields_]
    assert ct.sizeof(ddhf.ddhf_tuning) == 4 * len(fields)
