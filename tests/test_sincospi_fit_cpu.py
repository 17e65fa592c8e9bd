"""The sin/cos(pi x) polynomial coefficients compiled into the kernels are
the ones the committed fitting script produces (so they can be regenerated
from the mathematics), and the fitted polynomials are within FP32 accuracy
of sin and cos on the reduced range."""
import os
import re

import numpy as np

from paper_2603_08386_gb300 import fit_sincospi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def kernel_coefficients():
    src = open(os.path.join(ROOT, "paper_2603_08386_gb300", "csrc", "ddhf_internal.cuh")).read()
    body = src[src.index("void sincospi_reduced("):]
    body = body[:body.index("const int iq")]
    p = [float(v) for v in re.findall(r"float p = ([-0-9.e]+)f;", body)]
    p += [float(v) for v in re.findall(r"p = __fmaf_rn\(p, t, ([-0-9.e]+)f\);", body)]
    k = [float(v) for v in re.findall(r"float k = ([-0-9.e]+)f;", body)]
    k += [float(v) for v in re.findall(r"k = __fmaf_rn\(k, t, ([-0-9.e]+)f\);", body)]
    return np.array(p[::-1], np.float32), np.array(k[::-1], np.float32)


def test_kernel_coefficients_are_the_fit():
    P, C = fit_sincospi.fit()
    kp, kc = kernel_coefficients()
    assert kp.size == 5 and kc.size == 4
    np.testing.assert_array_equal(kp, P)
    np.testing.assert_array_equal(kc, C)


def test_fit_accuracy():
    P, C = fit_sincospi.fit()
    es, ec = fit_sincospi.max_rel_error(P, C)
    assert es < 2e-7 and ec < 2e-7, (es, ec)
