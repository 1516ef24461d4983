"""Physics validation of the CUDA path against the value the paper prints:
the drag coefficient of the Schaefer-Turek 2D-1 cylinder at Re = 20 with the
cylinder as an HLBM porous body (Sec. 5.1, reference c_D = 5.58)."""
import math
import os

import pytest

pytestmark = pytest.mark.gpu

H = pytest.importorskip("paper_2606_31707_b300.hlbm")
from paper_2606_31707_b300.drag_validation import run_case  # noqa: E402


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "sec5_1_schaefer_turek_drag.txt")
    ref, errs = None, {}
    for line in open(path):
        parts = line.split()
        if not parts or parts[0].startswith("#"):
            continue
        if parts[0] == "cd_reference":
            ref = float(parts[1])
        elif parts[0] == "hlbm_error":
            errs[int(parts[1])] = float(parts[2])
    return ref, errs


CD_REF, PAPER_ERR = _golden()


def test_schaefer_turek_drag_coefficient_converges_to_the_reference():
    c20 = run_case(20, 1.0, 4.0, H.FP32)
    c40 = run_case(40, 1.0, 4.0, H.FP32)
    c80 = run_case(80, 1.0, 4.0, H.FP32)
    for c in (c20, c40, c80):
        assert abs(c["Re"] - 20.0) < 0.05
        assert abs(c["cd"] - CD_REF) / CD_REF == pytest.approx(c["rel_err"])
        assert c["drag_change_last_window"] < 1e-5      # steady
    # the error falls with the resolution (the paper's HLBM: 0.73 % at N = 40,
    # 0.21 % at N = 80; here the Mach number also falls with N at tau = 1)
    assert c80["rel_err"] < c40["rel_err"] <= 0.025
    assert c80["rel_err"] <= 0.015
    # the same order of magnitude as the paper's own HLBM errors at these resolutions
    assert c40["rel_err"] <= 5 * PAPER_ERR[40] and c80["rel_err"] <= 5 * PAPER_ERR[80]
    # Richardson extrapolation, with the order observed among the three
    # resolutions themselves, lands near the reference
    p = math.log((c40["cd"] - c20["cd"]) / (c80["cd"] - c40["cd"])) / math.log(2.0)
    extrap = c80["cd"] + (c80["cd"] - c40["cd"]) / (2.0 ** p - 1.0)
    assert abs(extrap - CD_REF) / CD_REF <= 0.005
