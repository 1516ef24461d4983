"""The C-ABI library loads on a machine without a GPU and exports every
entry point that include/hlbm.h declares; host-side argument checks."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hlbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hlbm_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2606_31707_b300 import hlbm as H
    lib = H.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(H.EXPORTED)


def test_velocity_sets_match_the_paper_lattices():
    # D2Q9 / D3Q19 (Sec. 2.1) in the library's order: same set as the oracle's
    from oracle.lattice import velocity_set
    from paper_2606_31707_b300 import hlbm as H
    for q in (9, 19):
        xi, w = H.hlbm_velocity_set(q)
        oxi, ow, _ = velocity_set(q)
        got = sorted((tuple(v), round(x, 15)) for v, x in zip(xi, w))
        ref = sorted((tuple(v), round(x, 15)) for v, x in zip(oxi, ow))
        assert got == ref
        # opposite pairs (2k+1, 2k+2)
        for k in range(1, q, 2):
            assert (xi[k] == -xi[k + 1]).all()


def test_default_options_and_argument_checks_without_gpu():
    from paper_2606_31707_b300 import hlbm as H
    o = H.hlbm_default_options((200, 80, 1))
    assert o.ffa_x == 100 and list(o.diss_box) == [0, 200, 0, 80, 0, 1]
    assert o.accum_stride == 1 and o.check_every == 100
    # invalid arguments are rejected before any CUDA call
    for lattice, dims, tau in ((7, (10, 4, 1), 0.6), (9, (3, 4, 1), 0.6), (9, (10, 4, 2), 0.6),
                               (9, (10, 4, 1), 0.5), (19, (10, 4, 4), float("nan"))):
        with pytest.raises(H.HlbmError) as e:
            H.hlbm_create(lattice, dims, tau, 0.0)
        assert e.value.status == H.EINVAL
    # options: |u_in| < 0.5, tau_adj 0 or above 1/2, all finite
    for field, value in (("u_in", 0.7), ("u_in", float("nan")), ("tau_adj", 0.4),
                         ("tau_adj", -1.0), ("tau_adj", float("inf"))):
        o = H.hlbm_default_options((10, 4, 1))
        setattr(o, field, value)
        with pytest.raises(H.HlbmError) as e:
            H.hlbm_create(9, (10, 4, 1), 0.6, 0.0, o)
        assert e.value.status == H.EINVAL, (field, value)


def test_header_cites_the_paper_and_states_errors():
    src = open(os.path.join(ROOT, "include", "hlbm.h")).read()
    for key in ("Eq. adjoint_unsteady", "Eq. gradients_unsteady", "Sec. 4.2", "Sec. 4.3",
                "HLBM_EINVAL", "HLBM_ESTATE", "HLBM_ENONFINITE"):
        assert key in src


def test_option_and_stats_structs_match_the_header_layout(tmp_path):
    # the ctypes mirrors of hlbm_options / hlbm_stats against the C compiler's
    # layout of include/hlbm.h (sizes and every field offset)
    import ctypes
    import shutil
    import subprocess
    from paper_2606_31707_b300 import hlbm as H
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hlbm.h"', "int main(void) {"]
    for cname, cls in (("hlbm_options", H.hlbm_options), ("hlbm_stats", H.hlbm_stats)):
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in (("hlbm_options", H.hlbm_options), ("hlbm_stats", H.hlbm_stats)):
        assert got[(cname, "size")] == ctypes.sizeof(cls)
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_noalloc_wrapper_rejects_bad_buffers_before_any_launch():
    # the C side cannot check buffer sizes; the binding checks dtype, device,
    # contiguity and element counts and raises before calling it
    import torch
    from paper_2606_31707_b300 import hlbm as H
    dims = (8, 4, 1)
    f = torch.zeros(9 * 32, dtype=torch.float64)
    d = torch.zeros(32, dtype=torch.float64)
    J = torch.zeros(1, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        H.hlbm_objective_noalloc(9, dims, 0.7, 0.0, 0.05, H.OBJ_DISSIPATION, (0, 8, 0, 4, 0, 1),
                                 f, d, J)
    with pytest.raises(ValueError, match="required"):
        H.hlbm_objective_noalloc(9, dims, 0.7, 0.0, 0.05, H.OBJ_DISSIPATION, (0, 8, 0, 4, 0, 1),
                                 f, None, J)
