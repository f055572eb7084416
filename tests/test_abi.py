"""The C-ABI library loads, exports every symbol include/tgba.h declares, and rejects bad
arguments on the host before touching a device (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2410_04204_gb300 import build, tgba

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "tgba.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tgba_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    names = declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(tgba.SYMBOLS) == names


def test_argument_errors_are_host_side():
    bad = [dict(L=7, h_z=1.0, sectors=[0], max_qp=4),          # odd L
           dict(L=2, h_z=1.0, sectors=[0], max_qp=4),          # too short
           dict(L=122, h_z=1.0, sectors=[0], max_qp=4),        # too long
           dict(L=12, h_z=-1.0, sectors=[0], max_qp=4),        # h_z <= 0
           dict(L=12, h_z=1.0, sectors=[12], max_qp=4),        # m out of range
           dict(L=12, h_z=1.0, sectors=[0, 0], max_qp=4),      # repeated sector
           dict(L=12, h_z=1.0, sectors=[0], max_qp=17),        # too many quasiparticles
           dict(L=12, h_z=1.0, sectors=[0], max_qp=4, J=0.0)]  # J <= 0
    for kw in bad:
        with pytest.raises(tgba.TgbaError) as e:
            tgba.tgba_build_basis(**kw)
        assert e.value.code == tgba.TGBA_EINVAL, kw


def test_no_cpu_fallback_without_device():
    if tgba.tgba_device_count() > 0:
        pytest.skip("a CUDA device is present")
    with pytest.raises(tgba.TgbaError) as e:
        tgba.tgba_build_basis(12, 1.0, [0], 4)
    assert e.value.code == tgba.TGBA_ECUDA
    with pytest.raises(tgba.TgbaError) as e:
        tgba.tgba_fp64_peak(1)
    assert e.value.code == tgba.TGBA_ECUDA


def test_null_handles_rejected():
    with pytest.raises(tgba.TgbaError) as e:
        tgba.tgba_basis_totals(None)
    assert e.value.code == tgba.TGBA_EINVAL


def test_null_handles_rejected_by_every_handle_call():
    """Each entry point that takes a basis handle checks it on the host before anything else
    (no device needed): a null handle is TGBA_EINVAL."""
    lib = tgba.lib()
    calls = {
        "tgba_x_direct": (None, 0, None, 0, None, None),
        "tgba_z_elements": (None, 0, 0, 1, None, 0, None, None),
        "tgba_x_pairs": (None, 0, None, 0, None, None),
        "tgba_eigvals": (None, None, 0, None, None),
        "tgba_quench_correlators": (None, 0, 0.5, 0.1, 1.0, 1, 1.0, 2, 1, None, None, None, None, None),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == tgba.TGBA_EINVAL, name

