"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/tracker.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2107_01104_gb300 as trk
from paper_2107_01104_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    hdrs = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]
    names = set()
    for h in hdrs:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(tracker_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_abi():
    names = declared_functions()
    assert {"tracker_create", "tracker_interpolate", "tracker_advance", "tracker_adjoint"} <= names
    assert names == set(trk.ABI_FUNCTIONS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_loads_and_reports_errors_without_gpu(lib):
    trk.load_library()
    # argument errors are reported before any device call
    with pytest.raises(trk.TrackerError) as e:
        trk.tracker_create(12, I=6)          # N not a power of two
    assert e.value.status == trk.TRK_EINVAL
    with pytest.raises(trk.TrackerError):
        trk.tracker_create(64, I=5)          # unsupported kernel width
    with pytest.raises(trk.TrackerError):
        trk.tracker_create(64, family=trk.TRK_SPLINE, I=6, m=4)
    # queries on a NULL tracker return TRK_EINVAL without touching a device
    L = trk.load_library()
    assert L.tracker_field_texture(None) == trk.TRK_EINVAL
    assert L.tracker_last_step_kernel(None) == trk.TRK_EINVAL
    assert L.tracker_launch_count(None) == -1


def test_oracle_and_library_share_no_code():
    """The oracle neither includes nor links anything of the CUDA path, and vice versa."""
    osrc = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    assert "tracker.h" not in osrc and "coeffs.inc" not in osrc
    for f in os.listdir(os.path.join(ROOT, "paper_2107_01104_gb300", "csrc")):
        text = open(os.path.join(ROOT, "paper_2107_01104_gb300", "csrc", f)).read()
        assert "oracle" not in text.lower(), f
    for f in os.listdir(os.path.join(ROOT, "paper_2107_01104_gb300")):
        if f.endswith(".py"):
            text = open(os.path.join(ROOT, "paper_2107_01104_gb300", f)).read()
            assert "import oracle" not in text and "from oracle" not in text, f


def test_library_built_with_other_flags_is_rebuilt(lib):
    """A library made with extra nvcc flags (an experiment) is not reused by a
    plain build: the flags it was built with are recorded beside it."""
    if build.EXTRA:
        pytest.skip("extra nvcc flags set for this session")
    assert build.up_to_date()
    with open(build.STAMP) as fh:
        saved = fh.read()
    try:
        with open(build.STAMP, "w") as fh:
            fh.write("-DSOME_EXPERIMENT=1")
        assert not build.up_to_date()
        os.remove(build.STAMP)
        assert not build.up_to_date()
    finally:
        with open(build.STAMP, "w") as fh:
            fh.write(saved)
    assert build.up_to_date()
