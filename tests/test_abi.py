"""Host-side checks of the C ABI that need no GPU: the shared library loads, exports
every entry point include/ahs.h declares, and rejects bad arguments before any
CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def abi():
    from paper_2005_14454_gb300 import build, _abi
    build.build()
    return _abi


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ahs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ahs_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for want in ("ahs_create", "ahs_init", "ahs_step", "ahs_measure", "ahs_fields", "ahs_destroy"):
        assert want in syms


def test_library_exports_every_declared_symbol(abi):
    L = abi.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name
    assert set(declared_symbols()) <= set(abi.EXPORTS) | {"ahs_create"}


def test_obs_layout(abi):
    assert abi.lib().ahs_sizeof_obs() == ctypes.sizeof(abi.ahs_obs_t)


def test_strerror(abi):
    L = abi.lib()
    assert L.ahs_strerror(0) == b"ok"
    assert L.ahs_strerror(abi.AHS_EINVAL) == b"invalid argument"
    assert L.ahs_strerror(abi.AHS_ENONFINITE) == b"non-finite field value"
    assert L.ahs_strerror(12345) == b"unknown status"


@pytest.mark.parametrize("args", [
    (3, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, 1),        # N too small
    (1601, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, 1),     # N^3 would overflow 32-bit site offsets
    (16, -0.5, 0.1, 2.0, 1.0, 1.0, 0.0, 1),      # dx <= 0
    (16, 0.5, 0.0, 2.0, 1.0, 1.0, 0.0, 1),       # dt <= 0
    (16, 0.5, 0.1, 2.0, 0.0, 1.0, 0.0, 1),       # e0 = 0
    (16, 0.5, 0.1, 2.0, 1.0, 1.0, 0.0, 3),       # unknown era
    (16, 0.5, 0.1, float("nan"), 1.0, 1.0, 0.0, 1),
])
def test_create_rejects_bad_arguments(abi, args):
    L = abi.lib()
    assert not L.ahs_create(*args)
    assert L.ahs_last_error() == abi.AHS_EINVAL
    assert L.ahs_last_error_message()


def test_null_handle_is_rejected(abi):
    L = abi.lib()
    assert L.ahs_init(None, 1) == abi.AHS_EINVAL
    assert L.ahs_step(None, 1) == abi.AHS_EINVAL
    assert L.ahs_set_option(None, 0, 1.0) == abi.AHS_EINVAL
    L.ahs_destroy(None)


def test_binding_raises_without_library(tmp_path, abi):
    with pytest.raises(ImportError):
        abi.load(str(tmp_path / "missing.so"))


def test_binding_constants_match_the_header(abi):
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ahs.h")).read(), flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\b(AHS_[A-Z0-9_]+)\s*=\s*(-?\d+)", txt)}
    assert len(consts) > 30
    for name, value in consts.items():
        if name == "AHS_NOALLOC_MAX_ROWS":
            continue
        assert getattr(abi, name) == value, name
    assert consts["AHS_OPT_MOMENTA_IN_PLACE"] == 12


@pytest.mark.parametrize("args", [
    (0.0, 2.0, 1.0, 1.0, 0.0, 1, 1.0, 10.0, 0.0, 0.0, 0.9),           # dx <= 0
    (0.5, 2.0, 1.0, 1.0, 0.0, 3, 1.0, 10.0, 0.0, 0.0, 0.9),           # unknown era
    (0.5, 2.0, 1.0, 1.0, 0.0, 1, 1.0, 0.5, 0.0, 0.0, 0.9),            # tau_end < tau0
    (0.5, 2.0, 1.0, 1.0, 0.0, 1, 1.0, 10.0, 0.0, 0.0, 1.5),           # safety > 1
    (0.5, float("inf"), 1.0, 1.0, 0.0, 1, 1.0, 10.0, 0.0, 0.0, 0.9),  # non-finite coupling
])
def test_stable_dt_rejects_bad_arguments(abi, args):
    v = ctypes.c_double(-1.0)
    assert abi.lib().ahs_stable_dt(*args, ctypes.byref(v)) == abi.AHS_EINVAL
    assert v.value == -1.0
    assert abi.lib().ahs_stable_dt(0.5, 2.0, 1.0, 1.0, 0.0, 1, 1.0, 10.0, 0.0, 0.0, 0.9, None) == abi.AHS_EINVAL


def test_bounds_check_absent_from_the_production_build(abi):
    # the index checks exist only in the bounds-check build (_ahs_check.so); the
    # production library says so without touching the device
    c = ctypes.c_int64(-1)
    assert abi.lib().ahs_bounds_check(0, ctypes.byref(c)) == abi.AHS_ESTATE
    assert b"bounds-check build" in abi.lib().ahs_last_error_message()
    assert abi.lib().ahs_bounds_check(3, ctypes.byref(c)) == abi.AHS_EINVAL
