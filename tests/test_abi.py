"""The C-ABI library builds, loads and exports every symbol include/ncf.h
declares; host-only entry points behave without a GPU."""
import ctypes

import pytest

from paper_2609_03866_b300 import api, build


def test_library_builds_and_exports_declared_symbols():
    build.build()
    L = api.lib()
    names = api.declared_symbols()
    assert len(names) >= 9
    for n in names:
        assert hasattr(L, n), f"libncf.so does not export {n}"


def test_status_strings_and_default_options():
    assert api.status_name(0) == "NCF_OK"
    assert api.status_name(2) == "NCF_ENOTSORTED"
    assert api.status_name(9) == "NCF_EUNSUPPORTED"
    o = api.make_options()
    assert (o.kernel, o.path, o.precision, o.norm) == (0, 0, 0, 0)
    assert o.h == 1.0 and o.trunc_R == 0.0 and o.tol == 0.0


def test_create_without_a_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = api.lib().ncf_create(ctypes.byref(h), 0)
    assert rc == 5 and not h.value   # NCF_ECUDA, no context
    assert api.lib().ncf_last_error(None) == b"NULL context"
