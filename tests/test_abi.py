"""The C-ABI library builds, loads and exports every entry point of
include/bse.h; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "bse.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bse_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def L():
    from paper_1601_07728_gb300 import bse, build
    if not os.path.exists(bse.LIB_PATH):
        build.build()
    return bse.lib()


def test_exports_every_header_function(L):
    from paper_1601_07728_gb300 import bse
    names = header_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n
    assert sorted(bse.EXPORTS) == sorted(n for n in names)


def test_status_strings(L):
    assert L.bse_status_string(0) == b"BSE_OK"
    assert L.bse_status_string(7) == b"BSE_ERR_NAN"


def test_setup_rejects_bad_sizes_without_gpu(L):
    from paper_1601_07728_gb300 import bse
    d = bse.Desc()
    d.n_alpha = 0
    h = ctypes.c_void_p()
    assert L.bse_setup(ctypes.byref(h), ctypes.byref(d)) == bse.BSE_ERR_INVALID_ARG
    assert not h.value
    d.n_alpha = 1
    d.nk = (ctypes.c_int * 3)(2, 2, 17)
    assert L.bse_setup(ctypes.byref(h), ctypes.byref(d)) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_setup(None, ctypes.byref(d)) == bse.BSE_ERR_INVALID_ARG


def test_null_handle_calls(L):
    from paper_1601_07728_gb300 import bse
    assert L.bse_dim(None) == 0
    assert L.bse_apply_h(None, None, None, 1) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_last_error(None) == b"null handle"
    assert L.bse_autotune(None, 1, 1, None, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_set_tiles(None, 2, 4) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_set_wait_limit(None, 1.0) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_set_schedule(None, 2, 0, 0, 1) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_schedule(None) == -1
    assert L.bse_kernel_name(7) == b"one_pass"
    assert L.bse_haydock(None, None, 1, 1, 0, None, None, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_gmres(None, None, None, 1, 1e-6, 30, 100, 0, None, None, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_mlp_train(None, None, 1, None, 1, 1, 1, 1e-3, 0, 10, None, None) == bse.BSE_ERR_INVALID_ARG
    L.bse_destroy(None)


def test_set_up_projection_and_screening_reject_bad_sizes_without_gpu(L):
    from paper_1601_07728_gb300 import bse
    buf = (ctypes.c_double * 64)()
    nk = (ctypes.c_int * 3)(2, 2, 2)
    nx = (ctypes.c_int * 3)(2, 2, 2)
    p = ctypes.cast(buf, ctypes.c_void_p)
    # 9 bands on an 8-point grid, no projectors, 17 k-points along an axis
    assert L.bse_local_projection(p, nk, nx, 9, None, p, 1, 1.0, p, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_local_projection(p, nk, nx, 4, None, p, 0, 1.0, p, None) == bse.BSE_ERR_INVALID_ARG
    nk17 = (ctypes.c_int * 3)(2, 2, 17)
    assert L.bse_local_projection(p, nk17, nx, 4, None, p, 1, 1.0, p, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_local_projection(None, nk, nx, 4, None, p, 1, 1.0, p, None) == bse.BSE_ERR_INVALID_ARG
    # more frequency nodes or grid points than one launch covers, empty sizes, missing output
    assert L.bse_screening_chi0(p, p, 4, 4, 0.0, p, p, 70000, None, p, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_screening_chi0(p, p, 70000, 4, 0.0, p, p, 4, None, p, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_screening_chi0(p, p, 4, 0, 0.0, p, p, 4, None, p, None) == bse.BSE_ERR_INVALID_ARG
    assert L.bse_screening_chi0(p, p, 4, 4, 0.0, p, p, 4, None, None, None) == bse.BSE_ERR_INVALID_ARG


def test_header_cites_the_paper():
    txt = open(os.path.join(ROOT, "include", "bse.h")).read()
    for cite in ("Eq. 3", "Eq. 9", "Algorithm 1", "Eq. 14", "Eq. 2"):
        assert cite in txt


def test_binding_refuses_buffers_the_library_would_overrun():
    """The binding checks element type and size of every array it hands to the
    library, so a wrong array raises in Python instead of being read or
    written past its end."""
    from paper_1601_07728_gb300 import bse
    v = np.zeros((2, 10), dtype=np.complex128)
    assert bse._n_vectors(v, 10, "b") == 2 and bse._n_vectors(v[0], 10, "b") == 1
    for bad in (np.zeros((2, 9), dtype=np.complex128), np.zeros((1, 2, 10), dtype=np.complex128)):
        with pytest.raises(ValueError):
            bse._n_vectors(bad, 10, "b")
    assert bse._buf(v, "complex128", 20, "b") == v.ctypes.data
    with pytest.raises(ValueError):
        bse._buf(v, "complex128", 21, "b")
    with pytest.raises(TypeError):
        bse._buf(v.real.copy(), "complex128", 20, "b")
    with pytest.raises(TypeError):
        bse._buf(np.zeros(4, dtype=np.int64), "int32", 4, "steps")
    with pytest.raises(ValueError):
        bse._buf(None, "float64", 1, "a")
    torch = pytest.importorskip("torch")
    t = torch.zeros(6, dtype=torch.float64)
    assert bse._buf(t, "float64", 6, "a") == t.data_ptr()
    with pytest.raises(TypeError):
        bse._buf(t.float(), "float64", 6, "a")


def test_device_bytes_limit_must_be_a_number(L, monkeypatch):
    """A malformed BSE_DEVICE_BYTES_LIMIT is refused before any device work."""
    from paper_1601_07728_gb300 import bse
    d = bse.Desc()
    d.n_alpha = 1
    d.nk = (ctypes.c_int * 3)(1, 1, 1)
    d.n_bands = 1
    d.nx = (ctypes.c_int * 3)(1, 1, 2)
    dummy = np.zeros(8, dtype=np.complex128)
    d.u = d.e_nk = d.chi = d.w_rx = dummy.ctypes.data
    h = ctypes.c_void_p()
    monkeypatch.setenv("BSE_DEVICE_BYTES_LIMIT", "lots")
    assert L.bse_setup(ctypes.byref(h), ctypes.byref(d)) == bse.BSE_ERR_INVALID_ARG
    assert not h.value
