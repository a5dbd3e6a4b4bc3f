"""The allocation-free short-range entry point against the regular one.

bse_short_range_noalloc serves callers that may not call cudaMalloc where
they need the short-range term (for instance inside a host framework that
owns all device memory, or in a real-time loop that cannot afford an
allocation's synchronisation).  It uses a static 2 MiB device array as scratch instead of handle
memory.  Here its output is compared with bse_apply_h on a system whose band
energies, spin-orbit matrix and screened potential are zero, so that H psi is
exactly the short-range term; both paths run in FP64, so the FP64 parity
tolerance applies.  Two calls in a row check that the scratch left behind by
one call does not leak into the next; the oracle's short-range term and an
in-place call give the same result.  This file is collected last.
"""
import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import bse, synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-11


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def short_range_only_system(seed, **kw):
    s = S.tiny_system(seed, w_const=0.0, so=False, **kw)
    s.e_nk[:] = 0.0
    s.chi[:] = 0.0
    return s


@pytest.mark.parametrize("kw,n_vec", [
    (dict(n_alpha=6, nk=(4, 4, 2), n_bands=24, nx=(4, 4, 4), n_proj=36), 2),
    # the L2,3 workload's short-range shape: 6 core states, 8^3 k x 64 bands, 36 projectors
    (dict(n_alpha=6, nk=(8, 8, 8), n_bands=64, nx=(4, 4, 4), n_proj=36), 1),
])
def test_noalloc_matches_apply_h_twice(kw, n_vec):
    torch = pytest.importorskip("torch")
    s = short_range_only_system(81, **kw)
    sysg = bse.System(s, precision="fp64", max_vec=n_vec)
    rng = np.random.default_rng(17)
    psi = torch.from_numpy(S.complex_normal(rng, (n_vec, s.dim))).cuda()
    ref = sysg.apply_h(psi)
    torch.cuda.synchronize()
    ref_h = ref.cpu().numpy()
    a = torch.from_numpy(np.ascontiguousarray(s.a_proj.reshape(s.n_proj, -1))).cuda()
    m = torch.from_numpy(np.ascontiguousarray(s.m_sr)).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    # the oracle's short-range term on the same vectors (Sec. 3.2.2)
    ref_o = O.apply_sr(s, psi.cpu().numpy().reshape(n_vec, s.n_alpha, s.n_k, s.n_bands)).reshape(n_vec, -1)
    assert rel(ref_h, ref_o) < TOL
    for call in range(2):
        out = torch.full_like(psi, complex(7.0, -3.0))
        st = bse.short_range_noalloc(a, m, psi, out, s.n_alpha, stream=stream)
        torch.cuda.synchronize()
        assert st == bse.BSE_OK, call
        got = out.cpu().numpy()
        assert rel(got, ref_h) < TOL, call
        assert np.abs(got - ref_o).max() <= TOL * np.abs(ref_o).max(), call
    # in place: psi is read completely before out is written
    work = psi.clone()
    st = bse.short_range_noalloc(a, m, work, work, s.n_alpha, stream=stream)
    torch.cuda.synchronize()
    assert st == bse.BSE_OK
    assert rel(work.cpu().numpy(), ref_h) < TOL


def test_noalloc_rejects_out_overlapping_projectors():
    """out is written while A is read: an output that shares bytes with a_proj
    (or M) is refused before any work is enqueued."""
    torch = pytest.importorskip("torch")
    n_kb, n_proj, n_alpha = 64, 4, 1
    a = torch.zeros((n_proj, n_kb), dtype=torch.complex128, device="cuda")
    m = torch.zeros((n_alpha * n_proj, n_alpha * n_proj), dtype=torch.complex128, device="cuda")
    psi = torch.zeros((1, n_kb), dtype=torch.complex128, device="cuda")
    L = bse.lib()
    st = L.bse_short_range_noalloc(a.data_ptr(), m.data_ptr(), psi.data_ptr(), a[1].data_ptr(), n_alpha, n_kb,
                                   n_proj, 1, None)
    assert st == bse.BSE_ERR_INVALID_ARG
    st = L.bse_short_range_noalloc(a.data_ptr(), m.data_ptr(), psi.data_ptr(), m.data_ptr(), n_alpha, n_kb,
                                   n_proj, 1, None)
    assert st == bse.BSE_ERR_INVALID_ARG
    host = np.zeros((1, n_kb), dtype=np.complex128)   # host memory is refused as well
    st = L.bse_short_range_noalloc(a.data_ptr(), m.data_ptr(), psi.data_ptr(), host.ctypes.data, n_alpha, n_kb,
                                   n_proj, 1, None)
    assert st == bse.BSE_ERR_INVALID_ARG


def test_noalloc_rejects_oversize():
    torch = pytest.importorskip("torch")
    n_kb, n_proj, n_alpha = 2_000_000, 36, 6      # far beyond the 2 MiB scratch
    a = torch.zeros((n_proj, 8), dtype=torch.complex128, device="cuda")
    m = torch.zeros((n_alpha * n_proj, n_alpha * n_proj), dtype=torch.complex128, device="cuda")
    psi = torch.zeros((1, 8), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(psi)
    st = bse.lib().bse_short_range_noalloc(a.data_ptr(), m.data_ptr(), psi.data_ptr(), out.data_ptr(), n_alpha,
                                           n_kb, n_proj, 1, None)
    assert st == bse.BSE_ERR_INVALID_ARG
