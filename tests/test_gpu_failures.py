"""Failure detection on the GPU, made on purpose without faulting it.

* Bounded waits: every wait of the tensor-core pipeline is limited by
  %globaltimer.  With the limit set to 2 microseconds on a full-size L2,3
  launch (each 128-row tile takes several microseconds to stream), waits run
  out; the kernel then stops issuing, waits for its own copies and MMAs in
  flight, frees its tensor memory and returns, and the call reports
  BSE_ERR_TIMEOUT.  The next call on the same handle, with the limit back at
  2 s, must match the oracle.
* Out of memory: BSE_DEVICE_BYTES_LIMIT caps what bse_setup may allocate;
  caps below the handle's needs give BSE_ERR_OOM at different points of the
  set-up, and the device's free memory afterwards equals what it was before
  (nothing leaked).
"""
import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import bse, synth as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def l23():
    s = S.make_system("l23_multiplet")
    b = S.make_start_vectors(s, 1)
    return s, b, O.apply_h(s, b)


def test_tensor_core_wait_limit_times_out_and_handle_recovers(l23):
    s, b, ref = l23
    sysg = bse.System(s, precision="split_bf16", max_vec=1)
    sysg.set_wait_limit(2e-6)
    with pytest.raises(bse.BSEError) as e:
        sysg.apply_h(b)
    assert e.value.status == bse.BSE_ERR_TIMEOUT
    # the handle is still usable: normal limit, oracle-equal result, twice
    sysg.set_wait_limit(2.0)
    for _ in range(2):
        out = sysg.apply_h(b)
        assert rel(out[0], ref[0]) < 1e-5
        assert np.abs(out[0] - ref[0]).max() <= 1e-4 * np.abs(ref[0]).max()
    a, bc, steps, st = sysg.haydock(b[0], 5)
    assert st == bse.BSE_OK and steps[0] == 5
    sysg.close()


def test_wait_limit_range_checked():
    sysg = bse.System(S.tiny_system(3, n_alpha=1, nk=(2, 2, 2), n_bands=8, nx=(4, 4, 4)), precision="split_bf16")
    for bad in (0.0, 5e-7, 61.0, float("nan")):
        with pytest.raises(bse.BSEError) as e:
            sysg.set_wait_limit(bad)
        assert e.value.status == bse.BSE_ERR_INVALID_ARG
    sysg.close()


def test_device_memory_cap_gives_oom_without_leak(monkeypatch):
    torch = pytest.importorskip("torch")
    s = S.tiny_system(77, n_alpha=6, nk=(4, 4, 4), n_bands=64, nx=(16, 16, 16), n_proj=8)
    psi = S.make_start_vectors(s, 1)
    ref = O.apply_h(s, psi)
    monkeypatch.delenv("BSE_DEVICE_BYTES_LIMIT", raising=False)
    g = bse.System(s, precision="split_bf16")   # loads the device code once, outside the measurement
    g.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # u_nk alone is 268 MB as complex128 staging; the split-bf16 copies another 268 MB
    for cap in (1, 4096, 10 ** 6, 100 * 10 ** 6, 300 * 10 ** 6, 500 * 10 ** 6):
        monkeypatch.setenv("BSE_DEVICE_BYTES_LIMIT", str(cap))
        with pytest.raises(bse.BSEError) as e:
            bse.System(s, precision="split_bf16")
        assert e.value.status == bse.BSE_ERR_OOM, cap
    monkeypatch.setenv("BSE_DEVICE_BYTES_LIMIT", "12x")
    with pytest.raises(bse.BSEError) as e:
        bse.System(s, precision="split_bf16")
    assert e.value.status == bse.BSE_ERR_INVALID_ARG
    monkeypatch.delenv("BSE_DEVICE_BYTES_LIMIT")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < 8 * 2 ** 20, (free0, free1)
    # a cap above the need lets the set-up through, with the same result
    monkeypatch.setenv("BSE_DEVICE_BYTES_LIMIT", str(4 * 10 ** 9))
    g = bse.System(s, precision="split_bf16")
    out = g.apply_h(psi)
    g.close()
    assert rel(out[0], ref[0]) < 1e-5
