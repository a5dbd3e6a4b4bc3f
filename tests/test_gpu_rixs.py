"""RIXS two-step on the GPU (bse_rixs: GMRES absorption resolvent, emission,
final-state Haydock) against the oracle's two-step, element-wise.

* tiny core-hole / valence pair, FP64 and split-bf16 forms: the final-state
  Haydock coefficients and the RIXS spectra at three incoming energies;
* the emission entry point alone against the oracle's emission;
* the reduced L2,3 workload (6 core states, 4^3 k, 32 bands, 8^3 grid) with a
  10-state valence final state (a 3d shell), split-bf16, three incoming
  energies.
GMRES runs to 1e-10 (FP64) or 1e-6 (split-bf16: the operand rounding keeps
that operator linear only to ~1e-7, so its true residual stalls near there);
the oracle's to 1e-12.
"""
import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import bse, synth as S
from parity_check import close

pytestmark = pytest.mark.gpu


def oracle_rixs(core, val, d, b, z, n_steps):
    return O.rixs_two_step(core, val, d, b, z, n_steps, rtol=1e-12)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
def test_rixs_tiny_matches_oracle(prec):
    core = S.tiny_system(61, n_alpha=6, nk=(2, 2, 2), n_bands=10, nx=(6, 6, 6), n_proj=3)
    val, d = S.valence_final_state(core, n_v=4, seed=1)
    b = S.make_start_vectors(core, 1, seed=3)[0]
    z = np.array([3.0 + 0.4j, 11.5 + 0.4j, 19.0 + 1.0j])
    n_steps = 12
    gc = bse.System(core, precision=prec, max_vec=3)
    gv = bse.System(val, precision=prec, max_vec=3)
    rt = 1e-10 if prec == "fp64" else 1e-5   # tiny grid: the split-bf16 residual floor is near 1e-6
    a, bc, steps, it, rel, st = bse.rixs(gc, gv, b, z, d, n_steps, rtol=rt, restart=30, max_iter=2000)
    assert st == bse.BSE_OK and np.all(rel <= rt) and list(steps) == [n_steps] * 3
    ref = oracle_rixs(core, val, d, b, z, n_steps)
    om = np.linspace(-2.0, 35.0, 1000)
    tol_c = (1e-8, 1e-8) if prec == "fp64" else (1e-4, 1e-4)
    for j, (ao, bo, _) in enumerate(ref):
        close("rixs_tiny/%s/a/z%d" % (prec, j), a[j], ao, tol_c)
        close("rixs_tiny/%s/b/z%d" % (prec, j), bc[j], bo, tol_c)
        close("rixs_tiny/%s/spectrum/z%d" % (prec, j), bse.cf_spectrum(a[j], bc[j], steps[j], om, 0.3)[0],
              O.cf_spectrum(ao, bo, om, 0.3), tol_c)


def test_rixs_emission_entry_point():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    na, nv, nkb, nz = 6, 10, 777, 3
    d = S.complex_normal(rng, (nv, na))
    x = S.complex_normal(rng, (nz, na * nkb))
    dd, xd = torch.from_numpy(d).cuda(), torch.from_numpy(x).cuda()
    yd = torch.empty((nz, nv * nkb), dtype=torch.complex128, device="cuda")
    assert bse.rixs_emission(dd, xd, yd, na) == bse.BSE_OK
    torch.cuda.synchronize()
    close("rixs_emission", yd.cpu().numpy(), O.rixs_emission(d, x), (1e-14, 1e-14))
    # host memory is refused
    assert bse.rixs_emission(d, xd, yd, na) == bse.BSE_ERR_INVALID_ARG


def test_rixs_reduced_l23_split_bf16():
    core = S.reduced_l23(0)
    val, d = S.valence_final_state(core, n_v=10, seed=0)
    b = S.make_start_vectors(core, 1)[0]
    z = np.array([2.0 + 0.5j, 8.0 + 0.5j, 14.0 + 0.5j])
    n_steps = 15
    gc = bse.System(core, precision="split_bf16", max_vec=3)
    gv = bse.System(val, precision="split_bf16", max_vec=3)
    a, bc, steps, it, rel, st = bse.rixs(gc, gv, b, z, d, n_steps, rtol=1e-6, restart=30, max_iter=3000)
    assert st == bse.BSE_OK and np.all(rel <= 1e-6)
    ref = oracle_rixs(core, val, d, b, z, n_steps)
    om = np.linspace(-2.0, 35.0, 1000)
    for j, (ao, bo, _) in enumerate(ref):
        close("rixs_l23r/a/z%d" % j, a[j], ao, (1e-4, 1e-4))
        close("rixs_l23r/b/z%d" % j, bc[j], bo, (1e-4, 1e-4))
        close("rixs_l23r/spectrum/z%d" % j, bse.cf_spectrum(a[j], bc[j], steps[j], om, 0.3)[0],
              O.cf_spectrum(ao, bo, om, 0.3), (1e-4, 1e-4))
