"""Many-site workload at full size: 64 absorbing sites of uneven size (k mesh
n^3, n = 4..8; grid m^3, m = 12..20; 32..256 bands; 1 or 6 core states), 96.6
GB of complex64-equivalent u_nk drawn on the GPU, run in the split-bf16 form as
one graph-captured launch of 200 Haydock steps per site (bse_haydock_batch).

* every site completes its 200 steps, with the tiles chosen by rule and again
  after a per-site timed tile search (bse_autotune);
* the batched coefficients of sampled sites equal a single-site run of the
  same handle bit for bit (same kernels, fixed-order reductions);
* for sampled sites covering every mesh size 4..8 and both edge types, the
  200-step spectrum is within 1e-4 (relative L2 and per frequency point) of
  the spectrum of the plain FP64 GPU form for the same site, on 2000 omega in
  [-5, 30] eV with Gamma = 0.5 eV, and the batched run's first 20 Haydock
  coefficients and their 20-step spectrum match the FP64 oracle's own
  20-step run of that site.
"""
import copy
import time

import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import bse, synth as S
from parity_check import close

pytestmark = pytest.mark.gpu

N_SITES = 64
STEPS = 200


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def sampled_sites(cfgs):
    """Smallest site of each mesh size, plus the smallest 1s site."""
    size = lambda c: np.prod(c["nk"]) * np.prod(c["nx"]) * c["n_bands"]
    pick = set()
    for n in range(4, 9):
        cand = [i for i, c in enumerate(cfgs) if c["nk"][0] == n]
        if cand:
            pick.add(min(cand, key=lambda i: size(cfgs[i])))
    ones = [i for i, c in enumerate(cfgs) if c["n_alpha"] == 1]
    if ones:
        pick.add(min(ones, key=lambda i: size(cfgs[i])))
    return sorted(pick)


def test_64_uneven_sites_one_launch():
    torch = pytest.importorskip("torch")
    cfgs = [S.batched_site_config(i) for i in range(N_SITES)]
    systems, bs = [], []
    for i, cfg in enumerate(cfgs):
        s = S.make_system_device(cfg, site=i, name="sites64")
        systems.append(bse.System(s, precision="split_bf16", stream=torch.cuda.Stream().cuda_stream))
        bs.append(S.make_start_vectors(s, 1, seed=i))
        del s
        torch.cuda.empty_cache()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs, sts = bse.haydock_batch(systems, bs, STEPS)
    el = time.perf_counter() - t0
    print("64 sites x %d steps, tiles by rule: %.2f s, %.2f spectra/s" % (STEPS, el, N_SITES / el))
    assert np.all(sts == bse.BSE_OK)
    # per-site timed tile search, then the same batch again
    tiles = [g.autotune(n_vec=1, reps=3) for g in systems]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs, sts = bse.haydock_batch(systems, bs, STEPS)
    el = time.perf_counter() - t0
    print("64 sites x %d steps, tuned tiles: %.2f s, %.2f spectra/s; (split, stages) %s"
          % (STEPS, el, N_SITES / el, sorted(set(tiles))))
    assert np.all(sts == bse.BSE_OK)
    for a, bc, st in outs:
        assert st[0] == STEPS
    om = S.omega_grid()
    for i in sampled_sites(cfgs):
        a, bc, st = outs[i]
        a1, bc1, _, _ = systems[i].haydock(bs[i], STEPS)
        assert np.array_equal(a, a1) and np.array_equal(bc, bc1), i
        sig = bse.cf_spectrum(a, bc, st, om, 0.5)[0]
        s = S.make_system_device(cfgs[i], site=i, name="sites64")
        plain = bse.System(s, precision="fp64")
        # the oracle works on host arrays
        sh = copy.copy(s)
        sh.u = s.u.cpu().numpy()
        del s
        torch.cuda.empty_cache()
        a64, b64, s64, st64 = plain.haydock(bs[i], STEPS)
        plain.close()
        assert st64 == bse.BSE_OK and s64[0] == STEPS
        tag = "sites64/site%d_nk%d_na%d" % (i, cfgs[i]["nk"][0], cfgs[i]["n_alpha"])
        close(tag + "/spectrum200_vs_fp64_form", sig, bse.cf_spectrum(a64, b64, s64, om, 0.5)[0], (1e-4, 1e-4))
        ao, bo, nd, _ = O.haydock(lambda v: O.apply_h(sh, v), bs[i][0], 20)
        assert nd == 20
        del sh
        close(tag + "/prefix20_a_vs_oracle", a[0][:20], ao, (2e-5, 5e-5))
        close(tag + "/prefix20_b_vs_oracle", bc[0][:21], bo, (2e-5, 5e-5))
        close(tag + "/prefix20_spectrum_vs_oracle", bse.cf_spectrum(a[:, :20], bc[:, :21], [20], om, 0.5)[0],
              O.cf_spectrum(ao, bo, om, 0.5), (1e-4, 1e-4))
    for g in systems:
        g.close()
