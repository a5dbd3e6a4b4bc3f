"""Many absorbing sites of uneven size in one graph-captured launch
(bse_haydock_batch) against the oracle and against one-site runs."""
import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import bse, synth as S
from parity_check import close

pytestmark = pytest.mark.gpu

# uneven sites: core states 1 or 6, k meshes 2^3..4^3, bands, grids
SITES = [
    dict(seed=91, n_alpha=6, nk=(4, 4, 4), n_bands=40, nx=(6, 6, 6), n_proj=6),
    dict(seed=92, n_alpha=1, nk=(3, 3, 3), n_bands=70, nx=(5, 5, 5), n_proj=0),
    dict(seed=93, n_alpha=6, nk=(2, 2, 2), n_bands=24, nx=(7, 7, 7), n_proj=4),
    dict(seed=94, n_alpha=1, nk=(4, 4, 4), n_bands=33, nx=(6, 5, 4), n_proj=2),
    dict(seed=95, n_alpha=6, nk=(3, 3, 3), n_bands=16, nx=(4, 4, 4), n_proj=3),
]


@pytest.mark.parametrize("prec", ["split_bf16", "fp64"])
def test_batch_matches_single_and_oracle(prec):
    torch = pytest.importorskip("torch")
    systems, gpus, bs = [], [], []
    for kw in SITES:
        s = S.tiny_system(**kw)
        systems.append(s)
        gpus.append(bse.System(s, precision=prec, stream=torch.cuda.Stream().cuda_stream))
        bs.append(S.make_start_vectors(s, 1, seed=kw["seed"]))
    outs, sts = bse.haydock_batch(gpus, bs, 30)
    assert np.all(sts == bse.BSE_OK)
    tol = (1e-9, 1e-9) if prec == "fp64" else (2e-5, 5e-5)
    for i, (s, g, b, (a, bc, st)) in enumerate(zip(systems, gpus, bs, outs)):
        assert st[0] == 30
        a1, bc1, _, _ = g.haydock(b, 30)
        assert np.array_equal(a, a1) and np.array_equal(bc, bc1)   # same kernels, fixed-order sums
        ao, bo, _, _ = O.haydock(lambda v: O.apply_h(s, v), b[0], 30)
        close("batch/a20/%s/site%d" % (prec, i), a[0][:20], ao[:20], tol)
        close("batch/b21/%s/site%d" % (prec, i), bc[0][:21], bo[:21], tol)
