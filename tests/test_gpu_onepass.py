"""Schedules of the split-bf16 step (bse_set_schedule) against the oracle.

* two_pass_rowmajor: grid->band reads the row-major copy of U as an MN-major
  tensor-core operand instead of the transposed copy;
* one_pass: one persistent kernel walks the grid in slabs of 128 points:
  band->grid of every k, the k->R / x W / R->k sums of the slab's points and
  grid->band of every k, with per-slab counters between the CTAs.

Every comparison is element-wise (parity_check.close) at the split-bf16 bounds
of the two-pass step; both schedules change only the order of FP32 sums.
"""
from pathlib import Path

import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import bse, synth as S
from parity_check import close

pytestmark = pytest.mark.gpu

SHAPES = [
    dict(seed=91, n_alpha=6, nk=(4, 4, 4), n_bands=24, nx=(8, 8, 8), n_proj=3),    # 4 slabs
    dict(seed=92, n_alpha=1, nk=(8, 8, 8), n_bands=10, nx=(10, 10, 6), n_proj=0),  # 600 points: ragged last slab
    dict(seed=93, n_alpha=6, nk=(8, 8, 8), n_bands=6, nx=(8, 8, 4), n_proj=2),
    dict(seed=97, n_alpha=6, nk=(4, 4, 4), n_bands=64, nx=(8, 8, 4), n_proj=2),    # 2 Nb = 128: two K blocks
    dict(seed=98, n_alpha=6, nk=(8, 8, 8), n_bands=40, nx=(6, 6, 6), n_proj=1),    # Kp = 80: partial q block
]


@pytest.mark.parametrize("sched", ["two_pass_rowmajor", "one_pass"])
@pytest.mark.parametrize("kw", SHAPES)
def test_schedules_match_oracle(kw, sched):
    s = S.tiny_system(**kw)
    psi = S.complex_normal(np.random.default_rng(kw["seed"]), (1, s.dim))
    sysg = bse.System(s, precision="split_bf16", max_vec=1)
    sysg.set_schedule(sched)
    assert sysg.schedule == sched
    out = sysg.apply_h(psi)
    close("%s/apply_h/seed%d" % (sched, kw["seed"]), out[0], O.apply_h(s, psi)[0], "split_bf16")
    # fixed-order sums: a repeat is bit-identical
    assert np.array_equal(sysg.apply_h(psi), out)
    sysg.close()


@pytest.mark.parametrize("kw", [
    dict(seed=94, n_alpha=1, nk=(4, 4, 4), n_bands=80, nx=(6, 6, 4), n_proj=2),    # 2 Nb = 160: two M tiles
    dict(seed=95, n_alpha=2, nk=(2, 3, 2), n_bands=8, nx=(5, 4, 3), n_proj=1),     # any mesh, odd grid
])
def test_row_major_two_pass_other_shapes(kw):
    """The row-major two-pass schedule takes shapes the one-pass kernel does
    not: several 128-row M tiles of grid->band (q blocks beyond 2 Nb are
    zero-filled by the tensor map), non-cubic meshes and odd grids."""
    s = S.tiny_system(**kw)
    psi = S.complex_normal(np.random.default_rng(kw["seed"]), (2, s.dim))
    sysg = bse.System(s, precision="split_bf16", max_vec=2)
    sysg.set_schedule("two_pass_rowmajor")
    out = sysg.apply_h(psi)
    ref = O.apply_h(s, psi)
    for v in range(2):
        close("two_pass_rowmajor/seed%d/v%d" % (kw["seed"], v), out[v], ref[v], "split_bf16")
    sysg.close()


def test_one_pass_several_vectors_and_fallback():
    """N_alpha = 1: up to 8 vectors in one pass; 9 fall back to the two-pass step."""
    s = S.tiny_system(99, n_alpha=1, nk=(4, 4, 4), n_bands=16, nx=(8, 8, 4), n_proj=2)
    psi = S.complex_normal(np.random.default_rng(99), (9, s.dim))
    ref = O.apply_h(s, psi)
    sysg = bse.System(s, precision="split_bf16", max_vec=9)
    sysg.set_schedule("one_pass")
    for nv in (3, 8, 9):
        out = sysg.apply_h(psi[:nv])
        for v in range(nv):
            close("one_pass/nvec%d/v%d" % (nv, v), out[v], ref[v], "split_bf16")
    sysg.close()


@pytest.fixture(scope="module")
def l23():
    s = S.make_system("l23_multiplet")
    return s, S.make_start_vectors(s, 3)


@pytest.mark.parametrize("sched", ["two_pass_rowmajor", "one_pass"])
def test_l23_full_size(l23, sched):
    """Full-size L2,3 workload (6 core states, 8^3 k, 64 bands, 16^3 grid: 32
    slabs, 128 CTAs of 4 k points each for the one-pass kernel)."""
    s, b = l23
    sysg = bse.System(s, precision="split_bf16", max_vec=1)
    sysg.set_schedule(sched)
    for v in range(3):
        out = sysg.apply_h(b[v:v + 1])
        close("l23/%s/apply_h/v%d" % (sched, v), out[0], O.apply_h(s, b[v:v + 1])[0], "split_bf16")
    sysg.close()


@pytest.mark.parametrize("lag,stages,l2_hint", [(2, 5, True), (1, 4, True), (3, 3, False)])
def test_l23_one_pass_haydock(l23, lag, stages, l2_hint):
    """The one-pass step inside the captured Haydock loop (fused epilogue and
    update): 12-step prefix against the oracle, and 200 steps against the
    stored FP64 oracle spectrum (tests/golden, written by the oracle only)."""
    torch = pytest.importorskip("torch")
    s, b = l23
    stream = torch.cuda.Stream()
    sysg = bse.System(s, precision="split_bf16", max_vec=1, stream=stream.cuda_stream)
    sysg.set_schedule("one_pass", lag=lag, stages=stages, l2_hint=l2_hint)
    a, bc, steps, st = sysg.haydock(b[0], 12)
    ao, bo, _, _ = O.haydock(lambda v: O.apply_h(s, v), b[0], 12)
    assert st == bse.BSE_OK and steps[0] == 12
    close("l23/one_pass%d%d/prefix12_a" % (lag, stages), a[0], ao, (2e-5, 5e-5))
    close("l23/one_pass%d%d/prefix12_b" % (lag, stages), bc[0], bo, (2e-5, 5e-5))
    if lag == 2:
        g = np.load(Path(__file__).parent / "golden" / "l23_multiplet_haydock200.npz")
        a2, b2, st2, _ = sysg.haydock(b[0], 200)
        assert st2[0] == 200
        sg = bse.cf_spectrum(a2, b2, st2, g["omega"], 0.5)[0]
        close("l23/one_pass/spectrum200", sg, g["sigma"], (1e-4, 1e-4))
    sysg.close()


def test_one_pass_wait_limit_times_out_and_recovers(l23):
    """Every wait of the one-pass kernel (pipeline stages, the per-slab
    counters between CTAs) is bounded: at a 2 microsecond limit on the
    full-size workload waits run out, the call reports BSE_ERR_TIMEOUT, and
    the same handle then gives oracle-equal results (the counters were reset
    by the aborted launch)."""
    s, b = l23
    sysg = bse.System(s, precision="split_bf16", max_vec=1)
    sysg.set_schedule("one_pass")
    sysg.set_wait_limit(2e-6)
    with pytest.raises(bse.BSEError) as e:
        sysg.apply_h(b[:1])
    assert e.value.status == bse.BSE_ERR_TIMEOUT
    sysg.set_wait_limit(2.0)
    ref = O.apply_h(s, b[:1])[0]
    for r in range(2):
        close("l23/one_pass/after_timeout/%d" % r, sysg.apply_h(b[:1])[0], ref, "split_bf16")
    sysg.close()


def test_many_site_batch_keeps_two_pass():
    """Sites of a batch overlap on the GPU, so a handle set to the one-pass
    schedule runs the two-pass step there (its CTAs would wait on one another
    beside other sites' kernels): the batch equals single-site two-pass runs
    bit for bit and the oracle within the split-bf16 bounds."""
    torch = pytest.importorskip("torch")
    sites = [dict(seed=111, n_alpha=6, nk=(4, 4, 4), n_bands=24, nx=(8, 8, 4), n_proj=3),
             dict(seed=112, n_alpha=1, nk=(4, 4, 4), n_bands=40, nx=(6, 6, 6), n_proj=0)]
    systems, gpus, bs = [], [], []
    for kw in sites:
        s = S.tiny_system(**kw)
        systems.append(s)
        g = bse.System(s, precision="split_bf16", stream=torch.cuda.Stream().cuda_stream)
        g.set_schedule("one_pass")
        gpus.append(g)
        bs.append(S.make_start_vectors(s, 1, seed=kw["seed"]))
    outs, sts = bse.haydock_batch(gpus, bs, 20)
    assert np.all(sts == bse.BSE_OK)
    for i, (s, g, b, (a, bc, st)) in enumerate(zip(systems, gpus, bs, outs)):
        g.set_schedule("two_pass")
        a1, bc1, _, _ = g.haydock(b, 20)
        assert np.array_equal(a, a1) and np.array_equal(bc, bc1)
        ao, bo, _, _ = O.haydock(lambda v: O.apply_h(s, v), b[0], 20)
        close("batch_one_pass/a/site%d" % i, a[0], ao, (2e-5, 5e-5))
        g.close()


def test_schedule_arguments_checked():
    s = S.tiny_system(5, n_alpha=6, nk=(4, 4, 4), n_bands=24, nx=(8, 8, 4), n_proj=1)
    sysg = bse.System(s, precision="split_bf16")
    for kw in (dict(schedule=3), dict(schedule="one_pass", lag=4), dict(schedule="one_pass", stages=1),
               dict(schedule="one_pass", stages=6)):
        with pytest.raises(bse.BSEError) as e:
            sysg.set_schedule(**kw)
        assert e.value.status == bse.BSE_ERR_INVALID_ARG
    sysg.close()
    # 2 Nb > 128, a 2x3x2 mesh, a grid of 180 points (not whole 8-point
    # k-transform units): the one-pass kernel does not take them
    for kw in (dict(seed=6, n_alpha=1, nk=(4, 4, 4), n_bands=80, nx=(6, 6, 4), n_proj=0),
               dict(seed=7, n_alpha=2, nk=(2, 3, 2), n_bands=8, nx=(4, 4, 4), n_proj=1),
               dict(seed=9, n_alpha=1, nk=(4, 4, 4), n_bands=8, nx=(6, 6, 5), n_proj=0)):
        g = bse.System(S.tiny_system(**kw), precision="split_bf16")
        with pytest.raises(bse.BSEError) as e:
            g.set_schedule("one_pass")
        assert e.value.status == bse.BSE_ERR_UNSUPPORTED
        g.set_schedule("two_pass_rowmajor")   # any shape
        g.close()
    # other precisions: no-op
    g = bse.System(S.tiny_system(8, n_alpha=1, nk=(2, 2, 2), n_bands=8, nx=(4, 4, 4), n_proj=0), precision="fp64")
    g.set_schedule("one_pass")
    assert g.schedule == "two_pass"
    g.close()
