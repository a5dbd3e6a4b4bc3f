"""GPU kernels of the learned GMRES preconditioner against the FP64 oracle
(oracle/mlp_oracle.py): network outputs, loss gradient, Adam, and GMRES with
the preconditioner attached.

Tolerances: outputs and gradients are computed with FP16 weights and FP32
accumulation on the GPU versus FP64 arithmetic on the same FP16-rounded
weights in the oracle, so the difference is FP32 accumulation alone (a few
2^-24 per term, ~3e-7 recorded): 2e-6 relative L2 and 5e-6 per element
(relative to the largest entry) for outputs and for each parameter block of
the gradient (the H applications and probe statistics are FP64); Adam's FP32
update 1e-6; two GMRES solutions at true residual 1e-8 agree to 1e-6.  Every
comparison is recorded (parity_check.close).
"""
import numpy as np
import pytest

from oracle import bse_oracle as O
from oracle import mlp_oracle as M
from paper_1601_07728_gb300 import bse, synth as S
from parity_check import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    s = S.tiny_system(62, n_alpha=6, nk=(2, 2, 2), n_bands=10, nx=(4, 4, 4), n_proj=4)
    rng = np.random.default_rng(11)
    params = S.mlp_init(5).astype(np.float64)
    pr = M.unpack(params)
    pr["w3"] = pr["w3"] + 0.05 * rng.standard_normal(pr["w3"].shape)
    pr["b3"] = 0.05 * rng.standard_normal(pr["b3"].shape)
    flat = M.pack(M.fp16(pr)).astype(np.float32)
    return s, flat


def test_outputs_match_oracle(tiny):
    s, flat = tiny
    sysg = bse.System(s, precision="fp64")
    net = bse.MLP(flat)
    diag = O.jacobi_diag(s).reshape(-1)
    for om in (-2.0, 6.5):
        out = net.outputs(sysg, om, 0.5)
        ref, _ = M.forward(M.fp16(M.unpack(flat.astype(np.float64))), M.system_features(s, diag, om, 0.5))
        close("mlp/outputs/om%g" % om, out.astype(np.float64), ref, (2e-6, 5e-6))


@pytest.mark.parametrize("steps", [0, 1, 4])
def test_gradient_matches_oracle(tiny, steps):
    """Loss on three probes and its gradient against the oracle's: the plain
    approximate-inverse loss (steps = 0) and the k-step minimal-residual loss
    (forward and adjoint Krylov chains through FP64 applications of H)."""
    torch = pytest.importorskip("torch")
    s, flat = tiny
    sysg = bse.System(s, precision="fp64", max_vec=2)
    net = bse.MLP(flat)
    rng = np.random.default_rng(12)
    rs = S.complex_normal(rng, (3, s.dim))
    om, g = 4.0, 0.5
    loss, grad = net.loss_grad(sysg, om, g, torch.from_numpy(rs).cuda(), steps=steps)
    diag = O.jacobi_diag(s).reshape(-1)
    params = M.unpack(flat.astype(np.float64))
    feats = M.system_features(s, diag, om, g)
    happly = lambda v: O.apply_h(s, v)
    if steps == 0:
        lo, go = M.spai_grad(params, feats, diag, om + 1j * g, list(rs), happly)
    else:
        lo, go = M.krylov_grad(params, feats, diag, om + 1j * g, list(rs), happly, steps)
    assert loss == pytest.approx(lo, rel=1e-4)
    gg = M.unpack(grad.astype(np.float64))
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        close("mlp/grad%d/%s" % (steps, name), gg[name], go[name], (2e-6, 5e-6))


def test_adam_step_matches_oracle(tiny):
    s, flat = tiny
    net = bse.MLP(flat)
    rng = np.random.default_rng(13)
    grad = (rng.standard_normal(flat.size) * 0.1).astype(np.float32)
    net.adam_step(grad, 1e-3)
    net.adam_step(0.5 * grad, 1e-3)
    p = M.unpack(flat.astype(np.float64))
    z = {k: np.zeros_like(v) for k, v in p.items()}
    p1, m1, v1 = M.adam(p, M.unpack(grad.astype(np.float64)), z, z, 1, 1e-3)
    p2, _, _ = M.adam(p1, M.unpack(0.5 * grad.astype(np.float64)), m1, v1, 2, 1e-3)
    close("mlp/adam", net.params().astype(np.float64), M.pack(p2), (1e-6, 1e-6))


@pytest.fixture(scope="module")
def reduced():
    s = S.reduced_l23(0)
    return s, S.make_start_vectors(s, 1)[0]


TRAIN_Z = np.linspace(-3.0, 25.0, 8) + 0.5j
HELD_OUT_Z = np.array([2.0, 10.8, 17.8]) + 0.5j


@pytest.fixture(scope="module")
def trained(reduced):
    """Network trained on the GPU (probe harvest by GMRES, loss and gradient
    by the library's kernels, Adam) at eight shifts of the reduced L2,3 system."""
    s, b = reduced
    sysg = bse.System(s, precision="fp64", max_vec=4)
    net = bse.MLP(S.mlp_init(0))
    hist = net.train([sysg], [b], TRAIN_Z, epochs=10, batch=1, lr=1e-3, seed=1, steps=10)
    return net, hist


def test_training_reduces_loss(trained):
    """The mean sample loss (10-step minimal-residual form) falls over the epochs."""
    net, hist = trained
    assert np.all(np.isfinite(hist))
    assert hist[-1] < 0.95 * hist[0]


def test_trained_network_beats_prior_and_no_preconditioner(reduced, trained):
    """Gain of the trained network at shifts it was not trained on: GMRES(30)
    reaches the same solution (true residual 1e-8) in fewer iterations than
    with the untrained network (the damped diagonal it starts from) and than
    without a preconditioner."""
    s, b = reduced
    net, _ = trained
    sysg = bse.System(s, precision="fp64", max_vec=3)
    x0, it0, r0, st0 = sysg.gmres(b, HELD_OUT_Z, rtol=1e-8, restart=30, max_iter=3000, precond="none")
    prior = bse.MLP(S.mlp_init(0))
    bse.attach_mlp(sysg, prior)
    xp, itp, rp, stp = sysg.gmres(b, HELD_OUT_Z, rtol=1e-8, restart=30, max_iter=3000, precond="mlp")
    bse.attach_mlp(sysg, net)
    x1, it1, r1, st1 = sysg.gmres(b, HELD_OUT_Z, rtol=1e-8, restart=30, max_iter=3000, precond="mlp")
    assert st0 == bse.BSE_OK and stp == bse.BSE_OK and st1 == bse.BSE_OK
    for j in range(len(HELD_OUT_Z)):
        close("mlp/gmres_trained/z%d" % j, x1[j], x0[j], (1e-6, 1e-6))
    assert np.all(r1 <= 1e-8)
    assert np.all(it1 < it0), (it0, it1)
    assert np.all(it1 < itp), (itp, it1)


def test_gmres_with_prior_network(reduced):
    """The untrained network (last layer zero) is the damped diagonal
    1/(D - omega - i(Gamma + 4.5 eV)): GMRES converges to the same solution in
    fewer iterations than without preconditioning."""
    s, b = reduced
    sysg = bse.System(s, precision="fp64", max_vec=3)
    net = bse.MLP(S.mlp_init(0))
    bse.attach_mlp(sysg, net)
    z = HELD_OUT_Z
    x0, it0, r0, st0 = sysg.gmres(b, z, rtol=1e-8, restart=30, max_iter=3000, precond="none")
    x1, it1, r1, st1 = sysg.gmres(b, z, rtol=1e-8, restart=30, max_iter=3000, precond="mlp")
    assert st0 == bse.BSE_OK and st1 == bse.BSE_OK
    for j in range(3):
        close("mlp/gmres_prior/z%d" % j, x1[j], x0[j], (1e-6, 1e-6))
    assert np.all(it1 < it0)


def test_network_trained_on_seeded_variants_gains_on_held_out_seed():
    """Training on three seeded variants of the reduced L2,3 system (different
    u_nk, band energies, projectors and couplings) and evaluating on a fourth
    seed it never saw: GMRES(30) needs fewer iterations with the trained
    network than with its prior, and fewer with the prior than without a
    preconditioner, at the same solution."""
    train = [S.reduced_l23(seed) for seed in (1, 2, 3)]
    systems = [bse.System(t, precision="fp64", max_vec=4) for t in train]
    bs = [S.make_start_vectors(t, 1)[0] for t in train]
    net = bse.MLP(S.mlp_init(0))
    hist = net.train(systems, bs, TRAIN_Z, epochs=6, batch=2, lr=1e-3, seed=2, steps=10)
    assert np.all(np.isfinite(hist)) and hist[-1] < hist[0]
    for g in systems:
        g.close()
    held = S.reduced_l23(0)
    b = S.make_start_vectors(held, 1)[0]
    sysg = bse.System(held, precision="fp64", max_vec=3)
    x0, it0, r0, st0 = sysg.gmres(b, HELD_OUT_Z, rtol=1e-8, restart=30, max_iter=3000, precond="none")
    prior = bse.MLP(S.mlp_init(0))
    bse.attach_mlp(sysg, prior)
    xp, itp, rp, stp = sysg.gmres(b, HELD_OUT_Z, rtol=1e-8, restart=30, max_iter=3000, precond="mlp")
    bse.attach_mlp(sysg, net)
    x1, it1, r1, st1 = sysg.gmres(b, HELD_OUT_Z, rtol=1e-8, restart=30, max_iter=3000, precond="mlp")
    assert st0 == bse.BSE_OK and stp == bse.BSE_OK and st1 == bse.BSE_OK
    for j in range(len(HELD_OUT_Z)):
        close("mlp/gmres_heldout/z%d" % j, x1[j], x0[j], (1e-6, 1e-6))
    print("held-out seed: iterations none %s, prior %s, trained on 3 other seeds %s" % (it0, itp, it1))
    assert np.sum(it1) < np.sum(itp) < np.sum(it0), (it0, itp, it1)
