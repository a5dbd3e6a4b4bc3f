"""Pins of the learned-preconditioner oracle: finite-difference gradients,
the zero-network closed form, the low-rank operator against a dense matrix,
and one Adam step in closed form."""
import numpy as np
import pytest

from oracle import bse_oracle as O
from oracle import mlp_oracle as M
from paper_1601_07728_gb300 import synth as S


@pytest.fixture(scope="module")
def problem():
    s = S.tiny_system(61, n_alpha=6, nk=(2, 1, 2), n_bands=3, nx=(2, 2, 2), n_proj=3)
    diag = O.jacobi_diag(s).reshape(-1)
    z = 7.0 + 0.5j
    x = M.system_features(s, diag, z.real, z.imag)
    rng = np.random.default_rng(4)
    rs = [S.complex_normal(rng, (s.dim,)) for _ in range(2)]
    es = [S.complex_normal(rng, (s.dim,)) for _ in range(2)]
    params = M.unpack(S.mlp_init(3).astype(np.float64))
    params["w3"] = params["w3"] + 0.05 * rng.standard_normal(params["w3"].shape)
    params["b3"] = 0.05 * rng.standard_normal(params["b3"].shape)
    return s, diag, z, x, rs, es, params


def test_shapes():
    assert M.n_params() == S.mlp_init(0).size == 12 * 128 + 128 + 128 * 128 + 128 + 128 * 34 + 34


def test_gradient_matches_central_differences(problem):
    """Backpropagation against (L(w + h) - L(w - h)) / 2h of the FP64 network,
    at FP16-representable weights (where the FP16 network and the FP64 network
    coincide, so this is also the gradient the GPU's FP16-weight net has)."""
    s, diag, z, x, rs, es, params = problem
    p16 = M.fp16(params)
    tot, g = M.grad(p16, x, diag, z, rs, es)
    assert tot == pytest.approx(M.loss(p16, x, diag, z, rs, es), rel=1e-12)
    rng = np.random.default_rng(8)
    h = 1e-6
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        flat = p16[name].reshape(-1)
        for idx in rng.choice(flat.size, size=4, replace=False):
            up = {k: v.copy() for k, v in p16.items()}
            dn = {k: v.copy() for k, v in p16.items()}
            up[name].reshape(-1)[idx] += h
            dn[name].reshape(-1)[idx] -= h
            fd = (M.loss(up, x, diag, z, rs, es, quantize=False) - M.loss(dn, x, diag, z, rs, es, quantize=False)) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)


@pytest.mark.parametrize("scaled", [False, True])
def test_spai_gradient_matches_central_differences(problem, scaled):
    """Approximate-inverse loss sum_t |alpha_t (H - z) P r_t - r_t|^2/|r_t|^2 on
    residual probes (alpha_t = 1, or the minimal-residual scale):
    backpropagation (through two H applications per probe) against central
    differences of the FP64 network."""
    s, diag, z, x, rs, es, params = problem
    p16 = M.fp16(params)
    happly = lambda v: O.apply_h(s, v)
    tot, g = M.spai_grad(p16, x, diag, z, rs, happly, scaled=scaled)
    assert tot == pytest.approx(M.spai_loss(p16, x, diag, z, rs, happly, scaled=scaled), rel=1e-12)
    rng = np.random.default_rng(9)
    h = 1e-6
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        flat = p16[name].reshape(-1)
        for idx in rng.choice(flat.size, size=3, replace=False):
            up = {k: v.copy() for k, v in p16.items()}
            dn = {k: v.copy() for k, v in p16.items()}
            up[name].reshape(-1)[idx] += h
            dn[name].reshape(-1)[idx] -= h
            fd = (M.spai_loss(up, x, diag, z, rs, happly, quantize=False, scaled=scaled)
                  - M.spai_loss(dn, x, diag, z, rs, happly, quantize=False, scaled=scaled)) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)


@pytest.mark.parametrize("k", [1, 4])
def test_krylov_gradient_matches_central_differences(problem, k):
    """k-step minimal-residual loss: back-propagation through the forward and
    adjoint Krylov chains (2k applications of H per probe) against central
    differences of the FP64 network."""
    s, diag, z, x, rs, es, params = problem
    p16 = M.fp16(params)
    happly = lambda v: O.apply_h(s, v)
    tot, g = M.krylov_grad(p16, x, diag, z, rs, happly, k)
    assert tot == pytest.approx(M.krylov_loss(p16, x, diag, z, rs, happly, k), rel=1e-12)
    rng = np.random.default_rng(10 + k)
    h = 1e-6
    for name in ("w1", "b1", "w2", "b2", "w3", "b3"):
        flat = p16[name].reshape(-1)
        for idx in rng.choice(flat.size, size=3, replace=False):
            up = {kk: v.copy() for kk, v in p16.items()}
            dn = {kk: v.copy() for kk, v in p16.items()}
            up[name].reshape(-1)[idx] += h
            dn[name].reshape(-1)[idx] -= h
            fd = (M.krylov_loss(up, x, diag, z, rs, happly, k, quantize=False)
                  - M.krylov_loss(dn, x, diag, z, rs, happly, k, quantize=False)) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, idx, fd, an)


def test_krylov_loss_is_gmres_residual(problem):
    """The k-step loss on one probe equals the squared relative residual of k
    steps of right-preconditioned GMRES from x_0 = 0 for the right-hand side r
    (oracle GMRES, no restart), and one step equals the scaled approximate-
    inverse loss."""
    s, diag, z, x, rs, es, params = problem
    o, _ = M.forward(M.fp16(params), x)
    p, u, v = M.assemble(o, diag, z)
    happly = lambda vv: O.apply_h(s, vv)
    r = rs[0]
    k = 3
    a = lambda vv: happly(vv) - z * vv
    xg, it, rel = O.gmres(happly, r, z, lambda vv: M.apply(p, u, v, vv), rtol=1e-300, restart=k, max_iter=k)
    resid = np.linalg.norm(r - a(xg)) / np.linalg.norm(r)
    assert M.krylov_loss(params, x, diag, z, [r], happly, k) == pytest.approx(resid ** 2, rel=1e-8)
    assert M.krylov_loss(params, x, diag, z, rs, happly, 1) == pytest.approx(
        M.spai_loss(params, x, diag, z, rs, happly, scaled=True), rel=1e-10)


def test_spai_optimal_diagonal_closed_form():
    """For a diagonal P the approximate-inverse loss over all unit probes is
    |A diag(p) - I|_F^2, minimised column by column by
    p_j = conj(A_jj) / |A_:j|^2 -- the damped diagonal the network starts from
    approximates exactly this."""
    s = S.tiny_system(63, n_alpha=2, nk=(2, 1, 1), n_bands=3, nx=(2, 2, 2), n_proj=2)
    h = O.dense_h(s)
    z = 3.0 + 0.5j
    a = h - z * np.eye(s.dim)
    p_opt = np.conj(np.diag(a)) / (np.abs(a) ** 2).sum(0)
    f = lambda p: np.linalg.norm(a @ np.diag(p) - np.eye(s.dim)) ** 2
    rng = np.random.default_rng(2)
    for _ in range(5):
        dp = 1e-3 * (rng.standard_normal(s.dim) + 1j * rng.standard_normal(s.dim))
        assert f(p_opt + dp) > f(p_opt)


def test_zero_network_is_damped_diagonal(problem):
    """Last layer zero: P = diag(1 / (D - omega - i(Gamma + ETA0)))."""
    s, diag, z, x, rs, es, params = problem
    p0 = {k: v.copy() for k, v in params.items()}
    p0["w3"][:] = 0
    p0["b3"][:] = 0
    o, _ = M.forward(M.fp16(p0), x)
    p, u, v = M.assemble(o, diag, z)
    assert np.allclose(p, 1.0 / (diag - z.real - 1j * (z.imag + M.ETA0)), rtol=1e-14)
    assert np.abs(u).max() == 0 and np.abs(v).max() == 0


def test_scaled_loss_is_one_step_minimal_residual(problem):
    """The scaled per-probe term equals the squared residual reduction of one
    minimal-residual step min_a |r - a (H - z) P r|^2 / |r|^2, found here by a
    least-squares solve on the dense operator."""
    s, diag, z, x, rs, es, params = problem
    o, _ = M.forward(M.fp16(params), x)
    p, u, v = M.assemble(o, diag, z)
    a = O.dense_h(s) - z * np.eye(s.dim)
    pd = np.diag(p) + u @ v.conj().T / s.dim
    want = 0.0
    for r in rs:
        col = (a @ pd @ r)[:, None]
        coef = np.linalg.lstsq(col, r, rcond=None)[0]
        want += np.linalg.norm(r - col @ coef) ** 2 / np.linalg.norm(r) ** 2
    got = M.spai_loss(params, x, diag, z, rs, lambda v: O.apply_h(s, v), scaled=True)
    assert got == pytest.approx(want, rel=1e-10)
    assert 0.0 <= got <= len(rs)


def test_low_rank_operator_against_dense(problem):
    s, diag, z, x, rs, es, params = problem
    o, _ = M.forward(M.fp16(params), x)
    p, u, v = M.assemble(o, diag, z)
    dense = np.diag(p) + u @ v.conj().T / s.dim
    for r in rs:
        assert np.allclose(M.apply(p, u, v, r), dense @ r, rtol=1e-12, atol=1e-14)


def test_adam_first_step_closed_form():
    """First Adam step: m_hat = g, v_hat = g^2, so w -= lr g / (|g| + eps)."""
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g = {"w": np.array([0.3, -4.0, 1e-9])}
    z = {"w": np.zeros(3)}
    newp, m, v = M.adam(p, g, z, z, 1, 0.01)
    assert np.allclose(newp["w"], p["w"] - 0.01 * g["w"] / (np.abs(g["w"]) + 1e-8), rtol=1e-15)


def test_planted_wrong_silu_derivative_is_caught(problem, monkeypatch):
    monkeypatch.setattr(M, "dsilu", lambda x: 1.0 / (1.0 + np.exp(-x)))
    with pytest.raises(AssertionError):
        test_gradient_matches_central_differences(problem)
