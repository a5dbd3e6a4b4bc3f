"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here is independent of the oracle's own formulas: closed forms
(Eq. 2 resolvent of a diagonal or tridiagonal operator, supercell plane-wave
matrix elements of W), invariants (Hermiticity, moments, sum rule), library
routines on tiny inputs (eigh, solve) and brute-force loops.  The planted-
mistake tests at the end show that a plausible slip in the oracle fails one
of them.
"""
import math

import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import synth as S

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


TINY = [
    dict(seed=1),
    dict(seed=2, kshift=(0.5, 0.25, 0.0)),
    dict(seed=3, n_alpha=6, nk=(2, 2, 2), n_bands=4, nx=(2, 2, 3), n_proj=3),
    dict(seed=4, n_alpha=1, nk=(3, 1, 2), n_bands=2, nx=(3, 2, 1), n_proj=0),
]


# --- H psi --------------------------------------------------------------------

@pytest.mark.parametrize("kw", TINY)
def test_vectorised_equals_supercell_definition(kw):
    """The FFT/matmul route of Algorithm 1 equals H built from the definitions
    of its terms, with W_0 as the supercell potential's matrix between Bloch
    states accumulated point by point (no transforms, no band sums)."""
    s = S.tiny_system(**kw)
    rng = np.random.default_rng(7)
    for _ in range(2):
        psi = S.complex_normal(rng, (s.dim,))
        assert rel(O.apply_h(s, psi), O.apply_h_loop(s, psi)) < 1e-13


@pytest.mark.parametrize("kw", TINY)
def test_supercell_bloch_functions_orthonormal(kw):
    """phi_nk(x + R) = e^{ik.(x+R)} u_nk(x)/sqrt(Nk) over the supercell are
    orthonormal (orthonormal u_nk columns and sum_R e^{i(k'-k).R} = Nk delta_kk'),
    so W = c makes the supercell matrix c times the identity."""
    s = S.tiny_system(**kw)
    phi = O.bloch_on_supercell(s).reshape(-1, s.n_k * s.n_bands)
    assert np.abs(phi.conj().T @ phi - np.eye(s.n_k * s.n_bands)).max() < 1e-13
    s.w_rx = np.full_like(s.w_rx, -2.5)
    assert np.abs(O.w0_matrix_loop(s) + 2.5 * np.eye(s.n_k * s.n_bands)).max() < 1e-12


@pytest.mark.parametrize("kw", TINY)
def test_dense_h_hermitian(kw):
    s = S.tiny_system(**kw)
    h = O.dense_h(s)
    assert np.linalg.norm(h - h.conj().T) <= 1e-13 * np.linalg.norm(h)


@pytest.mark.parametrize("c", [0.0, -3.25, 1.7])
def test_constant_w_is_a_shift(c):
    """W(x,R) = c, no chi, no short range: H = diag(E_nk) + c*I exactly, because the
    u_nk columns are orthonormal and F_{R->k} F_{k->R} = 1 (Algorithm 1)."""
    s = S.tiny_system(5, kshift=(0.3, 0.0, 0.7), w_const=c, so=False, n_proj=0)
    h = O.dense_h(s)
    expect = np.diag(np.tile(s.e_nk.reshape(-1), s.n_alpha)).astype(np.complex128) + c * np.eye(s.dim)
    assert np.abs(h - expect).max() < 1e-12


def test_independent_particle_limit():
    """W = 0, M = 0: H = (E_nk delta_ab - chi_ab) delta_kk' delta_nn'."""
    s = S.tiny_system(6, n_alpha=6, nk=(2, 1, 2), n_bands=3, nx=(2, 2, 2), w_const=0.0, n_proj=0)
    h = O.dense_h(s)
    na, nk, nb = s.n_alpha, s.n_k, s.n_bands
    expect = np.zeros_like(h)
    for a in range(na):
        for b in range(na):
            for k in range(nk):
                for n in range(nb):
                    i, j = (a * nk + k) * nb + n, (b * nk + k) * nb + n
                    expect[i, j] = (s.e_nk[k, n] if a == b else 0.0) - s.chi[a, b]
    assert np.abs(h - expect).max() < 1e-13


@pytest.mark.parametrize("kshift", [(0.0, 0.0, 0.0), (0.5, 0.5, 0.5), (0.25, 0.0, 0.5)])
def test_plane_wave_supercell_matrix_elements(kshift):
    """With u_nk(x) = e^{iG_n.x}/sqrt(Nx), the state (n,k) is the supercell plane wave
    e^{i(k+G_n).(x+R)}/sqrt(Nx) (Eq. 8), so
    <n'k'|W_0|nk> = 1/(Nk Nx) sum_{x,R} W(x,R) e^{i(q-q').(x+R)},  q = k + G_n,
    summed directly over supercell positions (no FFT, no band sum)."""
    nk, nx, a = (2, 3, 2), (3, 2, 4), 7.4
    s = S.tiny_system(8, n_alpha=1, nk=nk, n_bands=4, nx=nx, n_proj=0, so=False, kshift=kshift)
    gvecs = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 1], [2, 1, 3]])
    jx = O._mesh_indices(nx)
    xpos = jx / np.asarray(nx) * a
    u = np.exp(1j * 2 * np.pi / a * (xpos @ gvecs.T)) / math.sqrt(s.n_x)     # [Nx][Nb]
    s.u = np.repeat(u[None], s.n_k, axis=0)
    s.e_nk = np.zeros_like(s.e_nk)
    h = O.dense_h(s)
    mk = O._mesh_indices(nk) + np.asarray(kshift)[None]
    kvec = 2 * np.pi * mk / (np.asarray(nk) * a)                            # [Nk][3]
    rpos = O._mesh_indices(nk) * a
    expect = np.zeros((s.n_k * 4, s.n_k * 4), dtype=np.complex128)
    for k in range(s.n_k):
        for n in range(4):
            q = kvec[k] + 2 * np.pi / a * gvecs[n]
            for k2 in range(s.n_k):
                for n2 in range(4):
                    q2 = kvec[k2] + 2 * np.pi / a * gvecs[n2]
                    acc = 0.0j
                    for r in range(s.n_k):
                        pos = xpos + rpos[r][None]
                        acc += np.sum(s.w_rx[r] * np.exp(1j * (pos @ (q - q2))))
                    expect[k2 * 4 + n2, k * 4 + n] = acc / (s.n_k * s.n_x)
    assert np.abs(h - expect).max() < 1e-12 * max(1.0, np.abs(expect).max())


def test_short_range_index_convention():
    """M with a single entry at (alpha0, p0),(alpha0, p0): V_SR psi lives on alpha0
    only and equals conj(A_p0) <A_p0^*|psi_alpha0> (Sec. 3.2.2 projection)."""
    s = S.tiny_system(9, n_alpha=3, n_proj=4, w_const=0.0, so=False)
    s.e_nk[:] = 0
    a0, p0 = 2, 1
    s.m_sr = np.zeros_like(s.m_sr)
    s.m_sr[a0 * 4 + p0, a0 * 4 + p0] = 1.0
    psi = S.complex_normal(np.random.default_rng(3), (s.dim,))
    out = O.apply_h(s, psi).reshape(3, s.n_k, s.n_bands)
    p = psi.reshape(3, s.n_k, s.n_bands)
    ap = s.a_proj[p0]
    expect = np.zeros_like(out)
    expect[a0] = np.conj(ap) * np.sum(ap * p[a0])
    assert np.abs(out - expect).max() < 1e-14


def test_short_range_spectrum_matches_m():
    """If the projector rows are orthonormal, the nonzero eigenvalues of V_SR are
    those of M (A (x) I is an isometry onto its range)."""
    s = S.tiny_system(10, n_alpha=2, nk=(2, 2, 1), n_bands=4, nx=(2, 2, 2), n_proj=3,
                      w_const=0.0, so=False)
    s.e_nk[:] = 0
    a = s.a_proj.reshape(3, -1)
    q, _ = np.linalg.qr(a.conj().T)
    s.a_proj = q.conj().T.reshape(s.a_proj.shape)
    ev = np.linalg.eigvalsh(O.dense_h(s))
    big = np.sort(ev[np.abs(ev) > 1e-10])
    assert np.allclose(big, np.sort(np.linalg.eigvalsh(s.m_sr)), atol=1e-12)


def test_jacobi_diag_is_diagonal_of_h():
    s = S.tiny_system(11, n_alpha=6, nk=(2, 1, 2), n_bands=3, nx=(2, 2, 2), n_proj=2)
    d = O.jacobi_diag(s).reshape(-1)
    assert np.abs(d - np.real(np.diag(O.dense_h(s)))).max() < 1e-12


# --- Haydock ------------------------------------------------------------------

def test_haydock_recovers_tridiagonal():
    """H tridiagonal in the basis e_0, e_1, ... with b = e_0: the recursion returns
    its diagonal and |off-diagonal| exactly (the Lanczos basis is e_i up to phases)."""
    rng = np.random.default_rng(0)
    n = 12
    d = rng.normal(size=n)
    off = rng.normal(size=n - 1) + 1j * rng.normal(size=n - 1)
    t = np.diag(d).astype(np.complex128) + np.diag(off, -1) + np.diag(np.conj(off), 1)
    e0 = np.zeros(n, dtype=np.complex128)
    e0[0] = 2.0
    a, b, nd, brk = O.haydock(lambda v: t @ v, e0, n - 1)
    assert nd == n - 1 and not brk
    assert np.allclose(a, d[: n - 1], atol=1e-12)
    assert np.allclose(b[1:], np.abs(off), atol=1e-12)
    assert b[0] == pytest.approx(2.0)


def test_cf_single_pole():
    """One step: sigma = (b0^2/pi) Gamma/((omega - a0)^2 + Gamma^2)."""
    om = np.linspace(-3, 3, 101)
    sig = O.cf_spectrum(np.array([0.4]), np.array([1.5, 0.0]), om, 0.3)
    assert np.allclose(sig, 1.5 ** 2 / np.pi * 0.3 / ((om - 0.4) ** 2 + 0.09), rtol=1e-13)


def test_cf_terminator_semicircle():
    """Constant chain a_i = a, b_i = c: g(z) = [(z-a) - sqrt((z-a)^2 - 4c^2)]/(2c^2)
    (semicircle); the terminated fraction reproduces it at any depth."""
    a0, c = 0.7, 1.3
    om = np.linspace(-4, 5, 301)
    z = om + 0.2j
    zz = z - a0
    r = np.sqrt(zz * zz - 4 * c * c)
    g = np.where(np.imag((zz - r) / (2 * c * c)) <= 0, (zz - r) / (2 * c * c), (zz + r) / (2 * c * c))
    for depth in (1, 3, 10):
        gt = O.cf_green(np.full(depth, a0), np.full(depth + 1, c), z, terminator=True)
        assert np.allclose(gt, g, rtol=1e-12, atol=1e-12)


@pytest.fixture(scope="module")
def kedge():
    s = S.make_system("k_edge_small")
    return s, O.dense_h(s), S.make_start_vectors(s, 1)[0]


def test_kedge_shapes(kedge):
    s, h, b = kedge
    assert s.dim == 128 and h.shape == (128, 128)


def test_haydock_full_equals_exact_diagonalisation(kedge):
    """N = 128 steps with full re-orthogonalisation: the continued fraction is the
    exact resolvent, so sigma equals the eigh spectrum (Eq. 1-2)."""
    s, h, b = kedge
    a, bb, nd, brk = O.haydock(lambda v: O.apply_h(s, v), b, s.dim, reorth=True)
    om = S.omega_grid()
    sig = O.cf_spectrum(a, bb, om, 0.5)
    ex = O.exact_spectrum(h, b, om, 0.5)
    assert rel(sig, ex) < 1e-10


def test_moments_of_continued_fraction(kedge):
    """<b|H^m|b> = |b|^2 (T^m)_00 for m <= 2n - 1, T = tridiag(a, b_1..b_{n-1})."""
    s, h, b = kedge
    n = 6
    a, bb, _, _ = O.haydock(lambda v: O.apply_h(s, v), b, n)
    t = np.diag(a) + np.diag(bb[1:n], 1) + np.diag(bb[1:n], -1)
    v = b.copy()
    tm = np.eye(n)
    for m in range(1, 2 * n):
        v = h @ v
        tm = tm @ t
        mom = np.vdot(b, v)
        assert abs(mom - bb[0] ** 2 * tm[0, 0]) <= 1e-9 * max(1.0, abs(mom))


def test_sum_rule(kedge):
    """Zeroth moment: the integral of sigma over a window equals
    sum_j w_j (1/pi)[atan((w_hi - E_j)/G) - atan((w_lo - E_j)/G)] and tends to <b|b>."""
    s, h, b = kedge
    a, bb, _, _ = O.haydock(lambda v: O.apply_h(s, v), b, s.dim, reorth=True)
    om = np.linspace(-5, 30, 200001)
    sig = O.cf_spectrum(a, bb, om, 0.5)
    integ = np.trapezoid(sig, om)
    ev, evec = np.linalg.eigh(h)
    w = np.abs(evec.conj().T @ b) ** 2
    closed = np.sum(w * (np.arctan((30 - ev) / 0.5) - np.arctan((-5 - ev) / 0.5))) / np.pi
    assert integ == pytest.approx(closed, rel=1e-8)
    assert closed == pytest.approx(np.vdot(b, b).real, rel=0.05)
    wide = np.linspace(-2000, 2000, 4_000_001)
    assert np.trapezoid(O.cf_spectrum(a, bb, wide, 0.5), wide) == pytest.approx(1.0, abs=2e-3)


def test_independent_particle_spectrum():
    """W = 0, M = 0: sigma is a closed-form sum of Lorentzians at E_nk + eig(-chi)."""
    s = S.tiny_system(12, n_alpha=6, nk=(2, 1, 1), n_bands=3, nx=(2, 2, 2), w_const=0.0, n_proj=0)
    b = S.make_start_vectors(s, 1)[0]
    ev_c, vec_c = np.linalg.eigh(-s.chi)
    bb = b.reshape(6, s.n_k, s.n_bands)
    proj = np.einsum("aj,akn->jkn", vec_c.conj(), bb)               # weights in eigenbasis
    om = np.linspace(-10, 30, 801)
    g = 0.5
    ex = np.zeros_like(om)
    for j in range(6):
        for k in range(s.n_k):
            for n in range(s.n_bands):
                e = s.e_nk[k, n] + ev_c[j]
                ex += abs(proj[j, k, n]) ** 2 * g / ((om - e) ** 2 + g * g) / np.pi
    a, b2, nd, _ = O.haydock(lambda v: O.apply_h(s, v), b, s.dim, reorth=True)
    assert rel(O.cf_spectrum(a, b2, om, g), ex) < 1e-10


# --- GMRES --------------------------------------------------------------------

@pytest.mark.parametrize("pre", [False, True])
@pytest.mark.parametrize("restart", [30, 7])
def test_gmres_solution_and_resolvent(kedge, pre, restart):
    s, h, b = kedge
    z = 6.0 + 0.5j
    d = O.jacobi_diag(s).reshape(-1)
    pc = (lambda v: v / (d - z)) if pre else None
    x, nmv, rr = O.gmres(lambda v: O.apply_h(s, v), b, z, pc, rtol=1e-10, restart=restart)
    assert rr <= 1e-10
    xs = np.linalg.solve(h - z * np.eye(s.dim), b)
    assert rel(x, xs) < 1e-8
    ev, evec = np.linalg.eigh(h)
    res = np.sum(np.abs(evec.conj().T @ b) ** 2 / (ev - z))
    assert abs(np.vdot(b, x) - res) < 1e-8 * abs(res)


def test_gmres_unrestarted_terminates_in_n_steps():
    """Without restarts GMRES is exact after at most N Arnoldi steps."""
    s = S.tiny_system(13, n_alpha=2, nk=(2, 1, 1), n_bands=3, nx=(2, 2, 2))
    b = S.make_start_vectors(s, 1)[0]
    x, nmv, rr = O.gmres(lambda v: O.apply_h(s, v), b, 1.0 + 0.1j, rtol=1e-12, restart=s.dim)
    assert nmv <= s.dim and rr < 1e-11


def test_gmres_spectrum_equals_haydock(kedge):
    """sigma(omega) = (1/pi) Im <b|x(omega + i Gamma)> equals the Haydock value."""
    s, h, b = kedge
    a, bb, _, _ = O.haydock(lambda v: O.apply_h(s, v), b, s.dim, reorth=True)
    for om in (-1.0, 4.0, 12.5):
        x, _, _ = O.gmres(lambda v: O.apply_h(s, v), b, om + 0.5j, rtol=1e-11)
        sg = np.imag(np.vdot(b, x)) / np.pi
        assert sg == pytest.approx(O.cf_spectrum(a, bb, np.array([om]), 0.5)[0], rel=1e-8)


# --- inputs (workload definitions) ----------------------------------------------

def test_spin_orbit_eigenvalues_golden():
    """-chi for the 5.7 eV L2,3 split: -1.9 eV (x4, L3) and +3.8 eV (x2, L2)."""
    from pathlib import Path
    g = np.loadtxt(Path(__file__).parent / "golden" / "so_l23_eigenvalues.txt")
    ev = np.sort(np.linalg.eigvalsh(-S.spin_orbit_p(5.7)))
    assert np.allclose(ev, np.sort(g), atol=1e-13)


def test_w_model_limits():
    eps = 5.0
    assert S.w_erf_hartree(np.array([0.0]), eps)[0] == pytest.approx(-2 / (0.5 * math.sqrt(math.pi) * eps))
    r = np.array([6.0, 9.0])
    assert np.allclose(S.w_erf_hartree(r, eps), -1.0 / (eps * r), rtol=1e-12)
    assert S.w_erf_hartree(np.array([1e-7]), eps)[0] == pytest.approx(-2 / (0.5 * math.sqrt(math.pi) * eps), rel=1e-9)


def test_bloch_orthonormal():
    s = S.make_system("k_edge_small")
    for k in range(s.n_k):
        assert np.abs(s.u[k].conj().T @ s.u[k] - np.eye(s.n_bands)).max() < 1e-13


def test_w_minimum_image():
    """W depends on the distance to the nearest core image in the nk*a supercell."""
    w = S.sample_w((2, 2, 2), (2, 2, 2), 4.0, 5.0)
    # R = 0, x = 0 -> r = 0 ; R = (1,0,0), x = (1/2 a,0,0): pos 6 in period 8 -> r = 2
    assert w[0, 0] == pytest.approx(S.w_erf_hartree(np.array([0.0]), 5.0)[0] * S.HARTREE_EV)
    ir = 4  # r = (1,0,0)
    ix = 4  # x = (1,0,0) grid index -> 2.0 bohr
    assert w[ir, ix] == pytest.approx(S.w_erf_hartree(np.array([2.0]), 5.0)[0] * S.HARTREE_EV)


# --- planted mistakes: each must be caught by a pin above -------------------------

def test_planted_conjugated_phase_is_caught(monkeypatch):
    good = O.kx_phase
    monkeypatch.setattr(O, "kx_phase", lambda nk, nx, ks=(0, 0, 0): np.conj(good(nk, nx, ks)))
    with pytest.raises(AssertionError):
        test_plane_wave_supercell_matrix_elements((0.0, 0.0, 0.0))


def test_planted_transposed_w_is_caught(monkeypatch):
    good = O.apply_w0

    def bad(s, psi):
        s2 = S.BSESystem(**{**s.__dict__})
        nkt, nxt = tuple(s.nk), tuple(s.nx)
        if nkt == nxt:
            s2.w_rx = s.w_rx.T.copy()
        else:                       # reverse the R axis ordering instead
            s2.w_rx = s.w_rx[::-1].copy()
        return good(s2, psi)

    monkeypatch.setattr(O, "apply_w0", bad)
    with pytest.raises(AssertionError):
        test_plane_wave_supercell_matrix_elements((0.0, 0.0, 0.0))


def test_planted_missing_normalisation_is_caught(monkeypatch):
    good = O.apply_w0
    monkeypatch.setattr(O, "apply_w0", lambda s, psi: good(s, psi) * np.prod(s.nk))
    with pytest.raises(AssertionError):
        test_constant_w_is_a_shift(-3.25)


def test_planted_sr_index_order_is_caught(monkeypatch):
    good = O.apply_sr

    def bad(s, psi):
        if s.a_proj is None:
            return good(s, psi)
        s2 = S.BSESystem(**{**s.__dict__})
        na, npj = s.n_alpha, s.a_proj.shape[0]
        perm = np.arange(na * npj).reshape(na, npj).T.reshape(-1)   # p slow instead of alpha
        s2.m_sr = s.m_sr[np.ix_(perm, perm)]
        return good(s2, psi)

    monkeypatch.setattr(O, "apply_sr", bad)
    with pytest.raises(AssertionError):
        test_short_range_index_convention()


def test_planted_haydock_missing_term_is_caught(monkeypatch):
    def bad(apply, b, n_steps, reorth=False, breakdown_tol=1e-12):
        b0 = np.linalg.norm(b)
        v = b / b0
        a_l, b_l = [], [b0]
        for i in range(n_steps):
            w = apply(v)
            ai = float(np.real(np.vdot(v, w)))
            a_l.append(ai)
            w = w - ai * v                      # b_i v_{i-1} dropped
            bn = float(np.linalg.norm(w))
            b_l.append(bn)
            v = w / bn
        return np.array(a_l), np.array(b_l), len(a_l), False

    monkeypatch.setattr(O, "haydock", bad)
    with pytest.raises(AssertionError):
        test_haydock_recovers_tridiagonal()


@pytest.mark.parametrize("reorth,tol", [(True, 1e-9), (False, 1e-6)])
def test_golden_haydock_regression(kedge, reorth, tol):
    """Stored oracle coefficients (written by tests/golden/make_golden.py) still hold."""
    from pathlib import Path
    s, h, b = kedge
    name = "k_edge_small_haydock_%s.txt" % ("reorth" if reorth else "plain")
    g = np.loadtxt(Path(__file__).parent / "golden" / name)
    a, bb, nd, _ = O.haydock(lambda v: O.apply_h(s, v), b, 100, reorth=reorth)
    assert nd == 100
    assert np.allclose(a, g[:100, 1], rtol=tol, atol=tol)
    assert np.allclose(bb, g[:, 2], rtol=tol, atol=tol)


def test_local_projection_against_loop_and_orthonormal_columns():
    """A[p][k][n] = dv sum_x conj(f_p(x)) e^{ik.x} u_nk(x): the vectorised
    oracle against an explicit loop, and with f_p = e^{ik0.x} u_{n0 k0} / dv
    (shifted mesh) the orthonormal columns give A[p][k0][n] = delta_{n n0}."""
    s = S.tiny_system(71, n_alpha=1, nk=(2, 1, 2), n_bands=3, nx=(3, 2, 2), n_proj=0, kshift=(0.5, 0.0, 0.25))
    rng = np.random.default_rng(2)
    f = S.complex_normal(rng, (4, s.n_x))
    dv = 0.37
    a = O.local_projection(s.u, s.nk, s.nx, f, dv, s.kshift)
    ph = O.kx_phase(s.nk, s.nx, s.kshift)
    for p in range(4):
        for k in range(s.n_k):
            for n in range(s.n_bands):
                ref = dv * sum(np.conj(f[p, x]) * ph[k, x] * s.u[k, x, n] for x in range(s.n_x))
                assert abs(a[p, k, n] - ref) < 1e-13
    k0, n0 = 3, 1
    f2 = (ph[k0] * s.u[k0, :, n0])[None, :] / dv
    a2 = O.local_projection(s.u, s.nk, s.nx, f2, dv, s.kshift)
    assert np.allclose(a2[0, k0], np.eye(s.n_bands)[n0], atol=1e-13)


def test_screening_chi0_equals_static_lindhard_form():
    """The imaginary-axis integral of G G (Sec. 3.3) against its closed form:
    (1/2 pi) int dt / ((a + i t)(b + i t)) = 1/(b - a) when a > 0 > b, 0 when
    a and b have the same sign, so chi0(r, r') = sum_{K occ, L empty}
    [psi_K(r) psi_K*(r') psi_L(r') psi_L*(r) + (K <-> L)] / (eps_K - eps_L)."""
    psi, eps = S.screening_grid_states(7, 6, seed=1)
    mu = float(np.sort(eps)[2] + np.sort(eps)[3]) / 2   # three states below mu, three above
    t, w = S.imag_axis_quadrature(600, scale=8.0)
    chi = O.screening_chi0(psi, eps, mu, t, w)
    ref = np.zeros((7, 7), dtype=np.complex128)
    for K in range(6):
        for L in range(6):
            if eps[K] < mu < eps[L]:
                pk, pl = psi[:, K], psi[:, L]
                term = (np.outer(pk, pk.conj()) * np.outer(pl, pl.conj()).T
                        + np.outer(pl, pl.conj()) * np.outer(pk, pk.conj()).T) / (eps[K] - eps[L])
                ref += term
    assert np.abs(ref).max() > 1e-3
    assert np.abs(chi - ref).max() < 1e-6 * np.abs(ref).max()
    # a system with every state on one side of mu does not respond
    chi_empty = O.screening_chi0(psi, eps + 20.0, mu, t, w)
    assert np.abs(chi_empty).max() < 1e-6 * np.abs(ref).max()


def test_local_projection_single_k_equals_shifted_one_point_mesh():
    """The projection at k-point m of an n_k mesh depends on k only through
    e^{ik.x}: a one-point mesh shifted by m / n_k gives the same phases, so
    the same coefficients (the identity the full-size GPU check samples by)."""
    s = S.make_system_from(dict(id=960, n_alpha=1, nk=(4, 2, 3), n_bands=5, nx=(6, 4, 5), cell=7.4, eps=5.0,
                                n_proj=0), 0)
    f = S.local_functions_on_grid(s.nx, s.cell, 2.5)
    dv = s.cell ** 3 / s.n_x
    a = O.local_projection(s.u, s.nk, s.nx, f, dv)
    for m in [(0, 0, 0), (3, 1, 2), (1, 0, 1)]:
        k = (m[0] * s.nk[1] + m[1]) * s.nk[2] + m[2]
        r = O.local_projection(s.u[k:k + 1], (1, 1, 1), s.nx, f, dv, tuple(m[d] / s.nk[d] for d in range(3)))
        assert np.abs(a[:, k, :] - r[:, 0, :]).max() < 1e-14 * max(1.0, np.abs(a).max())
    assert np.abs(a).max() > 0.1
