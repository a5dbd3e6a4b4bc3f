"""Pins of the structured short-range inputs (Sec. 3.2.2): Wigner 3j and
Gaunt factors against closed forms and orthogonality, the Slater x Gaunt
coupling matrix M (Hermitian, spin-diagonal, invariant under total orbital
rotations of electron and hole) and the dipole-shaped start vectors (only
the s and d local functions contribute from a p core level)."""
import math

import numpy as np
import pytest

from paper_1601_07728_gb300 import synth as S


def test_wigner3j_closed_forms_and_orthogonality():
    assert S.wigner3j(1, 1, 0, 0, 0, 0) == pytest.approx(-1 / math.sqrt(3), abs=1e-15)
    assert S.wigner3j(1, 1, 2, 0, 0, 0) == pytest.approx(math.sqrt(2 / 15), abs=1e-15)
    assert S.wigner3j(2, 2, 0, 1, -1, 0) == pytest.approx(-1 / math.sqrt(5), abs=1e-15)
    assert S.wigner3j(1, 1, 1, 0, 0, 0) == 0.0                  # odd sum with all m = 0
    # sum_{m1 m2} (2 j3 + 1) (j1 j2 j3; m1 m2 m3) (j1 j2 j3'; m1 m2 m3') = delta delta
    for j1, j2 in ((1, 2), (2, 3), (1, 1)):
        for j3 in range(abs(j1 - j2), j1 + j2 + 1):
            for j3p in range(abs(j1 - j2), j1 + j2 + 1):
                for m3 in range(-min(j3, j3p), min(j3, j3p) + 1):
                    s = sum((2 * j3 + 1) * S.wigner3j(j1, j2, j3, m1, m2, m3) * S.wigner3j(j1, j2, j3p, m1, m2, m3)
                            for m1 in range(-j1, j1 + 1) for m2 in range(-j2, j2 + 1))
                    assert s == pytest.approx(1.0 if j3 == j3p else 0.0, abs=1e-12)


def test_gaunt_identity_parity_and_dipole():
    for l in range(4):
        for m in range(-l, l + 1):
            for m2 in range(-l, l + 1):
                assert S.gaunt(l, m, 0, 0, l, m2) == pytest.approx(1.0 if m == m2 else 0.0, abs=1e-14)
    assert S.gaunt(1, 0, 1, 0, 1, 0) == 0.0                     # parity: l + k + l' odd
    assert S.gaunt(2, 1, 2, 1, 1, 0) == 0.0                     # parity again
    assert S.gaunt(0, 0, 1, 0, 1, 0) ** 2 == pytest.approx(1 / 3, abs=1e-14)   # |<s|C^1_0|p_0>|^2
    # sum_{q, m} |<l m|C^k_q|l' m'>|^2 = (2l + 1) (l k l'; 0 0 0)^2 for every m' (3j
    # orthogonality): p -> d dipole strength 5 * 2/15 = 2/3, p -> s 1/3, from each core m
    for mc in (-1, 0, 1):
        tot_d = sum(S.gaunt(2, m, 1, q, 1, mc) ** 2 for q in (-1, 0, 1) for m in range(-2, 3))
        tot_s = sum(S.gaunt(0, 0, 1, q, 1, mc) ** 2 for q in (-1, 0, 1))
        assert tot_d == pytest.approx(2 / 3, abs=1e-12)
        assert tot_s == pytest.approx(1 / 3, abs=1e-12)


@pytest.fixture(scope="module")
def mstruct():
    return S.structured_couplings(np.random.default_rng(5))


def _orbital_block(M):
    npj = len(S.local_functions())
    idx = [2 * (mc + 1) * npj + p for mc in (-1, 0, 1) for p in range(npj)]   # spin up
    return M[np.ix_(idx, idx)]


def _total_lplus():
    funcs = S.local_functions()
    npj = len(funcs)
    le = np.zeros((npj, npj))
    for p, (nu, l, m) in enumerate(funcs):
        if m < l:
            le[S.local_index(nu, l, m + 1), p] = math.sqrt(l * (l + 1) - m * (m + 1))
    lh = np.zeros((3, 3))
    for i, mc in enumerate((-1, 0, 1)):
        if mc < 1:
            lh[i + 1, i] = math.sqrt(2 - mc * (mc + 1))
    return np.kron(lh, np.eye(npj)) + np.kron(np.eye(3), le)


def test_coupling_matrix_hermitian_spin_diagonal_and_rotation_invariant(mstruct):
    M = mstruct
    npj = len(S.local_functions())
    assert np.abs(M - M.conj().T).max() < 1e-14
    for a in range(6):
        for b in range(6):
            if a % 2 != b % 2:   # different spin
                assert np.abs(M[a * npj:(a + 1) * npj, b * npj:(b + 1) * npj]).max() == 0.0
    orb = _orbital_block(M)
    lp = _total_lplus()
    lz = np.diag([mc + m for mc in (-1, 0, 1) for (_, _, m) in S.local_functions()])
    assert np.abs(orb @ lz - lz @ orb).max() < 1e-12
    assert np.abs(orb @ lp - lp @ orb).max() < 1e-12 * max(1.0, np.abs(orb).max())
    assert np.abs(orb).max() > 0.05                              # not trivially zero


def test_planted_phase_error_breaks_rotation_invariance(monkeypatch):
    real = S.gaunt
    monkeypatch.setattr(S, "gaunt", lambda l1, m1, k, q, l2, m2: real(l1, m1, k, q, l2, m2) * (-1) ** m1)
    orb = _orbital_block(S.structured_couplings(np.random.default_rng(5)))
    lp = _total_lplus()
    assert np.abs(orb @ lp - lp @ orb).max() > 1e-3


def test_dipole_vectors_see_only_s_and_d_functions():
    rng = np.random.default_rng(9)
    npj = len(S.local_functions())
    a = S.complex_normal(rng, (npj, 2, 5))
    b = S.dipole_start_vectors(a)
    a2 = a.copy()
    for p, (nu, l, m) in enumerate(S.local_functions()):
        if l in (1, 3):
            a2[p] = S.complex_normal(rng, (2, 5))
    assert np.allclose(S.dipole_start_vectors(a2), b, atol=1e-14)
    assert b.shape == (3, 6 * 10)
    assert np.allclose(np.linalg.norm(b, axis=1), 1.0)
    # spin-independent: both spin copies of each core m carry the same amplitudes
    bb = b.reshape(3, 6, 10)
    assert np.allclose(bb[:, 0::2], bb[:, 1::2])


def test_spherical_harmonics_closed_forms():
    rng = np.random.default_rng(3)
    th = rng.uniform(0, np.pi, 50)
    ph = rng.uniform(-np.pi, np.pi, 50)
    assert np.allclose(S.spherical_harmonic(0, 0, th, ph), 0.5 / math.sqrt(math.pi))
    assert np.allclose(S.spherical_harmonic(1, 0, th, ph), math.sqrt(3 / (4 * math.pi)) * np.cos(th))
    assert np.allclose(S.spherical_harmonic(1, 1, th, ph), -math.sqrt(3 / (8 * math.pi)) * np.sin(th) * np.exp(1j * ph))
    assert np.allclose(S.spherical_harmonic(1, -1, th, ph), math.sqrt(3 / (8 * math.pi)) * np.sin(th) * np.exp(-1j * ph))
    assert np.allclose(S.spherical_harmonic(2, 0, th, ph),
                       math.sqrt(5 / (16 * math.pi)) * (3 * np.cos(th) ** 2 - 1))
    assert np.allclose(S.spherical_harmonic(3, 3, th, ph),
                       -math.sqrt(35 / (64 * math.pi)) * np.sin(th) ** 3 * np.exp(3j * ph))


def test_spherical_harmonics_orthonormal_on_a_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi integrates products of Y_lm
    (l <= 3) exactly."""
    xg, wg = np.polynomial.legendre.leggauss(12)
    phis = np.linspace(0, 2 * np.pi, 16, endpoint=False)
    th = np.repeat(np.arccos(xg), len(phis))
    ph = np.tile(phis, len(xg))
    w = np.repeat(wg, len(phis)) * (2 * np.pi / len(phis))
    ys = [S.spherical_harmonic(l, m, th, ph) for l in range(4) for m in range(-l, l + 1)]
    g = np.array([[np.sum(w * np.conj(a) * b) for b in ys] for a in ys])
    assert np.abs(g - np.eye(16)).max() < 1e-12


def test_local_functions_vanish_outside_their_radius():
    f = S.local_functions_on_grid((6, 6, 6), 7.4, 2.0)
    assert f.shape == (64, 216)
    j = np.stack(np.meshgrid(*[np.arange(6)] * 3, indexing="ij"), -1).reshape(-1, 3) / 6.0
    r = np.linalg.norm((j - np.round(j)) * 7.4, axis=1)
    assert np.abs(f[:, r >= 2.0]).max() == 0.0
    assert np.abs(f[:, r < 2.0]).max() > 0.0


class _OneRadialIntegral:
    """Stands in for the generator's random stream: the `which`-th radial
    integral drawn is (scale / n_rad) * identity, every other one is zero.
    Draw order: F^0, F^2, then G^0 .. G^4."""

    def __init__(self, which):
        self.which, self.i = which, 0

    def standard_normal(self, shape):
        out = np.eye(shape[0]) if self.i == self.which else np.zeros(shape)
        self.i += 1
        return out


_NRAD = S.LOCAL_NU * (S.LOCAL_LMAX + 1)
_C = 0.5 / _NRAD            # the radial integral each pin turns on (scale 0.5)


def _diag_block(M, lsel):
    """Orbital diagonal entries [(m_c, nu, m)] of the spin-up block for local functions with l = lsel."""
    npj = len(S.local_functions())
    out = {}
    for ic, mc in enumerate((-1, 0, 1)):
        a = 2 * ic
        for p, (nu, l, m) in enumerate(S.local_functions()):
            if l == lsel:
                out[(mc, nu, m)] = M[a * npj + p, a * npj + p]
    return out


def test_monopole_direct_term_is_a_uniform_shift():
    """F^0 alone: <l m|C^0|l' m'> = delta, so the direct term is -F^0 times
    the identity in every orbital and spin index (sign of the direct term)."""
    M = S.structured_couplings(_OneRadialIntegral(0))
    assert np.abs(M - (-_C) * np.eye(M.shape[0])).max() < 1e-14


def test_quadrupole_direct_term_is_traceless():
    """F^2 alone: a rank-2 tensor operator has zero trace over m, so for each
    core m_c and radial function the diagonal of the l block sums to zero;
    s functions do not couple at all (<0 0|C^2|0 0> = 0)."""
    M = S.structured_couplings(_OneRadialIntegral(1))
    assert np.abs(M).max() > 1e-3
    for l in range(S.LOCAL_LMAX + 1):
        d = _diag_block(M, l)
        for mc in (-1, 0, 1):
            for nu in range(S.LOCAL_NU):
                tr = sum(d[(mc, nu, m)] for m in range(-l, l + 1))
                assert abs(tr) < 1e-14, (l, mc, nu, tr)
    for v in _diag_block(M, 0).values():
        assert v == 0.0


def test_dipole_exchange_closed_forms():
    """G^1 alone (exchange through the dipole multipole, p hole): an s
    electron sees G^1/3 on every diagonal entry, the traces over (m_c, m) of
    the d block are 2 G^1 (sum rule 3 (2 1 1; 0 0 0)^2 = 2/5 per m), and p and
    f electrons see nothing (parity, triangle rule)."""
    M = S.structured_couplings(_OneRadialIntegral(3))
    s = _diag_block(M, 0)
    for (mc, nu, m), v in s.items():
        assert abs(v - _C / 3) < 1e-14, (mc, nu, v)
    d = _diag_block(M, 2)
    for nu in range(S.LOCAL_NU):
        tr = sum(d[(mc, nu, m)] for mc in (-1, 0, 1) for m in range(-2, 3))
        assert abs(tr - 2 * _C) < 1e-13, (nu, tr)
    npj = len(S.local_functions())
    for p, (nu, l, m) in enumerate(S.local_functions()):
        if l in (1, 3):
            for a in range(6):
                assert np.abs(M[a * npj + p]).max() == 0.0
