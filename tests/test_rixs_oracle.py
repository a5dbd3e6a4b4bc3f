"""Pins of the oracle's RIXS two-step (absorption resolvent, emission,
final-state Haydock) against the Kramers-Heisenberg form built independently
from dense Hamiltonians:

  sigma(z_in, w) = (1/pi) sum_f |<f| (D (x) I) (z_in - H_core)^{-1} |b>|^2
                   Gamma_f / ((w - E_f)^2 + Gamma_f^2),

with (E_f, |f>) from eigh of the dense final-state H, the resolvent from eigh
of the dense core-hole H, and the emission operator as an explicit Kronecker
product.  A conjugated emission matrix (a plausible slip) fails the pin.
"""
import numpy as np
import pytest

from oracle import bse_oracle as O
from paper_1601_07728_gb300 import synth as S


def kramers_heisenberg(h_core, h_val, d_em, n_kb, b, z_in, omega, gamma_f):
    e, v = np.linalg.eigh(h_core)
    x = v @ ((v.conj().T @ b) / (z_in - e))                   # (z_in - H)^{-1} b
    y = np.kron(d_em, np.eye(n_kb)) @ x                        # hole alpha -> v, electron (k, n) kept
    ef, vf = np.linalg.eigh(h_val)
    w = np.abs(vf.conj().T @ y) ** 2
    om = np.asarray(omega)[:, None]
    return (w[None, :] * gamma_f / ((om - ef[None, :]) ** 2 + gamma_f ** 2)).sum(1) / np.pi, y


@pytest.fixture(scope="module")
def pair():
    core = S.tiny_system(61, n_alpha=6, nk=(2, 1, 2), n_bands=3, nx=(2, 2, 2), n_proj=2)
    val, d = S.valence_final_state(core, n_v=4, seed=1)
    b = S.make_start_vectors(core, 1, seed=3)[0]
    return core, val, d, b


def test_final_state_hamiltonian_is_hermitian(pair):
    _, val, _, _ = pair
    h = O.dense_h(val)
    assert np.linalg.norm(h - h.conj().T) <= 1e-13 * np.linalg.norm(h)


@pytest.mark.parametrize("z_in", [3.0 + 0.4j, 11.5 + 0.4j, 19.0 + 1.0j])
def test_rixs_two_step_equals_kramers_heisenberg(pair, z_in):
    core, val, d, b = pair
    om = np.linspace(-2.0, 35.0, 400)
    n_f = val.dim
    (a, bc, y), = O.rixs_two_step(core, val, d, b, [z_in], n_f + 3, rtol=1e-13, reorth=True)
    sig = O.cf_spectrum(a, bc, om, 0.3)
    ref, y_ref = kramers_heisenberg(O.dense_h(core), O.dense_h(val), d, core.n_k * core.n_bands, b, z_in, om, 0.3)
    assert np.linalg.norm(y - y_ref) <= 1e-10 * np.linalg.norm(y_ref)
    assert np.linalg.norm(sig - ref) <= 1e-9 * np.linalg.norm(ref)
    # zeroth moment: the final-state weight is |y|^2
    assert bc[0] ** 2 == pytest.approx(np.vdot(y_ref, y_ref).real, rel=1e-10)


def test_emission_moves_only_the_hole(pair):
    core, _, _, _ = pair
    rng = np.random.default_rng(2)
    x = S.complex_normal(rng, (2, core.dim))
    nkb = core.n_k * core.n_bands
    d = np.zeros((3, core.n_alpha), dtype=np.complex128)
    d[0, 4] = 1.0
    d[2, 1] = 0.5 - 0.25j
    y = O.rixs_emission(d, x).reshape(2, 3, nkb)
    xr = x.reshape(2, core.n_alpha, nkb)
    assert np.array_equal(y[:, 0], xr[:, 4])
    assert np.allclose(y[:, 1], 0.0)
    assert np.allclose(y[:, 2], (0.5 - 0.25j) * xr[:, 1], rtol=0, atol=1e-15)


def test_planted_conjugated_emission_fails_the_pin(pair):
    core, val, d, b = pair
    z_in = 11.5 + 0.4j
    om = np.linspace(-2.0, 35.0, 400)
    (a, bc, _), = O.rixs_two_step(core, val, d.conj(), b, [z_in], val.dim + 3, rtol=1e-13, reorth=True)
    ref, _ = kramers_heisenberg(O.dense_h(core), O.dense_h(val), d, core.n_k * core.n_bands, b, z_in, om, 0.3)
    assert np.linalg.norm(O.cf_spectrum(a, bc, om, 0.3) - ref) > 1e-3 * np.linalg.norm(ref)
