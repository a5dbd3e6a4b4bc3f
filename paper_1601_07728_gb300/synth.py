"""Seeded synthetic inputs for the core-excitation BSE Hamiltonian.

This module only *draws* inputs: Bloch functions u_nk(x), band energies E_nk,
the sampled screened core-hole potential W(x, R), the core spin-orbit matrix
chi, local-basis projections A and short-range couplings M, and start vectors.
It contains none of the Hamiltonian's arithmetic (no band->grid transform, no
Fourier transform over k, no Haydock or GMRES step), so both the FP64 CPU
oracle and the CUDA path can consume the same arrays without sharing code.

Shapes follow the exciton-vector layout psi[alpha][k][n] of Sec. 3.2 (Eq. 8):
    u      [Nk][Nx][Nb]   complex128, columns orthonormal per k (sum_x |u|^2 = 1)
    e_nk   [Nk][Nb]       float64, eV
    chi    [Na][Na]       complex128, eV (Hermitian core spin-orbit, Eq. 4)
    w_rx   [Nk][Nx]       float64, eV  (W(x, R) of Algorithm 1; R indexed like k)
    a_proj [Np][Nk][Nb]   complex128   (A^{nu l m}_{n k} of Eq. 14)
    m_sr   [Na*Np][Na*Np] complex128, eV, index (alpha, p) with alpha slow
Grid/mesh flattening: k = (m1*nk2 + m2)*nk3 + m3, same for R and for x.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HARTREE_EV = 27.211386245988  # CODATA 2018 Hartree energy in eV

# Configuration ids used in seeds: np.random.default_rng([config_id, site_id, stream_id]).
STREAM_U, STREAM_E, STREAM_A, STREAM_M, STREAM_B, STREAM_SITE = 1, 2, 3, 4, 5, 6


@dataclass
class BSESystem:
    n_alpha: int
    nk: tuple
    n_bands: int
    nx: tuple
    cell: float          # cubic cell side, bohr
    eps: float           # dielectric constant of the erf model potential
    u: np.ndarray
    e_nk: np.ndarray
    chi: np.ndarray
    w_rx: np.ndarray
    a_proj: np.ndarray | None
    m_sr: np.ndarray | None
    kshift: tuple = (0.0, 0.0, 0.0)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_k(self) -> int:
        return int(np.prod(self.nk))

    @property
    def n_x(self) -> int:
        return int(np.prod(self.nx))

    @property
    def n_proj(self) -> int:
        return 0 if self.a_proj is None else int(self.a_proj.shape[0])

    @property
    def dim(self) -> int:
        return self.n_alpha * self.n_k * self.n_bands


# Workload shapes (sizes, cell, screening) of the synthetic stand-ins for the
# paper's SrTiO3 / Alq3 systems.  "id" seeds the generator.
CONFIGS = {
    # 1s edge, single site, validated against dense diagonalisation (N = 128)
    "k_edge_small": dict(id=1, n_alpha=1, nk=(2, 2, 2), n_bands=16, nx=(8, 8, 8),
                         cell=7.4, eps=5.0, n_proj=0, so_split=None, m_scale=0.0),
    # L2,3 edge with multiplets: 6 core states, 8^3 k, 64 bands, 16^3 grid
    "l23_multiplet": dict(id=2, n_alpha=6, nk=(8, 8, 8), n_bands=64, nx=(16, 16, 16),
                          cell=7.4, eps=5.0, n_proj=36, so_split=5.7, m_scale=0.5),
    # the L2,3 physics on a smaller mesh (4^3 k, 32 bands, 8^3 grid): training
    # variants and small profiling cases
    "l23_reduced": dict(id=2, n_alpha=6, nk=(4, 4, 4), n_bands=32, nx=(8, 8, 8),
                        cell=7.4, eps=5.0, n_proj=36, so_split=5.7, m_scale=0.5),
    # SrTiO3 4x4x4-like supercell: 2^3 k, 1024 bands, 48^3 grid
    "supercell_48": dict(id=4, n_alpha=6, nk=(2, 2, 2), n_bands=1024, nx=(48, 48, 48),
                         cell=29.5, eps=6.0, n_proj=36, so_split=5.7, m_scale=0.5),
}


def rng_for(config_id: int, site_id: int, stream_id: int) -> np.random.Generator:
    return np.random.default_rng([int(config_id), int(site_id), int(stream_id)])


def complex_normal(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex normal with unit variance per entry (Re, Im ~ N(0, 1/2))."""
    s = np.sqrt(0.5)
    out = np.empty(shape, dtype=np.complex128)
    out.real = rng.standard_normal(shape) * s
    out.imag = rng.standard_normal(shape) * s
    return out


def orthonormal_bloch(rng: np.random.Generator, n_k: int, n_x: int, n_bands: int) -> np.ndarray:
    """u_nk(x) for each k: complex normal (Nx x Nb) with orthonormalised columns.

    Householder QR (numpy.linalg.qr) per k; phases fixed so R has a positive
    diagonal (makes the draw a deterministic function of the seed).
    """
    if n_bands > n_x:
        raise ValueError("need n_bands <= n_x for orthonormal columns")
    u = np.empty((n_k, n_x, n_bands), dtype=np.complex128)
    for k in range(n_k):
        g = complex_normal(rng, (n_x, n_bands))
        q, r = np.linalg.qr(g)
        d = np.diagonal(r)
        q *= (d / np.abs(d))[None, :]
        u[k] = q
    return u


def w_erf_hartree(r: np.ndarray, eps: float, a: float = 0.5) -> np.ndarray:
    """Model screened core-hole potential W(r) = -erf(r/a)/(eps*r) in Hartree.

    At r = 0 the limit -2/(a*sqrt(pi)*eps) is used.
    """
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = r < 1e-12
    rs = r[~small]
    from scipy.special import erf
    out[~small] = -erf(rs / a) / (eps * rs)
    out[small] = -2.0 / (a * math.sqrt(math.pi) * eps)
    return out


def sample_w(nk, nx, cell: float, eps: float, a: float = 0.5) -> np.ndarray:
    """W(x, R) in eV on the grid x_j = j*cell/nx and lattice R = r*cell.

    The core sits at the origin; the electron at x + R is taken at the nearest
    periodic image of the core in the (nk*cell)-periodic supercell
    (minimum-image convention).  Returns w_rx[R][x].
    """
    nk = tuple(int(v) for v in nk)
    nx = tuple(int(v) for v in nx)
    axes = []
    for d in range(3):
        xs = np.arange(nx[d]) * cell / nx[d]
        rs = np.arange(nk[d]) * cell
        pos = rs[:, None] + xs[None, :]          # [R_d][x_d]
        period = nk[d] * cell
        pos = np.mod(pos, period)
        pos = np.minimum(pos, period - pos)
        axes.append(pos)
    p0, p1, p2 = axes
    r2 = (p0[:, None, None, :, None, None] ** 2
          + p1[None, :, None, None, :, None] ** 2
          + p2[None, None, :, None, None, :] ** 2)
    r = np.sqrt(r2).reshape(int(np.prod(nk)), int(np.prod(nx)))
    return w_erf_hartree(r, eps, a) * HARTREE_EV


def spin_orbit_p(split_ev: float) -> np.ndarray:
    """chi = xi L.S for a p (l = 1) core level in the |m, sigma> basis, eV.

    Basis order alpha = 2*(m + 1) + s, m in (-1, 0, 1), s = 0 (up), 1 (down).
    The spin-orbit splitting between j = 1/2 and j = 3/2 is 3*xi/2, so
    xi = 2*split/3.  Eigenvalues: +xi/2 (x4, j = 3/2), -xi (x2, j = 1/2).
    """
    xi = 2.0 * split_ev / 3.0
    ms = (-1, 0, 1)
    sz = (0.5, -0.5)
    chi = np.zeros((6, 6), dtype=np.complex128)

    def idx(m, s):
        return 2 * (m + 1) + s

    for m in ms:
        for s in (0, 1):
            chi[idx(m, s), idx(m, s)] += xi * m * sz[s]
    # (L+ S- + L- S+)/2 ; L+|m> = sqrt(2 - m(m+1))|m+1>, S-|up> = |down>
    for m in ms:
        if m < 1:
            lp = math.sqrt(2 - m * (m + 1))
            # L+ S- : |m, up> -> |m+1, down>
            chi[idx(m + 1, 1), idx(m, 0)] += 0.5 * xi * lp
            chi[idx(m, 0), idx(m + 1, 1)] += 0.5 * xi * lp
    return chi


def random_hermitian(rng: np.random.Generator, n: int, scale: float) -> np.ndarray:
    g = complex_normal(rng, (n, n))
    return scale * 0.5 * (g + g.conj().T)


def make_system(name: str = "k_edge_small", site: int = 0, *, overrides: dict | None = None,
                u_dtype=np.complex128) -> BSESystem:
    """Draw one absorbing site of the named workload shape."""
    cfg = dict(CONFIGS[name])
    if overrides:
        cfg.update(overrides)
    return make_system_from(cfg, site=site, name=name)


def make_system_from(cfg: dict, site: int = 0, name: str = "custom", u=None) -> BSESystem:
    """Draw one site of shape cfg; u_nk may be supplied (e.g. drawn on the GPU)."""
    cid = int(cfg.get("id", 99))
    nk = tuple(int(v) for v in cfg["nk"])
    nx = tuple(int(v) for v in cfg["nx"])
    n_k, n_x = int(np.prod(nk)), int(np.prod(nx))
    nb, na = int(cfg["n_bands"]), int(cfg["n_alpha"])
    if u is None:
        u = orthonormal_bloch(rng_for(cid, site, STREAM_U), n_k, n_x, nb)
    e_nk = rng_for(cid, site, STREAM_E).uniform(0.0, 20.0, size=(n_k, nb))
    split = cfg.get("so_split")
    if na == 6 and split:
        chi = spin_orbit_p(float(split))
    else:
        chi = np.zeros((na, na), dtype=np.complex128)
    w = sample_w(nk, nx, float(cfg["cell"]), float(cfg["eps"]))
    if "w_const" in cfg:
        w = np.full_like(w, float(cfg["w_const"]))
    np_ = int(cfg.get("n_proj", 0))
    a_proj = m_sr = None
    if np_ > 0:
        ra = rng_for(cid, site, STREAM_A)
        a = complex_normal(ra, (np_, n_k * nb))
        a /= np.linalg.norm(a, axis=1, keepdims=True)
        a_proj = a.reshape(np_, n_k, nb)
        m_sr = random_hermitian(rng_for(cid, site, STREAM_M), na * np_, float(cfg.get("m_scale", 0.5)))
    ks = tuple(float(v) for v in cfg.get("kshift", (0.0, 0.0, 0.0)))
    return BSESystem(n_alpha=na, nk=nk, n_bands=nb, nx=nx, cell=float(cfg["cell"]),
                     eps=float(cfg["eps"]), u=u, e_nk=e_nk, chi=chi, w_rx=w,
                     a_proj=a_proj, m_sr=m_sr, kshift=ks, name=name, meta=dict(cfg))


# ---------------------------------------------------------------------------
# Structured short-range couplings (Sec. 3.2.2): local basis R_{nu,l} Y_{l,m}
# with 4 radial functions for each l = 0..3 (64 functions), a p core level,
# and M built from Slater-type radial integrals times Gaunt angular factors,
# so that only the multipoles allowed by the selection rules appear.
# ---------------------------------------------------------------------------
LOCAL_NU, LOCAL_LMAX = 4, 3


def wigner3j(j1: int, j2: int, j3: int, m1: int, m2: int, m3: int) -> float:
    """Wigner 3j symbol for integer arguments (Racah's closed form)."""
    if m1 + m2 + m3 != 0 or j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    f = math.factorial
    tri = f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3) / f(j1 + j2 + j3 + 1)
    pre = math.sqrt(tri * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3))
    s = 0.0
    for tt in range(0, j1 + j2 + j3 + 1):
        den = (tt, j3 - j2 + tt + m1, j3 - j1 + tt - m2, j1 + j2 - j3 - tt, j1 - tt - m1, j2 - tt + m2)
        if min(den) < 0:
            continue
        prod = 1
        for d in den:
            prod *= f(d)
        s += (-1) ** tt / prod
    return float((-1) ** (j1 - j2 - m3) * pre * s)


def gaunt(l1: int, m1: int, k: int, q: int, l2: int, m2: int) -> float:
    """<l1 m1| C^k_q |l2 m2> with C^k_q = sqrt(4 pi/(2k+1)) Y_kq."""
    return ((-1) ** m1 * math.sqrt((2 * l1 + 1) * (2 * l2 + 1)) * wigner3j(l1, k, l2, 0, 0, 0)
            * wigner3j(l1, k, l2, -m1, q, m2))


def local_index(nu: int, l: int, m: int) -> int:
    """Index p of the local function R_{nu,l} Y_{l,m}: nu slow, then l, then m."""
    return nu * (LOCAL_LMAX + 1) ** 2 + l * l + (l + m)


def local_functions():
    """[(nu, l, m)] in index order."""
    return [(nu, l, m) for nu in range(LOCAL_NU) for l in range(LOCAL_LMAX + 1) for m in range(-l, l + 1)]


def structured_couplings(rng: np.random.Generator, scale: float = 0.5) -> np.ndarray:
    """M [(alpha, p)][(alpha', p')] (alpha = 2 (m_c + 1) + s, p = local_index)
    for a p core hole and the 64 local functions, eV:
      M = -D + X,  both diagonal in the spin s,
      D = sum_{k=0,2} F^k_{nu l, nu' l'} sum_q (-1)^q <l m|C^k_q|l' m'> <1 m_c|C^k_-q|1 m_c'>
      X = sum_k G^k_{nu l, nu' l'} sum_q (-1)^q <l m|C^k_q|1 m_c'> <1 m_c|C^k_-q|l' m'>
    (direct and exchange multipoles of a scalar two-particle interaction, so
    M commutes with the total orbital angular momentum).  The radial
    integrals F^k, G^k are seeded symmetric positive semi-definite matrices
    over (nu, l) of scale `scale`."""
    funcs = local_functions()
    npj = len(funcs)
    nrad = LOCAL_NU * (LOCAL_LMAX + 1)
    rad = lambda nu, l: nu * (LOCAL_LMAX + 1) + l

    def radial():
        b = rng.standard_normal((nrad, nrad))
        return scale * (b @ b.T) / nrad

    fk = {k: radial() for k in (0, 2)}
    gk = {k: radial() for k in range(0, LOCAL_LMAX + 2)}
    mc_list = (-1, 0, 1)
    orb = np.zeros((3, npj, 3, npj))   # [m_c][p][m_c'][p']
    for ic, mc in enumerate(mc_list):
        for p, (nu, l, m) in enumerate(funcs):
            for jc, mc2 in enumerate(mc_list):
                for p2, (nu2, l2, m2) in enumerate(funcs):
                    if m + mc != m2 + mc2:
                        continue
                    v = 0.0
                    for k, f in fk.items():
                        q = m - m2
                        v -= f[rad(nu, l), rad(nu2, l2)] * (-1) ** q * gaunt(l, m, k, q, l2, m2) * gaunt(1, mc, k, -q, 1, mc2)
                    for k, g in gk.items():
                        q = m - mc2
                        v += g[rad(nu, l), rad(nu2, l2)] * (-1) ** q * gaunt(l, m, k, q, 1, mc2) * gaunt(1, mc, k, -q, l2, m2)
                    orb[ic, p, jc, p2] = v
    M = np.zeros((6 * npj, 6 * npj), dtype=np.complex128)
    for ic, mc in enumerate(mc_list):
        for jc, mc2 in enumerate(mc_list):
            for s in (0, 1):
                a, a2 = 2 * (mc + 1) + s, 2 * (mc2 + 1) + s
                M[a * npj:(a + 1) * npj, a2 * npj:(a2 + 1) * npj] = orb[ic, :, jc, :]
    return M


def dipole_start_vectors(a_proj: np.ndarray, qs=(-1, 0, 1), seed: int = 0) -> np.ndarray:
    """Start vectors b_q shaped by the dipole operator from the p core level
    into the local basis (Sec. 2, the x-ray matrix elements), one per
    polarisation component q:  b_q(alpha = (m_c, s), n, k) =
    sum_{nu, l in (0, 2), m} d_{nu l} <l m|C^1_q|1 m_c> conj(A^{nu l m}_{nk}),
    d_{nu l} seeded radial dipole integrals; each b_q normalised to 1.
    a_proj [64][Nk][Nb] -> b [len(qs)][6 * Nk * Nb]."""
    rng = np.random.default_rng([3, 7, int(seed)])
    d = rng.uniform(0.5, 1.5, size=(LOCAL_NU, LOCAL_LMAX + 1))
    npj, nk, nb = a_proj.shape
    out = np.zeros((len(qs), 6, nk * nb), dtype=np.complex128)
    a2 = a_proj.reshape(npj, nk * nb)
    for iq, q in enumerate(qs):
        for mc in (-1, 0, 1):
            acc = np.zeros(nk * nb, dtype=np.complex128)
            for nu in range(LOCAL_NU):
                for l in (0, 2):
                    for m in range(-l, l + 1):
                        gq = gaunt(l, m, 1, q, 1, mc)
                        if gq != 0.0:
                            acc += d[nu, l] * gq * np.conj(a2[local_index(nu, l, m)])
            for s in (0, 1):
                out[iq, 2 * (mc + 1) + s] = acc
        out[iq] /= np.linalg.norm(out[iq])
    return out.reshape(len(qs), -1)


def spherical_harmonic(l: int, m: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Y_{l,m}(theta, phi), orthonormal on the sphere, Condon-Shortley phase
    (associated Legendre functions by the standard upward recurrence)."""
    am = abs(m)
    x = np.cos(theta)
    somx2 = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    fact = 1.0
    for _ in range(am):
        pmm = -pmm * fact * somx2
        fact += 2.0
    if l == am:
        plm = pmm
    else:
        pmm1 = x * (2 * am + 1) * pmm
        if l == am + 1:
            plm = pmm1
        else:
            for ll in range(am + 2, l + 1):
                pll = (x * (2 * ll - 1) * pmm1 - (ll + am - 1) * pmm) / (ll - am)
                pmm, pmm1 = pmm1, pll
            plm = pmm1
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    y = norm * plm * np.exp(1j * am * phi)
    if m < 0:
        y = (-1) ** am * np.conj(y)
    return y


def local_functions_on_grid(nx, cell: float, rc: float, seed: int = 0) -> np.ndarray:
    """The 64 local functions f_p(x) = R_{nu,l}(r) Y_{l,m}(r^) sampled on the
    cell's grid x_d = j_d a / n_x_d, with r the minimum-image distance to the
    absorbing atom at the origin and f = 0 for r >= rc; radial functions
    R_{nu,l}(r) = r^l exp(-(r / s_nu)^2) with seeded widths s_nu < rc.
    Index order p = local_index(nu, l, m).  Returns [64][Nx] complex128."""
    rng = np.random.default_rng([3, 11, int(seed)])
    widths = np.sort(rng.uniform(0.15 * rc, 0.6 * rc, size=LOCAL_NU))
    j = np.stack(np.meshgrid(*[np.arange(n) for n in nx], indexing="ij"), -1).reshape(-1, 3)
    frac = j / np.asarray(nx, dtype=np.float64)
    frac = frac - np.round(frac)          # minimum image in the cell
    xyz = frac * cell
    r = np.linalg.norm(xyz, axis=1)
    theta = np.arccos(np.clip(np.where(r > 0, xyz[:, 2] / np.maximum(r, 1e-300), 1.0), -1.0, 1.0))
    phi = np.arctan2(xyz[:, 1], xyz[:, 0])
    inside = r < rc
    out = np.zeros((LOCAL_NU * (LOCAL_LMAX + 1) ** 2, len(r)), dtype=np.complex128)
    for nu, l, m in local_functions():
        rad = r ** l * np.exp(-(r / widths[nu]) ** 2)
        out[local_index(nu, l, m)] = np.where(inside, rad * spherical_harmonic(l, m, theta, phi), 0.0)
    return out


def imag_axis_quadrature(n: int, scale: float = 5.0):
    """Nodes t and weights w for integrals over t in (-inf, inf): Gauss-Legendre
    in u on (-1, 1) with t = scale * tan(pi u / 2)."""
    u, wu = np.polynomial.legendre.leggauss(n)
    t = scale * np.tan(0.5 * np.pi * u)
    w = wu * scale * 0.5 * np.pi / np.cos(0.5 * np.pi * u) ** 2
    return t, w


def screening_grid_states(n_r: int, n_states: int, seed: int = 0, e_range=(-10.0, 10.0)):
    """Bloch functions on a real-space grid around the core hole (n_r points,
    e.g. 36 angular x 25 radial = 900) for n_states band/k states: seeded
    complex normal values, and band energies uniform in e_range (eV)."""
    rng = rng_for(5, int(seed), STREAM_U)
    psi = complex_normal(rng, (n_r, n_states)) / math.sqrt(n_r)
    eps = rng_for(5, int(seed), STREAM_E).uniform(e_range[0], e_range[1], size=n_states)
    return psi, eps


def structured_system(cfg: dict, site: int = 0, name: str = "structured") -> BSESystem:
    """make_system_from with the 64-function local basis and structured M
    (structured_couplings); requires 6 core states."""
    c = dict(cfg)
    c["n_proj"] = LOCAL_NU * (LOCAL_LMAX + 1) ** 2
    s = make_system_from(c, site=site, name=name)
    if s.n_alpha != 6:
        raise ValueError("structured couplings need the 6 states of a p core level")
    s.m_sr = structured_couplings(rng_for(int(c.get("id", 99)), site, STREAM_M), float(c.get("m_scale", 0.5)))
    return s


STREAM_VAL = 7   # valence final state of the RIXS two-step


def valence_final_state(core: BSESystem, n_v: int = 10, seed: int = 0, w_scale: float = 0.5,
                        m_scale: float = 0.3, e_range=(2.0, 8.0)):
    """Final-state system of the RIXS two-step and its emission operator.

    The final state of resonant inelastic scattering has the core hole filled
    from the valence band: a valence hole v (one of n_v localised valence
    states, e.g. the 10 spin-orbitals of a 3d shell) with the photo-electron
    (n, k) left where the absorption put it.  Its Hamiltonian is taken of the
    same form as the core-hole one, with the hole index running over v:
    band energies E_nk, the hole term -chi_val with chi_val = -diag(eps_v) +
    a Hermitian hopping (hole binding energies eps_v ~ U[e_range] eV, so that
    energy losses are E_nk + eps_v), the long-range direct term with W scaled
    by w_scale (a valence hole is screened more and less localised than a
    core hole), and the short-range term through the same local functions
    with seeded Hermitian couplings of scale m_scale eV.  The emission
    operator D [n_v][n_alpha] (dipole matrix elements between the valence
    and core orbitals) is seeded complex normal with unit Frobenius norm per
    row.  Returns (final-state BSESystem, D)."""
    cid = int(core.meta.get("id", 99))
    rng = rng_for(cid, 5000 + seed, STREAM_VAL)
    eps_v = rng.uniform(e_range[0], e_range[1], size=n_v)
    hop = random_hermitian(rng, n_v, 0.25)
    chi = -np.diag(eps_v).astype(np.complex128) + hop
    a_proj = core.a_proj
    m_sr = None
    if a_proj is not None:
        m_sr = random_hermitian(rng, n_v * a_proj.shape[0], m_scale)
    d = complex_normal(rng, (n_v, core.n_alpha))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    meta = dict(core.meta)
    meta["id"] = cid + 500
    val = BSESystem(n_alpha=n_v, nk=core.nk, n_bands=core.n_bands, nx=core.nx, cell=core.cell, eps=core.eps,
                    u=core.u, e_nk=core.e_nk, chi=chi, w_rx=core.w_rx * w_scale, a_proj=a_proj, m_sr=m_sr,
                    kshift=core.kshift, name=core.name + "_valence", meta=meta)
    return val, d


def batched_site_config(site: int) -> dict:
    """Shape of one site of the many-site workload: k mesh n^3 with
    n ~ U{4..8}, grid m^3 with m ~ U{12..20}, Nb ~ U{32..256}, and 1 or 6 core
    states with probability 1/2 each.  L-edge sites (6 core states) carry the
    5.7 eV spin-orbit split and 36 local functions; 1s sites carry neither.
    Cell 7.4 bohr, epsilon 5."""
    r = rng_for(3, site, STREAM_SITE)
    n = int(r.integers(4, 9))
    m = int(r.integers(12, 21))
    nb = int(r.integers(32, 257))
    na = 6 if r.random() < 0.5 else 1
    return dict(id=3, n_alpha=na, nk=(n, n, n), n_bands=nb, nx=(m, m, m), cell=7.4, eps=5.0,
                n_proj=36 if na == 6 else 0, so_split=5.7 if na == 6 else None, m_scale=0.5)


def orthonormal_bloch_device(seed: int, n_k: int, n_x: int, n_bands: int, device="cuda", chunk: int = 32):
    """u_nk(x) drawn and orthonormalised on a GPU with torch, for workloads too
    large to draw on the host: complex normal (Nx x Nb) per k from a seeded
    torch generator, Householder QR (torch.linalg.qr), phases fixed so R has a
    positive diagonal.  A different random stream from orthonormal_bloch;
    returns a complex128 tensor [Nk][Nx][Nb] on the device, complete (the
    device is synchronised) when the call returns."""
    import torch
    if n_bands > n_x:
        raise ValueError("need n_bands <= n_x for orthonormal columns")
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    u = torch.empty((n_k, n_x, n_bands), dtype=torch.complex128, device=device)
    for k0 in range(0, n_k, chunk):
        k1 = min(n_k, k0 + chunk)
        g = torch.randn((k1 - k0, n_x, n_bands), dtype=torch.complex128, device=device, generator=gen)
        q, r = torch.linalg.qr(g)
        d = torch.diagonal(r, dim1=-2, dim2=-1)
        u[k0:k1] = q * (d / d.abs()).unsqueeze(-2)
        del g, q, r, d
    # the draw runs on torch's stream; consumers on other (non-blocking)
    # streams must not see it half-written
    torch.cuda.synchronize(device)
    return u


def make_system_device(cfg: dict, site: int = 0, name: str = "custom", device="cuda") -> BSESystem:
    """make_system_from with u_nk from orthonormal_bloch_device (a torch
    tensor on the device); every other array is drawn on the host as usual."""
    cid = int(cfg.get("id", 99))
    n_k = int(np.prod(cfg["nk"]))
    n_x = int(np.prod(cfg["nx"]))
    seed = (cid * 1000003 + int(site)) * 101 + STREAM_U
    u = orthonormal_bloch_device(seed, n_k, n_x, int(cfg["n_bands"]), device=device)
    return make_system_from(cfg, site=site, name=name, u=u)


def make_start_vectors(sysd: BSESystem, n_vec: int = 1, seed: int = 0) -> np.ndarray:
    """Start vectors b (dipole-operator stand-in): complex normal, unit norm each.

    Polarisations are independent seeds.  Shape [n_vec][Na*Nk*Nb].
    """
    cid = int(sysd.meta.get("id", 99))
    out = np.empty((n_vec, sysd.dim), dtype=np.complex128)
    for v in range(n_vec):
        g = complex_normal(rng_for(cid, 1000 + seed, STREAM_B * 100 + v), (sysd.dim,))
        out[v] = g / np.linalg.norm(g)
    return out


def omega_grid(n: int = 2000, lo: float = -5.0, hi: float = 30.0) -> np.ndarray:
    return np.linspace(lo, hi, n)


MLP_SHAPES = [((12, 128), "w1"), ((128,), "b1"), ((128, 128), "w2"), ((128,), "b2"), ((128, 34), "w3"),
              ((34,), "b3")]


def mlp_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the preconditioner network, packed as
    w1 [12][128], b1, w2 [128][128], b2, w3 [128][34], b3 (float32).
    Hidden weights ~ N(0, 1/fan_in); the last layer is zero except the eight
    V-factor outputs' imaginary/real columns (18..33), which start small so
    that the rank-8 term has a gradient."""
    rng = rng_for(77, seed, STREAM_SITE)
    parts = []
    for shp, name in MLP_SHAPES:
        if name == "w1":
            parts.append(rng.standard_normal(shp) / np.sqrt(12.0))
        elif name == "w2":
            parts.append(rng.standard_normal(shp) / np.sqrt(128.0))
        elif name == "w3":
            w = np.zeros(shp)
            w[:, 18:34] = rng.standard_normal((128, 16)) * 0.05 / np.sqrt(128.0)
            parts.append(w)
        else:
            parts.append(np.zeros(shp))
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def reduced_l23(seed: int = 0) -> BSESystem:
    """A seeded smaller variant of the L2,3 multiplet workload (4^3 k, 32
    bands, 8^3 grid, same physics) used to train the preconditioner."""
    return make_system("l23_multiplet", site=seed,
                       overrides=dict(nk=(4, 4, 4), n_bands=32, nx=(8, 8, 8)))


def tiny_system(seed: int, n_alpha=2, nk=(2, 1, 3), n_bands=3, nx=(2, 3, 2), *,
                n_proj=2, cell=7.4, eps=5.0, kshift=(0.0, 0.0, 0.0),
                w_const=None, so=True, m_scale=0.5) -> BSESystem:
    """Small random system with every term present (for oracle self-checks)."""
    cfg = dict(id=900 + seed, n_alpha=n_alpha, nk=nk, n_bands=n_bands, nx=nx, cell=cell,
               eps=eps, n_proj=n_proj, so_split=None, m_scale=m_scale, kshift=kshift)
    if w_const is not None:
        cfg["w_const"] = w_const
    s = make_system_from(cfg, site=0, name=f"tiny{seed}")
    if so:
        if n_alpha == 6:
            s.chi = spin_orbit_p(5.7)
        else:
            s.chi = random_hermitian(rng_for(900 + seed, 0, STREAM_SITE), n_alpha, 1.0)
    return s
