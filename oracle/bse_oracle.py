"""FP64 CPU oracle for the core-excitation BSE Hamiltonian (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module: only the test-suite, the smoke check of the package
entry file and the CPU-baseline leg of the benchmark use it.  It shares no
code with the CUDA path; both consume the same seeded input arrays.

Everything is plain NumPy/SciPy in float64 / complex128, written for a reader
to check against the paper by eye:

* H_BSE = H_e - H_h - V_D + V_X (Sec. 2, Eq. 3) acting on exciton vectors
  psi_{alpha, n, k} (Sec. 3.2, Eq. 8), with
    - H_e   -> band energies E_nk (Eq. 5, given as input),
    - H_h   -> core energy eps_c (taken as 0: energies relative to the edge) and
               the core spin-orbit matrix chi (Eq. 4); the lifetime Gamma is
               carried by the complex frequency z = omega + i*Gamma instead,
    - V_D long range -> W_0 through Algorithm 1 (Sec. 3.2.1, Eqs. 10-13),
    - short range (local direct + exchange) -> projections onto the local basis
      A^{nu l m}_{n k} of Eq. 14 and a Hermitian coupling matrix M (Sec. 3.2.2).
* Haydock recursion (Sec. 3.2, Eq. 9) and its continued fraction for the loss
  function of Eq. 1 with G(omega) = [omega - H]^{-1} (Eq. 2).
* GMRES for (H - z) x = b, the same resolvent applied to one right-hand side.
* RIXS two-step: the absorption resolvent at the incoming energy, the
  emission that moves the hole from the core to a valence state, and the
  Haydock recursion of the final-state Hamiltonian (reading below).

Readings where the paper is silent (also listed in the design notes):
  - the sampled W(x, R) is the signed potential energy in eV and is *added*
    (Algorithm 1 multiplies by W directly);
  - F_{k->R} carries e^{+i k.R} unnormalised, F_{R->k} carries e^{-i k.R}/Nk;
  - k = 2*pi*(m + s)/(nk*a) per axis, x = j*a/nx, R = r*a;
  - the core term enters H as -chi (from -H_h); eps_c = 0;
  - V_SR = (A (x) I_alpha)^H M (A (x) I_alpha), with M indexed (alpha, p),
    alpha slow;
  - RIXS final state: the same operator form with the hole index running over
    localised valence states; the photo-electron is a spectator of the
    emission.

Parity unpinned: none of the functions below; every one has a pin in the
oracle test-suite (closed forms, invariants, brute force, or library routines
on tiny inputs).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


# ----------------------------------------------------------------------------
# geometry helpers (Sec. 3.2, Eq. 8 / Eq. 13: positions entering e^{ik.x}, e^{ik.R})
# ----------------------------------------------------------------------------

def _mesh_indices(n3):
    """Integer triples (i1, i2, i3) of a flattened n1*n2*n3 mesh, last index fastest."""
    n1, n2, n3_ = (int(v) for v in n3)
    i1, i2, i3 = np.meshgrid(np.arange(n1), np.arange(n2), np.arange(n3_), indexing="ij")
    return np.stack([i1.ravel(), i2.ravel(), i3.ravel()], axis=1)


def kx_phase(nk, nx, kshift=(0.0, 0.0, 0.0)):
    """e^{i k.x} as [Nk][Nx]: k.x = 2*pi * sum_d (m_d + s_d) * j_d / (nk_d * nx_d)."""
    m = _mesh_indices(nk).astype(np.float64) + np.asarray(kshift, dtype=np.float64)[None, :]
    j = _mesh_indices(nx).astype(np.float64)
    kfrac = m / np.asarray(nk, dtype=np.float64)[None, :]       # k in units of 2*pi/a
    xfrac = j / np.asarray(nx, dtype=np.float64)[None, :]       # x in units of a
    return np.exp(1j * TWO_PI * (kfrac @ xfrac.T))


def kr_phase(nk, kshift=(0.0, 0.0, 0.0)):
    """e^{i k.R} as [Nk][NR]: k.R = 2*pi * sum_d (m_d + s_d) * r_d / nk_d (R indexed like k)."""
    m = _mesh_indices(nk).astype(np.float64) + np.asarray(kshift, dtype=np.float64)[None, :]
    r = _mesh_indices(nk).astype(np.float64)
    kfrac = m / np.asarray(nk, dtype=np.float64)[None, :]
    return np.exp(1j * TWO_PI * (kfrac @ r.T))


def _shape(s):
    return s.n_alpha, int(np.prod(s.nk)), s.n_bands, int(np.prod(s.nx))


# ----------------------------------------------------------------------------
# set-up projection, screening, and H psi from the definitions of its terms
# (tiny inputs only)
# ----------------------------------------------------------------------------

def local_projection(u, nk, nx, f, dv, kshift=(0.0, 0.0, 0.0)):
    """Projection of the Bloch functions onto the local basis (Sec. 3.2.2):
    A[p][k][n] = dv sum_x conj(f_p(x)) e^{i k.x} u_nk(x); u [Nk][Nx][Nb],
    f [Np][Nx] -> A [Np][Nk][Nb]."""
    ph = kx_phase(nk, nx, kshift)
    fc = np.conj(f)
    a = np.empty((f.shape[0], u.shape[0], u.shape[2]), dtype=np.complex128)
    for k in range(u.shape[0]):
        a[:, k, :] = dv * (fc @ (ph[k][:, None] * u[k]))
    return a


def screening_green(psi, eps, mu, t):
    """G_j(r, r') = sum_K psi(r, K) conj(psi(r', K)) / (mu + i t_j - eps_K)
    (the Green's function of Sec. 3.3 on the grid, imaginary frequencies)."""
    return np.stack([(psi / (mu + 1j * tj - eps)[None, :]) @ psi.conj().T for tj in t])


def screening_chi0(psi, eps, mu, t, w):
    """chi0(r, r') = (1/2 pi) sum_j w_j G_j(r, r') G_j(r', r): the frequency
    integral of the RPA chi^0 (Sec. 3.3) along omega' = mu + i t, static."""
    g = screening_green(psi, eps, mu, t)
    return np.einsum("j,jrc,jcr->rc", np.asarray(w, dtype=np.float64), g, g) / TWO_PI


def bloch_on_supercell(s):
    """Bloch functions phi_nk(x + R) = e^{i k.(x + R)} u_nk(x) / sqrt(Nk) on
    every point x + R of the Nk-cell supercell (Sec. 3.2, Eq. 8; R indexed like
    k), as [NR][Nx][Nk*Nb] with column (k, n), n fastest.  With orthonormal
    u_nk columns these are orthonormal over the supercell."""
    na, nk, nb, nx = _shape(s)
    ekx = kx_phase(s.nk, s.nx, s.kshift)            # [Nk][Nx]
    ekr = kr_phase(s.nk, s.kshift)                  # [Nk][NR]
    phi = np.empty((nk, nx, nk * nb), dtype=np.complex128)
    for r in range(nk):
        for k in range(nk):
            phase = ekr[k, r] * ekx[k, :] / np.sqrt(nk)                      # [Nx]
            phi[r, :, k * nb:(k + 1) * nb] = phase[:, None] * s.u[k]
    return phi


def w0_matrix_loop(s):
    """Matrix of the screened direct term in the Bloch basis, from its
    definition as a local potential on the supercell (Sec. 3.2.1: W(x, R) is
    the core-hole potential felt at the point x + R):
        <n k|W_0|n' k'> = sum over supercell points r = x + R of
                          conj(phi_nk(r)) W(r) phi_n'k'(r),
    accumulated one point at a time (each point adds a rank-one term).  The
    term does not act on the core index.  Tiny inputs only."""
    na, nk, nb, nx = _shape(s)
    phi = bloch_on_supercell(s)
    wm = np.zeros((nk * nb, nk * nb), dtype=np.complex128)
    for r in range(nk):
        for x in range(nx):
            f = phi[r, x]
            wm += s.w_rx[r, x] * np.outer(np.conj(f), f)
    return wm


def apply_sr_loop(s, psi):
    """Short-range term through the local basis (Sec. 3.2.2, Eq. 14), as loops:
    c_{alpha p} = sum_{n k} A_{p;nk} psi_{alpha n k};  c' = M c;
    psi'_{alpha n k} = sum_p conj(A_{p;nk}) c'_{alpha p}."""
    na, nk, nb, _ = _shape(s)
    out = np.zeros_like(psi)
    if s.a_proj is None:
        return out
    npj = s.a_proj.shape[0]
    c = np.zeros(na * npj, dtype=np.complex128)
    for a in range(na):
        for p in range(npj):
            acc = 0.0j
            for k in range(nk):
                for n in range(nb):
                    acc += s.a_proj[p, k, n] * psi[a, k, n]
            c[a * npj + p] = acc
    cp = np.zeros_like(c)
    for i in range(na * npj):
        acc = 0.0j
        for j in range(na * npj):
            acc += s.m_sr[i, j] * c[j]
        cp[i] = acc
    for a in range(na):
        for k in range(nk):
            for n in range(nb):
                acc = 0.0j
                for p in range(npj):
                    acc += np.conj(s.a_proj[p, k, n]) * cp[a * npj + p]
                out[a, k, n] = acc
    return out


def apply_h_loop(s, psi_flat):
    """H psi from the definitions of its terms (tiny inputs only):
    H = diag(E_nk) - chi (x) I + W_0 + V_SR, with W_0 taken as the matrix of
    the supercell potential between Bloch states (w0_matrix_loop) rather than
    by the transform steps of Algorithm 1."""
    na, nk, nb, _ = _shape(s)
    psi = psi_flat.reshape(na, nk, nb)
    out = np.zeros_like(psi)
    for a in range(na):
        for k in range(nk):
            for n in range(nb):
                acc = s.e_nk[k, n] * psi[a, k, n]
                for b in range(na):
                    acc -= s.chi[a, b] * psi[b, k, n]
                out[a, k, n] = acc
    wm = w0_matrix_loop(s)
    for a in range(na):
        out[a] += (wm @ psi[a].reshape(-1)).reshape(nk, nb)
    out += apply_sr_loop(s, psi)
    return out.reshape(-1)


# ----------------------------------------------------------------------------
# H psi: vectorised (per-k matmul + FFT over the k mesh)
# ----------------------------------------------------------------------------

def apply_w0(s, psi):
    """W_0 psi, Algorithm 1 with the x and alpha loops vectorised.
    psi: [V][Na][Nk][Nb] -> same.  Uses numpy matmul for the band sums and
    numpy FFTs for the k<->R sums (with the mesh-shift phase applied explicitly:
    sum_m e^{2pi i (m+s).r/nk} f_m = e^{2pi i s.r/nk} * Nk * ifftn(f)[r])."""
    nv = psi.shape[0]
    na, nk, nb, nx = _shape(s)
    ekx = kx_phase(s.nk, s.nx, s.kshift)                              # [Nk][Nx]
    ub = s.u * ekx[:, :, None]                                        # e^{ikx} u_nk(x)
    # phi[v, a, k, x] = sum_n ub[k, x, n] psi[v, a, k, n]
    phi = np.einsum("kxn,vakn->vakx", ub, psi, optimize=True)
    nkt = tuple(int(v) for v in s.nk)
    shp = (nv, na) + nkt + (nx,)
    phi = phi.reshape(shp)
    ax = (2, 3, 4)
    r = np.stack(np.meshgrid(*[np.arange(v) for v in nkt], indexing="ij"), axis=-1)
    sphase = np.exp(1j * TWO_PI * (r / np.asarray(nkt) * np.asarray(s.kshift)).sum(-1))
    phir = np.fft.ifftn(phi, axes=ax) * nk * sphase[None, None, :, :, :, None]
    w = s.w_rx.reshape(nkt + (nx,))
    phir = phir * w[None, None]
    phik = np.fft.fftn(phir * np.conj(sphase)[None, None, :, :, :, None], axes=ax) / nk
    phik = phik.reshape(nv, na, nk, nx)
    # psi'[v, a, k, n] = sum_x conj(ub[k, x, n]) phik[v, a, k, x]
    return np.einsum("kxn,vakx->vakn", np.conj(ub), phik, optimize=True)


def apply_sr(s, psi):
    """V_SR psi (Sec. 3.2.2): project in with A, couple with M, project out with A^H."""
    nv = psi.shape[0]
    na, nk, nb, _ = _shape(s)
    if s.a_proj is None:
        return np.zeros_like(psi)
    npj = s.a_proj.shape[0]
    a2 = s.a_proj.reshape(npj, nk * nb)
    c = np.einsum("pm,vam->vap", a2, psi.reshape(nv, na, nk * nb)).reshape(nv, na * npj)
    cp = (s.m_sr @ c.T).T.reshape(nv, na, npj)
    return np.einsum("pm,vap->vam", np.conj(a2), cp).reshape(nv, na, nk, nb)


def apply_h(s, psi):
    """H psi for one vector [N] or a batch [V][N] (N = Na*Nk*Nb, layout [alpha][k][n])."""
    single = psi.ndim == 1
    na, nk, nb, _ = _shape(s)
    p = np.asarray(psi, dtype=np.complex128).reshape(-1, na, nk, nb)
    out = s.e_nk[None, None, :, :] * p
    out -= np.einsum("ab,vbkn->vakn", s.chi, p)
    out += apply_w0(s, p)
    out += apply_sr(s, p)
    out = out.reshape(p.shape[0], -1)
    return out[0] if single else out


def dense_h(s, apply=None):
    """Explicit H (N x N) by applying H to each unit vector (tiny inputs)."""
    apply = apply or apply_h
    n = s.n_alpha * int(np.prod(s.nk)) * s.n_bands
    eye = np.eye(n, dtype=np.complex128)
    if apply is apply_h:
        return apply_h(s, eye).T.copy()
    return np.stack([apply(s, eye[j]) for j in range(n)], axis=1)


def jacobi_diag(s):
    """diag(H) for the Jacobi preconditioner, [Na][Nk][Nb] real:
    E_nk - chi_aa + sum_x |u_nk(x)|^2 Wbar(x) + sum_{pq} conj(A_p) M_{ap,aq} A_q,
    with Wbar(x) = (1/Nk) sum_R W(x, R) (the k = k' element of Algorithm 1)."""
    na, nk, nb, _ = _shape(s)
    wbar = s.w_rx.mean(axis=0)                                        # [Nx]
    lr = np.einsum("kxn,x->kn", np.abs(s.u) ** 2, wbar)
    d = s.e_nk[None] + lr[None] - np.real(np.diag(s.chi))[:, None, None]
    if s.a_proj is not None:
        npj = s.a_proj.shape[0]
        for a in range(na):
            mb = s.m_sr[a * npj:(a + 1) * npj, a * npj:(a + 1) * npj]
            d[a] += np.real(np.einsum("pkn,pq,qkn->kn", np.conj(s.a_proj), mb, s.a_proj))
    return d


# ----------------------------------------------------------------------------
# Haydock recursion and continued fraction (Sec. 3.2, Eq. 9; Eqs. 1-2)
# ----------------------------------------------------------------------------

def haydock(apply, b, n_steps, reorth=False, breakdown_tol=1e-12):
    """Lanczos/Haydock tridiagonalisation of H started from b.

    v_0 = b/|b|, b_0 = |b|;  for i = 0..n-1:
        w = H v_i;  a_i = Re<v_i|w>;  w -= a_i v_i + b_i v_{i-1} (i >= 1);
        optional full re-orthogonalisation, classical Gram-Schmidt applied twice;
        b_{i+1} = |w|;  stop if b_{i+1} <= tol*max(1, |a_i|);  v_{i+1} = w/b_{i+1}.
    Returns (a[n_done], b[n_done + 1], n_done, breakdown)."""
    b = np.asarray(b, dtype=np.complex128)
    b0 = np.linalg.norm(b)
    v = b / b0
    vprev = np.zeros_like(v)
    a_list, b_list = [], [b0]
    basis = [v] if reorth else None
    breakdown = False
    for i in range(n_steps):
        w = apply(v)
        ai = float(np.real(np.vdot(v, w)))
        a_list.append(ai)
        w = w - ai * v
        if i >= 1:
            w = w - b_list[i] * vprev
        if reorth:
            vb = np.stack(basis, axis=1)
            for _ in range(2):
                w = w - vb @ (vb.conj().T @ w)
        bn = float(np.linalg.norm(w))
        b_list.append(bn)
        if bn <= breakdown_tol * max(1.0, abs(ai)):
            breakdown = True
            break
        vprev, v = v, w / bn
        if reorth:
            basis.append(v)
    return np.array(a_list), np.array(b_list), len(a_list), breakdown


def cf_green(a, b, z, terminator=False):
    """g(z) = 1/(z - a_0 - b_1^2/(z - a_1 - ... - b_{n-1}^2/(z - a_{n-1} - t(z)))).

    b holds b_0..b_n (b_0 = |start vector| is not used here).  t = 0 without a
    terminator; with one, the chain is continued with constant (a_{n-1}, b_n):
    t = b_n^2 g_inf, g_inf = [(z-a) - sqrt((z-a)^2 - 4 b_n^2)]/(2 b_n^2), with
    the root chosen so Im g_inf <= 0 for Im z > 0.  Evaluated bottom-up."""
    z = np.asarray(z, dtype=np.complex128)
    n = len(a)
    t = np.zeros_like(z)
    if terminator and n >= 1 and len(b) > n and b[n] > 0:
        ainf, binf = a[n - 1], b[n]
        zz = z - ainf
        root = np.sqrt(zz * zz - 4.0 * binf * binf)
        g1 = (zz - root) / (2.0 * binf * binf)
        g2 = (zz + root) / (2.0 * binf * binf)
        ginf = np.where(np.imag(g1) <= 0, g1, g2)
        t = binf * binf * ginf
    d = z - a[n - 1] - t
    for i in range(n - 2, -1, -1):
        d = z - a[i] - (b[i + 1] ** 2) / d
    return 1.0 / d


def cf_spectrum(a, b, omega, gamma, terminator=False):
    """sigma(omega) = -(1/pi) b_0^2 Im g(omega + i*Gamma)  (Eq. 1 with Eq. 2)."""
    g = cf_green(a, b, np.asarray(omega) + 1j * gamma, terminator)
    return -(b[0] ** 2) / np.pi * np.imag(g)


def exact_spectrum(h, bvec, omega, gamma):
    """sigma(omega) = (1/pi) sum_j |<E_j|b>|^2 Gamma/((omega - E_j)^2 + Gamma^2) via eigh."""
    evals, evecs = np.linalg.eigh(h)
    wts = np.abs(evecs.conj().T @ bvec) ** 2
    om = np.asarray(omega)[:, None]
    return (wts[None, :] * gamma / ((om - evals[None, :]) ** 2 + gamma ** 2)).sum(1) / np.pi


# ----------------------------------------------------------------------------
# GMRES for (H - z) x = b (the resolvent of Eq. 2 applied to one vector)
# ----------------------------------------------------------------------------

def gmres(apply, b, z, precond=None, rtol=1e-6, restart=30, max_iter=3000):
    """Right-preconditioned restarted GMRES(m) with x_0 = 0.

    Solves (H - z) x = b.  Arnoldi by classical Gram-Schmidt applied twice,
    least squares by complex Givens rotations, x = x_0 + P (V y).  The true
    residual |b - (H - z) x| / |b| is recomputed at every restart and at exit.
    precond(v) -> P v (None = identity).  Returns (x, n_matvec, rel_resid)."""
    b = np.asarray(b, dtype=np.complex128)
    pc = precond if precond is not None else (lambda v: v)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    r = b.copy()
    n_mv = 0
    rel = 1.0
    while True:
        beta = np.linalg.norm(r)
        rel = beta / bnorm
        if rel <= rtol or n_mv >= max_iter:
            return x, n_mv, rel
        m = restart
        V = np.zeros((m + 1, b.size), dtype=np.complex128)
        Z = np.zeros((m, b.size), dtype=np.complex128)
        Hm = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = pc(V[j])
            w = apply(Z[j]) - z * Z[j]
            n_mv += 1
            h = np.zeros(j + 1, dtype=np.complex128)
            for _ in range(2):
                hh = V[: j + 1].conj() @ w
                w = w - V[: j + 1].T @ hh
                h += hh
            hn = np.linalg.norm(w)
            Hm[: j + 1, j] = h
            Hm[j + 1, j] = hn
            if hn > 0:
                V[j + 1] = w / hn
            for i in range(j):                       # previous rotations
                t1 = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                t2 = -np.conj(sn[i]) * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j], Hm[i + 1, j] = t1, t2
            aa, bb = Hm[j, j], Hm[j + 1, j]
            rr = np.hypot(abs(aa), abs(bb))
            if abs(aa) == 0.0:
                cs[j], sn[j] = 0.0, 1.0
                Hm[j, j] = bb
            else:
                cs[j] = abs(aa) / rr
                sn[j] = (aa / abs(aa)) * np.conj(bb) / rr
                Hm[j, j] = (aa / abs(aa)) * rr
            Hm[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            j_done = j + 1
            if abs(g[j + 1]) / bnorm <= rtol or n_mv >= max_iter or hn == 0:
                break
        y = np.zeros(j_done, dtype=np.complex128)
        for i in range(j_done - 1, -1, -1):           # back substitution
            y[i] = (g[i] - Hm[i, i + 1:j_done] @ y[i + 1:j_done]) / Hm[i, i]
        x = x + Z[:j_done].T @ y
        r = b - (apply(x) - z * x)


# ----------------------------------------------------------------------------
# RIXS two-step (resonant inelastic scattering, named with XES in the paper's
# abstract and conclusion as the next target of the same machinery; the
# final-state Hamiltonian is not given there -- the reading used: the same
# operator form with the hole index running over localised valence states,
# the photo-electron a spectator of the emission)
# ----------------------------------------------------------------------------

def rixs_emission(d_em, x):
    """Emission step: the hole moves from core state alpha to valence state v,
    the photo-electron (n, k) stays:  y[z][v][kn] = sum_alpha D[v][alpha] x[z][alpha][kn].
    x [Z][Na][Nk*Nb] (or [Z][Na*Nk*Nb]) -> y [Z][Nv*Nk*Nb]."""
    d_em = np.asarray(d_em, dtype=np.complex128)
    nv, na = d_em.shape
    x = np.asarray(x, dtype=np.complex128)
    z = x.shape[0]
    xr = x.reshape(z, na, -1)
    y = np.zeros((z, nv, xr.shape[2]), dtype=np.complex128)
    for v in range(nv):
        for a in range(na):
            y[:, v, :] += d_em[v, a] * xr[:, a, :]
    return y.reshape(z, -1)


def rixs_two_step(s_core, s_val, d_em, b, z_in, n_steps, rtol=1e-10, restart=30, max_iter=3000, reorth=False):
    """RIXS as absorption into the intermediate state, emission, final-state recursion:
      x(z_in) = (z_in - H_core)^{-1} b          (the resolvent of Eq. 2 at the incoming energy;
                                                 GMRES on (H_core - z_in) x' = b, x = -x')
      y = (D (x) I) x                           (emission, rixs_emission)
      a, b = Haydock(H_val, y)                  (Eq. 9 on the final-state Hamiltonian)
    sigma(z_in, omega_loss) = -(1/pi) |y|^2 Im g(omega_loss + i Gamma_f) then follows from
    cf_spectrum(a, b, omega_loss, Gamma_f).  Returns per incoming shift (a, b, y)."""
    out = []
    for z in np.atleast_1d(z_in):
        xp, _, rel = gmres(lambda v: apply_h(s_core, v), b, z, rtol=rtol, restart=restart, max_iter=max_iter)
        y = rixs_emission(d_em, -xp[None])[0]
        a, bc, _, _ = haydock(lambda v: apply_h(s_val, v), y, n_steps, reorth=reorth)
        out.append((a, bc, y))
    return out
