"""FP64 oracle of the learned GMRES preconditioner (test infrastructure only).

TEST INFRASTRUCTURE ONLY: used by the test-suite, never by the product path.

The paper has no preconditioner (it uses Haydock, Sec. 3.2); GMRES for
(H - z) x = b with z = omega + i Gamma applies the resolvent of Eq. 2 to one
vector.  The learned preconditioner is defined here step by step so the CUDA
kernels can be checked against it:

  rows j = (alpha, n, k) of the exciton vector (Eq. 8); per row and shift z
  features f_j (12 numbers, see ``features``) -> 3-layer network, width 128,
  SiLU activations, FP16-rounded weights -> 34 outputs o_j:
      sigma_j = i*ETA0 + SHIFT * (o_j0 + i o_j1)             (eV)
      p_j     = 1 / (D_j - z - sigma_j)      D = diag(H) (Jacobi diagonal)
      U_jq    = o_j(2+q)  + i o_j(10+q),   V_jq = o_j(18+q) + i o_j(26+q),  q < 8
  P r = p (.) r + U (V^H r) / N                (diagonal + rank 8)
  loss over (residual r_t, error e_t) pairs of a solve: sum_t |P r_t - e_t|^2 / |e_t|^2.

With the last layer zero, P is the damped diagonal 1/(D - omega - i(Gamma +
ETA0)).  Gradients are by hand-written backpropagation and are pinned against
central finite differences in the test-suite.
"""
from __future__ import annotations

import numpy as np

F_IN, WIDTH, F_OUT, RANK = 12, 128, 34, 8
ETA0 = 4.5      # eV, damping of the initial diagonal
SHIFT = 5.0     # eV per unit of the shift outputs
MAX_ALPHA = 6   # one-hot width of the core-state feature

PARAM_SHAPES = [("w1", (F_IN, WIDTH)), ("b1", (WIDTH,)), ("w2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
                ("w3", (WIDTH, F_OUT)), ("b3", (F_OUT,))]


def n_params():
    return int(sum(np.prod(s) for _, s in PARAM_SHAPES))


def unpack(flat):
    out, o = {}, 0
    for name, shp in PARAM_SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def pack(params):
    return np.concatenate([params[name].reshape(-1) for name, _ in PARAM_SHAPES])


def fp16(params):
    """The function the GPU evaluates: every parameter rounded to FP16."""
    return {k: v.astype(np.float16).astype(np.float64) for k, v in params.items()}


def features(diag, e_nk, chi_diag, a_norm, n_alpha, omega, gamma):
    """Per-row features, [N][12] with N = Na*Nk*Nb rows in [alpha][k][n] order:
      0 (D_j - omega)/10        1 gamma
      2 (E_nk - omega)/10       3 D_j - E_nk + chi_aa   (interaction part of the diagonal)
      4 chi_aa / 5              5 |A_{:,nk}|  (local-basis weight of the band state)
      6..11 one-hot alpha (alpha >= 6 folded into 5)."""
    na = n_alpha
    nkb = e_nk.size
    d = diag.reshape(na, nkb)
    x = np.zeros((na, nkb, F_IN))
    for a in range(na):
        x[a, :, 0] = (d[a] - omega) / 10.0
        x[a, :, 1] = gamma
        x[a, :, 2] = (e_nk.reshape(-1) - omega) / 10.0
        x[a, :, 3] = d[a] - e_nk.reshape(-1) + chi_diag[a]
        x[a, :, 4] = chi_diag[a] / 5.0
        x[a, :, 5] = a_norm.reshape(-1)
        x[a, :, 6 + min(a, MAX_ALPHA - 1)] = 1.0
    return x.reshape(na * nkb, F_IN)


def system_features(s, diag, omega, gamma):
    """features() for a synth.BSESystem and its Jacobi diagonal."""
    a_norm = np.zeros(s.n_k * s.n_bands) if s.a_proj is None else \
        np.sqrt((np.abs(s.a_proj.reshape(s.n_proj, -1)) ** 2).sum(0))
    return features(diag, s.e_nk, np.real(np.diag(s.chi)), a_norm, s.n_alpha, omega, gamma)


def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    sg = 1.0 / (1.0 + np.exp(-x))
    return sg + x * sg * (1.0 - sg)


def forward(params, x):
    """o = W3^T silu(W2^T silu(W1^T x + b1) + b2) + b3 for every row; returns (o, cache)."""
    z1 = x @ params["w1"] + params["b1"]
    h1 = silu(z1)
    z2 = h1 @ params["w2"] + params["b2"]
    h2 = silu(z2)
    o = h2 @ params["w3"] + params["b3"]
    return o, (x, z1, h1, z2, h2)


def assemble(o, diag, z):
    """(p, U, V) of P = diag(p) + U V^H / N from the network outputs."""
    sigma = 1j * ETA0 + SHIFT * (o[:, 0] + 1j * o[:, 1])
    p = 1.0 / (diag - z - sigma)
    u = o[:, 2:2 + RANK] + 1j * o[:, 2 + RANK:2 + 2 * RANK]
    v = o[:, 2 + 2 * RANK:2 + 3 * RANK] + 1j * o[:, 2 + 3 * RANK:2 + 4 * RANK]
    return p, u, v


def apply(p, u, v, r):
    """P r = p (.) r + U (V^H r) / N."""
    return p * r + u @ (v.conj().T @ r) / r.shape[0]


def loss(params, x, diag, z, rs, es, quantize=True):
    """sum_t |P r_t - e_t|^2 / |e_t|^2 with the FP16-rounded network
    (quantize=False evaluates the FP64 network as given)."""
    o, _ = forward(fp16(params) if quantize else params, x)
    p, u, v = assemble(o, diag, z)
    tot = 0.0
    for r, e in zip(rs, es):
        d = apply(p, u, v, r) - e
        tot += float(np.vdot(d, d).real / np.vdot(e, e).real)
    return tot


def grad(params, x, diag, z, rs, es, quantize=True):
    """(loss, dloss/dparams) by backpropagation through assemble and the network.

    With delta_t = P r_t - e_t, w_t = 2/|e_t|^2, c_t = V^H r_t / N and
    lambda_t = U^H delta_t (complex gradients g with dL = Re sum conj(g) dX):
      g_p = sum_t w_t delta_t conj(r_t);   g_U = sum_t w_t delta_t c_t^H;
      g_V = sum_t w_t r_t lambda_t^H / N;  dp = p^2 dsigma, dsigma = SHIFT (do0 + i do1)."""
    q16 = fp16(params) if quantize else params
    o, (x_, z1, h1, z2, h2) = forward(q16, x)
    p, u, v = assemble(o, diag, z)
    n = x.shape[0]
    g_p = np.zeros(n, dtype=np.complex128)
    g_u = np.zeros((n, RANK), dtype=np.complex128)
    g_v = np.zeros((n, RANK), dtype=np.complex128)
    tot = 0.0
    for r, e in zip(rs, es):
        c = v.conj().T @ r / n
        d = p * r + u @ c - e
        w = 2.0 / np.vdot(e, e).real
        tot += 0.5 * w * np.vdot(d, d).real
        g_p += w * d * np.conj(r)
        g_u += w * np.outer(d, np.conj(c))
        lam = u.conj().T @ d
        g_v += w * np.outer(r, np.conj(lam)) / n
    gs = np.conj(g_p) * p * p                                # dL = Re(conj(g_p) p^2 dsigma)
    do = np.zeros_like(o)
    do[:, 0] = SHIFT * np.real(gs)
    do[:, 1] = -SHIFT * np.imag(gs)
    do[:, 2:2 + RANK] = g_u.real
    do[:, 2 + RANK:2 + 2 * RANK] = g_u.imag
    do[:, 2 + 2 * RANK:2 + 3 * RANK] = g_v.real
    do[:, 2 + 3 * RANK:2 + 4 * RANK] = g_v.imag
    gr = {}
    gr["w3"] = h2.T @ do
    gr["b3"] = do.sum(0)
    dh2 = do @ q16["w3"].T
    dz2 = dh2 * dsilu(z2)
    gr["w2"] = h1.T @ dz2
    gr["b2"] = dz2.sum(0)
    dh1 = dz2 @ q16["w2"].T
    dz1 = dh1 * dsilu(z1)
    gr["w1"] = x_.T @ dz1
    gr["b1"] = dz1.sum(0)
    return tot, gr


def _outputs_grad(q16, cache, o, p, g_p, g_u, g_v):
    """Backpropagate per-row complex gradients of (p, U, V) through assemble and the network."""
    x_, z1, h1, z2, h2 = cache
    gs = np.conj(g_p) * p * p
    do = np.zeros_like(o)
    do[:, 0] = SHIFT * np.real(gs)
    do[:, 1] = -SHIFT * np.imag(gs)
    do[:, 2:2 + RANK] = g_u.real
    do[:, 2 + RANK:2 + 2 * RANK] = g_u.imag
    do[:, 2 + 2 * RANK:2 + 3 * RANK] = g_v.real
    do[:, 2 + 3 * RANK:2 + 4 * RANK] = g_v.imag
    gr = {"w3": h2.T @ do, "b3": do.sum(0)}
    dz2 = (do @ q16["w3"].T) * dsilu(z2)
    gr["w2"] = h1.T @ dz2
    gr["b2"] = dz2.sum(0)
    dz1 = (dz2 @ q16["w2"].T) * dsilu(z1)
    gr["w1"] = x_.T @ dz1
    gr["b1"] = dz1.sum(0)
    return gr


def _mr_scale(y, r, scaled):
    """alpha = <y, r>/|y|^2, the minimal-residual step along y, when scaled; else 1."""
    if not scaled:
        return 1.0
    yy = np.vdot(y, y).real
    return np.vdot(y, r) / yy if yy > 0 else 0.0


def spai_loss(params, x, diag, z, rs, apply_h, quantize=True, scaled=False):
    """Approximate-inverse loss on residual probes:
    sum_t |alpha_t (H - z) P r_t - r_t|^2 / |r_t|^2  (apply_h(v) = H v), with
    alpha_t = 1 or, when scaled, the minimal-residual scale that makes each
    term the residual reduction of one minimal-residual step with the
    preconditioned operator (1 - cos^2 of the angle between (H - z) P r_t and r_t)."""
    o, _ = forward(fp16(params) if quantize else params, x)
    p, u, v = assemble(o, diag, z)
    tot = 0.0
    for r in rs:
        y = apply(p, u, v, r)
        ay = apply_h(y) - z * y
        q = _mr_scale(ay, r, scaled) * ay - r
        tot += float(np.vdot(q, q).real / np.vdot(r, r).real)
    return tot


def spai_grad(params, x, diag, z, rs, apply_h, quantize=True, scaled=False):
    """(loss, gradient) of spai_loss.  With q_t = alpha_t (H - z) P r_t - r_t,
    g_t = (H - z)^H conj(alpha_t) q_t = (H - conj(z)) conj(alpha_t) q_t (H
    Hermitian; alpha_t is stationary, so it is held fixed), w_t = 2/|r_t|^2,
    c_t = V^H r_t / N, lambda_t = U^H g_t:
      g_p = sum_t w_t g_t conj(r_t); g_U = sum_t w_t g_t c_t^H; g_V = sum_t w_t r_t lambda_t^H / N."""
    q16 = fp16(params) if quantize else params
    o, cache = forward(q16, x)
    p, u, v = assemble(o, diag, z)
    n = x.shape[0]
    g_p = np.zeros(n, dtype=np.complex128)
    g_u = np.zeros((n, RANK), dtype=np.complex128)
    g_v = np.zeros((n, RANK), dtype=np.complex128)
    tot = 0.0
    for r in rs:
        c = v.conj().T @ r / n
        y = p * r + u @ c
        ay = apply_h(y) - z * y
        al = _mr_scale(ay, r, scaled)
        q = al * ay - r
        g = np.conj(al) * (apply_h(q) - np.conj(z) * q)
        w = 2.0 / np.vdot(r, r).real
        tot += 0.5 * w * np.vdot(q, q).real
        g_p += w * g * np.conj(r)
        g_u += w * np.outer(g, np.conj(c))
        g_v += w * np.outer(r, np.conj(u.conj().T @ g)) / n
    return tot, _outputs_grad(q16, cache, o, p, g_p, g_u, g_v)


def apply_adjoint(p, u, v, x):
    """P^H x = conj(p) x + V (U^H x) / N."""
    n = x.shape[0]
    return np.conj(p) * x + v @ (u.conj().T @ x) / n


def _krylov_residual(p, u, v, z, r, apply_h, k):
    """y_0 = r, y_i = (H - z) P y_{i-1}; c = argmin |r - sum_i c_i y_i| over the
    k vectors y_1..y_k (least squares, numpy.linalg.lstsq); returns (ys, c, res)."""
    ys = [r]
    for _ in range(k):
        t = apply(p, u, v, ys[-1])
        ys.append(apply_h(t) - z * t)
    kmat = np.stack(ys[1:], 1)
    c = np.linalg.lstsq(kmat, r, rcond=None)[0]
    return ys, c, r - kmat @ c


def krylov_loss(params, x, diag, z, rs, apply_h, k, quantize=True):
    """k-step minimal-residual loss on probes r_t:
    sum_t min_{deg q <= k, q(0) = 1} |q((H - z) P) r_t|^2 / |r_t|^2,
    the squared residual reduction of k steps of right-preconditioned GMRES
    started from residual r_t (k = 1: the scaled approximate-inverse loss)."""
    o, _ = forward(fp16(params) if quantize else params, x)
    p, u, v = assemble(o, diag, z)
    tot = 0.0
    for r in rs:
        _, _, res = _krylov_residual(p, u, v, z, r, apply_h, k)
        tot += float(np.vdot(res, res).real / np.vdot(r, r).real)
    return tot


def krylov_grad(params, x, diag, z, rs, apply_h, k, quantize=True):
    """(loss, gradient) of krylov_loss.  The least-squares coefficients c are
    stationary, so d|res|^2 = -2 Re <res, sum_i c_i dy_i>, and with
    dy_i = sum_{m<i} ((H - z)P)^m (H - z) dP y_{i-1-m}:
      dL_t = -w_t Re sum_{m + j <= k-1} c_{m+j+1} <q_m, dP y_j>,
    q_m = (H - z)^H s_m, s_0 = res, s_{m+1} = P^H q_m, w_t = 2/|r_t|^2.
    Summing over m first, G_j = -sum_m conj(c_{m+j+1}) q_m pairs with y_j
    exactly as g_t pairs with r_t in spai_grad."""
    q16 = fp16(params) if quantize else params
    o, cache = forward(q16, x)
    p, u, v = assemble(o, diag, z)
    n = x.shape[0]
    g_p = np.zeros(n, dtype=np.complex128)
    g_u = np.zeros((n, RANK), dtype=np.complex128)
    g_v = np.zeros((n, RANK), dtype=np.complex128)
    tot = 0.0
    for r in rs:
        ys, c, res = _krylov_residual(p, u, v, z, r, apply_h, k)
        w = 2.0 / np.vdot(r, r).real
        tot += 0.5 * w * np.vdot(res, res).real
        qs = []
        s = res
        for _ in range(k):
            q = apply_h(s) - np.conj(z) * s
            qs.append(q)
            s = apply_adjoint(p, u, v, q)
        for j in range(k):
            g = np.zeros(n, dtype=np.complex128)
            for m in range(k - j):
                g -= np.conj(c[m + j]) * qs[m]
            y = ys[j]
            g_p += w * g * np.conj(y)
            g_u += w * np.outer(g, np.conj(v.conj().T @ y / n))
            g_v += w * np.outer(y, np.conj(u.conj().T @ g)) / n
    return tot, _outputs_grad(q16, cache, o, p, g_p, g_u, g_v)


def adam(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (params, m, v)."""
    newp, newm, newv = {}, {}, {}
    for k in params:
        newm[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        newv[k] = beta2 * v[k] + (1 - beta2) * grads[k] ** 2
        mh = newm[k] / (1 - beta1 ** t)
        vh = newv[k] / (1 - beta2 ** t)
        newp[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return newp, newm, newv
