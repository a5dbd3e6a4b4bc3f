"""ctypes binding of libbse (include/bse.h): argument marshalling only.

Arrays may be numpy arrays (host) or torch CUDA tensors (device); the
library itself finds out which and stages host data.  Every step of H psi,
Haydock, GMRES and the spectrum runs in the library's CUDA kernels; there is
no Python or CPU fallback: if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbse.so")

BSE_OK, BSE_ERR_INVALID_ARG, BSE_ERR_OOM, BSE_ERR_CUDA, BSE_ERR_BREAKDOWN, BSE_ERR_NOT_CONVERGED, \
    BSE_ERR_TIMEOUT, BSE_ERR_NAN, BSE_ERR_UNSUPPORTED = range(9)
PREC = {"fp64": 0, "fp32": 1, "split_bf16": 2}
PRECOND = {"none": 0, "jacobi": 1, "mlp": 2}
GMRES_X0 = 0x100

# every function declared in include/bse.h
EXPORTS = ["bse_setup", "bse_destroy", "bse_dim", "bse_apply_h", "bse_haydock", "bse_cf_spectrum",
           "bse_gmres", "bse_jacobi_diag", "bse_launch_count", "bse_status_string", "bse_last_error",
           "bse_profile_enable", "bse_profile_read", "bse_kernel_name", "bse_short_range_noalloc",
           "bse_mlp_n_params", "bse_mlp_create", "bse_mlp_destroy", "bse_mlp_params", "bse_mlp_outputs",
           "bse_mlp_loss_grad", "bse_mlp_adam_step", "bse_mlp_train", "bse_gmres_set_mlp", "bse_haydock_batch", "bse_autotune", "bse_set_tiles", "bse_local_projection", "bse_screening_chi0", "bse_set_wait_limit", "bse_rixs", "bse_rixs_emission", "bse_set_slabs", "bse_slabs",
           "bse_set_schedule", "bse_schedule"]
KERNEL_KINDS = ["band_to_grid", "kconv", "grid_to_band", "sr_in", "sr_couple", "prep", "recursion", "one_pass"]
# schedules of the split-bf16 step (bse_set_schedule)
SCHEDULES = {"two_pass": 0, "two_pass_rowmajor": 1, "one_pass": 2}


class Desc(ctypes.Structure):
    _fields_ = [
        ("n_alpha", ctypes.c_int),
        ("nk", ctypes.c_int * 3),
        ("n_bands", ctypes.c_int),
        ("nx", ctypes.c_int * 3),
        ("n_proj", ctypes.c_int),
        ("max_vec", ctypes.c_int),
        ("kshift", ctypes.c_double * 3),
        ("u", ctypes.c_void_p),
        ("e_nk", ctypes.c_void_p),
        ("chi", ctypes.c_void_p),
        ("w_rx", ctypes.c_void_p),
        ("a_proj", ctypes.c_void_p),
        ("m_sr", ctypes.c_void_p),
        ("precision", ctypes.c_int),
        ("stream", ctypes.c_void_p),
    ]


_LIB = None


def lib():
    """Load libbse.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbse.so is not built (run paper_1601_07728_gb300/build.py)")
    L = ctypes.CDLL(LIB_PATH)
    vp, ci, cd, cll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    L.bse_setup.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Desc)]
    L.bse_setup.restype = ci
    L.bse_destroy.argtypes = [vp]
    L.bse_destroy.restype = None
    L.bse_dim.argtypes = [vp]
    L.bse_dim.restype = cll
    L.bse_apply_h.argtypes = [vp, vp, vp, ci]
    L.bse_apply_h.restype = ci
    L.bse_haydock.argtypes = [vp, vp, ci, ci, ci, vp, vp, vp]
    L.bse_haydock.restype = ci
    L.bse_cf_spectrum.argtypes = [vp, vp, vp, ci, ci, vp, ci, cd, ci, vp]
    L.bse_cf_spectrum.restype = ci
    L.bse_gmres.argtypes = [vp, vp, vp, ci, cd, ci, ci, ci, vp, vp, vp]
    L.bse_gmres.restype = ci
    L.bse_jacobi_diag.argtypes = [vp, vp]
    L.bse_jacobi_diag.restype = ci
    L.bse_launch_count.argtypes = [vp]
    L.bse_launch_count.restype = cll
    L.bse_status_string.argtypes = [ci]
    L.bse_status_string.restype = ctypes.c_char_p
    L.bse_last_error.argtypes = [vp]
    L.bse_last_error.restype = ctypes.c_char_p
    L.bse_profile_enable.argtypes = [vp, ci]
    L.bse_profile_enable.restype = ci
    L.bse_profile_read.argtypes = [vp, ci, ctypes.POINTER(cll), ctypes.POINTER(cd)]
    L.bse_profile_read.restype = ci
    L.bse_kernel_name.argtypes = [ci]
    L.bse_kernel_name.restype = ctypes.c_char_p
    L.bse_short_range_noalloc.argtypes = [vp, vp, vp, vp, ci, ci, ci, ci, vp]
    L.bse_short_range_noalloc.restype = ci
    L.bse_mlp_n_params.argtypes = []
    L.bse_mlp_n_params.restype = cll
    L.bse_mlp_create.argtypes = [ctypes.POINTER(vp), vp, cll]
    L.bse_mlp_create.restype = ci
    L.bse_mlp_destroy.argtypes = [vp]
    L.bse_mlp_destroy.restype = None
    L.bse_mlp_params.argtypes = [vp, vp]
    L.bse_mlp_params.restype = ci
    L.bse_mlp_outputs.argtypes = [vp, vp, cd, cd, vp]
    L.bse_mlp_outputs.restype = ci
    L.bse_mlp_loss_grad.argtypes = [vp, vp, cd, cd, ci, vp, ci, ctypes.POINTER(cd), vp]
    L.bse_mlp_loss_grad.restype = ci
    L.bse_mlp_adam_step.argtypes = [vp, vp, cd]
    L.bse_mlp_adam_step.restype = ci
    L.bse_mlp_train.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ci, vp, ci, ci, ci, cd, ci, ci, vp, vp]
    L.bse_mlp_train.restype = ci
    L.bse_gmres_set_mlp.argtypes = [vp, vp]
    L.bse_gmres_set_mlp.restype = ci
    L.bse_haydock_batch.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ci, ci, ci, ctypes.POINTER(vp),
                                    ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    L.bse_haydock_batch.restype = ci
    L.bse_autotune.argtypes = [vp, ci, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.bse_autotune.restype = ci
    L.bse_set_tiles.argtypes = [vp, ci, ci]
    L.bse_set_tiles.restype = ci
    L.bse_set_wait_limit.argtypes = [vp, cd]
    L.bse_set_wait_limit.restype = ci
    L.bse_set_slabs.argtypes = [vp, ci]
    L.bse_set_slabs.restype = ci
    L.bse_slabs.argtypes = [vp]
    L.bse_slabs.restype = ci
    L.bse_set_schedule.argtypes = [vp, ci, ci, ci, ci]
    L.bse_set_schedule.restype = ci
    L.bse_schedule.argtypes = [vp]
    L.bse_schedule.restype = ci
    L.bse_rixs.argtypes = [vp, vp, vp, vp, ci, vp, cd, ci, ci, ci, ci, vp, vp, vp, vp, vp]
    L.bse_rixs.restype = ci
    L.bse_rixs_emission.argtypes = [vp, ci, ci, cll, vp, ci, vp, vp]
    L.bse_rixs_emission.restype = ci
    L.bse_local_projection.argtypes = [vp, vp, vp, ci, vp, vp, ci, cd, vp, vp]
    L.bse_local_projection.restype = ci
    L.bse_screening_chi0.argtypes = [vp, vp, ci, ci, cd, vp, vp, ci, vp, vp, vp]
    L.bse_screening_chi0.restype = ci
    _LIB = L
    return L


class BSEError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__("%s %s" % (lib().bse_status_string(status).decode(), msg))


def _ptr(a):
    """Raw address of a numpy array or torch tensor (must be contiguous)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("expected numpy array or torch tensor")


_ELEM = {"complex128": np.complex128, "float64": np.float64, "int32": np.int32}


def _buf(a, elem, n, name):
    """Address of a buffer the library reads or writes n elements of: checks
    its element type and that it holds at least n elements, so that a wrong
    array is refused here instead of being overrun."""
    if a is None:
        raise ValueError("%s is required" % name)
    if isinstance(a, np.ndarray):
        ok, size = a.dtype == _ELEM[elem], a.size
    elif hasattr(a, "data_ptr"):
        ok, size = str(a.dtype) == "torch." + elem, a.numel()
    else:
        raise TypeError("%s: expected numpy array or torch tensor" % name)
    if not ok:
        raise TypeError("%s must hold %s elements, not %s" % (name, elem, a.dtype))
    if size < n:
        raise ValueError("%s holds %d elements, %d needed" % (name, size, n))
    return _ptr(a)


def _n_vectors(a, dim, name):
    """Number of N-vectors in a [N] or [V][N] array."""
    if a.ndim not in (1, 2) or a.shape[-1] != dim:
        raise ValueError("%s must be [%d] or [V][%d], got shape %s" % (name, dim, dim, tuple(a.shape)))
    return 1 if a.ndim == 1 else int(a.shape[0])


class System:
    """One absorbing site on the device (wraps a bse_handle)."""

    def __init__(self, s, precision="fp64", max_vec=1, stream=None):
        L = lib()
        self._keep = []

        def host(a, dt):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                self._keep.append(a)
                return a
            arr = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(arr)
            return arr

        d = Desc()
        d.n_alpha = s.n_alpha
        d.nk = (ctypes.c_int * 3)(*s.nk)
        d.n_bands = s.n_bands
        d.nx = (ctypes.c_int * 3)(*s.nx)
        d.n_proj = s.n_proj
        d.max_vec = int(max_vec)
        d.kshift = (ctypes.c_double * 3)(*s.kshift)
        d.u = _ptr(host(s.u, np.complex128))
        d.e_nk = _ptr(host(s.e_nk, np.float64))
        d.chi = _ptr(host(s.chi, np.complex128))
        d.w_rx = _ptr(host(s.w_rx, np.float64))
        d.a_proj = _ptr(host(s.a_proj, np.complex128))
        d.m_sr = _ptr(host(s.m_sr, np.complex128))
        d.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        d.stream = stream
        h = ctypes.c_void_p()
        st = L.bse_setup(ctypes.byref(h), ctypes.byref(d))
        self._keep = []
        if st != BSE_OK:
            raise BSEError(st, "bse_setup failed")
        self.h = h
        self.dim = int(L.bse_dim(h))
        self.precision = precision
        self.max_vec = int(max_vec)

    def close(self):
        if getattr(self, "h", None):
            lib().bse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, ok=(BSE_OK,)):
        if st not in ok:
            raise BSEError(st, lib().bse_last_error(self.h).decode())
        return st

    @property
    def launches(self):
        return int(lib().bse_launch_count(self.h))

    def apply_h(self, psi, out=None):
        """out = H psi; psi [N] or [V][N] complex128 (numpy or CUDA tensor)."""
        nv = _n_vectors(psi, self.dim, "psi")
        if out is None:
            out = np.empty_like(psi) if isinstance(psi, np.ndarray) else psi.new_empty(psi.shape)
        n = nv * self.dim
        self._check(lib().bse_apply_h(self.h, _buf(psi, "complex128", n, "psi"), _buf(out, "complex128", n, "out"),
                                      nv))
        return out

    def haydock(self, b, n_steps, reorth=False, a=None, bcoef=None, steps=None):
        """Haydock coefficients (a [V][n], b [V][n+1], steps_done [V], status)."""
        nv = _n_vectors(b, self.dim, "b")
        a = np.zeros((nv, n_steps)) if a is None else a
        bcoef = np.zeros((nv, n_steps + 1)) if bcoef is None else bcoef
        steps = np.zeros(nv, dtype=np.int32) if steps is None else steps
        st = lib().bse_haydock(self.h, _buf(b, "complex128", nv * self.dim, "b"), nv, int(n_steps),
                               int(bool(reorth)), _buf(a, "float64", nv * n_steps, "a"),
                               _buf(bcoef, "float64", nv * (n_steps + 1), "bcoef"), _buf(steps, "int32", nv, "steps"))
        self._check(st, (BSE_OK, BSE_ERR_BREAKDOWN))
        return a, bcoef, steps, st

    def gmres(self, b, z, rtol=1e-6, restart=30, max_iter=3000, precond="jacobi", x=None):
        """Solve (H - z_j) x_j = b for every z_j; returns (x [nz][N], iters, rel_resid, status)."""
        z = np.ascontiguousarray(np.atleast_1d(z), dtype=np.complex128)
        nz = z.shape[0]
        x = np.zeros((nz, self.dim), dtype=np.complex128) if x is None else x
        iters = np.zeros(nz, dtype=np.int32)
        rel = np.zeros(nz)
        st = lib().bse_gmres(self.h, _buf(b, "complex128", self.dim, "b"), _ptr(z), nz, float(rtol), int(restart),
                             int(max_iter), PRECOND[precond] if isinstance(precond, str) else int(precond),
                             _buf(x, "complex128", nz * self.dim, "x"), _ptr(iters), _ptr(rel))
        self._check(st, (BSE_OK, BSE_ERR_NOT_CONVERGED))
        return x, iters, rel, st

    def autotune(self, n_vec=1, reps=5):
        """Timed search of the tensor-core tile parameters; returns (split_k, stages), (0, 0) for other forms."""
        sp, sg = ctypes.c_int(), ctypes.c_int()
        self._check(lib().bse_autotune(self.h, int(n_vec), int(reps), ctypes.byref(sp), ctypes.byref(sg)))
        return sp.value, sg.value

    def set_tiles(self, split_k=0, stages=0):
        """Fix the tensor-core tile parameters (0 = the set-up rule)."""
        self._check(lib().bse_set_tiles(self.h, int(split_k), int(stages)))

    def set_slabs(self, slabs):
        """Number of x-slabs of the tensor-core step (1, 2 or 4)."""
        self._check(lib().bse_set_slabs(self.h, int(slabs)))

    @property
    def slabs(self):
        return int(lib().bse_slabs(self.h))

    def set_schedule(self, schedule, lag=0, stages=0, l2_hint=True):
        """Schedule of the split-bf16 step: "two_pass", "two_pass_rowmajor" or "one_pass"
        (one-pass pipeline lag and stages, 0 = defaults; L2 cache policy)."""
        sc = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
        flags = 1 if l2_hint else 0
        self._check(lib().bse_set_schedule(self.h, sc, int(lag), int(stages), flags))

    @property
    def schedule(self):
        v = int(lib().bse_schedule(self.h))
        return {b: a for a, b in SCHEDULES.items()}.get(v, v)

    def set_wait_limit(self, seconds):
        """Limit of every wait of the tensor-core pipeline (BSE_ERR_TIMEOUT beyond it)."""
        self._check(lib().bse_set_wait_limit(self.h, float(seconds)))

    def profile(self, enable=True):
        """Turn per-launch CUDA-event timing on (resets totals) or off."""
        self._check(lib().bse_profile_enable(self.h, int(bool(enable))))

    def profile_read(self):
        """{kernel class: (launches, total ms)} of the timed launches so far."""
        out = {}
        for k, name in enumerate(KERNEL_KINDS):
            n = ctypes.c_longlong()
            ms = ctypes.c_double()
            self._check(lib().bse_profile_read(self.h, k, ctypes.byref(n), ctypes.byref(ms)))
            out[name] = (int(n.value), float(ms.value))
        return out

    def jacobi_diag(self):
        d = np.empty(self.dim)
        self._check(lib().bse_jacobi_diag(self.h, _ptr(d)))
        return d


def cf_spectrum(a, bcoef, steps, omega, gamma, terminator=False):
    """sigma [V][n_omega] from Haydock coefficients, evaluated by the library's kernel."""
    a = np.ascontiguousarray(np.atleast_2d(a), dtype=np.float64)
    bcoef = np.ascontiguousarray(np.atleast_2d(bcoef), dtype=np.float64)
    steps = np.ascontiguousarray(np.atleast_1d(steps), dtype=np.int32)
    omega = np.ascontiguousarray(omega, dtype=np.float64)
    nv, ns = a.shape
    sig = np.zeros((nv, omega.size))
    st = lib().bse_cf_spectrum(_ptr(a), _ptr(bcoef), _ptr(steps), nv, ns, _ptr(omega), omega.size,
                               float(gamma), int(bool(terminator)), _ptr(sig))
    if st != BSE_OK:
        raise BSEError(st, "cf_spectrum failed")
    return sig


class MLP:
    """The learned GMRES preconditioner network (wraps a bse_mlp)."""

    def __init__(self, params):
        L = lib()
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = ctypes.c_void_p()
        st = L.bse_mlp_create(ctypes.byref(h), p.ctypes.data, p.size)
        if st != BSE_OK:
            raise BSEError(st, "bse_mlp_create failed")
        self.h = h
        self.n = int(L.bse_mlp_n_params())

    def close(self):
        if getattr(self, "h", None):
            lib().bse_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.n, dtype=np.float32)
        _chk(lib().bse_mlp_params(self.h, out.ctypes.data))
        return out

    def outputs(self, sysg, omega, gamma):
        out = np.empty((sysg.dim, 34), dtype=np.float32)
        sysg._check(lib().bse_mlp_outputs(sysg.h, self.h, float(omega), float(gamma), out.ctypes.data))
        return out

    def loss_grad(self, sysg, omega, gamma, r, steps=10):
        """(loss, grad [n]) on the device probe array r [T][N]: the k-step
        minimal-residual loss (steps = k >= 1) or the plain approximate-inverse loss (steps = 0)."""
        g = np.empty(self.n, dtype=np.float32)
        loss = ctypes.c_double()
        nt = _n_vectors(r, sysg.dim, "r")
        sysg._check(lib().bse_mlp_loss_grad(sysg.h, self.h, float(omega), float(gamma), nt,
                                            _buf(r, "complex128", nt * sysg.dim, "r"), int(steps),
                                            ctypes.byref(loss), g.ctypes.data))
        return loss.value, g

    def adam_step(self, grad, lr):
        g = np.ascontiguousarray(grad, dtype=np.float32)
        _chk(lib().bse_mlp_adam_step(self.h, g.ctypes.data, float(lr)))

    def train(self, systems, bs, z, epochs, batch, lr, seed=0, steps=10):
        """Harvest residual probes on each System and train; returns the mean loss per epoch."""
        n = len(systems)
        hs = (ctypes.c_void_p * n)(*[s.h.value for s in systems])
        keep = [np.ascontiguousarray(b, dtype=np.complex128) for b in bs]
        bp = (ctypes.c_void_p * n)(*[k.ctypes.data for k in keep])
        zz = np.ascontiguousarray(np.atleast_1d(z), dtype=np.complex128)
        hist = np.zeros(epochs)
        st = lib().bse_mlp_train(hs, bp, n, zz.ctypes.data, zz.size, int(epochs), int(batch), float(lr), int(seed),
                                 int(steps), self.h, hist.ctypes.data)
        if st != BSE_OK:
            raise BSEError(st, lib().bse_last_error(systems[0].h).decode())
        return hist


def haydock_batch(systems, bs, n_steps, outs=None):
    """bse_haydock_batch over Systems (each on its own stream); bs[s] [n_vec][N].
    Returns per site (a, bcoef, steps) and the per-site statuses."""
    n = len(systems)
    if len(bs) != n or (outs is not None and len(outs) != n):
        raise ValueError("one start-vector array (and output triple) per system")
    n_vec = _n_vectors(bs[0], systems[0].dim, "bs[0]")
    for i in range(n):
        if _n_vectors(bs[i], systems[i].dim, "bs[%d]" % i) != n_vec:
            raise ValueError("every site takes the same number of start vectors")
    if outs is None:
        outs = [(np.zeros((n_vec, n_steps)), np.zeros((n_vec, n_steps + 1)), np.zeros(n_vec, dtype=np.int32))
                for _ in range(n)]
    V = ctypes.c_void_p
    hs = (V * n)(*[s.h.value for s in systems])
    bp = (V * n)(*[_buf(b, "complex128", n_vec * sy.dim, "bs") for b, sy in zip(bs, systems)])
    ap = (V * n)(*[_buf(o[0], "float64", n_vec * n_steps, "a") for o in outs])
    bcp = (V * n)(*[_buf(o[1], "float64", n_vec * (n_steps + 1), "bcoef") for o in outs])
    sp = (V * n)(*[_buf(o[2], "int32", n_vec, "steps") for o in outs])
    sts = np.zeros(n, dtype=np.int32)
    st = lib().bse_haydock_batch(hs, bp, n, n_vec, int(n_steps), ap, bcp, sp, sts.ctypes.data)
    if st not in (BSE_OK, BSE_ERR_BREAKDOWN):
        raise BSEError(st, "bse_haydock_batch")
    return outs, sts


def _chk(st):
    if st != BSE_OK:
        raise BSEError(st)
    return st


def attach_mlp(sysg, mlp):
    """Attach (or detach with None) the network GMRES uses with precond="mlp".
    The System keeps a reference, so the network outlives its use by the handle."""
    sysg._check(lib().bse_gmres_set_mlp(sysg.h, mlp.h if mlp is not None else None))
    sysg._mlp = mlp


def local_projection(u, nk, nx, f, dv, kshift=(0.0, 0.0, 0.0), stream=None):
    """bse_local_projection: a [Np][Nk][Nb] = dv sum_x conj(f_p(x)) e^{ik.x} u_nk(x).
    u [Nk][Nx][Nb] and f [Np][Nx] are numpy arrays (a is returned on the host)
    or torch CUDA tensors (a is returned as a CUDA tensor, no staging)."""
    device = hasattr(u, "data_ptr")
    if not device:
        u = np.ascontiguousarray(u, dtype=np.complex128)
        f = np.ascontiguousarray(f, dtype=np.complex128)
    nkt, nxt, nb = u.shape
    npj = f.shape[0]
    if nkt != int(np.prod(nk)) or nxt != int(np.prod(nx)) or f.shape[-1] != nxt:
        raise ValueError("u must be [Nk][Nx][Nb] and f [Np][Nx] for the given meshes")
    if device:
        import torch
        a = torch.empty((npj, nkt, nb), dtype=torch.complex128, device=u.device)
    else:
        a = np.zeros((npj, nkt, nb), dtype=np.complex128)
    nk_a = (ctypes.c_int * 3)(*nk)
    nx_a = (ctypes.c_int * 3)(*nx)
    ks = (ctypes.c_double * 3)(*kshift)
    st = lib().bse_local_projection(_buf(u, "complex128", nkt * nxt * nb, "u"), nk_a, nx_a, nb, ks,
                                    _buf(f, "complex128", npj * nxt, "f"), npj, float(dv),
                                    _buf(a, "complex128", npj * nkt * nb, "a"), stream)
    _chk(st)
    return a


def screening_chi0(psi, eps, mu, t, w, want_green=False, stream=None):
    """bse_screening_chi0 on host arrays: returns chi0 [R][R] (and G [n_t][R][R] when want_green)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    t = np.ascontiguousarray(t, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    nr, ns = psi.shape
    chi = np.zeros((nr, nr), dtype=np.complex128)
    g = np.zeros((t.size, nr, nr), dtype=np.complex128) if want_green else None
    st = lib().bse_screening_chi0(psi.ctypes.data, eps.ctypes.data, nr, ns, float(mu), t.ctypes.data, w.ctypes.data,
                                  t.size, g.ctypes.data if g is not None else None, chi.ctypes.data, stream)
    _chk(st)
    return (chi, g) if want_green else chi


def short_range_noalloc(a_proj, m_sr, psi, out, n_alpha, stream=None):
    """out = V_SR psi through bse_short_range_noalloc (device arrays; nothing is
    allocated, the library's static scratch is used).  Returns the status code."""
    n_proj = a_proj.shape[0]
    n_kb = a_proj.shape[-1] if a_proj.ndim == 2 else int(np.prod(a_proj.shape[1:]))
    n_vec = 1 if psi.ndim == 1 else psi.shape[0]
    return lib().bse_short_range_noalloc(_ptr(a_proj), _ptr(m_sr), _ptr(psi), _ptr(out), int(n_alpha), int(n_kb),
                                         int(n_proj), int(n_vec), stream)


def rixs(core, val, b, z_in, d_em, n_steps, rtol=1e-6, restart=30, max_iter=3000, precond="none"):
    """RIXS two-step through bse_rixs: returns (a [nz][n], bcoef [nz][n+1], steps [nz],
    iters [nz], rel_resid [nz], status).  core and val are Systems on the same mesh."""
    z = np.ascontiguousarray(np.atleast_1d(z_in), dtype=np.complex128)
    nz = z.shape[0]
    d = np.ascontiguousarray(d_em, dtype=np.complex128)
    if d.shape != (val.dim // (core.dim // d.shape[1]), d.shape[1]):
        raise ValueError("d_em must be [n_v][n_alpha] of the two systems")
    a = np.zeros((nz, n_steps))
    bc = np.zeros((nz, n_steps + 1))
    steps = np.zeros(nz, dtype=np.int32)
    it = np.zeros(nz, dtype=np.int32)
    rel = np.zeros(nz)
    st = lib().bse_rixs(core.h, val.h, _buf(b, "complex128", core.dim, "b"), _ptr(z), nz, _ptr(d), float(rtol),
                        int(restart), int(max_iter), PRECOND[precond] if isinstance(precond, str) else int(precond),
                        int(n_steps), _ptr(a), _ptr(bc), _ptr(steps), _ptr(it), _ptr(rel))
    if st not in (BSE_OK, BSE_ERR_BREAKDOWN, BSE_ERR_NOT_CONVERGED):
        raise BSEError(st, lib().bse_last_error(core.h).decode())
    return a, bc, steps, it, rel, st


def rixs_emission(d_em, x, y, n_alpha, stream=None):
    """y = (D (x) I) x on device tensors through bse_rixs_emission; returns the status."""
    n_v = d_em.shape[0]
    n_z = 1 if x.ndim == 1 else x.shape[0]
    n_kb = (x.numel() if hasattr(x, "numel") else x.size) // (n_z * n_alpha)
    return lib().bse_rixs_emission(_ptr(d_em), int(n_v), int(n_alpha), int(n_kb), _ptr(x), int(n_z), _ptr(y),
                                   stream)
