/*
 * bse.h -- C ABI of the GB300 core-excitation Bethe-Salpeter hot path.
 *
 * The library applies the core-hole / photo-electron BSE Hamiltonian
 *     H = H_e - H_h - V_D + V_X                          (Sec. 2, Eq. 3)
 * to exciton vectors psi_{alpha,n,k} (Sec. 3.2, Eq. 8) and drives it inside
 * the Haydock recursion (Sec. 3.2, Eq. 9) and GMRES for (H - z) x = b with
 * z = omega + i*Gamma (the resolvent G(omega) = [omega - H]^{-1} of Eq. 2).
 * H is assembled from
 *   - diagonal band energies E_nk (Eq. 5) and the core spin-orbit matrix chi
 *     (Eq. 4), entering as  E_nk psi_{a n k} - sum_b chi_{ab} psi_{b n k};
 *     the core energy is the energy zero, the lifetime lives in z;
 *   - the long-range screened direct term W_0 (Sec. 3.2.1, Algorithm 1):
 *     band->grid sum with e^{ik.x} u_nk(x), k->R Fourier sum (e^{+ik.R},
 *     unnormalised), multiplication by W(x,R), R->k sum (e^{-ik.R}/Nk) and
 *     projection back with e^{-ik.x} u*_nk(x).  W is the signed potential
 *     energy in eV and is added;
 *   - the short-range direct + exchange term through the local basis of
 *     Eq. 14 (Sec. 3.2.2): c = (A (x) I_alpha) psi, c' = M c,
 *     psi' += (A (x) I_alpha)^H c'.
 *
 * Conventions
 *   Vector layout: psi[v][alpha][k][n], n fastest, complex interleaved
 *   (bse_c128 = {re, im}, identical to numpy / torch complex128).
 *   Meshes: k index = (m1*nk2 + m2)*nk3 + m3 with k_d = 2*pi*(m_d + s_d)/(nk_d a);
 *   the lattice vectors R are indexed the same way (R_d = r_d a); the grid
 *   x index = (j1*nx2 + j2)*nx3 + j3 with x_d = j_d a / nx_d.
 *   Energies in eV.
 *
 * Memory: every array argument of the compute calls may be a host pointer or
 * a device pointer; the library finds out with cudaPointerGetAttributes and
 * copies host data in and out on the handle's stream.  Caller buffers are
 * never freed or retained.  The library owns only the memory of its handles.
 *
 * Errors: every call returns a bse_status; no exception or abort crosses the
 * ABI.  bse_last_error() gives a message for the last failing call on a
 * handle.  Device-side conditions (Lanczos breakdown, NaN, GMRES not
 * converged) are collected in device status words and reported after the
 * call.  Calls on one handle are ordered on the handle's stream and are not
 * thread-safe against each other.
 */
#ifndef BSE_H
#define BSE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } bse_c128;

typedef enum {
  BSE_OK = 0,
  BSE_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, unsupported combination   */
  BSE_ERR_OOM = 2,           /* device allocation failed                          */
  BSE_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed                 */
  BSE_ERR_BREAKDOWN = 4,     /* (not an error) Haydock met an invariant subspace  */
  BSE_ERR_NOT_CONVERGED = 5, /* GMRES hit max_iter before rtol; best x returned   */
  BSE_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                      */
  BSE_ERR_NAN = 7,           /* NaN/Inf met in a recursion coefficient             */
  BSE_ERR_UNSUPPORTED = 8    /* shape/precision outside what the kernels support   */
} bse_status;

/* Arithmetic of the band<->grid contractions (Algorithm 1, first and last
 * lines).  The Haydock / GMRES recursion, inner products, diagonal, spin-orbit
 * and short-range terms are FP64 in every mode. */
typedef enum {
  BSE_PREC_FP64 = 0,        /* u complex128, FP64 FMA: the plain form                 */
  BSE_PREC_FP32 = 1,        /* u complex64, FP32 FMA, FP32 k-transforms               */
  BSE_PREC_SPLIT_BF16 = 2   /* u split into bf16 hi+lo, tcgen05 tensor-core MMAs with
                               3 products (hi*hi + hi*lo + lo*hi), FP32 accumulation */
} bse_precision;

typedef struct bse_handle bse_handle;

/* Description of one absorbing site.  All pointers are read during
 * bse_setup only (host or device memory); the caller keeps ownership. */
typedef struct {
  int n_alpha;           /* core states Na (1 for a 1s edge, 6 for L2,3)           */
  int nk[3];             /* k mesh; Nk = nk0*nk1*nk2                               */
  int n_bands;           /* conduction bands Nb                                     */
  int nx[3];             /* real-space grid per cell; Nx = nx0*nx1*nx2              */
  int n_proj;            /* local-basis functions Np (0: no short-range term)      */
  int max_vec;           /* largest n_vec processed in one pass (0 -> 1, at most
                            4096; split-bf16: max_vec*n_alpha <= 4096); larger
                            batches are processed in chunks of max_vec.  Wide
                            passes (2*max_vec*n_alpha > 256 operand rows) run
                            the tensor-core contractions in 256-row N tiles   */
  double kshift[3];      /* mesh shift s_d in units of the k spacing (0 = Gamma)   */
  const bse_c128* u;     /* [Nk][Nx][Nb] u_nk(x), columns orthonormal per k        */
  const double* e_nk;    /* [Nk][Nb] band energies, eV                             */
  const bse_c128* chi;   /* [Na][Na] Hermitian core spin-orbit matrix, eV          */
  const double* w_rx;    /* [Nk(R)][Nx] sampled W(x, R), eV                         */
  const bse_c128* a_proj;/* [Np][Nk][Nb] local-basis coefficients A (or NULL)      */
  const bse_c128* m_sr;  /* [Na*Np][Na*Np] Hermitian couplings, index (alpha,p)
                            with alpha slow, eV (or NULL)                           */
  int precision;         /* bse_precision                                           */
  void* stream;          /* cudaStream_t used by every call on the handle, or NULL */
} bse_system_desc;

/* Copies the system to the device (current CUDA device), folds e^{ik.x} into
 * u, converts it to the requested precision and precomputes diag(H).
 * Sizes: 1 <= Na <= 16, 1 <= Nb <= Nx, nk_d in 1..16, Np in 0..64.
 * Device-memory inputs are read on the handle's stream: work that produces
 * them on another stream must be complete (or ordered before it) when
 * bse_setup is called.  Returns after the set-up work has finished; the
 * caller may then free or reuse its arrays.
 * Memory budget: if the environment variable BSE_DEVICE_BYTES_LIMIT holds a
 * decimal byte count when bse_setup is called, the sum of the device
 * allocations bse_setup makes for the handle (its temporary staging
 * included) may not exceed it; a set-up that would returns BSE_ERR_OOM, as it
 * does when the device itself is out of memory.  A value that is not a
 * decimal number gives BSE_ERR_INVALID_ARG.
 * On failure *out is NULL and nothing is leaked. */
bse_status bse_setup(bse_handle** out, const bse_system_desc* desc);

/* Releases every device buffer of the handle.  NULL is ignored. */
void bse_destroy(bse_handle* h);

/* Vector length N = Na*Nk*Nb of the handle (0 for NULL). */
long long bse_dim(const bse_handle* h);

/* hpsi[v] = H psi[v] for v < n_vec, both [n_vec][N] complex128.  psi and hpsi
 * must not overlap.  Returns when the result is in hpsi (host) or enqueued on
 * the handle's stream (device output).  One call = n_vec matrix-vector
 * products (Eq. 9). */
bse_status bse_apply_h(bse_handle* h, const bse_c128* psi, bse_c128* hpsi, int n_vec);

/* Haydock recursion (Sec. 3.2, Eq. 9) started from b[v] ([n_vec][N]):
 *   v_0 = b/|b|, b_0 = |b|; w = H v_i; a_i = Re<v_i|w>;
 *   w -= a_i v_i + b_i v_{i-1}; optional full re-orthogonalisation (classical
 *   Gram-Schmidt, twice, FP64) against v_0..v_i; b_{i+1} = |w|;
 *   stop when b_{i+1} <= 1e-12 max(1, |a_i|); v_{i+1} = w / b_{i+1}.
 * Outputs (host or device): a [n_vec][n_steps], bcoef [n_vec][n_steps+1]
 * (bcoef[v][0] = |b_v|), steps_done [n_vec].  Entries past steps_done are 0.
 * All recursion arithmetic is FP64.  Returns BSE_ERR_BREAKDOWN (with valid
 * outputs) if any vector stopped early, BSE_ERR_NAN on a non-finite
 * coefficient.  reorth needs n_vec*(n_steps+1)*N*16 bytes of device memory. */
bse_status bse_haydock(bse_handle* h, const bse_c128* b, int n_vec, int n_steps, int reorth,
                       double* a, double* bcoef, int* steps_done);

/* Haydock runs of several absorbing sites at once (the per-site averaging of
 * Sec. 4.5).  hs[s] are independent handles (uneven sizes allowed), each
 * created with its own non-NULL stream; every site runs bse_haydock's
 * recursion (no re-orthogonalisation) on n_vec start vectors b[s].  All sites
 * are recorded into one CUDA graph -- a fork from a master stream to every
 * site stream, each site's full run, a join -- launched once, so kernels of
 * different sites overlap.  If the streams are not capturable (NULL or shared)
 * the sites run one after another.  Outputs per site as for bse_haydock;
 * site_status [n_sites] (host) receives each site's status; the return value
 * is the worst status other than BSE_ERR_BREAKDOWN. */
bse_status bse_haydock_batch(bse_handle* const* hs, const bse_c128* const* b, int n_sites, int n_vec,
                             int n_steps, double* const* a, double* const* bcoef, int* const* steps_done,
                             int* site_status);

/* Loss function from Haydock coefficients (Eqs. 1-2):
 *   sigma(omega) = -(1/pi) b_0^2 Im g(omega + i*gamma),
 *   g(z) = 1/(z - a_0 - b_1^2/(z - a_1 - ... - b_{n-1}^2/(z - a_{n-1} - t))),
 * t = 0, or (terminator != 0) the constant-chain tail continued with
 * (a_{n-1}, b_n).  a [n_vec][n_stride], bcoef [n_vec][n_stride+1],
 * steps [n_vec] (number of a_i used per vector; a count above n_stride is
 * taken as n_stride, zero or negative gives sigma = 0), omega [n_omega],
 * sigma [n_vec][n_omega].  Evaluated by a device kernel on the current
 * device's legacy default stream. */
bse_status bse_cf_spectrum(const double* a, const double* bcoef, const int* steps, int n_vec,
                           int n_stride, const double* omega, int n_omega, double gamma,
                           int terminator, double* sigma);

/* Preconditioner choice for bse_gmres (low byte of `precond`).  On the shifted
 * Hermitian operator H - z with Re z inside the spectrum a Jacobi right
 * preconditioner can slow GMRES down; NONE is often the better default. */
typedef enum { BSE_PRECOND_NONE = 0, BSE_PRECOND_JACOBI = 1, BSE_PRECOND_MLP = 2 } bse_precond;

/* Flag or-ed into `precond`: x holds the initial guess x_0 on entry (else
 * x_0 = 0).  Restarted GMRES carries only x between cycles, so calling with
 * max_iter = restart and this flag repeatedly reproduces one solve cycle by
 * cycle. */
#define BSE_GMRES_X0 0x100

/* Restarted right-preconditioned GMRES(restart) for (H - z_j) x_j = b, one
 * system per complex shift z_j = omega_j + i*Gamma_j, all n_z systems advanced
 * together (their H applications are batched; systems that have converged
 * drop out of the batch).  x_0 = 0 (or x on entry with BSE_GMRES_X0); Arnoldi by classical
 * Gram-Schmidt in FP64, repeated for a system where its first pass removed
 * more than half of |w|^2 (the DGKS test); Givens least squares; convergence when
 * the true residual |b - (H - z)x|/|b| <= rtol (recomputed at each restart and
 * at exit).  b [N], z [n_z] (bse_c128), x [n_z][N], iters [n_z] (H
 * applications spent on each system), rel_resid [n_z] (true residual).
 * Returns BSE_ERR_NOT_CONVERGED if a system hit max_iter.  Needs about
 * n_z*(restart+3)*N*16 bytes of device memory for the Krylov bases. */
bse_status bse_gmres(bse_handle* h, const bse_c128* b, const bse_c128* z, int n_z, double rtol,
                     int restart, int max_iter, int precond, bse_c128* x, int* iters,
                     double* rel_resid);

/* RIXS two-step (resonant inelastic x-ray scattering, named in the paper's
 * abstract and Sec. 5 as the next use of this machinery; the final-state
 * Hamiltonian is not given there).  Reading: the final state has the
 * core-hole Hamiltonian's form with the hole index running over n_v localised
 * valence states -- `val` is a handle set up with n_alpha = n_v on the same k
 * mesh and bands as `core` -- and the emission moves the hole while the
 * photo-electron (n, k) stays.  For every incoming shift z_j = omega_in + i
 * Gamma_c (z_in [n_z]):
 *   x_j = (z_j - H_core)^{-1} b          GMRES on (H_core - z_j) x' = b as in
 *                                        bse_gmres (x_0 = 0; precond, rtol,
 *                                        restart, max_iter as there), x = -x'
 *   y_j = (D (x) I) x_j                  y[v][kn] = sum_alpha D[v][alpha] x[alpha][kn]
 *   Haydock on H_val from y_j            n_steps steps, no re-orthogonalisation
 * and the RIXS spectrum at energy loss w is
 *   sigma_j(w) = -(1/pi) bcoef[j][0]^2 Im g_j(w + i Gamma_f)
 * (bse_cf_spectrum on a, bcoef, steps_done).  b [N_core], d_em [n_v][n_alpha]
 * (bse_c128), a [n_z][n_steps], bcoef [n_z][n_steps+1], steps_done [n_z],
 * iters [n_z], rel_resid [n_z]: host or device memory.  Allocates the n_z
 * intermediate and final-state vectors.  Returns BSE_ERR_INVALID_ARG for a
 * NULL argument or handles on different meshes/bands/devices,
 * BSE_ERR_NOT_CONVERGED if a GMRES solve stopped at max_iter (the outputs are
 * still written), BSE_ERR_BREAKDOWN if a final-state recursion stopped early
 * (valid outputs), and errors of the two drivers otherwise. */
bse_status bse_rixs(bse_handle* core, bse_handle* val, const bse_c128* b, const bse_c128* z_in, int n_z,
                    const bse_c128* d_em, double rtol, int restart, int max_iter, int precond, int n_steps,
                    double* a, double* bcoef, int* steps_done, int* iters, double* rel_resid);

/* Emission step of the RIXS two-step alone (device arrays, work on `stream`,
 * NULL = legacy default; returns without waiting):
 *   y[z][v][kn] = sum_alpha d_em[v][alpha] x[z][alpha][kn],
 * x [n_z][n_alpha][n_kb], y [n_z][n_v][n_kb], d_em [n_v][n_alpha], all
 * complex128 device memory; 1 <= n_v, n_alpha <= 16, 1 <= n_z <= 65535.
 * BSE_ERR_INVALID_ARG for bad sizes or non-device arrays. */
bse_status bse_rixs_emission(const bse_c128* d_em, int n_v, int n_alpha, long long n_kb, const bse_c128* x,
                             int n_z, bse_c128* y, void* stream);

/* ---- learned GMRES preconditioner (no counterpart in the paper) ----------
 * For every row j = (alpha, n, k) and shift z = omega + i*Gamma, 12 features
 *   (D_j-omega)/10, Gamma, (E_nk-omega)/10, D_j-E_nk+chi_aa, chi_aa/5,
 *   |A_{:,nk}|, one-hot alpha (6)          (D = diag(H) of bse_jacobi_diag)
 * pass a network dense(12,128)-SiLU-dense(128,128)-SiLU-dense(128,34) with FP16
 * weights and FP32 accumulation; its outputs o give
 *   p_j = 1/(D_j - z - sigma_j), sigma_j = i*4.5 eV + 5 eV*(o_0 + i o_1),
 *   U_jq = o_{2+q} + i o_{10+q},  V_jq = o_{18+q} + i o_{26+q}  (q < 8),
 * and GMRES uses the right preconditioner P = diag(p) + U V^H / N.  Parameters
 * are packed w1[12][128], b1[128], w2[128][128], b2[128], w3[128][34], b3[34]
 * (bse_mlp_n_params() floats, FP32 master copy).  Training minimises, over
 * residual probes r_t, the k-step minimal-residual loss
 *   sum_t min_{deg q <= k, q(0) = 1} |q((H - z) P) r_t|^2 / |r_t|^2,
 * the squared residual reduction of k steps of right-preconditioned GMRES
 * started from residual r_t (its gradient runs a forward and an adjoint
 * Krylov chain: 2k applications of H per probe); k = 0 selects the plain
 * approximate-inverse loss sum_t |(H - z) P r_t - r_t|^2 / |r_t|^2.  Adam
 * (beta 0.9/0.999, eps 1e-8).  Supports n_alpha <= 6. */
typedef struct bse_mlp bse_mlp;

long long bse_mlp_n_params(void);
/* Network on the current device from packed FP32 parameters (host or device). */
bse_status bse_mlp_create(bse_mlp** out, const float* params, long long n_params);
void bse_mlp_destroy(bse_mlp* m);
/* Current FP32 master parameters (host or device output). */
bse_status bse_mlp_params(const bse_mlp* m, float* out);
/* Network outputs o [N][34] (FP32) for the handle's system at one shift. */
bse_status bse_mlp_outputs(bse_handle* h, bse_mlp* m, double omega, double gamma, float* out);
/* Loss and its gradient with respect to the parameters (grad [n_params],
 * host or device, overwritten) for one shift and n_probes probes
 * r [n_probes][N] (device memory); krylov_steps k in 0..16 with
 * n_probes * max(k, 1) <= 64.  Costs 2 max(k, 1) applications of H per probe
 * (the handle's precision, in chunks of its max_vec). */
bse_status bse_mlp_loss_grad(bse_handle* h, bse_mlp* m, double omega, double gamma, int n_probes,
                             const bse_c128* r, int krylov_steps, double* loss, float* grad);
/* One Adam step with the given gradient (host or device). */
bse_status bse_mlp_adam_step(bse_mlp* m, const float* grad, double lr);
/* Harvest residual probes on each system (handles hs, start vectors bs [N]
 * each, host or device) for the n_z shifts z -- r = b and the true residuals
 * after 1, 2 and 4 restart cycles of unpreconditioned GMRES(30); probes with
 * |r| <= 1e-5 |b| (converged) are skipped -- then `epochs` passes over the
 * n_sys*n_z samples in a seeded shuffled order with one Adam step per `batch`
 * samples.  loss_per_epoch [epochs] (host) receives the mean sample loss. */
bse_status bse_mlp_train(bse_handle* const* hs, const bse_c128* const* bs, int n_sys, const bse_c128* z,
                         int n_z, int epochs, int batch, double lr, int seed, int krylov_steps, bse_mlp* m,
                         double* loss_per_epoch);
/* Attach (or detach with NULL) the network used by BSE_PRECOND_MLP; the caller
 * keeps ownership and must keep it alive while GMRES runs. */
bse_status bse_gmres_set_mlp(bse_handle* h, bse_mlp* m);

/* diag(H) [Na][Nk][Nb] (FP64): E_nk - chi_aa + sum_x |u_nk(x)|^2 Wbar(x)
 * + sum_pq conj(A_p) M_{ap,aq} A_q with Wbar(x) = mean_R W(x,R); the
 * diagonal of Algorithm 1 plus the short-range term.  Used by the Jacobi
 * preconditioner. */
bse_status bse_jacobi_diag(bse_handle* h, double* diag);

/* Projection of the Bloch functions onto the local basis around the
 * absorbing atom (Sec. 3.2.2, the expansion of phi_nk near the atom in
 * R_{nu,l} Y_{l,m}), the set-up step that produces a_proj for bse_setup:
 *   a[p][k][n] = dv * sum_x conj(f[p][x]) e^{i k.x} u[k][x][n],
 * u [Nk][Nx][Nb] (periodic parts, as for bse_setup), f [n_proj][Nx] the local
 * functions sampled on the cell's grid (zero outside their radius), k and x
 * indexed as in bse_setup, kshift [3] or NULL, dv the volume per grid point;
 * a [n_proj][Nk][Nb].  All complex128, host or device; FP64 arithmetic.
 * Work runs on `stream` (NULL: legacy default) and the call returns when a is
 * written.  Allocates staging copies of host arrays.  Returns
 * BSE_ERR_INVALID_ARG (before any device work) for a NULL u, nk, nx, f or a,
 * n_bands < 1, n_proj outside 1..4096, nk[d] outside 1..16, nx[d] < 1 or
 * n_bands > Nx; BSE_ERR_OOM or BSE_ERR_CUDA from staging or the launch. */
bse_status bse_local_projection(const bse_c128* u, const int* nk, const int* nx, int n_bands, const double* kshift,
                                const bse_c128* f, int n_proj, double dv, bse_c128* a, void* stream);

/* Screening stage (Sec. 3.3): the Green's function on the real-space grid
 * around the core hole along the imaginary axis and the static RPA response,
 *   G_j(r, r') = sum_K psi[r][K] conj(psi[r'][K]) / (mu + i t_j - eps[K]),
 *   chi0(r, r') = (1/2 pi) sum_j w_j G_j(r, r') G_j(r', r)
 * (the frequency integral of chi^0 along omega' = mu + i t with quadrature
 * nodes t [n_t] and weights w [n_t]); K = (n, k) runs over the n_states
 * band/k states.  psi [n_r][n_states] (the Bloch functions on the grid), eps
 * [n_states] eV, chi0 [n_r][n_r]; green [n_t][n_r][n_r] receives the G_j or
 * may be NULL.  Complex128 / FP64, host or device; work on `stream` (NULL:
 * legacy default), returns when the outputs are written.  Allocates staging
 * and the G_j scratch.  Returns BSE_ERR_INVALID_ARG (before any device work)
 * for a NULL psi, eps, t, w or chi0, n_r, n_states or n_t < 1, n_r > 65535 or
 * n_t > 65535; BSE_ERR_OOM or BSE_ERR_CUDA from staging or the launches.  A
 * node t_j = 0 with some eps[K] == mu sits on the integrand's pole and gives
 * non-finite values: the caller's nodes must avoid it (mu between two levels,
 * or t_j > 0). */
bse_status bse_screening_chi0(const bse_c128* psi, const double* eps, int n_r, int n_states, double mu,
                              const double* t, const double* w, int n_t, bse_c128* green, bse_c128* chi0,
                              void* stream);

/* Short-range (local direct + exchange) term alone, out = (A (x) I)^H M (A (x) I) psi,
 * computed without allocating memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc where they need
 * the term -- plug-ins whose host framework owns every device byte through
 * its own pool, and real-time loops that cannot afford the synchronisation an
 * allocation implies.  No handle is used.
 *   a_proj [n_proj][n_kb], m_sr [n_alpha*n_proj]^2 (index (alpha, p), alpha
 *   slow), psi and out [n_vec][n_alpha][n_kb], all complex128 DEVICE memory
 *   of the current device, owned by the caller; n_kb = Nk*Nb.  Arrays on
 *   another device, or host memory, give BSE_ERR_INVALID_ARG.  out may
 *   coincide with or overlap psi (in-place use: psi is read completely before
 *   out is written); out must not share bytes with a_proj or m_sr
 *   (BSE_ERR_INVALID_ARG).  Work is enqueued on `stream` (cudaStream_t, NULL =
 *   legacy default stream); the call returns without waiting for it.
 * Scratch: a 2 MiB array (131072 complex128 entries) compiled into the
 * library as a static device variable.  The call needs
 *   ceil(n_kb/64)*n_vec*n_alpha*n_proj + 2*n_vec*n_alpha*n_proj  entries
 * and returns BSE_ERR_INVALID_ARG (with a message on stderr) for anything
 * larger; n_proj must be in 1..64.
 * First call on a device: with CUDA's lazy module loading (the default), the
 * first call on each device -- and the first after that device's context was
 * reset -- loads the library's device code, and with it the 2 MiB array; that
 * one call therefore allocates device memory (the driver's module load), and
 * it looks up the array's device address with cudaGetSymbolAddress and caches
 * it per device and context.  Make that first call at set-up time, before any
 * stream capture begins; every later call allocates nothing, in this library
 * or in any library it calls, and the array stays resident until the process
 * exits (or the context is destroyed).
 * Every call shares the one array and it keeps the previous call's contents;
 * each call overwrites all the entries it reads, so nothing needs clearing.
 * Calls whose kernels overlap on the GPU (different streams, or host threads
 * using the same device) race on the scratch and must be serialised by the
 * caller. */
bse_status bse_short_range_noalloc(const bse_c128* a_proj, const bse_c128* m_sr, const bse_c128* psi,
                                   bse_c128* out, int n_alpha, int n_kb, int n_proj, int n_vec, void* stream);

/* Number of the library's own kernel launches since the handle was created
 * (every launch the compute calls enqueue is counted). */
long long bse_launch_count(const bse_handle* h);

/* Kernel classes timed by the profiling hook below. */
typedef enum {
  BSE_K_BAND_TO_GRID = 0,   /* Algorithm 1, band -> grid contraction                   */
  BSE_K_KCONV = 1,          /* Algorithm 1, k->R sum, x W(x,R), R->k sum               */
  BSE_K_GRID_TO_BAND = 2,   /* Algorithm 1, grid -> band + diagonal/spin-orbit/short range */
  BSE_K_SR_IN = 3,          /* Sec. 3.2.2 projection onto the local basis              */
  BSE_K_SR_COUPLE = 4,      /* Sec. 3.2.2 multiplet coupling c' = M c                  */
  BSE_K_PREP = 5,           /* operand preparation for the tensor-core form            */
  BSE_K_RECURSION = 6,      /* Haydock / GMRES vector kernels (Eq. 9)                  */
  BSE_K_ONE_PASS = 7,       /* Algorithm 1: both contractions and the k sums, one pass  */
  BSE_K_COUNT = 8
} bse_kernel_kind;

/* Tile search for the tensor-core form (no counterpart in the paper): times
 * H psi on n_vec (<= max_vec) internal test vectors, reps applications per
 * candidate, for every grid->band split-K factor in {1, 2, 4, 8, 16} (at most
 * one per 64-point K block of the grid), every pipeline depth in {3, 4, 6, 8}
 * stages that fits shared memory and, where bse_set_slabs allows it, 1 or 2
 * x-slabs, and keeps the fastest choice for the handle (split_out,
 * stages_out: host, may be NULL; the slab count stays on the handle).  The choice changes
 * only the order of the FP32 partial sums of grid->band.  Other precisions:
 * no-op, outputs 0.  Allocates its test vectors (and a larger partial-sum
 * buffer when needed) and synchronises the handle's stream, so call it
 * outside any stream capture, e.g. right after bse_setup. */
bse_status bse_autotune(bse_handle* h, int n_vec, int reps, int* split_out, int* stages_out);
/* Sets the tensor-core tile parameters directly (e.g. to reproduce a measured
 * configuration): split_k in 1..16 (0: the rule of bse_setup), stages 2..8
 * (0: the rule; more than fit shared memory are capped).  Other precisions:
 * no-op.  Synchronises the handle's stream; may reallocate the partial-sum
 * buffer. */
bse_status bse_set_tiles(bse_handle* h, int split_k, int stages);

/* Number of x-slabs of the tensor-core step (no counterpart in the paper):
 * with slabs = 2 or 4 the real-space grid is cut into that many slabs of
 * whole 128-point tiles; band->grid runs slab after slab on the handle's
 * stream, and as soon as a slab's band->grid is done its k->R / x W / R->k
 * transform and its grid->band contraction run on a second stream, so one
 * slab's transform overlaps the next slab's contractions; the split-K
 * partial sums of every slab meet in the grid->band epilogue.  Only the
 * order of FP32 partial sums changes.  slabs = 1 is the unsplit step.  Needs
 * the split-bf16 form, a 4^3 or 8^3 k mesh, an even grid and at least one
 * 128-point tile per slab (BSE_ERR_UNSUPPORTED otherwise; other precisions:
 * no-op); slabs outside {1, 2, 4}: BSE_ERR_INVALID_ARG.  Synchronises the
 * handle's stream; may reallocate the partial-sum buffer. */
bse_status bse_set_slabs(bse_handle* h, int slabs);
/* The handle's current slab count (0 for NULL). */
int bse_slabs(const bse_handle* h);

/* Schedule of the split-bf16 H psi step over U = e^{ik.x} u_nk(x) (Algorithm 1,
 * Sec. 3.2.1; the schedule is this library's, the paper distributes the same
 * sums over MPI ranks):
 *   BSE_SCHED_TWO_PASS (default): band->grid reads U row-major ([k][x][n]),
 *     grid->band reads a K-tiled transposed copy ([k][x/64][n][64]); U
 *     streams from HBM once per contraction;
 *   BSE_SCHED_TWO_PASS_ROWMAJOR: as above, but grid->band reads the row-major
 *     U as an MN-major tensor-core operand (the transposed copy unused);
 *   BSE_SCHED_ONE_PASS: one persistent kernel walks the grid in slabs of 128
 *     points; per slab it runs band->grid for every k, the k->R sum x W(x,R)
 *     R->k sum of the slab's points, and grid->band for every k reading the
 *     slab's U again while it is still in L2 -- so U streams from HBM once
 *     per H psi.  Its CTAs wait on one another (per-slab counters, every wait
 *     bounded by the limit of bse_set_wait_limit, BSE_ERR_TIMEOUT if one gives
 *     up), so it is used only where this handle's kernels run alone: the
 *     many-site batch keeps the two-pass step; one-pass steps of two handles
 *     must not run at the same time on different streams (each would hold
 *     SMs the other's CTAs wait for, until both give up with
 *     BSE_ERR_TIMEOUT).  It takes 2 Nb <= 128,
 *     N_alpha * n_vec <= 8, a 4^3 or 8^3 k mesh, a grid of a multiple of 8
 *     points and at most 4 k points per SM (BSE_ERR_UNSUPPORTED from this call otherwise; calls with
 *     more vectors fall back to the two-pass step).
 * In the one-pass kernel the grid->band tiles of a slab are issued, between
 * band->grid tiles of later slabs, as soon as the slab's k->R / x W / R->k
 * sums are complete on every CTA; lag (0 = default 2, else 1..3) bounds the
 * slabs read once but not yet twice to lag + 1 (fewer keep U in L2 between
 * its two reads, more hide the exchange between CTAs); stages (0 = default
 * 5, else 2..5): 36 KB pipeline stages of the one-pass kernel; flags (one pass): BSE_SCHED_L2_HINT = TMA cache policies that keep U
 * in L2 after its first read and drop it after the second.  Results differ from the two-pass step only in the order of
 * FP32 sums (no split-K partials).  Other precisions: no-op.  Synchronises
 * the handle's stream. */
enum { BSE_SCHED_TWO_PASS = 0, BSE_SCHED_TWO_PASS_ROWMAJOR = 1, BSE_SCHED_ONE_PASS = 2 };
enum { BSE_SCHED_L2_HINT = 1 };
bse_status bse_set_schedule(bse_handle* h, int schedule, int lag, int stages, int flags);
/* The handle's schedule (-1 for NULL). */
int bse_schedule(const bse_handle* h);

/* Failure-detection aid, no counterpart in the paper: every wait of the
 * tensor-core pipeline (a TMA copy landing, an MMA retiring, an accumulator
 * being drained) gives up after `seconds` (default 2 s, range 1e-6..60).  A
 * wait that gives up makes the kernel stop issuing work, wait for its own
 * copies and MMAs in flight (with a fixed 2 s bound), free its tensor memory
 * and return; the call reports BSE_ERR_TIMEOUT (its outputs are not valid)
 * and the handle stays usable.  Other precisions have no such waits.
 * Synchronises the handle's stream. */
bse_status bse_set_wait_limit(bse_handle* h, double seconds);

/* Measurement aid, no counterpart in the paper: when enabled, every kernel
 * launch of the handle is bracketed by CUDA events on the handle's stream
 * (a pool of 8192 launches; later launches are not timed).  bse_profile_read
 * waits for the stream, folds the recorded launches into per-class totals and
 * returns them for one class; bse_profile_enable(h, 1) also resets them. */
bse_status bse_profile_enable(bse_handle* h, int enable);
bse_status bse_profile_read(bse_handle* h, int kind, long long* launches, double* total_ms);
const char* bse_kernel_name(int kind);

/* Human-readable name of a status code (static storage). */
const char* bse_status_string(bse_status s);

/* Message of the last failing call on h ("" if none; static text for NULL). */
const char* bse_last_error(const bse_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* BSE_H */
