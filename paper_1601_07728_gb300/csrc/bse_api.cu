// C-ABI entry points of libbse (declared in include/bse.h): argument checks,
// host<->device staging, and dispatch to the device drivers.
#include "bse_internal.cuh"

#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

bool bse_is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bse_status bse_fail(bse_handle* h, bse_status s, const std::string& msg) {
  if (h && s != BSE_OK) h->err = msg;
  return s;
}

void bse_drop_graph(bse_handle* h) {
  if (h->hay_exec) cudaGraphExecDestroy(h->hay_exec);
  h->hay_exec = nullptr;
  h->hay_exec_launches = 0;
  for (auto& k : h->hay_key) k = 0;
}

bse_status bse_handle_malloc(bse_handle* h, void** p, size_t bytes, const char* what) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (h->dev_cap && h->dev_bytes + bytes > h->dev_cap)
    return bse_fail(h, BSE_ERR_OOM, std::string("device memory cap reached allocating ") + what);
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return bse_fail(h, BSE_ERR_OOM, std::string("cudaMalloc failed for ") + what);
  }
  h->dev_bytes += bytes;
  return BSE_OK;
}

bse_status bse_cuda_check(bse_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return BSE_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return bse_fail(h, e == cudaErrorMemoryAllocation ? BSE_ERR_OOM : BSE_ERR_CUDA, m);
}

// Timing events around one launch.  Inside a stream capture they become
// event-record nodes of the graph (external records), so a captured loop is
// timed as it runs, back to back, rather than launch by launch.
static void prof_record(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (s && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  else
    cudaEventRecord(e, s);
}

void bse_prof_begin(bse_handle* h, int kind) {
  if (!h->prof || h->ev_used + 2 > h->ev.size()) return;
  prof_record(h->ev[h->ev_used], h->cur ? h->cur : h->stream);
  h->ev_kind[h->ev_used / 2] = kind;
}

void bse_prof_end(bse_handle* h) {
  if (!h->prof || h->ev_used + 2 > h->ev.size()) return;
  prof_record(h->ev[h->ev_used + 1], h->cur ? h->cur : h->stream);
  h->ev_used += 2;
}

namespace {

// Device view of a caller array: either the caller's device pointer or a
// temporary device copy of host data (copied back on request).
struct Staged {
  void* dev = nullptr;
  bool owned = false;
  ~Staged() {
    if (owned && dev) cudaFree(dev);
  }
};

bse_status stage_in(bse_handle* h, Staged& s, const void* p, size_t bytes, bool copy, const char* what) {
  if (bse_is_device_ptr(p)) {
    s.dev = const_cast<void*>(p);
    return BSE_OK;
  }
  if (cudaMalloc(&s.dev, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    s.dev = nullptr;
    return bse_fail(h, BSE_ERR_OOM, std::string("cudaMalloc failed staging ") + what);
  }
  s.owned = true;
  if (copy && bytes) return bse_cuda_check(h, cudaMemcpyAsync(s.dev, p, bytes, cudaMemcpyHostToDevice, h->stream), what);
  return BSE_OK;
}

bse_status stage_out(bse_handle* h, Staged& s, void* p, size_t bytes, const char* what) {
  if (!s.owned || !bytes) return BSE_OK;
  return bse_cuda_check(h, cudaMemcpyAsync(p, s.dev, bytes, cudaMemcpyDeviceToHost, h->stream), what);
}

void free_handle(bse_handle* h) {
  if (!h) return;
  bse_drop_graph(h);
  void* ptrs[] = {h->e_nk, h->chi, h->a_proj, h->a_proj_f, h->m_sr, h->jdiag, h->twiddle, h->u, h->w, h->u_hi,
                  h->u_lo, h->ut_hi, h->ut_lo, h->phi, h->sr_c, h->sr_cp, h->sr_part, h->bpsi, h->psi_f, h->bphi,
                  h->part, h->tmap};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  bse_tc_free(h);
  if (h->io_in) cudaFree(h->io_in);
  if (h->io_out) cudaFree(h->io_out);
  if (h->ws) cudaFree(h->ws);
  if (h->mlp_anorm) cudaFree(h->mlp_anorm);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  for (cudaEvent_t e : h->ev_slab)
    if (e) cudaEventDestroy(e);
  if (h->ev_side2) cudaEventDestroy(h->ev_side2);
  if (h->side2) cudaStreamDestroy(h->side2);
  delete h;
}

#define TRY(x)                   \
  do {                           \
    bse_status _s = (x);         \
    if (_s != BSE_OK) return _s; \
  } while (0)

}  // namespace

extern "C" {

const char* bse_status_string(bse_status s) {
  switch (s) {
    case BSE_OK: return "BSE_OK";
    case BSE_ERR_INVALID_ARG: return "BSE_ERR_INVALID_ARG";
    case BSE_ERR_OOM: return "BSE_ERR_OOM";
    case BSE_ERR_CUDA: return "BSE_ERR_CUDA";
    case BSE_ERR_BREAKDOWN: return "BSE_ERR_BREAKDOWN";
    case BSE_ERR_NOT_CONVERGED: return "BSE_ERR_NOT_CONVERGED";
    case BSE_ERR_TIMEOUT: return "BSE_ERR_TIMEOUT";
    case BSE_ERR_NAN: return "BSE_ERR_NAN";
    case BSE_ERR_UNSUPPORTED: return "BSE_ERR_UNSUPPORTED";
  }
  return "BSE_ERR_UNKNOWN";
}

const char* bse_last_error(const bse_handle* h) {
  if (!h) return "null handle";
  return h->err.c_str();
}

long long bse_dim(const bse_handle* h) { return h ? h->N : 0; }

long long bse_launch_count(const bse_handle* h) { return h ? h->launches : 0; }

bse_status bse_setup(bse_handle** out, const bse_system_desc* d) {
  if (!out) return BSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d) return BSE_ERR_INVALID_ARG;
  bse_handle* h = new (std::nothrow) bse_handle();
  if (!h) return BSE_ERR_OOM;
  auto bad = [&](const char* m) {
    h->err = m;
    fprintf(stderr, "bse_setup: %s\n", m);
    free_handle(h);
    return BSE_ERR_INVALID_ARG;
  };
  if (d->n_alpha < 1 || d->n_alpha > BSE_MAX_ALPHA) return bad("n_alpha must be in 1..16");
  for (int i = 0; i < 3; ++i) {
    if (d->nk[i] < 1 || d->nk[i] > BSE_MAX_NK_AXIS) return bad("nk[d] must be in 1..16");
    if (d->nx[i] < 1) return bad("nx[d] must be >= 1");
  }
  if (d->n_bands < 1) return bad("n_bands must be >= 1");
  if (d->n_proj < 0 || d->n_proj > BSE_MAX_PROJ) return bad("n_proj must be in 0..64");
  if (!d->u || !d->e_nk || !d->chi || !d->w_rx) return bad("u, e_nk, chi and w_rx are required");
  if (d->n_proj > 0 && (!d->a_proj || !d->m_sr)) return bad("a_proj and m_sr are required when n_proj > 0");
  if (d->precision < BSE_PREC_FP64 || d->precision > BSE_PREC_SPLIT_BF16) return bad("unknown precision");
  if (d->max_vec < 0 || d->max_vec > 4096) return bad("max_vec must be in 0..4096");
  h->na = d->n_alpha;
  h->nb = d->n_bands;
  h->np = d->n_proj;
  h->prec = d->precision;
  h->max_vec = d->max_vec > 0 ? d->max_vec : 1;
  h->nk = 1;
  h->nx = 1;
  for (int i = 0; i < 3; ++i) {
    h->nk3[i] = d->nk[i];
    h->nx3[i] = d->nx[i];
    h->nk *= d->nk[i];
    h->nx *= d->nx[i];
    h->kshift[i] = d->kshift[i];
  }
  if (h->nb > h->nx) return bad("n_bands must not exceed the grid size Nx");
  h->N = (long long)h->na * h->nk * h->nb;
  h->stream = (cudaStream_t)d->stream;
  if (const char* cap = getenv("BSE_DEVICE_BYTES_LIMIT")) {
    char* end = nullptr;
    const unsigned long long v = strtoull(cap, &end, 10);
    if (end == cap || *end != '\0') return bad("BSE_DEVICE_BYTES_LIMIT must be a decimal byte count");
    h->dev_cap = (size_t)v;
  }
  if (h->prec == BSE_PREC_SPLIT_BF16) {
    if ((long long)h->max_vec * h->na > 4096) return bad("split-bf16 form needs max_vec*n_alpha <= 4096");
  }
  if (cudaGetDevice(&h->dev) != cudaSuccess) {
    cudaGetLastError();
    h->err = "no CUDA device";
    free_handle(h);
    return BSE_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    h->err = "stream/event creation failed";
    free_handle(h);
    return BSE_ERR_CUDA;
  }
  bse_status s = bse_setup_device(h, d);
  if (s != BSE_OK) {
    fprintf(stderr, "bse_setup: %s (%s)\n", h->err.c_str(), bse_status_string(s));
    free_handle(h);
    return s;
  }
  *out = h;
  return BSE_OK;
}

void bse_destroy(bse_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

bse_status bse_apply_h(bse_handle* h, const bse_c128* psi, bse_c128* hpsi, int n_vec) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (!psi || !hpsi || n_vec < 0) return bse_fail(h, BSE_ERR_INVALID_ARG, "apply_h: bad arguments");
  if (n_vec == 0) return BSE_OK;
  if ((const void*)psi == (void*)hpsi) return bse_fail(h, BSE_ERR_INVALID_ARG, "apply_h: psi and hpsi overlap");
  const size_t bytes = (size_t)n_vec * h->N * sizeof(double2);
  const bool din = bse_is_device_ptr(psi), dout = bse_is_device_ptr(hpsi);
  if ((!din || !dout) && h->io_cap < bytes) {
    if (h->io_in) cudaFree(h->io_in);
    if (h->io_out) cudaFree(h->io_out);
    h->io_in = h->io_out = nullptr;
    h->io_cap = 0;
    if (cudaMalloc(&h->io_in, bytes) != cudaSuccess || cudaMalloc(&h->io_out, bytes) != cudaSuccess) {
      cudaGetLastError();
      return bse_fail(h, BSE_ERR_OOM, "apply_h: staging allocation failed");
    }
    h->io_cap = bytes;
  }
  const double2* dp = din ? (const double2*)psi : (const double2*)h->io_in;
  double2* dq = dout ? (double2*)hpsi : (double2*)h->io_out;
  if (!din) TRY(bse_cuda_check(h, cudaMemcpyAsync((void*)dp, psi, bytes, cudaMemcpyHostToDevice, h->stream), "psi copy-in"));
  for (int v0 = 0; v0 < n_vec; v0 += h->max_vec) {
    int nv = n_vec - v0 < h->max_vec ? n_vec - v0 : h->max_vec;
    TRY(bse_apply_device(h, dp + (size_t)v0 * h->N, dq + (size_t)v0 * h->N, nv));
  }
  if (!dout) {
    TRY(bse_cuda_check(h, cudaMemcpyAsync(hpsi, dq, bytes, cudaMemcpyDeviceToHost, h->stream), "hpsi copy-out"));
    TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "apply_h sync"));
    TRY(bse_tc_status(h));
  }
  return BSE_OK;
}

bse_status bse_haydock(bse_handle* h, const bse_c128* b, int n_vec, int n_steps, int reorth, double* a,
                       double* bcoef, int* steps_done) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (!b || !a || !bcoef || !steps_done || n_vec < 1 || n_steps < 1)
    return bse_fail(h, BSE_ERR_INVALID_ARG, "haydock: bad arguments");
  Staged sb, sa, sbb, ss;
  TRY(stage_in(h, sb, b, (size_t)n_vec * h->N * sizeof(double2), true, "b"));
  TRY(stage_in(h, sa, a, (size_t)n_vec * n_steps * sizeof(double), false, "a"));
  TRY(stage_in(h, sbb, bcoef, (size_t)n_vec * (n_steps + 1) * sizeof(double), false, "bcoef"));
  TRY(stage_in(h, ss, steps_done, (size_t)n_vec * sizeof(int), false, "steps_done"));
  bse_status s = bse_haydock_device(h, (const double2*)sb.dev, n_vec, n_steps, reorth, (double*)sa.dev,
                                    (double*)sbb.dev, (int*)ss.dev);
  if (s != BSE_OK && s != BSE_ERR_BREAKDOWN && s != BSE_ERR_NAN) return s;
  TRY(stage_out(h, sa, a, (size_t)n_vec * n_steps * sizeof(double), "a copy-out"));
  TRY(stage_out(h, sbb, bcoef, (size_t)n_vec * (n_steps + 1) * sizeof(double), "b copy-out"));
  TRY(stage_out(h, ss, steps_done, (size_t)n_vec * sizeof(int), "steps copy-out"));
  TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "haydock sync"));
  TRY(bse_tc_status(h));
  return s;
}

bse_status bse_haydock_batch(bse_handle* const* hs, const bse_c128* const* b, int n_sites, int n_vec, int n_steps,
                             double* const* a, double* const* bcoef, int* const* steps_done, int* site_status) {
  if (!hs || !b || !a || !bcoef || !steps_done || !site_status || n_sites < 1 || n_vec < 1 || n_steps < 1)
    return BSE_ERR_INVALID_ARG;
  for (int s = 0; s < n_sites; ++s)
    if (!hs[s] || !b[s] || !a[s] || !bcoef[s] || !steps_done[s]) return BSE_ERR_INVALID_ARG;
  std::vector<Staged> sb(n_sites), sa(n_sites), sbb(n_sites), ss(n_sites);
  std::vector<const double2*> bd(n_sites);
  std::vector<double*> ad(n_sites), bcd(n_sites);
  std::vector<int*> sd(n_sites);
  for (int s = 0; s < n_sites; ++s) {
    bse_handle* h = hs[s];
    TRY(stage_in(h, sb[s], b[s], (size_t)n_vec * h->N * sizeof(double2), true, "b"));
    TRY(stage_in(h, sa[s], a[s], (size_t)n_vec * n_steps * sizeof(double), false, "a"));
    TRY(stage_in(h, sbb[s], bcoef[s], (size_t)n_vec * (n_steps + 1) * sizeof(double), false, "bcoef"));
    TRY(stage_in(h, ss[s], steps_done[s], (size_t)n_vec * sizeof(int), false, "steps_done"));
    TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "batch staging"));
    bd[s] = (const double2*)sb[s].dev;
    ad[s] = (double*)sa[s].dev;
    bcd[s] = (double*)sbb[s].dev;
    sd[s] = (int*)ss[s].dev;
  }
  std::vector<bse_status> st(n_sites, BSE_OK);
  bse_status worst = bse_haydock_batch_device(hs, bd.data(), n_sites, n_vec, n_steps, ad.data(), bcd.data(),
                                              sd.data(), st.data());
  for (int s = 0; s < n_sites; ++s) {
    bse_handle* h = hs[s];
    site_status[s] = st[s];
    TRY(stage_out(h, sa[s], a[s], (size_t)n_vec * n_steps * sizeof(double), "a copy-out"));
    TRY(stage_out(h, sbb[s], bcoef[s], (size_t)n_vec * (n_steps + 1) * sizeof(double), "b copy-out"));
    TRY(stage_out(h, ss[s], steps_done[s], (size_t)n_vec * sizeof(int), "steps copy-out"));
    TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "batch sync"));
  }
  return worst;
}

bse_status bse_cf_spectrum(const double* a, const double* bcoef, const int* steps, int n_vec, int n_stride,
                           const double* omega, int n_omega, double gamma, int terminator, double* sigma) {
  if (!a || !bcoef || !steps || !omega || !sigma || n_vec < 1 || n_stride < 1 || n_omega < 0)
    return BSE_ERR_INVALID_ARG;
  if (n_omega == 0) return BSE_OK;
  bse_handle tmp;  // error sink + default stream
  Staged sa, sb, ss, so, sg;
  TRY(stage_in(&tmp, sa, a, (size_t)n_vec * n_stride * sizeof(double), true, "a"));
  TRY(stage_in(&tmp, sb, bcoef, (size_t)n_vec * (n_stride + 1) * sizeof(double), true, "bcoef"));
  TRY(stage_in(&tmp, ss, steps, (size_t)n_vec * sizeof(int), true, "steps"));
  TRY(stage_in(&tmp, so, omega, (size_t)n_omega * sizeof(double), true, "omega"));
  TRY(stage_in(&tmp, sg, sigma, (size_t)n_vec * n_omega * sizeof(double), false, "sigma"));
  // counts in steps above n_stride are clamped by the kernel
  TRY(bse_cf_device((const double*)sa.dev, (const double*)sb.dev, (const int*)ss.dev, n_vec, n_stride,
                    (const double*)so.dev, n_omega, gamma, terminator, (double*)sg.dev, tmp.stream));
  TRY(stage_out(&tmp, sg, sigma, (size_t)n_vec * n_omega * sizeof(double), "sigma copy-out"));
  TRY(bse_cuda_check(&tmp, cudaStreamSynchronize(tmp.stream), "cf sync"));
  return BSE_OK;
}

bse_status bse_local_projection(const bse_c128* u, const int* nk, const int* nx, int n_bands, const double* kshift,
                                const bse_c128* f, int n_proj, double dv, bse_c128* a, void* stream) {
  if (!u || !nk || !nx || !f || !a || n_bands < 1 || n_proj < 1 || n_proj > 4096) return BSE_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (nk[d] < 1 || nk[d] > BSE_MAX_NK_AXIS || nx[d] < 1) return BSE_ERR_INVALID_ARG;
  const size_t nkt = (size_t)nk[0] * nk[1] * nk[2], nxt = (size_t)nx[0] * nx[1] * nx[2];
  if ((size_t)n_bands > nxt) return BSE_ERR_INVALID_ARG;
  bse_handle tmp;   // error sink
  tmp.stream = (cudaStream_t)stream;
  Staged su, sf, sa;
  TRY(stage_in(&tmp, su, u, nkt * nxt * n_bands * sizeof(double2), true, "u"));
  TRY(stage_in(&tmp, sf, f, (size_t)n_proj * nxt * sizeof(double2), true, "f"));
  TRY(stage_in(&tmp, sa, a, (size_t)n_proj * nkt * n_bands * sizeof(double2), false, "a"));
  TRY(bse_local_projection_device((const double2*)su.dev, nk, nx, n_bands, kshift, (const double2*)sf.dev, n_proj, dv,
                                  (double2*)sa.dev, tmp.stream));
  TRY(stage_out(&tmp, sa, a, (size_t)n_proj * nkt * n_bands * sizeof(double2), "a copy-out"));
  TRY(bse_cuda_check(&tmp, cudaStreamSynchronize(tmp.stream), "local projection sync"));
  return BSE_OK;
}

bse_status bse_screening_chi0(const bse_c128* psi, const double* eps, int n_r, int n_states, double mu,
                              const double* t, const double* w, int n_t, bse_c128* green, bse_c128* chi0,
                              void* stream) {
  if (!psi || !eps || !t || !w || !chi0 || n_r < 1 || n_states < 1 || n_t < 1) return BSE_ERR_INVALID_ARG;
  if (n_r > 65535 || n_t > 65535) return BSE_ERR_INVALID_ARG;   // grid y and z extents of the G_j launch
  bse_handle tmp;   // error sink
  tmp.stream = (cudaStream_t)stream;
  const size_t nrr = (size_t)n_r * n_r;
  Staged sp, se, st_, sw, sc, sg;
  TRY(stage_in(&tmp, sp, psi, (size_t)n_r * n_states * sizeof(double2), true, "psi"));
  TRY(stage_in(&tmp, se, eps, (size_t)n_states * sizeof(double), true, "eps"));
  TRY(stage_in(&tmp, st_, t, (size_t)n_t * sizeof(double), true, "t"));
  TRY(stage_in(&tmp, sw, w, (size_t)n_t * sizeof(double), true, "w"));
  TRY(stage_in(&tmp, sc, chi0, nrr * sizeof(double2), false, "chi0"));
  if (green) {
    TRY(stage_in(&tmp, sg, green, (size_t)n_t * nrr * sizeof(double2), false, "green"));
  } else {
    TRY(stage_in(&tmp, sg, nullptr, (size_t)n_t * nrr * sizeof(double2), false, "green (scratch)"));
  }
  TRY(bse_screening_device((const double2*)sp.dev, (const double*)se.dev, n_r, n_states, mu, (const double*)st_.dev,
                           (const double*)sw.dev, n_t, (double2*)sg.dev, (double2*)sc.dev, tmp.stream));
  if (green) TRY(stage_out(&tmp, sg, green, (size_t)n_t * nrr * sizeof(double2), "green copy-out"));
  TRY(stage_out(&tmp, sc, chi0, nrr * sizeof(double2), "chi0 copy-out"));
  TRY(bse_cuda_check(&tmp, cudaStreamSynchronize(tmp.stream), "screening sync"));
  return BSE_OK;
}

bse_status bse_gmres(bse_handle* h, const bse_c128* b, const bse_c128* z, int n_z, double rtol, int restart,
                     int max_iter, int precond, bse_c128* x, int* iters, double* rel_resid) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (!b || !z || !x || !iters || !rel_resid || n_z < 1 || restart < 1 || max_iter < 1 || !(rtol > 0))
    return bse_fail(h, BSE_ERR_INVALID_ARG, "gmres: bad arguments");
  const int pkind = precond & 0xff;
  if ((precond & ~(0xff | BSE_GMRES_X0)) != 0 ||
      (pkind != BSE_PRECOND_NONE && pkind != BSE_PRECOND_JACOBI && pkind != BSE_PRECOND_MLP))
    return bse_fail(h, BSE_ERR_INVALID_ARG, "gmres: unknown preconditioner");
  Staged sb, sz, sx, si, sr;
  TRY(stage_in(h, sb, b, (size_t)h->N * sizeof(double2), true, "b"));
  TRY(stage_in(h, sz, z, (size_t)n_z * sizeof(double2), true, "z"));
  TRY(stage_in(h, sx, x, (size_t)n_z * h->N * sizeof(double2), false, "x"));
  TRY(stage_in(h, si, iters, (size_t)n_z * sizeof(int), false, "iters"));
  TRY(stage_in(h, sr, rel_resid, (size_t)n_z * sizeof(double), false, "rel_resid"));
  bse_status s = bse_gmres_device(h, (const double2*)sb.dev, (const double2*)sz.dev, n_z, rtol, restart,
                                  max_iter, precond, (double2*)sx.dev, (int*)si.dev, (double*)sr.dev);
  if (s != BSE_OK && s != BSE_ERR_NOT_CONVERGED) return s;
  TRY(stage_out(h, sx, x, (size_t)n_z * h->N * sizeof(double2), "x copy-out"));
  TRY(stage_out(h, si, iters, (size_t)n_z * sizeof(int), "iters copy-out"));
  TRY(stage_out(h, sr, rel_resid, (size_t)n_z * sizeof(double), "rel copy-out"));
  TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "gmres sync"));
  TRY(bse_tc_status(h));
  return s;
}

bse_status bse_gmres_set_mlp(bse_handle* h, bse_mlp* m) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (m && h->na > 6) return bse_fail(h, BSE_ERR_UNSUPPORTED, "learned preconditioner supports up to 6 core states");
  h->mlp = m;
  return BSE_OK;
}

const char* bse_kernel_name(int kind) {
  static const char* names[BSE_K_COUNT] = {"band_to_grid", "kconv", "grid_to_band", "sr_in",
                                           "sr_couple", "prep", "recursion", "one_pass"};
  return (kind >= 0 && kind < BSE_K_COUNT) ? names[kind] : "unknown";
}

bse_status bse_profile_enable(bse_handle* h, int enable) {
  if (!h) return BSE_ERR_INVALID_ARG;
  TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "profile sync"));
  bse_drop_graph(h);   // a cached graph has no profiling events in it
  if (enable && h->ev.empty()) {
    h->ev.resize(2 * 8192);
    h->ev_kind.resize(8192);
    for (auto& e : h->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return bse_cuda_check(h, cudaGetLastError(), "event create");
  }
  h->prof = enable != 0;
  h->ev_used = 0;
  if (enable)
    for (int k = 0; k < BSE_K_COUNT; ++k) {
      h->prof_count[k] = 0;
      h->prof_ms[k] = 0;
    }
  return BSE_OK;
}

bse_status bse_profile_read(bse_handle* h, int kind, long long* launches, double* total_ms) {
  if (!h || kind < 0 || kind >= BSE_K_COUNT || !launches || !total_ms) return BSE_ERR_INVALID_ARG;
  TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "profile sync"));
  for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) == cudaSuccess) {
      h->prof_count[h->ev_kind[i / 2]]++;
      h->prof_ms[h->ev_kind[i / 2]] += ms;
    } else {
      cudaGetLastError();
    }
  }
  h->ev_used = 0;
  *launches = h->prof_count[kind];
  *total_ms = h->prof_ms[kind];
  return BSE_OK;
}

bse_status bse_jacobi_diag(bse_handle* h, double* diag) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (!diag) return bse_fail(h, BSE_ERR_INVALID_ARG, "jacobi_diag: NULL output");
  TRY(bse_cuda_check(h, cudaMemcpyAsync(diag, h->jdiag, (size_t)h->N * sizeof(double), cudaMemcpyDefault, h->stream),
                     "jacobi copy"));
  return bse_cuda_check(h, cudaStreamSynchronize(h->stream), "jacobi sync");
}

}  // extern "C"
