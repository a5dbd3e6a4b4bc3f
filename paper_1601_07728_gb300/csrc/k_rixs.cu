// RIXS two-step on the device: the absorption resolvent at each incoming
// energy (GMRES on the core-hole Hamiltonian), the emission that moves the
// hole from the core states to the valence states with the photo-electron a
// spectator, and the Haydock recursion of the final-state Hamiltonian for
// every incoming energy at once.  The paper names RIXS as the target of the
// same machinery (abstract, Sec. 5) without giving the final-state
// Hamiltonian; the final state used here has the core-hole Hamiltonian's
// form with the hole index running over localised valence states.
#include "bse_internal.cuh"

#include <stdio.h>

namespace {

// y[z][v][kn] = scale * sum_a D[v][a] x[z][a][kn]; one thread per (kn, z),
// all n_v outputs of a point from one read of its n_alpha inputs.
__global__ void __launch_bounds__(256) rixs_emission_kernel(const double2* __restrict__ d, int nv, int na,
                                                            long long nkb, const double2* __restrict__ x,
                                                            double2* __restrict__ y, double scale) {
  __shared__ double2 ds[BSE_MAX_ALPHA * BSE_MAX_ALPHA];
  for (int i = threadIdx.x; i < nv * na; i += blockDim.x)
    ds[i] = make_double2(scale * d[i].x, scale * d[i].y);
  __syncthreads();
  const int z = blockIdx.y;
  const double2* xz = x + (size_t)z * na * nkb;
  double2* yz = y + (size_t)z * nv * nkb;
  for (long long kn = blockIdx.x * (long long)blockDim.x + threadIdx.x; kn < nkb;
       kn += (long long)gridDim.x * blockDim.x) {
    double2 xa[BSE_MAX_ALPHA];
#pragma unroll
    for (int a = 0; a < BSE_MAX_ALPHA; ++a)
      if (a < na) xa[a] = xz[(size_t)a * nkb + kn];
    for (int v = 0; v < nv; ++v) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int a = 0; a < BSE_MAX_ALPHA; ++a) {
        if (a < na) {
          const double2 q = ds[v * na + a];
          re += q.x * xa[a].x - q.y * xa[a].y;
          im += q.x * xa[a].y + q.y * xa[a].x;
        }
      }
      yz[(size_t)v * nkb + kn] = make_double2(re, im);
    }
  }
}

bse_status launch_emission(const double2* d, int nv, int na, long long nkb, const double2* x, int n_z, double2* y,
                           double scale, cudaStream_t st) {
  const long long blocks = (nkb + 255) / 256;
  const dim3 g((unsigned)(blocks < 2048 ? blocks : 2048), (unsigned)n_z);
  rixs_emission_kernel<<<g, 256, 0, st>>>(d, nv, na, nkb, x, y, scale);
  return cudaGetLastError() == cudaSuccess ? BSE_OK : BSE_ERR_CUDA;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" bse_status bse_rixs_emission(const bse_c128* d_em, int n_v, int n_alpha, long long n_kb,
                                        const bse_c128* x, int n_z, bse_c128* y, void* stream) {
  if (!d_em || !x || !y || n_v < 1 || n_v > BSE_MAX_ALPHA || n_alpha < 1 || n_alpha > BSE_MAX_ALPHA || n_kb < 1 ||
      n_z < 1 || n_z > 65535) {
    fprintf(stderr, "bse_rixs_emission: bad arguments\n");
    return BSE_ERR_INVALID_ARG;
  }
  if (!bse_is_device_ptr(d_em) || !bse_is_device_ptr(x) || !bse_is_device_ptr(y)) {
    fprintf(stderr, "bse_rixs_emission: every array must be device memory\n");
    return BSE_ERR_INVALID_ARG;
  }
  return launch_emission((const double2*)d_em, n_v, n_alpha, n_kb, (const double2*)x, n_z, (double2*)y, 1.0,
                         (cudaStream_t)stream);
}

extern "C" bse_status bse_rixs(bse_handle* core, bse_handle* val, const bse_c128* b, const bse_c128* z_in, int n_z,
                               const bse_c128* d_em, double rtol, int restart, int max_iter, int precond,
                               int n_steps, double* a, double* bcoef, int* steps_done, int* iters,
                               double* rel_resid) {
  if (!core || !val) return BSE_ERR_INVALID_ARG;
  if (!b || !z_in || !d_em || !a || !bcoef || !steps_done || !iters || !rel_resid || n_z < 1 || n_steps < 1 ||
      restart < 1 || max_iter < 1 || !(rtol > 0))
    return bse_fail(core, BSE_ERR_INVALID_ARG, "rixs: bad arguments");
  if (val->nk != core->nk || val->nb != core->nb || val->dev != core->dev)
    return bse_fail(core, BSE_ERR_INVALID_ARG, "rixs: the final-state handle must share the k mesh and bands");
  const long long nkb = (long long)core->nk * core->nb;
  const size_t nz = (size_t)n_z;
  // the caller's arrays: inputs to the device, outputs back where they live
  const bool d_b = bse_is_device_ptr(b), d_z = bse_is_device_ptr(z_in), d_d = bse_is_device_ptr(d_em);
  DevBuf sb, sz, sd, sx, sy, sa, sbc, ss, si, sr;
  auto need = [&](DevBuf& buf, size_t bytes, const char* what) -> bse_status {
    if (cudaMalloc(&buf.p, bytes ? bytes : 16) != cudaSuccess) {
      cudaGetLastError();
      buf.p = nullptr;
      return bse_fail(core, BSE_ERR_OOM, std::string("rixs: cudaMalloc failed for ") + what);
    }
    return BSE_OK;
  };
  bse_status s = BSE_OK;
  cudaStream_t st = core->stream;
  const double2* bd = (const double2*)b;
  const double2* zd = (const double2*)z_in;
  const double2* dd = (const double2*)d_em;
  if (!d_b) {
    if ((s = need(sb, (size_t)core->N * sizeof(double2), "b")) != BSE_OK) return s;
    cudaMemcpyAsync(sb.p, b, (size_t)core->N * sizeof(double2), cudaMemcpyHostToDevice, st);
    bd = (const double2*)sb.p;
  }
  if (!d_z) {
    if ((s = need(sz, nz * sizeof(double2), "z")) != BSE_OK) return s;
    cudaMemcpyAsync(sz.p, z_in, nz * sizeof(double2), cudaMemcpyHostToDevice, st);
    zd = (const double2*)sz.p;
  }
  if (!d_d) {
    if ((s = need(sd, (size_t)val->na * core->na * sizeof(double2), "d_em")) != BSE_OK) return s;
    cudaMemcpyAsync(sd.p, d_em, (size_t)val->na * core->na * sizeof(double2), cudaMemcpyHostToDevice, st);
    dd = (const double2*)sd.p;
  }
  if ((s = need(sx, nz * core->N * sizeof(double2), "intermediate states")) != BSE_OK) return s;
  if ((s = need(sy, nz * val->N * sizeof(double2), "final-state start vectors")) != BSE_OK) return s;
  const bool d_a = bse_is_device_ptr(a), d_bc = bse_is_device_ptr(bcoef), d_s = bse_is_device_ptr(steps_done),
             d_i = bse_is_device_ptr(iters), d_r = bse_is_device_ptr(rel_resid);
  double* ad = a;
  double* bcd = bcoef;
  int* sdd = steps_done;
  int* id = iters;
  double* rd = rel_resid;
  if (!d_a && (s = need(sa, nz * n_steps * sizeof(double), "a")) != BSE_OK) return s;
  if (!d_bc && (s = need(sbc, nz * (n_steps + 1) * sizeof(double), "bcoef")) != BSE_OK) return s;
  if (!d_s && (s = need(ss, nz * sizeof(int), "steps")) != BSE_OK) return s;
  if (!d_i && (s = need(si, nz * sizeof(int), "iters")) != BSE_OK) return s;
  if (!d_r && (s = need(sr, nz * sizeof(double), "rel_resid")) != BSE_OK) return s;
  if (!d_a) ad = (double*)sa.p;
  if (!d_bc) bcd = (double*)sbc.p;
  if (!d_s) sdd = (int*)ss.p;
  if (!d_i) id = (int*)si.p;
  if (!d_r) rd = (double*)sr.p;
  // 1. absorption: (H_core - z) x' = b for every incoming shift; the
  //    intermediate state is x = (z - H_core)^{-1} b = -x'
  const int pk = precond & 0xff;   // x_0 = 0 always: an initial-guess flag is ignored
  if (pk != BSE_PRECOND_NONE && pk != BSE_PRECOND_JACOBI && pk != BSE_PRECOND_MLP)
    return bse_fail(core, BSE_ERR_INVALID_ARG, "rixs: unknown preconditioner");
  const bse_status sg = bse_gmres_device(core, bd, zd, n_z, rtol, restart, max_iter, pk, (double2*)sx.p, id, rd);
  if (sg != BSE_OK && sg != BSE_ERR_NOT_CONVERGED) return sg;
  // 2. emission on the final state's stream, after the absorption
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bse_fail(core, BSE_ERR_CUDA, "rixs: event creation failed");
  }
  cudaEventRecord(ev, st);
  cudaStreamWaitEvent(val->stream, ev, 0);
  cudaEventDestroy(ev);
  s = launch_emission(dd, val->na, core->na, nkb, (const double2*)sx.p, n_z, (double2*)sy.p, -1.0, val->stream);
  val->launches++;
  if (s != BSE_OK) return bse_fail(core, s, "rixs: emission launch failed");
  // 3. final-state recursion, every incoming energy as one start vector
  const bse_status sh = bse_haydock_device(val, (const double2*)sy.p, n_z, n_steps, 0, ad, bcd, sdd);
  if (sh != BSE_OK && sh != BSE_ERR_BREAKDOWN) return bse_fail(core, sh, "rixs: final-state Haydock: " + val->err);
  if (!d_a) cudaMemcpyAsync(a, ad, nz * n_steps * sizeof(double), cudaMemcpyDeviceToHost, val->stream);
  if (!d_bc) cudaMemcpyAsync(bcoef, bcd, nz * (n_steps + 1) * sizeof(double), cudaMemcpyDeviceToHost, val->stream);
  if (!d_s) cudaMemcpyAsync(steps_done, sdd, nz * sizeof(int), cudaMemcpyDeviceToHost, val->stream);
  if (!d_i) cudaMemcpyAsync(iters, id, nz * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!d_r) cudaMemcpyAsync(rel_resid, rd, nz * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(val->stream) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return bse_cuda_check(core, cudaGetLastError(), "rixs sync");
  s = bse_tc_status(core);
  if (s == BSE_OK) s = bse_tc_status(val);
  if (s != BSE_OK) return s;
  if (sg == BSE_ERR_NOT_CONVERGED) return sg;
  return sh;
}
