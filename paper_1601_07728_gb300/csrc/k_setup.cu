// One-time set-up of a BSE system on the device: copies, e^{ik.x} folding,
// precision conversion and the diagonal of H used by the Jacobi
// preconditioner (Sec. 3.2.1 Algorithm 1 diagonal + Sec. 3.2.2 short range).
#include "bse_internal.cuh"

#include <math.h>
#include <stdio.h>

#include <vector>

namespace {

// u[k][x][n] *= e^{i k.x},  k.x / 2pi = sum_d (m_d + s_d) j_d / (nk_d nx_d)   (Eq. 13)
__global__ void fold_phase_kernel(double2* __restrict__ u, int nk0, int nk1, int nk2, int nx0,
                                  int nx1, int nx2, int nb, double s0, double s1, double s2) {
  const int nx = nx0 * nx1 * nx2;
  const int kx = blockIdx.y;  // k index
  const int m2 = kx % nk2, m1 = (kx / nk2) % nk1, m0 = kx / (nk1 * nk2);
  for (int x = blockIdx.x; x < nx; x += gridDim.x) {
    const int j2 = x % nx2, j1 = (x / nx2) % nx1, j0 = x / (nx1 * nx2);
    double f = (m0 + s0) * j0 / ((double)nk0 * nx0) + (m1 + s1) * j1 / ((double)nk1 * nx1) +
               (m2 + s2) * j2 / ((double)nk2 * nx2);
    f -= floor(f);
    double sn, cs;
    sincospi(2.0 * f, &sn, &cs);
    double2* row = u + ((size_t)kx * nx + x) * nb;
    for (int n = threadIdx.x; n < nb; n += blockDim.x) {
      double2 v = row[n];
      row[n] = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
    }
  }
}

__global__ void to_float2_kernel(const double2* __restrict__ in, float2* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void to_float_kernel(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// bf16 split of a double: hi = bf16(v), lo = bf16(v - hi)
__device__ __forceinline__ void split_bf16(double v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn((float)v);
  lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
}

// u [Nk][Nx][Nb] complex -> hi/lo [Nk][Nx][Kp] (re/im interleaved, rows zero-padded to Kp)
__global__ void split_rows_kernel(const double2* __restrict__ u, __nv_bfloat16* __restrict__ hi,
                                  __nv_bfloat16* __restrict__ lo, size_t nrows, int nb, int kp) {
  const size_t n = nrows * (size_t)kp;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t row = i / kp;
    const int q = (int)(i % kp);
    if (q < 2 * nb) {
      const double2 v = u[row * nb + (q >> 1)];
      split_bf16((q & 1) ? v.y : v.x, hi[i], lo[i]);
    } else {
      hi[i] = __float2bfloat16_rn(0.f);
      lo[i] = __float2bfloat16_rn(0.f);
    }
  }
}

// u [Nk][Nx][Nb] complex -> hi/lo K-tiled transpose [Nk][ceil(Nx/64)][2Nb][64]:
// element (k, row 2n+u, x) at ((k*X64 + x/64)*2Nb + row)*64 + x%64 (x padding zeroed by the caller)
__global__ void split_transpose_kernel(const double2* __restrict__ u, __nv_bfloat16* __restrict__ hi,
                                       __nv_bfloat16* __restrict__ lo, int nx, int nb) {
  __shared__ double2 tile[32][33];
  const int k = blockIdx.z;
  const int x0 = blockIdx.x * 32, n0 = blockIdx.y * 32;
  const double2* uk = u + (size_t)k * nx * nb;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int x = x0 + r, n = n0 + threadIdx.x;
    tile[r][threadIdx.x] = (x < nx && n < nb) ? uk[(size_t)x * nb + n] : make_double2(0, 0);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int n = n0 + r, x = x0 + threadIdx.x;
    if (n < nb && x < nx) {
      double2 v = tile[threadIdx.x][r];
      const size_t x64 = (size_t)(nx + 63) / 64;
      const size_t o = (((size_t)k * x64 + x / 64) * (2 * (size_t)nb) + 2 * n) * 64 + (x % 64);
      split_bf16(v.x, hi[o], lo[o]);
      split_bf16(v.y, hi[o + 64], lo[o + 64]);
    }
  }
}

// wbar[x] = (1/Nk) sum_R W(x, R)
__global__ void wbar_kernel(const double* __restrict__ w, double* __restrict__ wbar, int nk, int nx) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < nx; x += gridDim.x * blockDim.x) {
    double s = 0;
    for (int r = 0; r < nk; ++r) s += w[(size_t)r * nx + x];
    wbar[x] = s / nk;
  }
}

// lr[k][n] = sum_x |u_nk(x)|^2 wbar(x)
__global__ void diag_lr_kernel(const double2* __restrict__ u, const double* __restrict__ wbar,
                               double* __restrict__ lr, int nx, int nb) {
  const int k = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nb) return;
  const double2* uk = u + (size_t)k * nx * nb;
  double s = 0;
  for (int x = 0; x < nx; ++x) {
    double2 v = uk[(size_t)x * nb + n];
    s += (v.x * v.x + v.y * v.y) * wbar[x];
  }
  lr[(size_t)k * nb + n] = s;
}

// d[a][kn] = E[kn] - Re chi_aa + lr[kn] + sum_pq conj(A_p[kn]) M_{ap,aq} A_q[kn]
__global__ void diag_total_kernel(const double* __restrict__ e, const double2* __restrict__ chi,
                                  const double* __restrict__ lr, const double2* __restrict__ a,
                                  const double2* __restrict__ m, double* __restrict__ d, int na,
                                  int nkb, int np) {
  const int al = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nkb; i += gridDim.x * blockDim.x) {
    double v = e[i] - chi[al * na + al].x + lr[i];
    if (np > 0) {
      double sr = 0;
      for (int p = 0; p < np; ++p) {
        double2 ap = a[(size_t)p * nkb + i];
        double2 t = make_double2(0, 0);
        for (int q = 0; q < np; ++q) {
          double2 mm = m[(size_t)(al * np + p) * (na * np) + al * np + q];
          double2 aq = a[(size_t)q * nkb + i];
          t.x += mm.x * aq.x - mm.y * aq.y;
          t.y += mm.x * aq.y + mm.y * aq.x;
        }
        sr += ap.x * t.x + ap.y * t.y;  // Re(conj(ap) * t)
      }
      v += sr;
    }
    d[(size_t)al * nkb + i] = v;
  }
}

template <typename T>
bse_status dev_alloc(bse_handle* h, T** p, size_t bytes, const char* what) {
  void* q = nullptr;
  const bse_status s = bse_handle_malloc(h, &q, bytes, what);
  *p = (T*)q;
  return s;
}

#define TRY(x)                          \
  do {                                  \
    bse_status _s = (x);                \
    if (_s != BSE_OK) return _s;        \
  } while (0)

}  // namespace

bse_status bse_setup_device(bse_handle* h, const bse_system_desc* d) {
  const size_t nkb = (size_t)h->nk * h->nb;
  const size_t nu = (size_t)h->nk * h->nx * h->nb;
  cudaStream_t st = h->stream;

  TRY(dev_alloc(h, &h->e_nk, nkb * sizeof(double), "e_nk"));
  TRY(dev_alloc(h, &h->chi, (size_t)h->na * h->na * sizeof(double2), "chi"));
  TRY(dev_alloc(h, &h->jdiag, (size_t)h->na * nkb * sizeof(double), "jdiag"));
  TRY(dev_alloc(h, &h->twiddle, 3 * 16 * 2 * sizeof(double), "twiddle"));
  TRY(bse_cuda_check(h, cudaMemcpyAsync(h->e_nk, d->e_nk, nkb * sizeof(double), cudaMemcpyDefault, st), "copy e_nk"));
  TRY(bse_cuda_check(h, cudaMemcpyAsync(h->chi, d->chi, (size_t)h->na * h->na * sizeof(double2), cudaMemcpyDefault, st), "copy chi"));
  if (h->np > 0) {
    TRY(dev_alloc(h, &h->a_proj, (size_t)h->np * nkb * sizeof(double2), "a_proj"));
    TRY(dev_alloc(h, &h->m_sr, (size_t)h->na * h->np * h->na * h->np * sizeof(double2), "m_sr"));
    TRY(bse_cuda_check(h, cudaMemcpyAsync(h->a_proj, d->a_proj, (size_t)h->np * nkb * sizeof(double2), cudaMemcpyDefault, st), "copy a_proj"));
    if (h->prec != BSE_PREC_FP64) {
      TRY(dev_alloc(h, &h->a_proj_f, (size_t)h->np * nkb * sizeof(float2), "a_proj (fp32)"));
      BSE_PROF(h, BSE_K_PREP, to_float2_kernel<<<1024, 256, 0, st>>>(h->a_proj, h->a_proj_f, (size_t)h->np * nkb));
    }
    TRY(bse_cuda_check(h, cudaMemcpyAsync(h->m_sr, d->m_sr, (size_t)h->na * h->np * h->na * h->np * sizeof(double2), cudaMemcpyDefault, st), "copy m_sr"));
    TRY(dev_alloc(h, &h->sr_c, (size_t)h->max_vec * h->na * h->np * sizeof(double2), "sr_c"));
    TRY(dev_alloc(h, &h->sr_cp, (size_t)h->max_vec * h->na * h->np * sizeof(double2), "sr_cp"));
    const size_t nblk = (nkb + 63) / 64;
    TRY(dev_alloc(h, &h->sr_part, nblk * h->max_vec * h->na * h->np * sizeof(double2), "sr_part"));
  }

  // twiddles e^{+2 pi i j / n} per axis (host libm, FP64)
  {
    std::vector<double> tw(3 * 16 * 2, 0.0);
    for (int ax = 0; ax < 3; ++ax)
      for (int j = 0; j < h->nk3[ax]; ++j) {
        double ang = 2.0 * M_PI * (double)j / (double)h->nk3[ax];
        tw[(ax * 16 + j) * 2 + 0] = cos(ang);
        tw[(ax * 16 + j) * 2 + 1] = sin(ang);
      }
    TRY(bse_cuda_check(h, cudaMemcpyAsync(h->twiddle, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice, st), "copy twiddle"));
    TRY(bse_cuda_check(h, cudaStreamSynchronize(st), "sync twiddle"));
  }

  // U (FP64) with the phase folded in
  double2* u64 = nullptr;
  double *w64 = nullptr, *wbar = nullptr, *lr = nullptr;
  TRY(dev_alloc(h, &u64, nu * sizeof(double2), "u (fp64 staging)"));
  bse_status s = BSE_OK;
  do {
    if ((s = dev_alloc(h, &w64, (size_t)h->nk * h->nx * sizeof(double), "w")) != BSE_OK) break;
    if ((s = dev_alloc(h, &wbar, (size_t)h->nx * sizeof(double), "wbar")) != BSE_OK) break;
    if ((s = dev_alloc(h, &lr, nkb * sizeof(double), "lr")) != BSE_OK) break;
    if ((s = bse_cuda_check(h, cudaMemcpyAsync(u64, d->u, nu * sizeof(double2), cudaMemcpyDefault, st), "copy u")) != BSE_OK) break;
    if ((s = bse_cuda_check(h, cudaMemcpyAsync(w64, d->w_rx, (size_t)h->nk * h->nx * sizeof(double), cudaMemcpyDefault, st), "copy w")) != BSE_OK) break;
    {
      dim3 g((unsigned)(h->nx < 4096 ? h->nx : 4096), (unsigned)h->nk);
      BSE_PROF(h, BSE_K_PREP, fold_phase_kernel<<<g, 128, 0, st>>>(u64, h->nk3[0], h->nk3[1], h->nk3[2], h->nx3[0], h->nx3[1],
                                           h->nx3[2], h->nb, h->kshift[0], h->kshift[1], h->kshift[2]));
      BSE_PROF(h, BSE_K_PREP, wbar_kernel<<<(h->nx + 255) / 256, 256, 0, st>>>(w64, wbar, h->nk, h->nx));
      dim3 g2((unsigned)((h->nb + 127) / 128), (unsigned)h->nk);
      BSE_PROF(h, BSE_K_PREP, diag_lr_kernel<<<g2, 128, 0, st>>>(u64, wbar, lr, h->nx, h->nb));
      dim3 g3((unsigned)((nkb + 255) / 256 < 2048 ? (nkb + 255) / 256 : 2048), (unsigned)h->na);
      BSE_PROF(h, BSE_K_PREP, diag_total_kernel<<<g3, 256, 0, st>>>(h->e_nk, h->chi, lr, h->a_proj, h->m_sr, h->jdiag, h->na,
                                            (int)nkb, h->np));
    }
    if ((s = bse_cuda_check(h, cudaGetLastError(), "setup kernels")) != BSE_OK) break;

    const size_t nphi = (size_t)h->nk * h->nx * h->max_vec * h->na;
    if (h->prec == BSE_PREC_FP64) {
      h->u = u64;
      u64 = nullptr;
      h->w = w64;
      w64 = nullptr;
      if ((s = dev_alloc(h, (double2**)&h->phi, nphi * sizeof(double2), "phi")) != BSE_OK) break;
    } else {
      float* wf = nullptr;
      if ((s = dev_alloc(h, &wf, (size_t)h->nk * h->nx * sizeof(float), "w (fp32)")) != BSE_OK) break;
      h->w = wf;
      BSE_PROF(h, BSE_K_PREP, to_float_kernel<<<1024, 256, 0, st>>>(w64, wf, (size_t)h->nk * h->nx));
      if ((s = dev_alloc(h, (float2**)&h->phi, nphi * sizeof(float2), "phi")) != BSE_OK) break;
      if (h->prec == BSE_PREC_FP32) {
        float2* uf = nullptr;
        if ((s = dev_alloc(h, &uf, nu * sizeof(float2), "u (fp32)")) != BSE_OK) break;
        h->u = uf;
        BSE_PROF(h, BSE_K_PREP, to_float2_kernel<<<4096, 256, 0, st>>>(u64, uf, nu));
      } else {
        const size_t nr = 2 * nu;
        const int kp = (2 * h->nb + 7) / 8 * 8;   // bf16 rows padded to 16 bytes
        const size_t nrp = (size_t)h->nk * h->nx * kp;
        if ((s = dev_alloc(h, &h->u_hi, nrp * sizeof(__nv_bfloat16), "u_hi")) != BSE_OK) break;
        if ((s = dev_alloc(h, &h->u_lo, nrp * sizeof(__nv_bfloat16), "u_lo")) != BSE_OK) break;
        const size_t ntp = (size_t)h->nk * ((h->nx + 63) / 64) * 64 * 2 * h->nb;   // K-tiled, x padded to 64
        (void)nr;
        if ((s = dev_alloc(h, &h->ut_hi, ntp * sizeof(__nv_bfloat16), "ut_hi")) != BSE_OK) break;
        if ((s = dev_alloc(h, &h->ut_lo, ntp * sizeof(__nv_bfloat16), "ut_lo")) != BSE_OK) break;
        cudaMemsetAsync(h->ut_hi, 0, ntp * sizeof(__nv_bfloat16), st);
        cudaMemsetAsync(h->ut_lo, 0, ntp * sizeof(__nv_bfloat16), st);
        BSE_PROF(h, BSE_K_PREP, split_rows_kernel<<<4096, 256, 0, st>>>(u64, h->u_hi, h->u_lo, (size_t)h->nk * h->nx, h->nb, kp));
        dim3 gt((unsigned)((h->nx + 31) / 32), (unsigned)((h->nb + 31) / 32), (unsigned)h->nk);
        BSE_PROF(h, BSE_K_PREP, split_transpose_kernel<<<gt, dim3(32, 8), 0, st>>>(u64, h->ut_hi, h->ut_lo, h->nx, h->nb));
      }
      if ((s = bse_cuda_check(h, cudaGetLastError(), "conversion kernels")) != BSE_OK) break;
    }
    if ((s = bse_cuda_check(h, cudaStreamSynchronize(st), "setup sync")) != BSE_OK) break;
    if (h->prec == BSE_PREC_SPLIT_BF16) {
      if ((s = bse_tc_prepare(h)) != BSE_OK) break;
    }
  } while (0);
  if (u64) cudaFree(u64);
  if (w64) cudaFree(w64);
  if (wbar) cudaFree(wbar);
  if (lr) cudaFree(lr);
  return s;
}
