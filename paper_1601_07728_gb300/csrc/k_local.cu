// Set-up projection of the Bloch functions onto the local basis around the
// absorbing atom (Sec. 3.2.2): with the local functions f_p(x) = R_{nu,l}(r)
// Y_{l,m}(r^) sampled on the real-space grid of one cell (core at the origin,
// minimum image),
//     A[p][k][n] = dv * sum_x conj(f_p(x)) e^{i k.x} u_nk(x),
// a complex GEMM per k (N_p x N_x times N_x x N_b) in FP64.  It runs once per
// system, before bse_setup (whose short-range term takes A as input).
#include "bse_internal.cuh"

namespace {

constexpr int LP = 16, LN = 16, LX = 32;   // projector, band and grid tile of one 256-thread block

__global__ void __launch_bounds__(256) local_proj_kernel(const double2* __restrict__ u, const double2* __restrict__ f,
                                                         int nk0, int nk1, int nk2, int nx0, int nx1, int nx2,
                                                         int nb, int np, double s0, double s1, double s2,
                                                         double dv, double2* __restrict__ a) {
  __shared__ double2 Fs[LP][LX + 1];
  __shared__ double2 Us[LX][LN + 1];
  __shared__ double2 ph[LX];
  const int k = blockIdx.x, n0 = blockIdx.y * LN, p0 = blockIdx.z * LP;
  const int tp = threadIdx.x / LN, tn = threadIdx.x % LN;
  const int nx = nx0 * nx1 * nx2, nkt = nk0 * nk1 * nk2;
  const int m2 = k % nk2, m1 = (k / nk2) % nk1, m0 = k / (nk1 * nk2);
  double ar = 0.0, ai = 0.0;
  for (int x0 = 0; x0 < nx; x0 += LX) {
    if (threadIdx.x < LX) {
      const int x = x0 + threadIdx.x;
      double sn = 0.0, cs = 1.0;
      if (x < nx) {
        const int j2 = x % nx2, j1 = (x / nx2) % nx1, j0 = x / (nx1 * nx2);
        double fr = (m0 + s0) * j0 / ((double)nk0 * nx0) + (m1 + s1) * j1 / ((double)nk1 * nx1) +
                    (m2 + s2) * j2 / ((double)nk2 * nx2);
        fr -= floor(fr);
        sincospi(2.0 * fr, &sn, &cs);
      }
      ph[threadIdx.x] = make_double2(cs, sn);
    }
    for (int e = threadIdx.x; e < LP * LX; e += blockDim.x) {
      const int pp = e / LX, xx = e % LX, p = p0 + pp, x = x0 + xx;
      const double2 v = (p < np && x < nx) ? f[(size_t)p * nx + x] : make_double2(0.0, 0.0);
      Fs[pp][xx] = make_double2(v.x, -v.y);   // conj(f)
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LX * LN; e += blockDim.x) {
      const int xx = e / LN, nn = e % LN, x = x0 + xx, n = n0 + nn;
      double2 v = make_double2(0.0, 0.0);
      if (x < nx && n < nb) {
        const double2 w = u[((size_t)k * nx + x) * nb + n], c = ph[xx];
        v = make_double2(w.x * c.x - w.y * c.y, w.x * c.y + w.y * c.x);   // e^{ik.x} u
      }
      Us[xx][nn] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int xx = 0; xx < LX; ++xx) {
      const double2 fv = Fs[tp][xx], uv = Us[xx][tn];
      ar += fv.x * uv.x - fv.y * uv.y;
      ai += fv.x * uv.y + fv.y * uv.x;
    }
    __syncthreads();
  }
  const int p = p0 + tp, n = n0 + tn;
  if (p < np && n < nb) a[((size_t)p * nkt + k) * nb + n] = make_double2(ar * dv, ai * dv);
}

}  // namespace

bse_status bse_local_projection_device(const double2* u, const int* nk, const int* nx, int nb, const double* kshift,
                                       const double2* f, int np, double dv, double2* a, cudaStream_t st) {
  const int nkt = nk[0] * nk[1] * nk[2];
  const dim3 g((unsigned)nkt, (unsigned)((nb + LN - 1) / LN), (unsigned)((np + LP - 1) / LP));
  local_proj_kernel<<<g, 256, 0, st>>>(u, f, nk[0], nk[1], nk[2], nx[0], nx[1], nx[2], nb, np,
                                       kshift ? kshift[0] : 0.0, kshift ? kshift[1] : 0.0, kshift ? kshift[2] : 0.0,
                                       dv, a);
  return cudaGetLastError() == cudaSuccess ? BSE_OK : BSE_ERR_CUDA;
}
