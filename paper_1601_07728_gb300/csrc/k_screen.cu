// Screening stage (Sec. 3.3): Green's function on the real-space grid around
// the core hole along the imaginary frequency axis and the static RPA
// response from it,
//   G_j(r, r') = sum_K psi(r, K) conj(psi(r', K)) / (mu + i t_j - eps_K),
//   chi0(r, r') = (1/2 pi) sum_j w_j G_j(r, r') G_j(r', r),
// (Eqs. for chi^0 and G with omega' = mu + i t, d omega' = i dt), K = (n, k)
// running over bands and k-points.  G_j for all frequencies is one batched
// complex GEMM psi diag(d_j) psi^H in FP64 (tiles of psi staged in shared
// memory, the diagonal applied while staging); chi0 is an element-wise pass.
#include "bse_internal.cuh"

namespace {

constexpr int GT = 32, GK = 16;   // output tile GT x GT, K chunk GK; 256 threads, 4 outputs each

__global__ void __launch_bounds__(256) green_kernel(const double2* __restrict__ psi, const double* __restrict__ eps,
                                                    int nr, int nkk, double mu, const double* __restrict__ t,
                                                    double2* __restrict__ G) {
  __shared__ double2 As[GT][GK + 1];   // psi(r, K) d_j(K)
  __shared__ double2 Bs[GT][GK + 1];   // conj(psi(r', K))
  const int j = blockIdx.z, r0 = blockIdx.y * GT, c0 = blockIdx.x * GT;
  const int tr = threadIdx.x / 8, tc = threadIdx.x % 8;   // rows r0 + tr, columns c0 + tc + 8 q
  const double tj = t[j];
  double ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
  for (int k0 = 0; k0 < nkk; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += blockDim.x) {
      const int rr = e / GK, kk = e % GK, r = r0 + rr, K = k0 + kk;
      double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
      if (K < nkk) {
        // d = 1 / (mu - eps + i t) = (mu - eps - i t) / ((mu - eps)^2 + t^2)
        const double x = mu - eps[K], den = x * x + tj * tj;
        const double dr = x / den, di = -tj / den;
        if (r < nr) {
          const double2 p = psi[(size_t)r * nkk + K];
          a = make_double2(p.x * dr - p.y * di, p.x * di + p.y * dr);
        }
        const int c = c0 + rr;
        if (c < nr) {
          const double2 q = psi[(size_t)c * nkk + K];
          b = make_double2(q.x, -q.y);
        }
      }
      As[rr][kk] = a;
      Bs[rr][kk] = b;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GK; ++kk) {
      const double2 a = As[tr][kk];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 b = Bs[tc + 8 * q][kk];
        ar[q] += a.x * b.x - a.y * b.y;
        ai[q] += a.x * b.y + a.y * b.x;
      }
    }
    __syncthreads();
  }
  const int r = r0 + tr;
  if (r < nr) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + tc + 8 * q;
      if (c < nr) G[((size_t)j * nr + r) * nr + c] = make_double2(ar[q], ai[q]);
    }
  }
}

// chi0[r][c] = (1/2 pi) sum_j w_j G_j[r][c] G_j[c][r]
__global__ void chi0_kernel(const double2* __restrict__ G, const double* __restrict__ w, int nr, int nt,
                            double2* __restrict__ chi) {
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e >= (size_t)nr * nr) return;
  const int r = (int)(e / nr), c = (int)(e % nr);
  double sr = 0.0, si = 0.0;
  for (int j = 0; j < nt; ++j) {
    const double2 a = G[((size_t)j * nr + r) * nr + c], b = G[((size_t)j * nr + c) * nr + r];
    sr += w[j] * (a.x * b.x - a.y * b.y);
    si += w[j] * (a.x * b.y + a.y * b.x);
  }
  const double s = 1.0 / (2.0 * 3.14159265358979323846);
  chi[e] = make_double2(sr * s, si * s);
}

}  // namespace

bse_status bse_screening_device(const double2* psi, const double* eps, int nr, int nkk, double mu, const double* t,
                                const double* w, int nt, double2* G, double2* chi, cudaStream_t st) {
  const dim3 g((unsigned)((nr + GT - 1) / GT), (unsigned)((nr + GT - 1) / GT), (unsigned)nt);
  green_kernel<<<g, 256, 0, st>>>(psi, eps, nr, nkk, mu, t, G);
  const size_t n = (size_t)nr * nr;
  chi0_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, w, nr, nt, chi);
  return cudaGetLastError() == cudaSuccess ? BSE_OK : BSE_ERR_CUDA;
}
