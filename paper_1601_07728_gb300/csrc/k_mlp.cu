// Learned GMRES preconditioner: inference and training on the GPU.
//
// For each row j = (alpha, n, k) of the exciton vector (Sec. 3.2, Eq. 8) and
// shift z = omega + i Gamma, 12 features -> dense(12,128)+SiLU ->
// dense(128,128)+SiLU -> dense(128,34) give
//     p_j = 1 / (D_j - z - sigma_j),  sigma_j = i ETA0 + SHIFT (o_j0 + i o_j1)
//     U_jq = o_j(2+q) + i o_j(10+q),  V_jq = o_j(18+q) + i o_j(26+q)      (q < 8)
// and the right preconditioner P = diag(p) + U V^H / N of GMRES for
// (H - z) x = b (the resolvent of Eq. 2).  Weights are stored in FP16 and every
// product accumulates in FP32; the FP32 master copy, Adam moments and
// gradients live next to them.  Training minimises, over residual probes r_t
// harvested from unpreconditioned GMRES histories, the k-step minimal-residual
// loss sum_t min_{deg q <= k, q(0)=1} |q((H - z)P) r_t|^2/|r_t|^2 (the residual
// reduction of k steps of preconditioned GMRES; k = 0 selects the plain
// approximate-inverse loss |(H - z)P r_t - r_t|^2/|r_t|^2).  Every reduction
// is a fixed-order two-stage sum.
#include "bse_internal.cuh"

#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace {

constexpr int F_IN = 12, WID = 128, F_OUT = 34, RANK = 8;
constexpr float ETA0 = 4.5f, SHIFT = 5.0f;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + F_IN * WID, OFF_W2 = OFF_B1 + WID, OFF_B2 = OFF_W2 + WID * WID,
              OFF_W3 = OFF_B2 + WID, OFF_B3 = OFF_W3 + WID * F_OUT, NPARAM = OFF_B3 + F_OUT;
constexpr int RB = 64;        // rows per dense-layer block
constexpr int NRED = 128;     // blocks of the row reductions
constexpr int WG_BLOCKS = 64; // blocks of the weight-gradient reduction

__device__ __forceinline__ float silu_f(float x) { return x / (1.f + __expf(-x)); }
__device__ __forceinline__ float dsilu_f(float x) {
  const float s = 1.f / (1.f + __expf(-x));
  return s + x * s * (1.f - s);
}

// a_norm[kn] = sqrt(sum_p |A[p][kn]|^2)
__global__ void mlp_anorm(const double2* __restrict__ a, int np, int nkb, float* __restrict__ out) {
  const int kn = blockIdx.x * blockDim.x + threadIdx.x;
  if (kn >= nkb) return;
  double s = 0;
  for (int p = 0; p < np; ++p) {
    const double2 v = a[(size_t)p * nkb + kn];
    s += v.x * v.x + v.y * v.y;
  }
  out[kn] = (float)sqrt(s);
}

__global__ void mlp_features(const double* __restrict__ jdiag, const double* __restrict__ e_nk,
                             const double2* __restrict__ chi, const float* __restrict__ a_norm, int na, int nkb,
                             double omega, double gamma, float* __restrict__ X) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= na * nkb) return;
  const int a = row / nkb, kn = row % nkb;
  const double D = jdiag[row], E = e_nk[kn], ca = chi[a * na + a].x;
  float* x = X + (size_t)row * F_IN;
  x[0] = (float)((D - omega) / 10.0);
  x[1] = (float)gamma;
  x[2] = (float)((E - omega) / 10.0);
  x[3] = (float)(D - E + ca);
  x[4] = (float)(ca / 5.0);
  x[5] = a_norm ? a_norm[kn] : 0.f;
  for (int q = 0; q < 6; ++q) x[6 + q] = (q == (a < 5 ? a : 5)) ? 1.f : 0.f;
}

// Z = X W + b (W [in][out] FP16), H = silu(Z) when H != nullptr.  64 rows per block.
__global__ void __launch_bounds__(256) mlp_dense(const float* __restrict__ X, int in, const __half* __restrict__ W,
                                                 const __half* __restrict__ b, int out, float* __restrict__ Z,
                                                 float* __restrict__ H, int rows) {
  extern __shared__ __align__(16) float dsm[];
  const int outp = (out + 3) & ~3;
  float* Xs = dsm;             // [RB][in]
  float* Ws = dsm + RB * in;   // [in][outp]
  const int r0 = blockIdx.x * RB;
  for (int e = threadIdx.x; e < RB * in; e += blockDim.x) {
    const int r = e / in, k = e % in;
    Xs[e] = (r0 + r < rows) ? X[(size_t)(r0 + r) * in + k] : 0.f;
  }
  for (int e = threadIdx.x; e < in * outp; e += blockDim.x) {
    const int k = e / outp, o = e % outp;
    Ws[e] = o < out ? __half2float(W[k * out + o]) : 0.f;
  }
  __syncthreads();
  const int ng = outp / 4;
  for (int idx = threadIdx.x; idx < RB * ng; idx += blockDim.x) {
    const int r = idx / ng, cg = idx % ng;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int k = 0; k < in; ++k) {
      const float xv = Xs[r * in + k];
      const float4 w4 = *reinterpret_cast<const float4*>(&Ws[k * outp + 4 * cg]);
      a0 = fmaf(xv, w4.x, a0);
      a1 = fmaf(xv, w4.y, a1);
      a2 = fmaf(xv, w4.z, a2);
      a3 = fmaf(xv, w4.w, a3);
    }
    const float acc[4] = {a0, a1, a2, a3};
    if (r0 + r < rows) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int col = 4 * cg + q;
        if (col < out) {
          const float zv = acc[q] + __half2float(b[col]);
          Z[(size_t)(r0 + r) * out + col] = zv;
          if (H) H[(size_t)(r0 + r) * out + col] = silu_f(zv);
        }
      }
    }
  }
}

// dX = dZ W^T, then dZprev = dX * silu'(Zprev):  dZ [rows][out], W [in][out] -> dZprev [rows][in]
__global__ void __launch_bounds__(256) mlp_dense_bwd(const float* __restrict__ dZ, int out,
                                                     const __half* __restrict__ W, int in,
                                                     const float* __restrict__ Zprev, float* __restrict__ dZprev,
                                                     int rows) {
  extern __shared__ __align__(16) float dsm[];
  const int inp = (in + 3) & ~3;
  float* Ds = dsm;              // [RB][out]
  float* Wt = dsm + RB * out;   // [out][inp] = W^T
  const int r0 = blockIdx.x * RB;
  for (int e = threadIdx.x; e < RB * out; e += blockDim.x) {
    const int r = e / out, o = e % out;
    Ds[e] = (r0 + r < rows) ? dZ[(size_t)(r0 + r) * out + o] : 0.f;
  }
  for (int e = threadIdx.x; e < out * inp; e += blockDim.x) {
    const int o = e / inp, i = e % inp;
    Wt[e] = i < in ? __half2float(W[i * out + o]) : 0.f;
  }
  __syncthreads();
  const int ng = inp / 4;
  for (int idx = threadIdx.x; idx < RB * ng; idx += blockDim.x) {
    const int r = idx / ng, cg = idx % ng;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int o = 0; o < out; ++o) {
      const float dv = Ds[r * out + o];
      const float4 w4 = *reinterpret_cast<const float4*>(&Wt[o * inp + 4 * cg]);
      a0 = fmaf(dv, w4.x, a0);
      a1 = fmaf(dv, w4.y, a1);
      a2 = fmaf(dv, w4.z, a2);
      a3 = fmaf(dv, w4.w, a3);
    }
    const float acc[4] = {a0, a1, a2, a3};
    if (r0 + r < rows) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int col = 4 * cg + q;
        if (col < in) {
          const size_t o = (size_t)(r0 + r) * in + col;
          dZprev[o] = acc[q] * dsilu_f(Zprev[o]);
        }
      }
    }
  }
}

// part[blk][(in+1)*out]: sum over this block's rows of X[r][i] dZ[r][o] (i = in: bias, X = 1)
constexpr int WG_PER = 65;   // outputs per thread (>= ceil(129*128/256))
__global__ void __launch_bounds__(256) mlp_wgrad(const float* __restrict__ X, int in, const float* __restrict__ dZ,
                                                 int out, int rows, float* __restrict__ part) {
  __shared__ float Xs[32][WID + 1];
  __shared__ float Ds[32][WID];
  const int nout = (in + 1) * out;
  float acc[WG_PER];
#pragma unroll
  for (int j = 0; j < WG_PER; ++j) acc[j] = 0.f;
  const int per = (rows + gridDim.x - 1) / gridDim.x;
  const int rbeg = blockIdx.x * per, rend = min(rows, rbeg + per);
  for (int c0 = rbeg; c0 < rend; c0 += 32) {
    for (int e = threadIdx.x; e < 32 * (in + 1); e += blockDim.x) {
      const int r = e / (in + 1), i = e % (in + 1);
      Xs[r][i] = (c0 + r < rend) ? (i < in ? X[(size_t)(c0 + r) * in + i] : 1.f) : 0.f;
    }
    for (int e = threadIdx.x; e < 32 * out; e += blockDim.x) {
      const int r = e / out, o = e % out;
      Ds[r][o] = (c0 + r < rend) ? dZ[(size_t)(c0 + r) * out + o] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < WG_PER; ++j) {
      const int e = threadIdx.x + 256 * j;
      if (e < nout) {
        const int i = e / out, o = e % out;
        float s = acc[j];
        for (int r = 0; r < 32; ++r) s = fmaf(Xs[r][i], Ds[r][o], s);
        acc[j] = s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < WG_PER; ++j) {
    const int e = threadIdx.x + 256 * j;
    if (e < nout) part[(size_t)blockIdx.x * nout + e] = acc[j];
  }
}

// grad[w_off + i*out + o] += sum_blk part (i < in), grad[b_off + o] += bias row
__global__ void mlp_wgrad_reduce(const float* __restrict__ part, int nblk, int in, int out, float* __restrict__ grad,
                                 int w_off, int b_off) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int nout = (in + 1) * out;
  if (e >= nout) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += part[(size_t)b * nout + e];
  const int i = e / out, o = e % out;
  if (i < in)
    grad[w_off + i * out + o] += s;
  else
    grad[b_off + o] += s;
}

// p, U, V from the network outputs (FP32)
__global__ void pc_assemble(const float* __restrict__ O, const double* __restrict__ jdiag, double zr, double zi, int N,
                            float2* __restrict__ p, float2* __restrict__ u, float2* __restrict__ v) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const float* o = O + (size_t)j * F_OUT;
  // p = 1 / (D - z - sigma), sigma = i ETA0 + SHIFT (o0 + i o1)
  const float dr = (float)(jdiag[j] - zr) - SHIFT * o[0];
  const float di = (float)(-zi) - ETA0 - SHIFT * o[1];
  const float den = dr * dr + di * di;
  p[j] = make_float2(dr / den, -di / den);
  for (int q = 0; q < RANK; ++q) {
    u[(size_t)j * RANK + q] = make_float2(o[2 + q], o[2 + RANK + q]);
    v[(size_t)j * RANK + q] = make_float2(o[2 + 2 * RANK + q], o[2 + 3 * RANK + q]);
  }
}

// block partials over rows of (sum_j conj(V_jq) r_tj  [q < 8],  sum_j |e_tj|^2): part[blk][t][9]
__global__ void __launch_bounds__(256) pc_red_c(const float2* __restrict__ v, const double2* __restrict__ r,
                                                const double2* __restrict__ e, int N, double2* __restrict__ part) {
  const int t = blockIdx.y;
  double cr[RANK + 1], ci[RANK + 1];
#pragma unroll
  for (int q = 0; q <= RANK; ++q) cr[q] = ci[q] = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    const double2 rr = r[(size_t)t * N + j], ee = e[(size_t)t * N + j];
#pragma unroll
    for (int q = 0; q < RANK; ++q) {
      const float2 vv = v[(size_t)j * RANK + q];
      cr[q] += vv.x * rr.x + vv.y * rr.y;
      ci[q] += vv.x * rr.y - vv.y * rr.x;
    }
    cr[RANK] += ee.x * ee.x + ee.y * ee.y;
  }
  __shared__ double sr[8][RANK + 1], si[8][RANK + 1];
#pragma unroll
  for (int q = 0; q <= RANK; ++q) {
    for (int off = 16; off > 0; off >>= 1) {
      cr[q] += __shfl_xor_sync(0xffffffffu, cr[q], off);
      ci[q] += __shfl_xor_sync(0xffffffffu, ci[q], off);
    }
    if ((threadIdx.x & 31) == 0) {
      sr[threadIdx.x >> 5][q] = cr[q];
      si[threadIdx.x >> 5][q] = ci[q];
    }
  }
  __syncthreads();
  if (threadIdx.x <= RANK) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += sr[w][threadIdx.x];
      b += si[w][threadIdx.x];
    }
    part[((size_t)blockIdx.x * gridDim.y + t) * (RANK + 1) + threadIdx.x] = make_double2(a, b);
  }
}

// out[t][q] = sum_blk part[blk][t][q]
__global__ void pc_red_finish(const double2* __restrict__ part, int nblk, int T, double2* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= T * (RANK + 1)) return;
  double a = 0, b = 0;
  for (int blk = 0; blk < nblk; ++blk) {
    const double2 v = part[(size_t)blk * T * (RANK + 1) + e];
    a += v.x;
    b += v.y;
  }
  out[e] = make_double2(a, b);
}

// partials of (lambda_tq = sum_j conj(U_jq) g_tj,  sum_j |q_tj|^2)
__global__ void __launch_bounds__(256) pc_red_spai(const float2* __restrict__ u, const double2* __restrict__ G,
                                                   const double2* __restrict__ Q, int N, double2* __restrict__ part) {
  const int t = blockIdx.y;
  double lr[RANK + 1], li[RANK + 1];
#pragma unroll
  for (int q = 0; q <= RANK; ++q) lr[q] = li[q] = 0.0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    const double2 gg = G[(size_t)t * N + j], qq = Q[(size_t)t * N + j];
#pragma unroll
    for (int q = 0; q < RANK; ++q) {
      const float2 uu = u[(size_t)j * RANK + q];
      lr[q] += uu.x * gg.x + uu.y * gg.y;   // conj(u) g
      li[q] += uu.x * gg.y - uu.y * gg.x;
    }
    lr[RANK] += qq.x * qq.x + qq.y * qq.y;
  }
  __shared__ double sr[8][RANK + 1], si[8][RANK + 1];
#pragma unroll
  for (int q = 0; q <= RANK; ++q) {
    for (int off = 16; off > 0; off >>= 1) {
      lr[q] += __shfl_xor_sync(0xffffffffu, lr[q], off);
      li[q] += __shfl_xor_sync(0xffffffffu, li[q], off);
    }
    if ((threadIdx.x & 31) == 0) {
      sr[threadIdx.x >> 5][q] = lr[q];
      si[threadIdx.x >> 5][q] = li[q];
    }
  }
  __syncthreads();
  if (threadIdx.x <= RANK) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += sr[w][threadIdx.x];
      b += si[w][threadIdx.x];
    }
    part[((size_t)blockIdx.x * gridDim.y + t) * (RANK + 1) + threadIdx.x] = make_double2(a, b);
  }
}

// dO per row from T (vector r_t, adjoint g_t) pairs and their statistics (C:
// V^H r and |r|^2, L: U^H g): g_p = sum_t w_t g_t conj(r_t), g_U = sum_t w_t
// g_t c_t^H, g_V = sum_t w_t r_t lambda_t^H / N.  Weights: wts[t] when given,
// else w_t = 2/|r_t|^2 (0 for |r_t|^2 <= r2_min).
__global__ void pc_dout(const float2* __restrict__ p, const float2* __restrict__ u, const double2* __restrict__ C,
                        const double2* __restrict__ L, const double2* __restrict__ r, const double2* __restrict__ G,
                        int T, int N, double r2_min, const double* __restrict__ wts, float* __restrict__ dO) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const float2 pp = p[j];
  float gpx = 0.f, gpy = 0.f;
  float gux[RANK] = {0}, guy[RANK] = {0}, gvx[RANK] = {0}, gvy[RANK] = {0};
  for (int t = 0; t < T; ++t) {
    float w;
    if (wts) {
      w = (float)wts[t];
      if (w == 0.f) continue;
    } else {
      const double r2 = C[t * (RANK + 1) + RANK].x;
      if (!(r2 > r2_min)) continue;   // residuals of an already converged solve carry no information
      w = (float)(2.0 / r2);
    }
    float2 c[RANK];
#pragma unroll
    for (int q = 0; q < RANK; ++q) {
      const double2 cc = C[t * (RANK + 1) + q];
      c[q] = make_float2((float)(cc.x / N), (float)(cc.y / N));
    }
    const double2 rr = r[(size_t)t * N + j], gg = G[(size_t)t * N + j];
    const float rx = (float)rr.x, ry = (float)rr.y;
    const float dx = (float)gg.x, dy = (float)gg.y;
    // g_p += w delta conj(r)
    gpx += w * (dx * rx + dy * ry);
    gpy += w * (dy * rx - dx * ry);
#pragma unroll
    for (int q = 0; q < RANK; ++q) {
      // g_u += w delta conj(c)
      gux[q] += w * (dx * c[q].x + dy * c[q].y);
      guy[q] += w * (dy * c[q].x - dx * c[q].y);
      // g_v += w r conj(lambda) / N
      const double2 ll = L[t * (RANK + 1) + q];
      const float lx = (float)ll.x, ly = (float)ll.y;
      gvx[q] += w * (rx * lx + ry * ly) / N;
      gvy[q] += w * (ry * lx - rx * ly) / N;
    }
  }
  // gs = conj(g_p) p^2
  const float p2x = pp.x * pp.x - pp.y * pp.y, p2y = 2.f * pp.x * pp.y;
  const float gsx = gpx * p2x + gpy * p2y, gsy = gpx * p2y - gpy * p2x;
  float* d = dO + (size_t)j * F_OUT;
  d[0] = SHIFT * gsx;
  d[1] = -SHIFT * gsy;
#pragma unroll
  for (int q = 0; q < RANK; ++q) {
    d[2 + q] = gux[q];
    d[2 + RANK + q] = guy[q];
    d[2 + 2 * RANK + q] = gvx[q];
    d[2 + 3 * RANK + q] = gvy[q];
  }
}

__global__ void mlp_adam_k(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                           float* __restrict__ g, __half* __restrict__ w16, int n, float lr, float scale, float bc1,
                           float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gg = g[i] * scale;
  const float mm = 0.9f * m[i] + 0.1f * gg;
  const float vv = 0.999f * v[i] + 0.001f * gg * gg;
  m[i] = mm;
  v[i] = vv;
  const float nw = w[i] - lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
  w[i] = nw;
  w16[i] = __float2half_rn(nw);
  g[i] = 0.f;
}

__global__ void to_half(const float* __restrict__ w, __half* __restrict__ w16, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) w16[i] = __float2half_rn(w[i]);
}

// ---- GMRES application of P = diag(p) + U V^H / N to packed vectors ----
// part[s][blk][q] = sum_j conj(V_s,jq) x_s,j   (system of slot s = idx[s])
__global__ void __launch_bounds__(256) pc_apply_red(const double2* __restrict__ x, long long xstride,
                                                    const float2* __restrict__ V, long long fstride, long long N,
                                                    const int* __restrict__ idx, double2* __restrict__ part) {
  const int s = blockIdx.y, sys = idx ? idx[s] : s;
  const double2* xs = x + (size_t)(idx ? sys : s) * xstride;
  const float2* vs = V + (size_t)sys * fstride * N * RANK;
  // FP32 products and per-thread sums (V is FP32; FP64 here would make this
  // pass FP64-bound), FP64 across the block and the grid
  float fr[RANK], fi[RANK];
#pragma unroll
  for (int q = 0; q < RANK; ++q) fr[q] = fi[q] = 0.f;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
    const double2 xd = xs[j];
    const float2 xx = make_float2((float)xd.x, (float)xd.y);
#pragma unroll
    for (int q = 0; q < RANK; ++q) {
      const float2 vv = vs[j * RANK + q];
      fr[q] += vv.x * xx.x + vv.y * xx.y;
      fi[q] += vv.x * xx.y - vv.y * xx.x;
    }
  }
  double cr[RANK], ci[RANK];
#pragma unroll
  for (int q = 0; q < RANK; ++q) {
    cr[q] = fr[q];
    ci[q] = fi[q];
  }
  __shared__ double sr[8][RANK], si[8][RANK];
#pragma unroll
  for (int q = 0; q < RANK; ++q) {
    for (int off = 16; off > 0; off >>= 1) {
      cr[q] += __shfl_xor_sync(0xffffffffu, cr[q], off);
      ci[q] += __shfl_xor_sync(0xffffffffu, ci[q], off);
    }
    if ((threadIdx.x & 31) == 0) {
      sr[threadIdx.x >> 5][q] = cr[q];
      si[threadIdx.x >> 5][q] = ci[q];
    }
  }
  __syncthreads();
  if (threadIdx.x < RANK) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += sr[w][threadIdx.x];
      b += si[w][threadIdx.x];
    }
    part[((size_t)s * gridDim.x + blockIdx.x) * RANK + threadIdx.x] = make_double2(a, b);
  }
}

// y_s = p (.) x_s + U c_s / N with c_s = sum_blk part[s][blk]; add != 0: y += (...)
__global__ void pc_apply(const double2* __restrict__ x, long long xstride, long long fstride,
                         const float2* __restrict__ pv,
                         const float2* __restrict__ U, const double2* __restrict__ part, int nblk, long long N,
                         const int* __restrict__ idx, double2* __restrict__ y, long long ystride, int add) {
  const int s = blockIdx.y, sys = idx ? idx[s] : s;
  __shared__ float2 c[RANK];
  if (threadIdx.x < RANK) {
    double a = 0, b = 0;
    for (int blk = 0; blk < nblk; ++blk) {
      const double2 v = part[((size_t)s * nblk + blk) * RANK + threadIdx.x];
      a += v.x;
      b += v.y;
    }
    c[threadIdx.x] = make_float2((float)(a / N), (float)(b / N));
  }
  __syncthreads();
  const double2* xs = x + (size_t)(idx ? sys : s) * xstride;
  double2* ys = y + (size_t)s * ystride;
  const float2* ps = pv + (size_t)sys * fstride * N;
  const float2* us = U + (size_t)sys * fstride * N * RANK;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
    const double2 xx = xs[j];
    const float2 pp = ps[j];
    double rx = pp.x * xx.x - pp.y * xx.y, ry = pp.x * xx.y + pp.y * xx.x;
    float lx = 0.f, ly = 0.f;
#pragma unroll
    for (int q = 0; q < RANK; ++q) {
      const float2 uu = us[j * RANK + q];
      lx += uu.x * c[q].x - uu.y * c[q].y;
      ly += uu.x * c[q].y + uu.y * c[q].x;
    }
    rx += lx;
    ry += ly;
    if (add) {
      const double2 o = ys[j];
      ys[j] = make_double2(o.x + rx, o.y + ry);
    } else {
      ys[j] = make_double2(rx, ry);
    }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
struct bse_mlp {
  float* w = nullptr;     // FP32 master [NPARAM]
  __half* w16 = nullptr;  // FP16 weights used by every kernel
  float* m = nullptr;
  float* v = nullptr;
  float* g = nullptr;     // accumulated gradient
  long long t = 0;        // Adam steps taken
  size_t rows_cap = 0;
  float* act = nullptr;   // X, Z1, H1, Z2, H2, O, dO, dA, dB for rows_cap rows
  float* wpart = nullptr; // WG_BLOCKS * 129 * 128
  double2* red = nullptr; // reduction scratch
  double2* stats = nullptr;
  size_t red_cap = 0, stats_cap = 0;   // entries
  double2* probe = nullptr;   // P r, (H - z) P r - r, (H - conj z)(...) for the probes
  size_t probe_cap = 0;
};

bse_status bse_mlp_apply(bse_handle* h, const float2* p, const float2* u, const float2* v, const double2* x,
                         long long xstride, int ns, const int* idx, double2* y, long long ystride, int add,
                         double2* part, long long fstride);

namespace {

template <typename T>
bool dmalloc(T** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

void mlp_free(bse_mlp* m) {
  if (!m) return;
  void* ptrs[] = {m->w, m->w16, m->m, m->v, m->g, m->act, m->wpart, m->red, m->stats, m->probe};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete m;
}

struct Act {
  float *X, *Z1, *H1, *Z2, *H2, *O, *dO, *dA, *dB;
};

bse_status ensure_rows(bse_handle* h, bse_mlp* m, size_t rows, Act* a) {
  const size_t per = F_IN + 4 * WID + F_OUT + F_OUT + 2 * WID;
  if (m->rows_cap < rows) {
    if (m->act) cudaFree(m->act);
    m->act = nullptr;
    m->rows_cap = 0;
    if (!dmalloc(&m->act, rows * per * sizeof(float))) return bse_fail(h, BSE_ERR_OOM, "mlp activations");
    m->rows_cap = rows;
  }
  float* p = m->act;
  a->X = p;
  p += rows * F_IN;
  a->Z1 = p;
  p += rows * WID;
  a->H1 = p;
  p += rows * WID;
  a->Z2 = p;
  p += rows * WID;
  a->H2 = p;
  p += rows * WID;
  a->O = p;
  p += rows * F_OUT;
  a->dO = p;
  p += rows * F_OUT;
  a->dA = p;
  p += rows * WID;
  a->dB = p;
  return BSE_OK;
}

size_t dense_smem(int in, int out) { return (size_t)(RB * in + in * ((out + 3) & ~3)) * sizeof(float); }

bse_status ensure_anorm(bse_handle* h) {
  if (h->mlp_anorm || h->np == 0) return BSE_OK;
  const int nkb = h->nk * h->nb;
  if (!dmalloc(&h->mlp_anorm, (size_t)nkb * sizeof(float))) return bse_fail(h, BSE_ERR_OOM, "a_norm");
  BSE_PROF(h, BSE_K_PREP, mlp_anorm<<<(nkb + 255) / 256, 256, 0, h->stream>>>(h->a_proj, h->np, nkb, h->mlp_anorm));
  return BSE_OK;
}

// features + 3 dense layers for shift z over every row of the handle's system
bse_status forward(bse_handle* h, bse_mlp* m, double omega, double gamma, Act* a) {
  const int N = (int)h->N;
  if (ensure_rows(h, m, (size_t)N, a) != BSE_OK) return BSE_ERR_OOM;
  if (ensure_anorm(h) != BSE_OK) return BSE_ERR_OOM;
  cudaStream_t st = h->stream;
  BSE_PROF(h, BSE_K_PREP,
           mlp_features<<<(N + 255) / 256, 256, 0, st>>>(h->jdiag, h->e_nk, h->chi, h->mlp_anorm, h->na,
                                                         h->nk * h->nb, omega, gamma, a->X));
  const int g = (N + RB - 1) / RB;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem(WID, WID));
    cudaFuncSetAttribute(mlp_dense_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem(WID, WID));
    attr = true;
  }
  BSE_PROF(h, BSE_K_PREP,
           mlp_dense<<<g, 256, dense_smem(F_IN, WID), st>>>(a->X, F_IN, m->w16 + OFF_W1, m->w16 + OFF_B1, WID, a->Z1,
                                                            a->H1, N));
  BSE_PROF(h, BSE_K_PREP,
           mlp_dense<<<g, 256, dense_smem(WID, WID), st>>>(a->H1, WID, m->w16 + OFF_W2, m->w16 + OFF_B2, WID, a->Z2,
                                                           a->H2, N));
  BSE_PROF(h, BSE_K_PREP,
           mlp_dense<<<g, 256, dense_smem(WID, F_OUT), st>>>(a->H2, WID, m->w16 + OFF_W3, m->w16 + OFF_B3, F_OUT,
                                                             a->O, nullptr, N));
  return bse_cuda_check(h, cudaGetLastError(), "mlp forward");
}

// q = HY - z Y - R, or q = HY - z Y when R is null  (HY is in Q on entry)
__global__ void spai_q(double2* __restrict__ Q, const double2* __restrict__ Y, const double2* __restrict__ R,
                       double zr, double zi, size_t n) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    const double2 hy = Q[j], y = Y[j];
    const double2 r = R ? R[j] : make_double2(0.0, 0.0);
    Q[j] = make_double2(hy.x - (zr * y.x - zi * y.y) - r.x, hy.y - (zr * y.y + zi * y.x) - r.y);
  }
}

// g = HQ - conj(z) q  (HQ is in G on entry)
__global__ void spai_g(double2* __restrict__ G, const double2* __restrict__ Q, double zr, double zi, size_t n) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    const double2 hq = G[j], q = Q[j];
    G[j] = make_double2(hq.x - (zr * q.x + zi * q.y), hq.y - (zr * q.y - zi * q.x));
  }
}

// ---- k-step minimal-residual loss ----
constexpr int KMAX = 16;   // largest number of Krylov steps of the loss

// partials of <Y_i, Y_j> (i = 0..j) per probe t for one j: part[blk][t][i][j], Y [(k+1)][T][N]
template <int NI>
__global__ void __launch_bounds__(256) ks_dots(const double2* __restrict__ Y, int T, int N, int j, int k,
                                               double2* __restrict__ part) {
  const int t = blockIdx.y;
  double ar[NI], ai[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) ar[i] = ai[i] = 0.0;
  const size_t tn = (size_t)T * N;
  const double2* yj = Y + (size_t)j * tn + (size_t)t * N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    const double2 b = yj[e];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      if (i <= j) {
        const double2 a = Y[(size_t)i * tn + (size_t)t * N + e];
        ar[i] += a.x * b.x + a.y * b.y;   // conj(a) b
        ai[i] += a.x * b.y - a.y * b.x;
      }
    }
  }
  __shared__ double sr[8][NI], si[8][NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    for (int off = 16; off > 0; off >>= 1) {
      ar[i] += __shfl_xor_sync(0xffffffffu, ar[i], off);
      ai[i] += __shfl_xor_sync(0xffffffffu, ai[i], off);
    }
    if ((threadIdx.x & 31) == 0) {
      sr[threadIdx.x >> 5][i] = ar[i];
      si[threadIdx.x >> 5][i] = ai[i];
    }
  }
  __syncthreads();
  if (threadIdx.x <= j && threadIdx.x < NI) {
    double a = 0, b = 0;
    for (int w = 0; w < 8; ++w) {
      a += sr[w][threadIdx.x];
      b += si[w][threadIdx.x];
    }
    part[(((size_t)blockIdx.x * T + t) * (k + 1) + threadIdx.x) * (k + 1) + j] = make_double2(a, b);
  }
}

// gram[t][i][j] = sum_blk part[blk][t][i][j] for i <= j (fixed order)
__global__ void ks_dots_finish(const double2* __restrict__ part, int nblk, int T, int k, double2* __restrict__ gram) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int per = (k + 1) * (k + 1);
  if (e >= T * per) return;
  const int i = (e % per) / (k + 1), j = e % (k + 1);
  if (i > j) return;
  double a = 0, b = 0;
  for (int blk = 0; blk < nblk; ++blk) {
    const double2 v = part[(size_t)blk * T * per + e];
    a += v.x;
    b += v.y;
  }
  gram[e] = make_double2(a, b);
}

// out_t = (x0 ? x0_t : 0) + sum_{i < n} coef[t][i] X_i,t   (X_i,t = X + i*xs + t*N; coef [T][KMAX])
__global__ void ks_lincomb(double2* __restrict__ out, const double2* __restrict__ x0, const double2* __restrict__ X,
                           size_t xs, int n, const double2* __restrict__ coef, int T, int N) {
  const int t = blockIdx.y;
  __shared__ double2 cf[KMAX];
  if (threadIdx.x < KMAX) cf[threadIdx.x] = coef[t * KMAX + threadIdx.x];
  __syncthreads();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N; e += gridDim.x * blockDim.x) {
    double2 acc = x0 ? x0[(size_t)t * N + e] : make_double2(0.0, 0.0);
    for (int i = 0; i < n; ++i) {
      const double2 c = cf[i], v = X[(size_t)i * xs + (size_t)t * N + e];
      acc.x += c.x * v.x - c.y * v.y;
      acc.y += c.x * v.y + c.y * v.x;
    }
    out[(size_t)t * N + e] = acc;
  }
}

// Y = HT - z T (HT in Y on entry); conj != 0: Y = HT - conj(z) T
__global__ void ks_shift(double2* __restrict__ Y, const double2* __restrict__ Tv, double zr, double zi, size_t n) {
  for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n; j += (size_t)gridDim.x * blockDim.x) {
    const double2 hy = Y[j], y = Tv[j];
    Y[j] = make_double2(hy.x - (zr * y.x - zi * y.y), hy.y - (zr * y.y + zi * y.x));
  }
}

__global__ void conj_f2(const float2* __restrict__ a, float2* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2(a[i].x, -a[i].y);
}

bse_status apply_h_chunks(bse_handle* h, const double2* in, double2* out, int n) {
  for (int v0 = 0; v0 < n; v0 += h->max_vec) {
    const int nv = std::min(h->max_vec, n - v0);
    const bse_status s = bse_apply_device(h, in + (size_t)v0 * h->N, out + (size_t)v0 * h->N, nv);
    if (s != BSE_OK) return s;
  }
  return BSE_OK;
}

// backward through the three layers from dO (per-row output gradients), into m->g
bse_status backward(bse_handle* h, bse_mlp* m, const Act& a) {
  cudaStream_t st = h->stream;
  const int N = (int)h->N;
  const int g = (N + RB - 1) / RB;
  BSE_PROF(h, BSE_K_PREP, mlp_wgrad<<<WG_BLOCKS, 256, 0, st>>>(a.H2, WID, a.dO, F_OUT, N, m->wpart));
  BSE_PROF(h, BSE_K_PREP,
           mlp_wgrad_reduce<<<((WID + 1) * F_OUT + 255) / 256, 256, 0, st>>>(m->wpart, WG_BLOCKS, WID, F_OUT, m->g,
                                                                              OFF_W3, OFF_B3));
  BSE_PROF(h, BSE_K_PREP,
           mlp_dense_bwd<<<g, 256, dense_smem(F_OUT, WID), st>>>(a.dO, F_OUT, m->w16 + OFF_W3, WID, a.Z2, a.dA, N));
  BSE_PROF(h, BSE_K_PREP, mlp_wgrad<<<WG_BLOCKS, 256, 0, st>>>(a.H1, WID, a.dA, WID, N, m->wpart));
  BSE_PROF(h, BSE_K_PREP,
           mlp_wgrad_reduce<<<((WID + 1) * WID + 255) / 256, 256, 0, st>>>(m->wpart, WG_BLOCKS, WID, WID, m->g,
                                                                            OFF_W2, OFF_B2));
  BSE_PROF(h, BSE_K_PREP,
           mlp_dense_bwd<<<g, 256, dense_smem(WID, WID), st>>>(a.dA, WID, m->w16 + OFF_W2, WID, a.Z1, a.dB, N));
  BSE_PROF(h, BSE_K_PREP, mlp_wgrad<<<WG_BLOCKS, 256, 0, st>>>(a.X, F_IN, a.dB, WID, N, m->wpart));
  BSE_PROF(h, BSE_K_PREP,
           mlp_wgrad_reduce<<<((F_IN + 1) * WID + 255) / 256, 256, 0, st>>>(m->wpart, WG_BLOCKS, F_IN, WID, m->g,
                                                                             OFF_W1, OFF_B1));
  return bse_cuda_check(h, cudaGetLastError(), "mlp backward");
}

bse_status ensure_probe(bse_handle* h, bse_mlp* m, size_t n) {
  if (m->probe_cap >= n) return BSE_OK;
  if (m->probe) cudaFree(m->probe);
  m->probe = nullptr;
  m->probe_cap = 0;
  if (!dmalloc(&m->probe, n * sizeof(double2))) return bse_fail(h, BSE_ERR_OOM, "probe buffers");
  m->probe_cap = n;
  return BSE_OK;
}

bool grow(double2** buf, size_t* cap, size_t n) {
  if (*cap >= n) return true;
  double2* b = nullptr;
  if (!dmalloc(&b, n * sizeof(double2))) return false;
  cudaFree(*buf);
  *buf = b;
  *cap = n;
  return true;
}

// Plain approximate-inverse loss sum_t |(H - z) P r_t - r_t|^2 / |r_t|^2 over
// the T probes r [T][N] (device); gradient accumulated into m->g.
bse_status loss_grad_spai(bse_handle* h, bse_mlp* m, double omega, double gamma, int T, const double2* r, float2* p,
                          float2* u, float2* v, double* loss_out, double r2_min) {
  Act a;
  bse_status s = forward(h, m, omega, gamma, &a);
  if (s != BSE_OK) return s;
  const int N = (int)h->N;
  cudaStream_t st = h->stream;
  const size_t tn = (size_t)T * N;
  if ((s = ensure_probe(h, m, 3 * tn)) != BSE_OK) return s;
  double2 *Y = m->probe, *Q = Y + tn, *G = Q + tn;
  BSE_PROF(h, BSE_K_PREP, pc_assemble<<<(N + 255) / 256, 256, 0, st>>>(a.O, h->jdiag, omega, gamma, N, p, u, v));
  double2* part = m->red;
  // Y = P r, Q = (H - z) Y - r, G = (H - conj z) Q: two applications of H per probe
  s = bse_mlp_apply(h, p, u, v, r, N, T, nullptr, Y, N, 0, part, 0);
  if (s == BSE_OK) s = apply_h_chunks(h, Y, Q, T);
  if (s != BSE_OK) return s;
  const int ge = (int)std::min<size_t>((tn + 255) / 256, 4096);
  BSE_PROF(h, BSE_K_PREP, spai_q<<<ge, 256, 0, st>>>(Q, Y, r, omega, gamma, tn));
  s = apply_h_chunks(h, Q, G, T);
  if (s != BSE_OK) return s;
  BSE_PROF(h, BSE_K_PREP, spai_g<<<ge, 256, 0, st>>>(G, Q, omega, gamma, tn));
  double2* C = m->stats;
  double2* L = m->stats + T * (RANK + 1);
  BSE_PROF(h, BSE_K_PREP, pc_red_c<<<dim3(NRED, T), 256, 0, st>>>(v, r, r, N, part));
  BSE_PROF(h, BSE_K_PREP, pc_red_finish<<<1, 256, 0, st>>>(part, NRED, T, C));
  BSE_PROF(h, BSE_K_PREP, pc_red_spai<<<dim3(NRED, T), 256, 0, st>>>(u, G, Q, N, part));
  BSE_PROF(h, BSE_K_PREP, pc_red_finish<<<1, 256, 0, st>>>(part, NRED, T, L));
  BSE_PROF(h, BSE_K_PREP,
           pc_dout<<<(N + 255) / 256, 256, 0, st>>>(p, u, C, L, r, G, T, N, r2_min, nullptr, a.dO));
  if ((s = backward(h, m, a)) != BSE_OK) return s;
  if (loss_out) {
    std::vector<double2> hs(2 * T * (RANK + 1));
    bse_status cs = bse_cuda_check(
        h, cudaMemcpyAsync(hs.data(), m->stats, hs.size() * sizeof(double2), cudaMemcpyDeviceToHost, st), "loss");
    if (cs != BSE_OK) return cs;
    cs = bse_cuda_check(h, cudaStreamSynchronize(st), "loss sync");
    if (cs != BSE_OK) return cs;
    double tot = 0;
    for (int t = 0; t < T; ++t) {
      const double e2 = hs[t * (RANK + 1) + RANK].x;
      if (e2 > r2_min) tot += hs[T * (RANK + 1) + t * (RANK + 1) + RANK].x / e2;
    }
    *loss_out = tot;
  }
  return bse_cuda_check(h, cudaGetLastError(), "mlp loss/grad");
}

// Solve the k x k Hermitian system G c = hv (row-major G, FP64) by Cholesky on
// the diagonally scaled matrix; a vanishing pivot adds a small ridge and retries.
bool solve_gram(std::vector<double2> G, std::vector<double2> hv, int k, std::vector<double2>& c) {
  std::vector<double> sc(k);
  for (int i = 0; i < k; ++i) sc[i] = G[i * k + i].x > 0 ? 1.0 / sqrt(G[i * k + i].x) : 1.0;
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      G[i * k + j].x *= sc[i] * sc[j];
      G[i * k + j].y *= sc[i] * sc[j];
    }
  for (int attempt = 0; attempt < 4; ++attempt) {
    const double ridge = attempt ? pow(10.0, -14 + 3 * attempt) : 0.0;
    std::vector<double2> Lm(G);
    for (int i = 0; i < k; ++i) Lm[i * k + i].x += ridge;
    bool ok = true;
    for (int j = 0; j < k && ok; ++j) {   // L L^H, lower triangle
      double d = Lm[j * k + j].x;
      for (int q = 0; q < j; ++q) d -= Lm[j * k + q].x * Lm[j * k + q].x + Lm[j * k + q].y * Lm[j * k + q].y;
      if (!(d > 1e-300)) {
        ok = false;
        break;
      }
      const double ljj = sqrt(d);
      Lm[j * k + j] = make_double2(ljj, 0.0);
      for (int i = j + 1; i < k; ++i) {
        double2 s = Lm[i * k + j];   // G_ij (scaled); G Hermitian: use the lower entry G[i][j]
        for (int q = 0; q < j; ++q) {
          const double2 a = Lm[i * k + q], b = Lm[j * k + q];   // s -= a conj(b)
          s.x -= a.x * b.x + a.y * b.y;
          s.y -= a.y * b.x - a.x * b.y;
        }
        Lm[i * k + j] = make_double2(s.x / ljj, s.y / ljj);
      }
    }
    if (!ok) continue;
    std::vector<double2> y(k);
    for (int i = 0; i < k; ++i) {   // L y = sc * hv
      double2 s = make_double2(hv[i].x * sc[i], hv[i].y * sc[i]);
      for (int q = 0; q < i; ++q) {
        const double2 a = Lm[i * k + q], b = y[q];
        s.x -= a.x * b.x - a.y * b.y;
        s.y -= a.x * b.y + a.y * b.x;
      }
      y[i] = make_double2(s.x / Lm[i * k + i].x, s.y / Lm[i * k + i].x);
    }
    c.assign(k, make_double2(0.0, 0.0));
    for (int i = k - 1; i >= 0; --i) {   // L^H x = y
      double2 s = y[i];
      for (int q = i + 1; q < k; ++q) {
        const double2 a = Lm[q * k + i], b = c[q];   // conj(L[q][i]) x_q
        s.x -= a.x * b.x + a.y * b.y;
        s.y -= a.x * b.y - a.y * b.x;
      }
      c[i] = make_double2(s.x / Lm[i * k + i].x, s.y / Lm[i * k + i].x);
    }
    for (int i = 0; i < k; ++i) c[i] = make_double2(c[i].x * sc[i], c[i].y * sc[i]);
    return true;
  }
  return false;
}

// k-step minimal-residual loss sum_t min_{deg q <= k, q(0)=1} |q((H - z)P) r_t|^2/|r_t|^2
// over the T probes r [T][N] (device) and its gradient into m->g.
//   forward chain  Y_0 = r, Y_i = (H - z) P Y_{i-1} (k applications of H);
//   least squares  c = argmin |r - sum_i c_i Y_i| from the FP64 Gram matrix;
//   adjoint chain  s_0 = r - sum c_i Y_i, Q_m = (H - conj z) s_m, s_{m+1} = P^H Q_m;
//   pairs          (Y_j, G_j), G_j = -sum_m conj(c_{m+j+1}) Q_m, weight 2/|r_t|^2.
bse_status loss_grad_krylov(bse_handle* h, bse_mlp* m, double omega, double gamma, int T, const double2* r,
                            float2* p, float2* u, float2* v, double* loss_out, double r2_min, int k) {
  Act a;
  bse_status s = forward(h, m, omega, gamma, &a);
  if (s != BSE_OK) return s;
  const int N = (int)h->N;
  cudaStream_t st = h->stream;
  const size_t tn = (size_t)T * N;
  // Y [k+1][T][N], Q [k][T][N], GJ [k][T][N], Tt [T][N]
  if ((s = ensure_probe(h, m, (size_t)(3 * k + 2) * tn)) != BSE_OK) return s;
  double2* Y = m->probe;
  double2* Q = Y + (size_t)(k + 1) * tn;
  double2* GJ = Q + (size_t)k * tn;
  double2* Tt = GJ + (size_t)k * tn;
  const int per = (k + 1) * (k + 1);
  const int TT = k * T;
  cudaStreamSynchronize(st);   // the scratch below may be reallocated
  if (!grow(&m->red, &m->red_cap, std::max((size_t)NRED * T * per, (size_t)NRED * TT * (RANK + 1))) ||
      !grow(&m->stats, &m->stats_cap, (size_t)T * per + (size_t)T * KMAX + TT + 2 * (size_t)TT * (RANK + 1)))
    return bse_fail(h, BSE_ERR_OOM, "k-step loss scratch");
  double2* part = m->red;
  float2* pc = (float2*)a.dA;   // conj(p): the first N float2 of a scratch activation, free until backward
  BSE_PROF(h, BSE_K_PREP, pc_assemble<<<(N + 255) / 256, 256, 0, st>>>(a.O, h->jdiag, omega, gamma, N, p, u, v));
  BSE_PROF(h, BSE_K_PREP, conj_f2<<<(N + 255) / 256, 256, 0, st>>>(p, pc, N));
  const int ge = (int)std::min<size_t>((tn + 255) / 256, 4096);
  cudaMemcpyAsync(Y, r, tn * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  for (int i = 1; i <= k; ++i) {
    s = bse_mlp_apply(h, p, u, v, Y + (size_t)(i - 1) * tn, N, T, nullptr, Tt, N, 0, part, 0);
    if (s == BSE_OK) s = apply_h_chunks(h, Tt, Y + (size_t)i * tn, T);
    if (s != BSE_OK) return s;
    BSE_PROF(h, BSE_K_PREP, ks_shift<<<ge, 256, 0, st>>>(Y + (size_t)i * tn, Tt, omega, gamma, tn));
  }
  // Gram matrix <Y_i, Y_j>, 0 <= i <= j <= k
  for (int j = 0; j <= k; ++j)
    BSE_PROF(h, BSE_K_PREP, ks_dots<KMAX + 1><<<dim3(NRED, T), 256, 0, st>>>(Y, T, N, j, k, part));
  double2* gram = m->stats;   // [T][k+1][k+1]
  BSE_PROF(h, BSE_K_PREP, ks_dots_finish<<<(T * per + 255) / 256, 256, 0, st>>>(part, NRED, T, k, gram));
  std::vector<double2> hg((size_t)T * per);
  s = bse_cuda_check(h, cudaMemcpyAsync(hg.data(), gram, hg.size() * sizeof(double2), cudaMemcpyDeviceToHost, st),
                     "gram");
  if (s == BSE_OK) s = bse_cuda_check(h, cudaStreamSynchronize(st), "gram sync");
  if (s != BSE_OK) return s;
  // host: least-squares coefficients, loss, pair weights and adjoint coefficients
  std::vector<double2> cres((size_t)T * KMAX, make_double2(0.0, 0.0));
  std::vector<double> wts((size_t)k * T, 0.0);
  std::vector<std::vector<double2>> cs(T);
  double tot = 0.0;
  for (int t = 0; t < T; ++t) {
    const double2* gt = hg.data() + (size_t)t * per;
    auto at = [&](int i, int j) {   // <Y_i, Y_j> for any i, j (Hermitian completion)
      if (i <= j) return gt[i * (k + 1) + j];
      const double2 q = gt[j * (k + 1) + i];
      return make_double2(q.x, -q.y);
    };
    const double r2 = at(0, 0).x;
    cs[t].assign(k, make_double2(0.0, 0.0));
    if (!(r2 > r2_min)) continue;   // probe of an already converged solve
    std::vector<double2> G((size_t)k * k), hv(k);
    for (int i = 0; i < k; ++i) {
      for (int j = 0; j < k; ++j) G[i * k + j] = at(i + 1, j + 1);
      hv[i] = at(i + 1, 0);   // <Y_i, r>
    }
    if (!solve_gram(G, hv, k, cs[t])) continue;
    // |res|^2 = |r|^2 - Re(c^H h) at the least-squares optimum
    double ch = 0.0;
    for (int i = 0; i < k; ++i) ch += cs[t][i].x * hv[i].x + cs[t][i].y * hv[i].y;
    tot += std::max(0.0, r2 - ch) / r2;
    for (int j = 0; j < k; ++j) wts[(size_t)j * T + t] = 2.0 / r2;
    for (int i = 0; i < k; ++i) cres[(size_t)t * KMAX + i] = make_double2(-cs[t][i].x, -cs[t][i].y);
  }
  if (loss_out) *loss_out = tot;
  double2* dcoef = m->stats + (size_t)T * per;   // [T][KMAX] coefficient staging
  double* dwts = (double*)(dcoef + (size_t)T * KMAX);
  s = bse_cuda_check(h, cudaMemcpyAsync(dcoef, cres.data(), cres.size() * sizeof(double2), cudaMemcpyHostToDevice, st),
                     "coefficients");
  if (s != BSE_OK) return s;
  // residual s_0 = r - sum_i c_i Y_i (into Tt), adjoint chain into Q
  const dim3 gl((unsigned)std::min((N + 255) / 256, 512), (unsigned)T);
  BSE_PROF(h, BSE_K_PREP, ks_lincomb<<<gl, 256, 0, st>>>(Tt, Y, Y + tn, tn, k, dcoef, T, N));
  for (int mm = 0; mm < k; ++mm) {
    s = apply_h_chunks(h, Tt, Q + (size_t)mm * tn, T);
    if (s != BSE_OK) return s;
    BSE_PROF(h, BSE_K_PREP, ks_shift<<<ge, 256, 0, st>>>(Q + (size_t)mm * tn, Tt, omega, -gamma, tn));
    if (mm + 1 < k) {   // s_{m+1} = P^H Q_m = conj(p) Q_m + V (U^H Q_m) / N
      s = bse_mlp_apply(h, pc, v, u, Q + (size_t)mm * tn, N, T, nullptr, Tt, N, 0, part, 0);
      if (s != BSE_OK) return s;
    }
  }
  // G_j = -sum_{m <= k-1-j} conj(c_{m+j+1}) Q_m
  for (int j = 0; j < k; ++j) {
    std::vector<double2> cj((size_t)T * KMAX, make_double2(0.0, 0.0));
    for (int t = 0; t < T; ++t)
      for (int mm = 0; mm + j < k; ++mm) {
        const double2 c = cs[t][mm + j];
        cj[(size_t)t * KMAX + mm] = make_double2(-c.x, c.y);
      }
    s = bse_cuda_check(h, cudaMemcpyAsync(dcoef, cj.data(), cj.size() * sizeof(double2), cudaMemcpyHostToDevice, st),
                       "adjoint coefficients");
    if (s != BSE_OK) return s;
    BSE_PROF(h, BSE_K_PREP,
             ks_lincomb<<<gl, 256, 0, st>>>(GJ + (size_t)j * tn, nullptr, Q, tn, k - j, dcoef, T, N));
    // the next iteration overwrites dcoef: wait for this combination
    s = bse_cuda_check(h, cudaStreamSynchronize(st), "adjoint sync");
    if (s != BSE_OK) return s;
  }
  // k*T pairs (Y_j, G_j) with their statistics, then dO and the backward pass
  s = bse_cuda_check(h, cudaMemcpyAsync(dwts, wts.data(), wts.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                     "pair weights");
  if (s != BSE_OK) return s;
  double2* C = m->stats + (size_t)T * per + (size_t)T * KMAX + TT;   // after the weights (TT doubles)
  double2* L = C + (size_t)TT * (RANK + 1);
  BSE_PROF(h, BSE_K_PREP, pc_red_c<<<dim3(NRED, TT), 256, 0, st>>>(v, Y, Y, N, part));
  BSE_PROF(h, BSE_K_PREP, pc_red_finish<<<(TT * (RANK + 1) + 255) / 256, 256, 0, st>>>(part, NRED, TT, C));
  BSE_PROF(h, BSE_K_PREP, pc_red_spai<<<dim3(NRED, TT), 256, 0, st>>>(u, GJ, GJ, N, part));
  BSE_PROF(h, BSE_K_PREP, pc_red_finish<<<(TT * (RANK + 1) + 255) / 256, 256, 0, st>>>(part, NRED, TT, L));
  BSE_PROF(h, BSE_K_PREP,
           pc_dout<<<(N + 255) / 256, 256, 0, st>>>(p, u, C, L, Y, GJ, TT, N, 0.0, dwts, a.dO));
  if ((s = backward(h, m, a)) != BSE_OK) return s;
  s = bse_cuda_check(h, cudaStreamSynchronize(st), "loss/grad sync");
  if (s != BSE_OK) return s;
  return bse_cuda_check(h, cudaGetLastError(), "mlp k-step loss/grad");
}

// krylov_steps = 0: plain approximate-inverse loss; >= 1: k-step minimal-residual loss
bse_status loss_grad(bse_handle* h, bse_mlp* m, double omega, double gamma, int T, const double2* r, float2* p,
                     float2* u, float2* v, double* loss_out, double r2_min, int krylov_steps) {
  if (krylov_steps <= 0) return loss_grad_spai(h, m, omega, gamma, T, r, p, u, v, loss_out, r2_min);
  return loss_grad_krylov(h, m, omega, gamma, T, r, p, u, v, loss_out, r2_min, krylov_steps);
}

}  // namespace

// preconditioner factors for n_z shifts (a14): p [n_z][N], U, V [n_z][N][8] (float2, device)
bse_status bse_mlp_factors(bse_handle* h, bse_mlp* m, const double2* z_host, int n_z, float2* p, float2* u,
                           float2* v) {
  const long long N = h->N;
  for (int i = 0; i < n_z; ++i) {
    Act a;
    bse_status s = forward(h, m, z_host[i].x, z_host[i].y, &a);
    if (s != BSE_OK) return s;
    BSE_PROF(h, BSE_K_PREP,
             pc_assemble<<<(int)((N + 255) / 256), 256, 0, h->stream>>>(a.O, h->jdiag, z_host[i].x, z_host[i].y,
                                                                         (int)N, p + (size_t)i * N,
                                                                         u + (size_t)i * N * RANK,
                                                                         v + (size_t)i * N * RANK));
  }
  return bse_cuda_check(h, cudaGetLastError(), "mlp factors");
}

// y[s] (=|+=) P_{idx[s]} x[s'] for ns packed systems (x rows indexed by idx when x_by_system)
bse_status bse_mlp_apply(bse_handle* h, const float2* p, const float2* u, const float2* v, const double2* x,
                         long long xstride, int ns, const int* idx, double2* y, long long ystride, int add,
                         double2* part, long long fstride) {
  if (ns <= 0) return BSE_OK;
  const long long N = h->N;
  BSE_PROF(h, BSE_K_RECURSION,
           pc_apply_red<<<dim3(NRED, ns), 256, 0, h->stream>>>(x, xstride, v, fstride, N, idx, part));
  BSE_PROF(h, BSE_K_RECURSION,
           pc_apply<<<dim3(NRED, ns), 256, 0, h->stream>>>(x, xstride, fstride, p, u, part, NRED, N, idx, y, ystride,
                                                           add));
  return bse_cuda_check(h, cudaGetLastError(), "mlp apply");
}

size_t bse_mlp_apply_scratch(int ns) { return (size_t)ns * NRED * RANK * sizeof(double2); }

extern "C" {

bse_status bse_mlp_create(bse_mlp** out, const float* params, long long n_params) {
  if (!out) return BSE_ERR_INVALID_ARG;
  *out = nullptr;
  if (!params || n_params != NPARAM) return BSE_ERR_INVALID_ARG;
  bse_mlp* m = new (std::nothrow) bse_mlp();
  if (!m) return BSE_ERR_OOM;
  const size_t nb = (size_t)NPARAM * sizeof(float);
  if (!dmalloc(&m->w, nb) || !dmalloc(&m->w16, (size_t)NPARAM * sizeof(__half)) || !dmalloc(&m->m, nb) ||
      !dmalloc(&m->v, nb) || !dmalloc(&m->g, nb) ||
      !dmalloc(&m->wpart, (size_t)WG_BLOCKS * (WID + 1) * WID * sizeof(float)) ||
      !dmalloc(&m->red, (size_t)NRED * 64 * (RANK + 1) * sizeof(double2)) ||
      !dmalloc(&m->stats, (size_t)3 * 64 * (RANK + 1) * sizeof(double2))) {
    mlp_free(m);
    return BSE_ERR_OOM;
  }
  m->red_cap = (size_t)NRED * 64 * (RANK + 1);
  m->stats_cap = (size_t)3 * 64 * (RANK + 1);
  if (cudaMemcpy(m->w, params, nb, cudaMemcpyDefault) != cudaSuccess) {
    cudaGetLastError();
    mlp_free(m);
    return BSE_ERR_CUDA;
  }
  cudaMemset(m->m, 0, nb);
  cudaMemset(m->v, 0, nb);
  cudaMemset(m->g, 0, nb);
  to_half<<<(NPARAM + 255) / 256, 256>>>(m->w, m->w16, NPARAM);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    mlp_free(m);
    return BSE_ERR_CUDA;
  }
  *out = m;
  return BSE_OK;
}

void bse_mlp_destroy(bse_mlp* m) {
  cudaDeviceSynchronize();
  mlp_free(m);
}

long long bse_mlp_n_params(void) { return NPARAM; }

bse_status bse_mlp_params(const bse_mlp* m, float* out) {
  if (!m || !out) return BSE_ERR_INVALID_ARG;
  return cudaMemcpy(out, m->w, (size_t)NPARAM * sizeof(float), cudaMemcpyDefault) == cudaSuccess ? BSE_OK
                                                                                                  : BSE_ERR_CUDA;
}

bse_status bse_mlp_outputs(bse_handle* h, bse_mlp* m, double omega, double gamma, float* out) {
  if (!h || !m || !out) return BSE_ERR_INVALID_ARG;
  if (h->na > BSE_MAX_ALPHA) return bse_fail(h, BSE_ERR_UNSUPPORTED, "mlp");
  Act a;
  bse_status s = forward(h, m, omega, gamma, &a);
  if (s != BSE_OK) return s;
  s = bse_cuda_check(h, cudaMemcpyAsync(out, a.O, (size_t)h->N * F_OUT * sizeof(float), cudaMemcpyDefault, h->stream),
                     "outputs copy");
  if (s != BSE_OK) return s;
  return bse_cuda_check(h, cudaStreamSynchronize(h->stream), "outputs sync");
}

bse_status bse_mlp_loss_grad(bse_handle* h, bse_mlp* m, double omega, double gamma, int n_probes, const bse_c128* r,
                             int krylov_steps, double* loss, float* grad) {
  if (!h || !m || !r || !loss || !grad || n_probes < 1 || n_probes > 64 || krylov_steps < 0 ||
      krylov_steps > KMAX || n_probes * std::max(krylov_steps, 1) > 64)
    return h ? bse_fail(h, BSE_ERR_INVALID_ARG, "mlp_loss_grad: bad arguments") : BSE_ERR_INVALID_ARG;
  if (!bse_is_device_ptr(r)) return bse_fail(h, BSE_ERR_INVALID_ARG, "mlp_loss_grad: r must be device memory");
  const int n_pairs = n_probes;
  const long long N = h->N;
  float2 *p = nullptr, *u = nullptr, *v = nullptr;
  if (!dmalloc(&p, (size_t)N * sizeof(float2)) || !dmalloc(&u, (size_t)N * RANK * sizeof(float2)) ||
      !dmalloc(&v, (size_t)N * RANK * sizeof(float2))) {
    cudaFree(p);
    cudaFree(u);
    return bse_fail(h, BSE_ERR_OOM, "mlp_loss_grad scratch");
  }
  cudaMemsetAsync(m->g, 0, (size_t)NPARAM * sizeof(float), h->stream);
  bse_status s = loss_grad(h, m, omega, gamma, n_pairs, (const double2*)r, p, u, v, loss, 0.0, krylov_steps);
  if (s == BSE_OK)
    s = bse_cuda_check(h, cudaMemcpyAsync(grad, m->g, (size_t)NPARAM * sizeof(float), cudaMemcpyDefault, h->stream),
                       "grad copy");
  if (s == BSE_OK) s = bse_cuda_check(h, cudaStreamSynchronize(h->stream), "grad sync");
  cudaMemsetAsync(m->g, 0, (size_t)NPARAM * sizeof(float), h->stream);
  cudaFree(p);
  cudaFree(u);
  cudaFree(v);
  return s;
}

bse_status bse_mlp_adam_step(bse_mlp* m, const float* grad, double lr) {
  if (!m || !grad) return BSE_ERR_INVALID_ARG;
  if (cudaMemcpy(m->g, grad, (size_t)NPARAM * sizeof(float), cudaMemcpyDefault) != cudaSuccess) return BSE_ERR_CUDA;
  m->t += 1;
  const float bc1 = 1.f - powf(0.9f, (float)m->t), bc2 = 1.f - powf(0.999f, (float)m->t);
  mlp_adam_k<<<(NPARAM + 255) / 256, 256>>>(m->w, m->m, m->v, m->g, m->w16, NPARAM, (float)lr, 1.f, bc1, bc2);
  return cudaDeviceSynchronize() == cudaSuccess ? BSE_OK : BSE_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// training: harvest GMRES histories on each system, then epochs of Adam
// ---------------------------------------------------------------------------
// r = b - (H x - z x)  for one system (hx = H x)
__global__ void residual_from_x(const double2* __restrict__ b, const double2* __restrict__ hx,
                                const double2* __restrict__ x, const double2* __restrict__ z, long long N,
                                double2* __restrict__ r) {
  const double2 zz = *z;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (long long)gridDim.x * blockDim.x) {
    const double2 xx = x[j], hh = hx[j], bb = b[j];
    r[j] = make_double2(bb.x - hh.x + zz.x * xx.x - zz.y * xx.y, bb.y - hh.y + zz.x * xx.y + zz.y * xx.x);
  }
}

// out[s] = |x_s|^2 (one block per row, fixed-order reduction)
__global__ void __launch_bounds__(256) sq_norm_rows(const double2* __restrict__ x, long long N, double* out) {
  const double2* xs = x + (size_t)blockIdx.x * N;
  double acc = 0;
  for (long long j = threadIdx.x; j < N; j += blockDim.x) acc += xs[j].x * xs[j].x + xs[j].y * xs[j].y;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ double sw[8];
  if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < 8; ++w) s += sw[w];
    out[blockIdx.x] = s;
  }
}

extern "C" bse_status bse_mlp_train(bse_handle* const* hs, const bse_c128* const* bs, int n_sys,
                                    const bse_c128* z, int n_z, int epochs, int batch, double lr, int seed,
                                    int krylov_steps, bse_mlp* m, double* loss_per_epoch) {
  if (!hs || !bs || !z || !m || n_sys < 1 || n_z < 1 || epochs < 1 || batch < 1 || !(lr > 0) ||
      krylov_steps < 0 || krylov_steps > KMAX)
    return BSE_ERR_INVALID_ARG;
  // residual probes r_t of unpreconditioned GMRES(30) after 0 (r = b), 1, 2 and 4 restart cycles
  const int cycles[4] = {0, 1, 2, 4};
  const int T = 4;
  struct Sample {
    int sys, zi;
  };
  std::vector<double2*> R(n_sys, nullptr);
  std::vector<double> b2(n_sys, 0.0);   // |b|^2 per system
  std::vector<double2> zh(n_z);
  for (int i = 0; i < n_z; ++i) zh[i] = make_double2(z[i].re, z[i].im);
  bse_status st = BSE_OK;
  // ---- harvest ----
  for (int s = 0; s < n_sys && st == BSE_OK; ++s) {
    bse_handle* h = hs[s];
    const long long N = h->N;
    double2 *bd = nullptr, *zd = nullptr, *x = nullptr, *hx = nullptr;
    int* it = nullptr;
    double* rr = nullptr;
    if (!dmalloc(&bd, N * sizeof(double2)) || !dmalloc(&zd, n_z * sizeof(double2)) ||
        !dmalloc(&x, (size_t)n_z * N * sizeof(double2)) || !dmalloc(&hx, (size_t)n_z * N * sizeof(double2)) ||
        !dmalloc(&it, n_z * sizeof(int)) || !dmalloc(&rr, n_z * sizeof(double)) ||
        !dmalloc(&R[s], (size_t)n_z * T * N * sizeof(double2))) {
      st = bse_fail(h, BSE_ERR_OOM, "training harvest");
    }
    if (st == BSE_OK) {
      cudaMemcpyAsync(bd, bs[s], N * sizeof(double2), cudaMemcpyDefault, h->stream);
      cudaMemcpyAsync(zd, zh.data(), n_z * sizeof(double2), cudaMemcpyHostToDevice, h->stream);
      sq_norm_rows<<<1, 256, 0, h->stream>>>(bd, N, rr);
      BSE_LAUNCHED(h);
      st = bse_cuda_check(h, cudaMemcpyAsync(&b2[s], rr, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "|b|^2");
    }
    int done = 0;
    for (int c = 0; c < T && st == BSE_OK; ++c) {
      if (cycles[c] == 0) {
        for (int i = 0; i < n_z; ++i)
          cudaMemcpyAsync(R[s] + ((size_t)i * T + c) * N, bd, N * sizeof(double2), cudaMemcpyDeviceToDevice,
                          h->stream);
        continue;
      }
      const int more = cycles[c] - done;
      bse_status g = bse_gmres_device(h, bd, zd, n_z, 1e-300, 30, 30 * more,
                                      done ? (BSE_PRECOND_NONE | BSE_GMRES_X0) : BSE_PRECOND_NONE, x, it, rr);
      if (g != BSE_OK && g != BSE_ERR_NOT_CONVERGED) {
        st = g;
        break;
      }
      done = cycles[c];
      for (int v0 = 0; v0 < n_z && st == BSE_OK; v0 += h->max_vec) {
        const int nv = std::min(h->max_vec, n_z - v0);
        st = bse_apply_device(h, x + (size_t)v0 * N, hx + (size_t)v0 * N, nv);
      }
      for (int i = 0; i < n_z && st == BSE_OK; ++i) {
        residual_from_x<<<256, 256, 0, h->stream>>>(bd, hx + (size_t)i * N, x + (size_t)i * N, zd + i, N,
                                                    R[s] + ((size_t)i * T + c) * N);
        BSE_LAUNCHED(h);
      }
    }
    if (st == BSE_OK) st = bse_cuda_check(h, cudaStreamSynchronize(h->stream), "harvest sync");
    cudaFree(bd);
    cudaFree(zd);
    cudaFree(x);
    cudaFree(hx);
    cudaFree(it);
    cudaFree(rr);
  }
  // ---- epochs ----
  std::vector<Sample> samples;
  for (int s = 0; s < n_sys; ++s)
    for (int i = 0; i < n_z; ++i) samples.push_back({s, i});
  long long maxN = 0;
  for (int s = 0; s < n_sys; ++s) maxN = std::max(maxN, hs[s]->N);
  float2 *p = nullptr, *u = nullptr, *v = nullptr;
  if (st == BSE_OK && (!dmalloc(&p, (size_t)maxN * sizeof(float2)) ||
                       !dmalloc(&u, (size_t)maxN * RANK * sizeof(float2)) ||
                       !dmalloc(&v, (size_t)maxN * RANK * sizeof(float2))))
    st = BSE_ERR_OOM;
  uint64_t rng = 0x9E3779B97F4A7C15ull ^ (uint64_t)seed;
  for (int ep = 0; ep < epochs && st == BSE_OK; ++ep) {
    for (size_t i = samples.size(); i > 1; --i) {   // Fisher-Yates with a 64-bit LCG
      rng = rng * 6364136223846793005ull + 1442695040888963407ull;
      std::swap(samples[i - 1], samples[(rng >> 33) % i]);
    }
    double tot = 0;
    int inb = 0;
    for (size_t k = 0; k < samples.size() && st == BSE_OK; ++k) {
      bse_handle* h = hs[samples[k].sys];
      const long long N = h->N;
      const int zi = samples[k].zi;
      double l = 0;
      // probes with |r| <= 1e-5 |b| belong to an already converged solve and are skipped
      st = loss_grad(h, m, zh[zi].x, zh[zi].y, T, R[samples[k].sys] + (size_t)zi * T * N, p, u, v, &l,
                     1e-10 * b2[samples[k].sys], krylov_steps);
      tot += l;
      if (++inb == batch || k + 1 == samples.size()) {
        m->t += 1;
        const float bc1 = 1.f - powf(0.9f, (float)m->t), bc2 = 1.f - powf(0.999f, (float)m->t);
        mlp_adam_k<<<(NPARAM + 255) / 256, 256, 0, h->stream>>>(m->w, m->m, m->v, m->g, m->w16, NPARAM, (float)lr,
                                                                1.f / inb, bc1, bc2);
        BSE_LAUNCHED(h);
        inb = 0;
      }
    }
    if (loss_per_epoch) loss_per_epoch[ep] = tot / samples.size();
  }
  for (int s = 0; s < n_sys; ++s) {
    cudaStreamSynchronize(hs[s]->stream);
    cudaFree(R[s]);
  }
  cudaFree(p);
  cudaFree(u);
  cudaFree(v);
  return st;
}
