// k -> R Fourier sum, multiplication by W(x, R) and R -> k sum of Algorithm 1
// (Sec. 3.2.1), applied to every column (x, c) of phi[k][c][x]:
//     phi'(x, k) = (1/Nk) sum_R e^{-ik.R} W(x, R) sum_k' e^{+ik'.R} phi(x, k').
// The 3-D transform over the k mesh is done axis by axis.
//
// kconv_cubic<T, N, BF16>: cubic mesh N x N x N (N <= 8).  One CTA owns one
// column c and 16 consecutive x; thread (g, xl) works on whole pencils, so each
// 1-D transform runs in registers.  The first forward pass is fused into the
// global load, the multiplication by W sits between the forward and inverse
// transforms along the last axis, and the last inverse pass is fused into the
// store (either complex T in place, or the bf16 hi/lo planes the tensor-core
// grid->band GEMM reads).
// kconv_generic<T, BF16>: any mesh with axes <= 16, one pass per axis in
// shared memory with explicit sums.
#include "bse_internal.cuh"
#include "dft_dev.cuh"

namespace {


constexpr int XC = 16;   // consecutive x per CTA

template <typename T, int N, bool BF16>
__global__ void __launch_bounds__(256) kconv_cubic(typename CT<T>::t* __restrict__ phi, const T* __restrict__ w,
                                                   const double* __restrict__ twiddle, __nv_bfloat16* __restrict__ hi,
                                                   __nv_bfloat16* __restrict__ lo, int nx, int nc, int nnmax) {
  typedef typename CT<T>::t C;
  constexpr int NK = N * N * N, NP = N * N;           // points, pencils per axis
  constexpr int PPT = (NP + 15) / 16;                  // pencils per thread
  extern __shared__ __align__(16) unsigned char kc_smem[];
  C* S = reinterpret_cast<C*>(kc_smem);               // [NK][XC]
  const int xl = threadIdx.x & (XC - 1), g = threadIdx.x >> 4;
  const int c = blockIdx.y, x0 = blockIdx.x * XC, x = x0 + xl;
  const bool xin = x < nx;
  C tw[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    tw[j].x = (T)twiddle[2 * j];   // axis-0 twiddles (cubic mesh: every axis the same)
    tw[j].y = (T)twiddle[2 * j + 1];
  }
  const size_t colstride = (size_t)nc * nx;   // distance between consecutive k in phi
  C* base = phi + (size_t)c * nx + x;
  // pass A: global load (all of this thread's pencils first, so the loads are
  // in flight together) + forward transform along axis 2 (k = (m0 N + m1) N + m2)
  {
    C va[PPT][N];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = g + 16 * i;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        if (xin && p < NP) {
          va[i][j] = base[(size_t)(p * N + j) * colstride];
        } else {
          va[i][j].x = 0;
          va[i][j].y = 0;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = g + 16 * i;
      if (p < NP) {
        dftN<T, N, +1>(va[i], tw);
#pragma unroll
        for (int j = 0; j < N; ++j) S[(p * N + j) * XC + xl] = va[i][j];
      }
    }
  }
  __syncthreads();
  // pass B: forward along axis 1; pencil p = (m0, m2): k = m0 N^2 + j N + m2
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + 16 * i;
    if (p < NP) {
      const int kb = (p / N) * NP + (p % N);
      C v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = S[(kb + j * N) * XC + xl];
      dftN<T, N, +1>(v, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) S[(kb + j * N) * XC + xl] = v[j];
    }
  }
  __syncthreads();
  // pass C: forward along axis 0, times W(x, R)/Nk, inverse along axis 0; p = (m1, m2): k = j N^2 + p
  const T inv = (T)1 / (T)NK;
  T wr[PPT][N];   // W(x, R) of this thread's pencils, loaded ahead of the transforms
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + 16 * i;
#pragma unroll
    for (int j = 0; j < N; ++j) wr[i][j] = (xin && p < NP) ? w[(size_t)(j * NP + p) * nx + x] * inv : (T)0;
  }
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + 16 * i;
    if (p < NP) {
      C v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = S[(j * NP + p) * XC + xl];
      dftN<T, N, +1>(v, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        v[j].x *= wr[i][j];
        v[j].y *= wr[i][j];
      }
      dftN<T, N, -1>(v, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) S[(j * NP + p) * XC + xl] = v[j];
    }
  }
  __syncthreads();
  // pass D: inverse along axis 1
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + 16 * i;
    if (p < NP) {
      const int kb = (p / N) * NP + (p % N);
      C v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = S[(kb + j * N) * XC + xl];
      dftN<T, N, -1>(v, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) S[(kb + j * N) * XC + xl] = v[j];
    }
  }
  __syncthreads();
  // pass E: inverse along axis 2 + store
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + 16 * i;
    if (p < NP) {
      C v[N];
#pragma unroll
      for (int j = 0; j < N; ++j) v[j] = S[(p * N + j) * XC + xl];
      dftN<T, N, -1>(v, tw);
      if (xin) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int k = p * N + j;
          if constexpr (BF16) {
            // K-tiled planes [k][x/64][row][64], rows 2c (re) and 2c+1 (im)
            const size_t o = (((size_t)k * ((nx + 63) >> 6) + (x >> 6)) * nnmax + 2 * c) * 64 + (x & 63);
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf((float)v[j].x, h0, l0);
            split_bf((float)v[j].y, h1, l1);
            hi[o] = h0;
            lo[o] = l0;
            hi[o + 64] = h1;
            lo[o + 64] = l1;
          } else {
            base[(size_t)k * colstride] = v[j];
          }
        }
      }
    }
  }
}

// kconv_cubic2<N, BF16, XW>: the FP32 transform of kconv_cubic with two
// consecutive x per thread (even Nx): every shared-memory and global access
// moves 16 bytes (two complex64), the bf16 planes are written as bf16 pairs,
// so the memory and address instructions per point are halved while the
// transform arithmetic is unchanged.  CTA: one column c and XW consecutive x
// (XW/2 pairs); 256 threads = XW/2 pairs x 512/XW pencil groups.  XW is
// chosen so that every thread owns whole pencils and the shared tile
// (N^3 x XW complex64) stays small enough for several CTAs per SM.
template <int N, bool BF16, int XW>
__global__ void __launch_bounds__(256) kconv_cubic2(float2* __restrict__ phi, const float* __restrict__ w,
                                                    const double* __restrict__ twiddle,
                                                    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                                    int nx, int nc, int nnmax, int x0) {
  constexpr int NK = N * N * N, NP = N * N;
  constexpr int XP = XW / 2;                 // x pairs per CTA
  constexpr int NG = 256 / XP;               // pencil groups
  constexpr int PPT = (NP + NG - 1) / NG;    // pencils per thread
  static_assert(XW <= 64 && 64 % XW == 0, "an x pair must not straddle a 64-point K block");
  extern __shared__ __align__(16) unsigned char kc_smem[];
  float4* S = reinterpret_cast<float4*>(kc_smem);   // [NK][XP], each entry (x, x+1)
  const int xp = threadIdx.x & (XP - 1), g = threadIdx.x / XP;
  const int c = blockIdx.y, x = x0 + blockIdx.x * XW + 2 * xp;
  const bool xin = x < nx;                   // Nx even: then x + 1 < Nx as well
  float2 tw[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    tw[j].x = (float)twiddle[2 * j];
    tw[j].y = (float)twiddle[2 * j + 1];
  }
  const size_t colstride = (size_t)nc * nx;
  float2* base = phi + (size_t)c * nx + x;
  // pass A: global load + forward transform along axis 2
  {
    float2 va[PPT][N], vb[PPT][N];
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = g + NG * i;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (xin && p < NP) q = *reinterpret_cast<const float4*>(base + (size_t)(p * N + j) * colstride);
        va[i][j] = make_float2(q.x, q.y);
        vb[i][j] = make_float2(q.z, q.w);
      }
    }
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      const int p = g + NG * i;
      if (p < NP) {
        dftN<float, N, +1>(va[i], tw);
        dftN<float, N, +1>(vb[i], tw);
#pragma unroll
        for (int j = 0; j < N; ++j) S[(p * N + j) * XP + xp] = make_float4(va[i][j].x, va[i][j].y, vb[i][j].x, vb[i][j].y);
      }
    }
  }
  __syncthreads();
  // pass B: forward along axis 1; pencil p = (m0, m2): k = m0 N^2 + j N + m2
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + NG * i;
    if (p < NP) {
      const int kb = (p / N) * NP + (p % N);
      float2 va[N], vb[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float4 q = S[(kb + j * N) * XP + xp];
        va[j] = make_float2(q.x, q.y);
        vb[j] = make_float2(q.z, q.w);
      }
      dftN<float, N, +1>(va, tw);
      dftN<float, N, +1>(vb, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) S[(kb + j * N) * XP + xp] = make_float4(va[j].x, va[j].y, vb[j].x, vb[j].y);
    }
  }
  __syncthreads();
  // pass C: forward along axis 0, times W(x, R)/Nk, inverse along axis 0; p = (m1, m2): k = j N^2 + p
  const float inv = 1.f / (float)NK;
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + NG * i;
    if (p < NP) {
      float2 wr[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        wr[j] = xin ? *reinterpret_cast<const float2*>(w + (size_t)(j * NP + p) * nx + x) : make_float2(0.f, 0.f);
        wr[j].x *= inv;
        wr[j].y *= inv;
      }
      float2 va[N], vb[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float4 q = S[(j * NP + p) * XP + xp];
        va[j] = make_float2(q.x, q.y);
        vb[j] = make_float2(q.z, q.w);
      }
      dftN<float, N, +1>(va, tw);
      dftN<float, N, +1>(vb, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        va[j].x *= wr[j].x;
        va[j].y *= wr[j].x;
        vb[j].x *= wr[j].y;
        vb[j].y *= wr[j].y;
      }
      dftN<float, N, -1>(va, tw);
      dftN<float, N, -1>(vb, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) S[(j * NP + p) * XP + xp] = make_float4(va[j].x, va[j].y, vb[j].x, vb[j].y);
    }
  }
  __syncthreads();
  // pass D: inverse along axis 1
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + NG * i;
    if (p < NP) {
      const int kb = (p / N) * NP + (p % N);
      float2 va[N], vb[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float4 q = S[(kb + j * N) * XP + xp];
        va[j] = make_float2(q.x, q.y);
        vb[j] = make_float2(q.z, q.w);
      }
      dftN<float, N, -1>(va, tw);
      dftN<float, N, -1>(vb, tw);
#pragma unroll
      for (int j = 0; j < N; ++j) S[(kb + j * N) * XP + xp] = make_float4(va[j].x, va[j].y, vb[j].x, vb[j].y);
    }
  }
  __syncthreads();
  // pass E: inverse along axis 2 + store
#pragma unroll
  for (int i = 0; i < PPT; ++i) {
    const int p = g + NG * i;
    if (p < NP) {
      float2 va[N], vb[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const float4 q = S[(p * N + j) * XP + xp];
        va[j] = make_float2(q.x, q.y);
        vb[j] = make_float2(q.z, q.w);
      }
      dftN<float, N, -1>(va, tw);
      dftN<float, N, -1>(vb, tw);
      if (xin) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const int k = p * N + j;
          if constexpr (BF16) {
            // K-tiled planes [k][x/64][row][64], rows 2c (re) and 2c+1 (im); x, x+1 in one 64-block
            const size_t o = (((size_t)k * ((nx + 63) >> 6) + (x >> 6)) * nnmax + 2 * c) * 64 + (x & 63);
            __nv_bfloat16 h0, l0, h1, l1, h2, l2, h3, l3;
            split_bf(va[j].x, h0, l0);
            split_bf(vb[j].x, h1, l1);
            split_bf(va[j].y, h2, l2);
            split_bf(vb[j].y, h3, l3);
            *reinterpret_cast<__nv_bfloat162*>(hi + o) = __halves2bfloat162(h0, h1);
            *reinterpret_cast<__nv_bfloat162*>(lo + o) = __halves2bfloat162(l0, l1);
            *reinterpret_cast<__nv_bfloat162*>(hi + o + 64) = __halves2bfloat162(h2, h3);
            *reinterpret_cast<__nv_bfloat162*>(lo + o + 64) = __halves2bfloat162(l2, l3);
          } else {
            *reinterpret_cast<float4*>(base + (size_t)k * colstride) = make_float4(va[j].x, va[j].y, vb[j].x, vb[j].y);
          }
        }
      }
    }
  }
}

// kconv_plane8<BF16>: the 8^3 mesh with one shared-memory round trip for the
// two outer axes.  CTA: one column c and 16 consecutive x, 128 threads.
//   pass A: thread (x, g) transforms the axis-2 pencils p = g + 8i (i < 8,
//           p = (m0, m1)) straight from global memory and writes them to the
//           shared tile S[k][x];
//   pass P: thread (x, m2) holds the whole (m0, m1) plane of its m2 and x:
//           forward along axes 1 and 0, times W(x, R)/Nk, inverse along
//           axes 0 and 1, all in registers, and writes the plane back;
//   pass E: as pass A, the inverse along axis 2 fused into the store.
// Shared-memory traffic per point: one write and one read in each half (four
// accesses, against eight for the pencil-per-pass form).
template <bool BF16>
__global__ void __launch_bounds__(128) kconv_plane8(float2* __restrict__ phi, const float* __restrict__ w,
                                                    __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                                    int nx, int nc, int nnmax, int x0) {
  constexpr int N = 8, NP = 64, NK = 512, XW = 16;
  extern __shared__ __align__(16) unsigned char kp_smem[];
  float2* S = reinterpret_cast<float2*>(kp_smem);   // [NK][XW]
  const int xl = threadIdx.x & (XW - 1), g = threadIdx.x >> 4;   // g in 0..7
  const int c = blockIdx.y, x = x0 + blockIdx.x * XW + xl;
  const bool xin = x < nx;
  const size_t colstride = (size_t)nc * nx;
  float2* base = phi + (size_t)c * nx + x;
  float2 tw[N];   // unused by the radix-8 butterfly; kept for the dftN signature
#pragma unroll
  for (int j = 0; j < N; ++j) tw[j] = make_float2(0.f, 0.f);
  // pass A: pencils p = g + 8i along axis 2 (k = p*8 + j)
#pragma unroll 2
  for (int i = 0; i < 8; ++i) {
    const int p = g + 8 * i;
    float2 v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = xin ? base[(size_t)(p * N + j) * colstride] : make_float2(0.f, 0.f);
    dftN<float, N, +1>(v, tw);
#pragma unroll
    for (int j = 0; j < N; ++j) S[(p * N + j) * XW + xl] = v[j];
  }
  __syncthreads();
  // pass P: the plane (m0, m1) of m2 = g; k = (m0*8 + m1)*8 + m2
  {
    const int m2 = g;
    float2 pl[N][N];   // [m0][m1]
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) pl[a][b] = S[((a * N + b) * N + m2) * XW + xl];
    // forward along axis 1 (m1), then axis 0 (m0)
#pragma unroll
    for (int a = 0; a < N; ++a) dftN<float, N, +1>(pl[a], tw);
#pragma unroll
    for (int b = 0; b < N; ++b) {
      float2 col[N];
#pragma unroll
      for (int a = 0; a < N; ++a) col[a] = pl[a][b];
      dftN<float, N, +1>(col, tw);
      // times W(x, R)/Nk, R = (r0, r1, r2) = (a, b, m2), then the inverse along axis 0
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const float wv = xin ? w[(size_t)((a * N + b) * N + m2) * nx + x] * (1.f / (float)NK) : 0.f;
        col[a].x *= wv;
        col[a].y *= wv;
      }
      dftN<float, N, -1>(col, tw);
#pragma unroll
      for (int a = 0; a < N; ++a) pl[a][b] = col[a];
    }
    // inverse along axis 1
#pragma unroll
    for (int a = 0; a < N; ++a) dftN<float, N, -1>(pl[a], tw);
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int b = 0; b < N; ++b) S[((a * N + b) * N + m2) * XW + xl] = pl[a][b];
  }
  __syncthreads();
  // pass E: inverse along axis 2 + store
#pragma unroll 2
  for (int i = 0; i < 8; ++i) {
    const int p = g + 8 * i;
    float2 v[N];
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = S[(p * N + j) * XW + xl];
    dftN<float, N, -1>(v, tw);
    if (xin) {
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int k = p * N + j;
        if constexpr (BF16) {
          const size_t o = (((size_t)k * ((nx + 63) >> 6) + (x >> 6)) * nnmax + 2 * c) * 64 + (x & 63);
          __nv_bfloat16 h0, l0, h1, l1;
          split_bf(v[j].x, h0, l0);
          split_bf(v[j].y, h1, l1);
          hi[o] = h0;
          lo[o] = l0;
          hi[o + 64] = h1;
          lo[o + 64] = l1;
        } else {
          base[(size_t)k * colstride] = v[j];
        }
      }
    }
  }
}

// Generic mesh: one shared-memory pass per axis with explicit sums; CTA owns
// XC consecutive x of one column c.  S[k][xl].
template <typename T, int SIGN>
__device__ void axis_pass(typename CT<T>::t* S, const typename CT<T>::t* tw, int nk, int len, int stride) {
  typedef typename CT<T>::t C;
  const int nlines = (nk / len) * XC;
  for (int wv = threadIdx.x; wv < nlines; wv += blockDim.x) {
    const int xl = wv & (XC - 1), line = wv / XC;
    const int inner = line % stride, outer = line / stride;
    const int b = outer * stride * len + inner;
    C v[BSE_MAX_NK_AXIS];
#pragma unroll
    for (int j = 0; j < BSE_MAX_NK_AXIS; ++j)
      if (j < len) v[j] = S[(b + j * stride) * XC + xl];
    for (int q = 0; q < len; ++q) {
      C acc;
      acc.x = 0;
      acc.y = 0;
#pragma unroll
      for (int j = 0; j < BSE_MAX_NK_AXIS; ++j) {
        if (j < len) {
          C t = tw[(j * q) % len];
          if (SIGN < 0) t.y = -t.y;
          C p = cmulc(t, v[j]);
          acc.x += p.x;
          acc.y += p.y;
        }
      }
      S[(b + q * stride) * XC + xl] = acc;
    }
  }
}

template <typename T, bool BF16>
__global__ void __launch_bounds__(256) kconv_generic(typename CT<T>::t* __restrict__ phi, const T* __restrict__ w,
                                                     const double* __restrict__ twiddle,
                                                     __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                                     int nk0, int nk1, int nk2, int nx, int nc, int nnmax) {
  typedef typename CT<T>::t C;
  extern __shared__ __align__(16) unsigned char kg_smem[];
  C* tw = reinterpret_cast<C*>(kg_smem);   // [3][16]
  C* S = tw + 48;                          // [Nk][XC]
  const int nk = nk0 * nk1 * nk2;
  const int c = blockIdx.y, x0 = blockIdx.x * XC;
  for (int i = threadIdx.x; i < 48; i += blockDim.x) {
    tw[i].x = (T)twiddle[2 * i];
    tw[i].y = (T)twiddle[2 * i + 1];
  }
  const size_t colstride = (size_t)nc * nx;
  for (int e = threadIdx.x; e < nk * XC; e += blockDim.x) {
    const int k = e / XC, xl = e % XC, x = x0 + xl;
    C z;
    z.x = 0;
    z.y = 0;
    S[e] = x < nx ? phi[(size_t)k * colstride + (size_t)c * nx + x] : z;
  }
  __syncthreads();
  axis_pass<T, +1>(S, tw + 32, nk, nk2, 1);
  __syncthreads();
  axis_pass<T, +1>(S, tw + 16, nk, nk1, nk2);
  __syncthreads();
  axis_pass<T, +1>(S, tw, nk, nk0, nk1 * nk2);
  __syncthreads();
  const T inv = (T)1 / (T)nk;
  for (int e = threadIdx.x; e < nk * XC; e += blockDim.x) {
    const int r = e / XC, x = x0 + e % XC;
    const T wv = x < nx ? w[(size_t)r * nx + x] * inv : (T)0;
    S[e].x *= wv;
    S[e].y *= wv;
  }
  __syncthreads();
  axis_pass<T, -1>(S, tw + 32, nk, nk2, 1);
  __syncthreads();
  axis_pass<T, -1>(S, tw + 16, nk, nk1, nk2);
  __syncthreads();
  axis_pass<T, -1>(S, tw, nk, nk0, nk1 * nk2);
  __syncthreads();
  for (int e = threadIdx.x; e < nk * XC; e += blockDim.x) {
    const int k = e / XC, x = x0 + e % XC;
    if (x >= nx) continue;
    if constexpr (BF16) {
      const size_t o = (((size_t)k * ((nx + 63) >> 6) + (x >> 6)) * nnmax + 2 * c) * 64 + (x & 63);
      __nv_bfloat16 h0, l0, h1, l1;
      split_bf((float)S[e].x, h0, l0);
      split_bf((float)S[e].y, h1, l1);
      hi[o] = h0;
      lo[o] = l0;
      hi[o + 64] = h1;
      lo[o + 64] = l1;
    } else {
      phi[(size_t)k * colstride + (size_t)c * nx + x] = S[e];
    }
  }
}

template <typename T, int N, bool BF16>
void launch_cubic(bse_handle* h, dim3 g, typename CT<T>::t* phi, const T* w, __nv_bfloat16* hi, __nv_bfloat16* lo,
                  int nc, int nnmax) {
  const size_t smem = (size_t)N * N * N * XC * sizeof(typename CT<T>::t);
  cudaFuncSetAttribute(kconv_cubic<T, N, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  BSE_PROF(h, BSE_K_KCONV,
           kconv_cubic<T, N, BF16><<<g, 256, smem, h->stream>>>(phi, w, h->twiddle, hi, lo, h->nx, nc, nnmax));
}

template <int N, bool BF16, int XW>
void launch_cubic2(bse_handle* h, float2* phi, const float* w, __nv_bfloat16* hi, __nv_bfloat16* lo, int nc,
                   int nnmax, int x0, int x1, cudaStream_t st) {
  const size_t smem = (size_t)N * N * N * XW * sizeof(float2);
  const dim3 g((unsigned)((x1 - x0 + XW - 1) / XW), (unsigned)nc);
  cudaFuncSetAttribute(kconv_cubic2<N, BF16, XW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  BSE_PROF(h, BSE_K_KCONV,
           kconv_cubic2<N, BF16, XW><<<g, 256, smem, st>>>(phi, w, h->twiddle, hi, lo, h->nx, nc, nnmax, x0));
}

template <bool BF16>
void launch_plane8(bse_handle* h, float2* phi, const float* w, __nv_bfloat16* hi, __nv_bfloat16* lo, int nc,
                   int nnmax, int x0, int x1, cudaStream_t st) {
  const size_t smem = (size_t)512 * 16 * sizeof(float2);
  const dim3 g((unsigned)((x1 - x0 + 15) / 16), (unsigned)nc);
  cudaFuncSetAttribute(kconv_plane8<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  BSE_PROF(h, BSE_K_KCONV, kconv_plane8<BF16><<<g, 128, smem, st>>>(phi, w, hi, lo, h->nx, nc, nnmax, x0));
}

// x range [x0, x1) on stream st: only the pencil and plane forms take a
// part of the grid (x-slabs of the tensor-core step); the others the whole
template <typename T, bool BF16>
bse_status launch(bse_handle* h, int nc, __nv_bfloat16* hi, __nv_bfloat16* lo, int nnmax, int x0, int x1,
                  cudaStream_t st) {
  typedef typename CT<T>::t C;
  C* phi = (C*)h->phi;
  const T* w = (const T*)h->w;
  const dim3 g((unsigned)((h->nx + XC - 1) / XC), (unsigned)nc);
  const int n = h->nk3[0];
  if constexpr (sizeof(T) == sizeof(float)) {
    // wide passes (more than 128 columns) on the 8^3 mesh: the plane form
    // (1200 columns of the L2,3 workload: 26.1 vs 28.0 ms per H application);
    // narrow ones keep the pencil form (6 columns: 59 vs 82 us)
    if (n == 8 && h->nk3[1] == 8 && h->nk3[2] == 8 && nc > 128) {
      launch_plane8<BF16>(h, (float2*)phi, (const float*)w, hi, lo, nc, nnmax, x0, x1, st);
      return bse_cuda_check(h, cudaGetLastError(), "k-transform launch");
    }
    if (h->nk3[1] == n && h->nk3[2] == n && (n == 4 || n == 8) && h->nx % 2 == 0) {
      // FP32, even Nx: two x per thread, 16 x per CTA (measured against 8 x
      // per CTA at four CTAs per SM on the 8^3 mesh: 59 vs 90 us)
      if (n == 8)
        launch_cubic2<8, BF16, 16>(h, (float2*)phi, (const float*)w, hi, lo, nc, nnmax, x0, x1, st);
      else
        launch_cubic2<4, BF16, 16>(h, (float2*)phi, (const float*)w, hi, lo, nc, nnmax, x0, x1, st);
      return bse_cuda_check(h, cudaGetLastError(), "k-transform launch");
    }
  }
  if (x0 != 0 || x1 != h->nx || st != h->stream)
    return bse_fail(h, BSE_ERR_UNSUPPORTED, "k-transform of part of the grid needs the 4^3 or 8^3 FP32 forms");
  if (h->nk3[1] == n && h->nk3[2] == n && n <= 8) {
#define KCUBIC(NN)                                                  \
  case NN:                                                          \
    launch_cubic<T, NN, BF16>(h, g, phi, w, hi, lo, nc, nnmax);     \
    break;
    switch (n) {
      KCUBIC(1)
      KCUBIC(2)
      KCUBIC(3)
      KCUBIC(4)
      KCUBIC(5)
      KCUBIC(6)
      KCUBIC(7)
      KCUBIC(8)
    }
#undef KCUBIC
  } else {
    const size_t smem = (48 + (size_t)h->nk * XC) * sizeof(C);
    if (smem > 220 * 1024) return bse_fail(h, BSE_ERR_UNSUPPORTED, "k mesh too large for the shared-memory transform");
    cudaFuncSetAttribute(kconv_generic<T, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    BSE_PROF(h, BSE_K_KCONV,
             kconv_generic<T, BF16><<<g, 256, smem, h->stream>>>(phi, w, h->twiddle, hi, lo, h->nk3[0], h->nk3[1],
                                                                 h->nk3[2], h->nx, nc, nnmax));
  }
  return bse_cuda_check(h, cudaGetLastError(), "k-transform launch");
}

}  // namespace

// phi[k][c][x] in place (FP64 / FP32 forms)
bse_status bse_kconv_inplace(bse_handle* h, int n_vec) {
  const int nc = n_vec * h->na;
  if (h->prec == BSE_PREC_FP64) return launch<double, false>(h, nc, nullptr, nullptr, 0, 0, h->nx, h->stream);
  return launch<float, false>(h, nc, nullptr, nullptr, 0, 0, h->nx, h->stream);
}

// phi[k][c][x] (FP32) -> bf16 hi/lo planes [k][2c+s][x] with row stride nnmax,
// for x in [x0, x1) on stream st
bse_status bse_kconv_split(bse_handle* h, int n_vec, __nv_bfloat16* hi, __nv_bfloat16* lo, int nnmax, int x0, int x1,
                           cudaStream_t st) {
  return launch<float, true>(h, n_vec * h->na, hi, lo, nnmax, x0, x1, st);
}

bool bse_kconv_takes_slabs(const bse_handle* h) {
  const int n = h->nk3[0];
  return h->prec != BSE_PREC_FP64 && h->nk3[1] == n && h->nk3[2] == n && (n == 4 || n == 8) && h->nx % 2 == 0;
}
