// H psi on the device: SIMT band<->grid contractions (FP64 and FP32 forms),
// the k->R / x W / R->k transform, and the short-range projector terms.
//
// Algorithm 1 (Sec. 3.2.1), with the loop over x and alpha turned inside out:
//   band->grid  phi[k][x][c]  = sum_n  U[k][x][n] psi[c][k][n]   (U = e^{ik.x} u, first line)
//   k-conv      phi[.][x][c]  = F_{R->k} W(x,R) F_{k->R} phi[.][x][c]         (lines 3-5)
//   grid->band  out[c][k][n]  = sum_x conj(U[k][x][n]) phi[k][x][c]           (last line)
// with c = v*Na + alpha the column index (vector v, core state alpha).  The
// grid->band kernel also adds E_nk psi - chi psi (Eqs. 3-5) and the short-range
// projection out (Sec. 3.2.2) in FP64, so one pass writes H psi.
#include "bse_internal.cuh"

namespace {

template <typename T> struct Cx { typedef typename cvec<T>::type type; };

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

template <typename C> __device__ __forceinline__ C from_d2(double2 v) {
  C r;
  r.x = v.x;
  r.y = v.y;
  return r;
}

// ---------------------------------------------------------------------------
// band -> grid:  phi[k][x][c0+cc] = sum_n U[k][x][n] psi[c0+cc][k][n]
// grid (ceil(Nx/64), Nk), 256 threads: row = t&63, column group g = t>>6.
// ---------------------------------------------------------------------------
template <typename T, int CC>
__global__ void __launch_bounds__(256) b2g_simt(const typename Cx<T>::type* __restrict__ U,
                                                const double2* __restrict__ psi,
                                                typename Cx<T>::type* __restrict__ phi, int nk,
                                                int nx, int nb, int c0, int ncc, int nc_total) {
  typedef typename Cx<T>::type C;
  __shared__ C Us[64][33];
  __shared__ C Ps[CC][32];
  const int t = threadIdx.x, row = t & 63, g = t >> 6;
  const int k = blockIdx.y, x0 = blockIdx.x * 64;
  C acc[CC / 4];
#pragma unroll
  for (int i = 0; i < CC / 4; ++i) acc[i] = czero<C>();
  const C* Uk = U + (size_t)k * nx * nb;
  for (int n0 = 0; n0 < nb; n0 += 32) {
    for (int e = t; e < 64 * 32; e += 256) {
      int r = e >> 5, j = e & 31, x = x0 + r, n = n0 + j;
      Us[r][j] = (x < nx && n < nb) ? Uk[(size_t)x * nb + n] : czero<C>();
    }
    for (int e = t; e < CC * 32; e += 256) {
      int cc = e >> 5, j = e & 31, n = n0 + j;
      Ps[cc][j] = (cc < ncc && n < nb) ? from_d2<C>(psi[((size_t)(c0 + cc) * nk + k) * nb + n]) : czero<C>();
    }
    __syncthreads();
#pragma unroll 4
    for (int j = 0; j < 32; ++j) {
      C u = Us[row][j];
#pragma unroll
      for (int i = 0; i < CC / 4; ++i) cmac(acc[i], u, Ps[g + 4 * i][j]);
    }
    __syncthreads();
  }
  const int x = x0 + row;
  if (x < nx) {
#pragma unroll
    for (int i = 0; i < CC / 4; ++i) {
      int cc = g + 4 * i;
      if (cc < ncc) phi[((size_t)k * nx + x) * nc_total + c0 + cc] = acc[i];
    }
  }
}

// ---------------------------------------------------------------------------
// k-convolution with W (Algorithm 1, lines 3-5) on CC consecutive columns of
// phi[k][col], col = x*Nc + c:  phi <- (1/Nk) F^- ( W(x, R) * F^+ phi ).
// F^{+/-} are 3-D DFTs over the (nk0, nk1, nk2) mesh, computed axis by axis in
// shared memory with explicit sums (nk_d <= 16).
// ---------------------------------------------------------------------------
// radix-2 8-point DFT in registers: v_q <- sum_j e^{SIGN 2 pi i j q / 8} v_j
template <typename T, int SIGN>
__device__ __forceinline__ void dft8_simt(typename Cx<T>::type* v) {
  typedef typename Cx<T>::type C;
  const T r = (T)0.70710678118654752440;
  auto add = [](C a, C b) { C o; o.x = a.x + b.x; o.y = a.y + b.y; return o; };
  auto sub = [](C a, C b) { C o; o.x = a.x - b.x; o.y = a.y - b.y; return o; };
  auto mi = [](C a) { C o; o.x = -SIGN * a.y; o.y = SIGN * a.x; return o; };   // times SIGN*i
  C a0 = add(v[0], v[4]), a1 = sub(v[0], v[4]), a2 = add(v[2], v[6]), a3 = sub(v[2], v[6]);
  C a4 = add(v[1], v[5]), a5 = sub(v[1], v[5]), a6 = add(v[3], v[7]), a7 = sub(v[3], v[7]);
  C e0 = add(a0, a2), e2 = sub(a0, a2), e1 = add(a1, mi(a3)), e3 = sub(a1, mi(a3));
  C o0 = add(a4, a6), o2 = sub(a4, a6), o1 = add(a5, mi(a7)), o3 = sub(a5, mi(a7));
  C t1, t3;
  t1.x = r * (o1.x - SIGN * o1.y);
  t1.y = r * (o1.y + SIGN * o1.x);
  C t2 = mi(o2);
  t3.x = r * (-o3.x - SIGN * o3.y);
  t3.y = r * (-o3.y + SIGN * o3.x);
  v[0] = add(e0, o0);
  v[4] = sub(e0, o0);
  v[1] = add(e1, t1);
  v[5] = sub(e1, t1);
  v[2] = add(e2, t2);
  v[6] = sub(e2, t2);
  v[3] = add(e3, t3);
  v[7] = sub(e3, t3);
}

template <typename T, int SIGN>
__device__ __forceinline__ void dft_axis(typename Cx<T>::type* S, const typename Cx<T>::type* tw, int nk,
                                         int len, int stride, int CCn) {
  typedef typename Cx<T>::type C;
  const int nlines = (nk / len) * CCn;
  for (int w = threadIdx.x; w < nlines; w += blockDim.x) {
    int cc = w % CCn, line = w / CCn;
    // line -> base k index: split line into (outer, inner) around the axis
    int inner = line % stride, outer = line / stride;
    int base = outer * stride * len + inner;
    if (len == 1) continue;
    if (len == 8) {
      C v8[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v8[j] = S[(size_t)(base + j * stride) * CCn + cc];
      dft8_simt<T, SIGN>(v8);
#pragma unroll
      for (int j = 0; j < 8; ++j) S[(size_t)(base + j * stride) * CCn + cc] = v8[j];
      continue;
    }
    C v[BSE_MAX_NK_AXIS];
#pragma unroll
    for (int j = 0; j < BSE_MAX_NK_AXIS; ++j)
      if (j < len) v[j] = S[(size_t)(base + j * stride) * CCn + cc];
    for (int q = 0; q < len; ++q) {
      C acc = czero<C>();
#pragma unroll
      for (int j = 0; j < BSE_MAX_NK_AXIS; ++j) {
        if (j < len) {
          C t = tw[(j * q) % len];
          if (SIGN < 0) t.y = -t.y;
          cmac(acc, t, v[j]);
        }
      }
      S[(size_t)(base + q * stride) * CCn + cc] = acc;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) kconv_simt(typename Cx<T>::type* __restrict__ phi,
                                                  const T* __restrict__ w,
                                                  const double* __restrict__ twiddle, int nk0,
                                                  int nk1, int nk2, int nx, int nc, int CCn) {
  typedef typename Cx<T>::type C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);   // [3][16]
  C* S = tw + 48;                           // [Nk][CCn]
  const int nk = nk0 * nk1 * nk2;
  const long long ncol = (long long)nx * nc;
  const long long col0 = (long long)blockIdx.x * CCn;
  for (int i = threadIdx.x; i < 48; i += blockDim.x) {
    C t;
    t.x = (T)twiddle[2 * i];
    t.y = (T)twiddle[2 * i + 1];
    tw[i] = t;
  }
  for (int e = threadIdx.x; e < nk * CCn; e += blockDim.x) {
    int k = e / CCn, cc = e % CCn;
    long long col = col0 + cc;
    S[e] = (col < ncol) ? phi[(size_t)k * ncol + col] : czero<C>();
  }
  __syncthreads();
  // F_{k->R}: e^{+ik.R}
  dft_axis<T, +1>(S, tw + 32, nk, nk2, 1, CCn);
  __syncthreads();
  dft_axis<T, +1>(S, tw + 16, nk, nk1, nk2, CCn);
  __syncthreads();
  dft_axis<T, +1>(S, tw + 0, nk, nk0, nk1 * nk2, CCn);
  __syncthreads();
  // times W(x, R)
  const T inv = (T)1 / (T)nk;
  for (int e = threadIdx.x; e < nk * CCn; e += blockDim.x) {
    int r = e / CCn, cc = e % CCn;
    long long col = col0 + cc;
    if (col < ncol) {
      T wv = w[(size_t)r * nx + (int)(col / nc)] * inv;
      S[e].x *= wv;
      S[e].y *= wv;
    }
  }
  __syncthreads();
  // F_{R->k}: e^{-ik.R} (1/Nk applied above)
  dft_axis<T, -1>(S, tw + 32, nk, nk2, 1, CCn);
  __syncthreads();
  dft_axis<T, -1>(S, tw + 16, nk, nk1, nk2, CCn);
  __syncthreads();
  dft_axis<T, -1>(S, tw + 0, nk, nk0, nk1 * nk2, CCn);
  __syncthreads();
  for (int e = threadIdx.x; e < nk * CCn; e += blockDim.x) {
    int k = e / CCn, cc = e % CCn;
    long long col = col0 + cc;
    if (col < ncol) phi[(size_t)k * ncol + col] = S[e];
  }
}

// ---------------------------------------------------------------------------
// grid -> band + diagonal + spin-orbit + short-range out, FP64 epilogue:
// out[c][k][n] = sum_x conj(U[k][x][n]) phi[k][x][c] + E_kn psi[c][k][n]
//              - sum_b chi[a][b] psi[(v,b)][k][n] + sum_p conj(A[p][kn]) c'[v][a][p]
// grid (ceil(Nb/64), Nk), 256 threads: n = t&63, x group xg = t>>6.
// ---------------------------------------------------------------------------
template <typename T, int CC>
__global__ void __launch_bounds__(256) g2b_simt(
    const typename Cx<T>::type* __restrict__ U, const typename Cx<T>::type* __restrict__ phi,
    const double2* __restrict__ psi, double2* __restrict__ out, const double* __restrict__ e_nk,
    const double2* __restrict__ chi, const double2* __restrict__ a_proj,
    const double2* __restrict__ srcp, int nk, int nx, int nb, int na, int np, int c0, int ncc,
    int nc_total) {
  typedef typename Cx<T>::type C;
  __shared__ C Fs[32][CC];
  __shared__ C red[4][64][CC];
  const int t = threadIdx.x, nl = t & 63, xg = t >> 6;
  const int k = blockIdx.y, n = blockIdx.x * 64 + nl;
  C acc[CC];
#pragma unroll
  for (int i = 0; i < CC; ++i) acc[i] = czero<C>();
  const C* Uk = U + (size_t)k * nx * nb;
  for (int x0 = 0; x0 < nx; x0 += 32) {
    for (int e = t; e < 32 * CC; e += 256) {
      int xi = e / CC, cc = e % CC, x = x0 + xi;
      Fs[xi][cc] = (x < nx && cc < ncc) ? phi[((size_t)k * nx + x) * nc_total + c0 + cc] : czero<C>();
    }
    __syncthreads();
    if (n < nb) {
      for (int xi = xg; xi < 32; xi += 4) {
        int x = x0 + xi;
        if (x < nx) {
          C u = Uk[(size_t)x * nb + n];
#pragma unroll
          for (int cc = 0; cc < CC; ++cc) cmac_conj(acc[cc], u, Fs[xi][cc]);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int cc = 0; cc < CC; ++cc) red[xg][nl][cc] = acc[cc];
  __syncthreads();
  if (xg != 0 || n >= nb) return;
  const size_t kn = (size_t)k * nb + n;
  const double e = e_nk[kn];
  for (int cc = 0; cc < ncc; ++cc) {
    const int c = c0 + cc, v = c / na, a = c % na;
    double2 lr = make_double2(0, 0);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      lr.x += (double)red[g][nl][cc].x;
      lr.y += (double)red[g][nl][cc].y;
    }
    const double2 ps = psi[((size_t)c * nk + k) * nb + n];
    double2 val = make_double2(lr.x + e * ps.x, lr.y + e * ps.y);
    for (int b = 0; b < na; ++b) {
      double2 ch = chi[a * na + b];
      double2 pb = psi[((size_t)(v * na + b) * nk + k) * nb + n];
      val.x -= ch.x * pb.x - ch.y * pb.y;
      val.y -= ch.x * pb.y + ch.y * pb.x;
    }
    if (np > 0) {
      const double2* cp = srcp + (size_t)v * na * np + (size_t)a * np;
      for (int p = 0; p < np; ++p) {
        double2 ap = a_proj[(size_t)p * nk * nb + kn];
        double2 q = cp[p];
        val.x += ap.x * q.x + ap.y * q.y;
        val.y += ap.x * q.y - ap.y * q.x;
      }
    }
    out[((size_t)c * nk + k) * nb + n] = val;
  }
}

// ---------------------------------------------------------------------------
// short range (Sec. 3.2.2): c[c][p] = sum_{kn} A[p][kn] psi[c][kn];  c' = M c
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) sr_in_kernel(const double2* __restrict__ a_proj,
                                                    const double2* __restrict__ psi,
                                                    double2* __restrict__ src, int nkb, int np) {
  const int p = blockIdx.x, c = blockIdx.y;
  const double2* ap = a_proj + (size_t)p * nkb;
  const double2* pc = psi + (size_t)c * nkb;
  double re = 0, im = 0;
  for (int i = threadIdx.x; i < nkb; i += blockDim.x) {
    double2 a = ap[i], q = pc[i];
    re += a.x * q.x - a.y * q.y;
    im += a.x * q.y + a.y * q.x;
  }
  __shared__ double sre[256], sim[256];
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sre[threadIdx.x] += sre[threadIdx.x + s];
      sim[threadIdx.x] += sim[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) src[(size_t)c * np + p] = make_double2(sre[0], sim[0]);
}

// c'[v][i] = sum_j M[i][j] c[v][j],  i, j over (alpha, p), alpha slow
__global__ void __launch_bounds__(256) sr_couple_kernel(const double2* __restrict__ m,
                                                        const double2* __restrict__ src,
                                                        double2* __restrict__ srcp, int dimm) {
  const int v = blockIdx.x;
  const double2* cv = src + (size_t)v * dimm;
  for (int i = threadIdx.x; i < dimm; i += blockDim.x) {
    double re = 0, im = 0;
    const double2* mr = m + (size_t)i * dimm;
    for (int j = 0; j < dimm; ++j) {
      double2 a = mr[j], q = cv[j];
      re += a.x * q.x - a.y * q.y;
      im += a.x * q.y + a.y * q.x;
    }
    srcp[(size_t)v * dimm + i] = make_double2(re, im);
  }
}

// Split-K projection onto the local basis: block b sums kn in [b*SRK, (b+1)*SRK)
// for up to SRC columns and all Np functions; part[b][c][p].
constexpr int SRK = 64, SRC = 16;
__global__ void __launch_bounds__(256) sr_in_partial(const double2* __restrict__ a_proj,
                                                     const double2* __restrict__ psi,
                                                     double2* __restrict__ part, int nkb, int np, int nc) {
  extern __shared__ __align__(16) unsigned char sr_smem[];
  double2* As = reinterpret_cast<double2*>(sr_smem);   // [np][SRK + 1]
  double2* Ps = As + (size_t)np * (SRK + 1);            // [SRC][SRK + 1]
  const int b = blockIdx.x, c0 = blockIdx.y * SRC;
  const int ncc = nc - c0 < SRC ? nc - c0 : SRC;
  const int k0 = b * SRK;
  for (int e = threadIdx.x; e < np * SRK; e += blockDim.x) {
    const int p = e / SRK, i = e % SRK;
    As[p * (SRK + 1) + i] = (k0 + i < nkb) ? a_proj[(size_t)p * nkb + k0 + i] : make_double2(0, 0);
  }
  for (int e = threadIdx.x; e < ncc * SRK; e += blockDim.x) {
    const int c = e / SRK, i = e % SRK;
    Ps[c * (SRK + 1) + i] = (k0 + i < nkb) ? psi[(size_t)(c0 + c) * nkb + k0 + i] : make_double2(0, 0);
  }
  __syncthreads();
  for (int o = threadIdx.x; o < ncc * np; o += blockDim.x) {
    const int c = o / np, p = o % np;
    double re = 0, im = 0;
#pragma unroll 8
    for (int i = 0; i < SRK; ++i) {
      const double2 a = As[p * (SRK + 1) + i], q = Ps[c * (SRK + 1) + i];
      re += a.x * q.x - a.y * q.y;
      im += a.x * q.y + a.y * q.x;
    }
    part[((size_t)b * nc + c0 + c) * np + p] = make_double2(re, im);
  }
}

// c[o] = sum_b part[b][o]  (fixed order), o over (c, p)
__global__ void sr_reduce(const double2* __restrict__ part, double2* __restrict__ src, int nblk, int nout) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double re = 0, im = 0;
  for (int b = 0; b < nblk; ++b) {
    const double2 t = part[(size_t)b * nout + o];
    re += t.x;
    im += t.y;
  }
  src[o] = make_double2(re, im);
}

// c'[v][i] = sum_j M[i][j] c[v][j]: one warp per row i
__global__ void __launch_bounds__(256) sr_couple_warp(const double2* __restrict__ m, const double2* __restrict__ src,
                                                      double2* __restrict__ srcp, int dimm) {
  const int v = blockIdx.y;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= dimm) return;
  const double2* mr = m + (size_t)i * dimm;
  const double2* cv = src + (size_t)v * dimm;
  double re = 0, im = 0;
  for (int j = lane; j < dimm; j += 32) {
    const double2 a = mr[j], q = cv[j];
    re += a.x * q.x - a.y * q.y;
    im += a.x * q.y + a.y * q.x;
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  if (lane == 0) srcp[(size_t)v * dimm + i] = make_double2(re, im);
}

template <typename T>
bse_status apply_simt(bse_handle* h, const double2* psi, double2* hpsi, int n_vec) {
  typedef typename Cx<T>::type C;
  cudaStream_t st = h->stream;
  const int nc = n_vec * h->na;
  const C* U = (const C*)h->u;
  C* phi = (C*)h->phi;
  constexpr int CCB = 8;   // columns per band->grid pass
  constexpr int CCG = 8;   // columns per grid->band pass
  for (int c0 = 0; c0 < nc; c0 += CCB) {
    dim3 g((unsigned)((h->nx + 63) / 64), (unsigned)h->nk);
    BSE_PROF(h, BSE_K_BAND_TO_GRID, b2g_simt<T, CCB><<<g, 256, 0, st>>>(U, psi, phi, h->nk, h->nx, h->nb, c0,
                                        nc - c0 < CCB ? nc - c0 : CCB, nc));
  }
  {
    int ccn = (int)(sizeof(T) == 8 ? 12288 : 24576) / h->nk;  // ~ <=196 KB of shared memory
    if (ccn > 64) ccn = 64;
    if (ccn < 1) ccn = 1;
    long long ncol = (long long)h->nx * nc;
    size_t sm = (size_t)(48 + (size_t)h->nk * ccn) * sizeof(C);
    cudaFuncSetAttribute(kconv_simt<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    BSE_PROF(h, BSE_K_KCONV, kconv_simt<T><<<(unsigned)((ncol + ccn - 1) / ccn), 256, sm, st>>>(
        phi, (const T*)h->w, h->twiddle, h->nk3[0], h->nk3[1], h->nk3[2], h->nx, nc, ccn));
  }
  for (int c0 = 0; c0 < nc; c0 += CCG) {
    dim3 g((unsigned)((h->nb + 63) / 64), (unsigned)h->nk);
    BSE_PROF(h, BSE_K_GRID_TO_BAND, g2b_simt<T, CCG><<<g, 256, 0, st>>>(U, phi, psi, hpsi, h->e_nk, h->chi, h->a_proj, h->sr_cp,
                                        h->nk, h->nx, h->nb, h->na, h->np, c0,
                                        nc - c0 < CCG ? nc - c0 : CCG, nc));
  }
  return bse_cuda_check(h, cudaGetLastError(), "apply (SIMT)");
}

}  // namespace

bse_status bse_sr_terms(bse_handle* h, const double2* psi, int n_vec) {
  if (h->np <= 0) return BSE_OK;
  cudaStream_t st = h->stream;
  const int nc = n_vec * h->na;
  const int nkb = h->nk * h->nb;
  if (h->sr_part) {
    const int nblk = (nkb + SRK - 1) / SRK;
    dim3 g((unsigned)nblk, (unsigned)((nc + SRC - 1) / SRC));
    const size_t smem = (size_t)(h->np + SRC) * (SRK + 1) * sizeof(double2);
    cudaFuncSetAttribute(sr_in_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    BSE_PROF(h, BSE_K_SR_IN, sr_in_partial<<<g, 256, smem, st>>>(h->a_proj, psi, h->sr_part, nkb, h->np, nc));
    const int nout = nc * h->np;
    BSE_PROF(h, BSE_K_SR_IN, sr_reduce<<<(nout + 255) / 256, 256, 0, st>>>(h->sr_part, h->sr_c, nblk, nout));
  } else {
    dim3 g((unsigned)h->np, (unsigned)nc);
    BSE_PROF(h, BSE_K_SR_IN, sr_in_kernel<<<g, 256, 0, st>>>(h->a_proj, psi, h->sr_c, nkb, h->np));
  }
  const int dimm = h->na * h->np;
  dim3 gc((unsigned)((dimm + 7) / 8), (unsigned)n_vec);
  BSE_PROF(h, BSE_K_SR_COUPLE, sr_couple_warp<<<gc, 256, 0, st>>>(h->m_sr, h->sr_c, h->sr_cp, dimm));
  return bse_cuda_check(h, cudaGetLastError(), "short-range kernels");
}

bse_status bse_apply_device(bse_handle* h, const double2* psi, double2* hpsi, int n_vec) {
  bse_status s = bse_sr_terms(h, psi, n_vec);
  if (s != BSE_OK) return s;
  switch (h->prec) {
    case BSE_PREC_FP64: return apply_simt<double>(h, psi, hpsi, n_vec);
    case BSE_PREC_FP32: return apply_simt<float>(h, psi, hpsi, n_vec);
    case BSE_PREC_SPLIT_BF16: {
      s = bse_tc_band_to_grid(h, psi, n_vec);
      if (s != BSE_OK) return s;
      s = bse_kconv_bf16(h, n_vec);
      if (s != BSE_OK) return s;
      return bse_tc_grid_to_band(h, psi, hpsi, n_vec);
    }
    default: return bse_fail(h, BSE_ERR_UNSUPPORTED, "unknown precision");
  }
}
