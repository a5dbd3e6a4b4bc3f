// H psi on the device: SIMT band<->grid contractions (FP64 and FP32 forms)
// and the short-range projector terms.
//
// Algorithm 1 (Sec. 3.2.1), with the loop over x and alpha turned inside out:
//   band->grid  phi[k][c][x]  = sum_n  U[k][x][n] psi[c][k][n]   (U = e^{ik.x} u)
//   k-conv      phi[k][c][x]  <- F_{R->k} W(x,R) F_{k->R} phi     (k_kconv.cu)
//   grid->band  out[c][k][n]  = sum_x conj(U[k][x][n]) phi[k][c][x]
// with c = v*Na + alpha the column index (vector v, core state alpha).  The
// grid->band kernel also adds E_nk psi - chi psi (Eqs. 3-5) and the short-range
// projection out (Sec. 3.2.2), so one pass writes H psi.
//
// Arithmetic: the FP64 form does everything in FP64.  The reduced-precision
// forms accumulate the short-range projections and the spin-orbit product in
// FP32 (FP64 throughput on this part is a small fraction of FP32) and keep
// E_nk psi and the final sums in FP64.
#include "bse_internal.cuh"

bse_status bse_kconv_inplace(bse_handle* h, int n_vec);

namespace {

template <typename T> struct Cx { typedef typename cvec<T>::type type; };

template <typename C> __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

template <typename C> __device__ __forceinline__ C from_d2(double2 v) {
  C r;
  r.x = v.x;
  r.y = v.y;
  return r;
}
template <typename C> __device__ __forceinline__ C from_d2(float2 v) {
  C r;
  r.x = v.x;
  r.y = v.y;
  return r;
}

// ---------------------------------------------------------------------------
// band -> grid:  phi[k][c0+cc][x] = sum_n U[k][x][n] psi[c0+cc][k][n]
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
      if (cc < ncc) phi[((size_t)k * nc_total + c0 + cc) * nx + x] = acc[i];
    }
  }
}

// ---------------------------------------------------------------------------
// grid -> band + diagonal + spin-orbit + short-range out:
// out[c][k][n] = sum_x conj(U[k][x][n]) phi[k][c][x] + E_kn psi[c][k][n]
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
  __shared__ C Fs[CC][32];
  __shared__ C red[4][64][CC];
  const int t = threadIdx.x, nl = t & 63, xg = t >> 6;
  const int k = blockIdx.y, n = blockIdx.x * 64 + nl;
  C acc[CC];
#pragma unroll
  for (int i = 0; i < CC; ++i) acc[i] = czero<C>();
  const C* Uk = U + (size_t)k * nx * nb;
  for (int x0 = 0; x0 < nx; x0 += 32) {
    for (int e = t; e < 32 * CC; e += 256) {
      int cc = e >> 5, xi = e & 31, x = x0 + xi;
      Fs[cc][xi] = (x < nx && cc < ncc) ? phi[((size_t)k * nc_total + c0 + cc) * nx + x] : czero<C>();
    }
    __syncthreads();
    if (n < nb) {
      for (int xi = xg; xi < 32; xi += 4) {
        int x = x0 + xi;
        if (x < nx) {
          C u = Uk[(size_t)x * nb + n];
#pragma unroll
          for (int cc = 0; cc < CC; ++cc) cmac_conj(acc[cc], u, Fs[cc][xi]);
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
    C lr = czero<C>();
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      lr.x += red[g][nl][cc].x;
      lr.y += red[g][nl][cc].y;
    }
    const double2 ps = psi[((size_t)c * nk + k) * nb + n];
    C rest = czero<C>();   // -chi psi + short-range out, in T
    for (int b = 0; b < na; ++b) {
      const C ch = from_d2<C>(chi[a * na + b]);
      const C pb = from_d2<C>(psi[((size_t)(v * na + b) * nk + k) * nb + n]);
      rest.x -= ch.x * pb.x - ch.y * pb.y;
      rest.y -= ch.x * pb.y + ch.y * pb.x;
    }
    if (np > 0) {
      const double2* cp = srcp + (size_t)v * na * np + (size_t)a * np;
      for (int p = 0; p < np; ++p) {
        const C ap = from_d2<C>(a_proj[(size_t)p * nk * nb + kn]);
        const C q = from_d2<C>(cp[p]);
        rest.x += ap.x * q.x + ap.y * q.y;
        rest.y += ap.x * q.y - ap.y * q.x;
      }
    }
    out[((size_t)c * nk + k) * nb + n] =
        make_double2((double)lr.x + (double)rest.x + e * ps.x, (double)lr.y + (double)rest.y + e * ps.y);
  }
}

// ---------------------------------------------------------------------------
// short range (Sec. 3.2.2): c[c][p] = sum_{kn} A[p][kn] psi[c][kn];  c' = M c
// Split-K projection: block b sums kn in [b*SRK*srt, (b+1)*SRK*srt) in srt
// shared-memory tiles of SRK for up to SRC columns and all Np functions,
// accumulating in registers; part[b][c][p] (accumulated in T).  srt is as
// large as keeps about two blocks per SM busy: longer blocks mean fewer
// partials for the FP64 reduction (sr_reduce).
// ---------------------------------------------------------------------------
constexpr int SRK = 64, SRC = 16, SRT_MAX = 8, SRO = 4;   // SRO: outputs per thread (SRC * Np <= 16 * 64 = 256 * SRO)
template <typename T, typename AT, typename PT>
__global__ void __launch_bounds__(256) sr_in_partial(const AT* __restrict__ a_proj,
                                                     const PT* __restrict__ psi,
                                                     double2* __restrict__ part, int nkb, int np, int nc,
                                                     int srt) {
  typedef typename Cx<T>::type C;
  extern __shared__ __align__(16) unsigned char sr_smem[];
  C* As = reinterpret_cast<C*>(sr_smem);   // [np][SRK + 1]
  C* Ps = As + (size_t)np * (SRK + 1);     // [SRC][SRK + 1]
  const int b = blockIdx.x, c0 = blockIdx.y * SRC;
  const int ncc = nc - c0 < SRC ? nc - c0 : SRC;
  C acc[SRO];
#pragma unroll
  for (int r = 0; r < SRO; ++r) acc[r] = czero<C>();
  for (int tile = 0; tile < srt; ++tile) {
    const int k0 = (b * srt + tile) * SRK;
    if (k0 >= nkb) break;   // uniform across the block
    for (int e = threadIdx.x; e < np * SRK; e += blockDim.x) {
      const int p = e / SRK, i = e % SRK;
      As[p * (SRK + 1) + i] = (k0 + i < nkb) ? from_d2<C>(a_proj[(size_t)p * nkb + k0 + i]) : czero<C>();
    }
    for (int e = threadIdx.x; e < ncc * SRK; e += blockDim.x) {
      const int c = e / SRK, i = e % SRK;
      Ps[c * (SRK + 1) + i] = (k0 + i < nkb) ? from_d2<C>(psi[(size_t)(c0 + c) * nkb + k0 + i]) : czero<C>();
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SRO; ++r) {
      const int o = threadIdx.x + r * blockDim.x;
      if (o < ncc * np) {
        const int c = o / np, p = o % np;
#pragma unroll 8
        for (int i = 0; i < SRK; ++i) cmac(acc[r], As[p * (SRK + 1) + i], Ps[c * (SRK + 1) + i]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < SRO; ++r) {
    const int o = threadIdx.x + r * blockDim.x;
    if (o < ncc * np) {
      const int c = o / np, p = o % np;
      part[((size_t)b * nc + c0 + c) * np + p] = make_double2((double)acc[r].x, (double)acc[r].y);
    }
  }
}

// c[o] = sum_b part[b][o], one block of 128 threads per output o (fixed order)
__global__ void __launch_bounds__(128) sr_reduce(const double2* __restrict__ part, double2* __restrict__ src,
                                                 int nblk, int nout) {
  const int o = blockIdx.x;
  double re = 0, im = 0;
  for (int b = threadIdx.x; b < nblk; b += 128) {
    const double2 t = part[(size_t)b * nout + o];
    re += t.x;
    im += t.y;
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  __shared__ double sr[4], si[4];
  if ((threadIdx.x & 31) == 0) {
    sr[threadIdx.x >> 5] = re;
    si[threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) src[o] = make_double2(sr[0] + sr[1] + sr[2] + sr[3], si[0] + si[1] + si[2] + si[3]);
}

// c'[v][i] = sum_j M[i][j] c[v][j]: one warp per row i (FP64)
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
    BSE_PROF(h, BSE_K_BAND_TO_GRID,
             b2g_simt<T, CCB><<<g, 256, 0, st>>>(U, psi, phi, h->nk, h->nx, h->nb, c0,
                                                 nc - c0 < CCB ? nc - c0 : CCB, nc));
  }
  bse_status s = bse_kconv_inplace(h, n_vec);
  if (s != BSE_OK) return s;
  if (h->np > 0) cudaStreamWaitEvent(st, h->ev_join, 0);   // short-range c' ready
  for (int c0 = 0; c0 < nc; c0 += CCG) {
    dim3 g((unsigned)((h->nb + 63) / 64), (unsigned)h->nk);
    BSE_PROF(h, BSE_K_GRID_TO_BAND,
             g2b_simt<T, CCG><<<g, 256, 0, st>>>(U, phi, psi, hpsi, h->e_nk, h->chi, h->a_proj, h->sr_cp, h->nk,
                                                 h->nx, h->nb, h->na, h->np, c0, nc - c0 < CCG ? nc - c0 : CCG,
                                                 nc));
  }
  return bse_cuda_check(h, cudaGetLastError(), "apply (SIMT)");
}

template <typename T>
void launch_sr_in(bse_handle* h, const double2* psi, int nc, int nkb, int nblk, int srt) {
  typedef typename Cx<T>::type C;
  dim3 g((unsigned)nblk, (unsigned)((nc + SRC - 1) / SRC));
  const size_t smem = (size_t)(h->np + SRC) * (SRK + 1) * sizeof(C);
  if (h->a_proj_f && h->psi_f && h->prec == BSE_PREC_SPLIT_BF16) {
    // tensor-core form: FP32 projectors and the FP32 psi of the operand pass
    cudaFuncSetAttribute(sr_in_partial<T, float2, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    BSE_PROF(h, BSE_K_SR_IN,
             (sr_in_partial<T, float2, float2><<<g, 256, smem, h->side>>>(h->a_proj_f, h->psi_f, h->sr_part, nkb,
                                                                           h->np, nc, srt)));
  } else if (h->a_proj_f) {   // FP32 form: FP32 copy of the projectors (half the bytes)
    cudaFuncSetAttribute(sr_in_partial<T, float2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    BSE_PROF(h, BSE_K_SR_IN,
             (sr_in_partial<T, float2, double2><<<g, 256, smem, h->side>>>(h->a_proj_f, psi, h->sr_part, nkb, h->np,
                                                                            nc, srt)));
  } else {
    cudaFuncSetAttribute(sr_in_partial<T, double2, double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    BSE_PROF(h, BSE_K_SR_IN,
             (sr_in_partial<T, double2, double2><<<g, 256, smem, h->side>>>(h->a_proj, psi, h->sr_part, nkb, h->np,
                                                                             nc, srt)));
  }
}

}  // namespace

// Short-range coefficients c' = M (A (x) I) psi on the side stream, forked
// from and joined back (ev_join) to the handle's stream; the consumer of
// sr_cp waits on ev_join.
bse_status bse_sr_terms(bse_handle* h, const double2* psi, int n_vec) {
  if (h->np <= 0) return BSE_OK;
  cudaStream_t st = h->side;
  cudaEventRecord(h->ev_fork, h->stream);
  cudaStreamWaitEvent(st, h->ev_fork, 0);
  h->cur = st;
  const int nc = n_vec * h->na;
  const int nkb = h->nk * h->nb;
  const int tiles = (nkb + SRK - 1) / SRK;
  const int cgroups = (nc + SRC - 1) / SRC;
  int srt = tiles * cgroups / 304;   // keep >= ~2 blocks per SM of 152
  srt = srt < 1 ? 1 : (srt > SRT_MAX ? SRT_MAX : srt);
  const int nblk = (tiles + srt - 1) / srt;
  if (h->prec == BSE_PREC_FP64)
    launch_sr_in<double>(h, psi, nc, nkb, nblk, srt);
  else
    launch_sr_in<float>(h, psi, nc, nkb, nblk, srt);
  const int nout = nc * h->np;
  BSE_PROF(h, BSE_K_SR_IN, sr_reduce<<<nout, 128, 0, st>>>(h->sr_part, h->sr_c, nblk, nout));
  const int dimm = h->na * h->np;
  dim3 gc((unsigned)((dimm + 7) / 8), (unsigned)n_vec);
  BSE_PROF(h, BSE_K_SR_COUPLE, sr_couple_warp<<<gc, 256, 0, st>>>(h->m_sr, h->sr_c, h->sr_cp, dimm));
  h->cur = nullptr;
  cudaEventRecord(h->ev_join, st);
  return bse_cuda_check(h, cudaGetLastError(), "short-range kernels");
}

bool bse_apply_fuses_dot(const bse_handle* h) { return h->prec == BSE_PREC_SPLIT_BF16; }

bse_status bse_apply_device(bse_handle* h, const double2* psi, double2* hpsi, int n_vec, const bse_dotfuse* fuse) {
  bse_status s;
  switch (h->prec) {
    case BSE_PREC_FP64:
      if (fuse) return BSE_ERR_UNSUPPORTED;
      s = bse_sr_terms(h, psi, n_vec);
      if (s != BSE_OK) return s;
      return apply_simt<double>(h, psi, hpsi, n_vec);
    case BSE_PREC_FP32:
      if (fuse) return BSE_ERR_UNSUPPORTED;
      s = bse_sr_terms(h, psi, n_vec);
      if (s != BSE_OK) return s;
      return apply_simt<float>(h, psi, hpsi, n_vec);
    case BSE_PREC_SPLIT_BF16: {
      // the operand pass runs first: it may rescale psi in place (lazy Haydock
      // normalisation), and the short-range side stream forks after it
      if (!(fuse && fuse->operand_ready)) {
        s = bse_tc_prep(h, psi, n_vec, fuse);
        if (s != BSE_OK) return s;
      }
      s = bse_sr_terms(h, psi, n_vec);
      if (s != BSE_OK) return s;
      // one pass over U (a handle running alone; sizes the one-pass kernel takes)
      if (h->sched == BSE_SCHED_ONE_PASS && !h->concurrent && n_vec <= h->op_max_vec)
        return bse_tc_apply_onepass(h, psi, hpsi, n_vec, fuse, h->np > 0);
      if (h->slabs > 1) return bse_tc_apply_slabbed(h, psi, hpsi, n_vec, fuse, h->np > 0);
      s = bse_tc_band_to_grid(h, n_vec);
      if (s != BSE_OK) return s;
      s = bse_kconv_bf16(h, n_vec);
      if (s != BSE_OK) return s;
      return bse_tc_grid_to_band(h, psi, hpsi, n_vec, fuse, h->np > 0);
    }
    default: return bse_fail(h, BSE_ERR_UNSUPPORTED, "unknown precision");
  }
}
