// Krylov drivers on the device, all recursion arithmetic in FP64:
//   Haydock / Lanczos recursion (Sec. 3.2, Eq. 9) with optional classical
//   Gram-Schmidt re-orthogonalisation, the continued-fraction loss function
//   (Eqs. 1-2), and restarted right-preconditioned GMRES for (H - z) x = b.
// Reductions are two-stage and deterministic: fixed per-block partial sums,
// then one block per vector sums the partials in a fixed tree order.
#include "bse_internal.cuh"

#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

namespace {

constexpr int RB = 256;      // threads per reduction block
constexpr int NBLK = 296;    // partial-sum blocks per vector (2 x 148)

// Blocks per vector of a norm over nv vectors of length N: about 4096
// elements per block, but at least ~608 blocks in all (four per SM of 152),
// at most NBLK -- so that many short vectors (GMRES over many shifts) do not
// pay a block reduction per few dozen elements.
inline int norm_blocks(long long N, int nv) {
  long long nb = (N + 4095) / 4096;
  const long long fill = (608 + nv - 1) / nv;
  if (nb < fill) nb = fill;
  if (nb > NBLK) nb = NBLK;
  const long long cap = (N + 255) / 256;
  if (nb > cap) nb = cap;
  return (int)(nb < 1 ? 1 : nb);
}
constexpr int UBLK = 296;    // blocks per vector of the Haydock update (its |w|^2 partials are reduced again by every block of the next operand pass)

enum { ST_BREAKDOWN = 1, ST_NAN = 2, ST_TIMEOUT = BSE_ST_TIMEOUT };

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// block-wide sum of a double2 (RB threads)
__device__ double2 block_sum2(double2 v) {
  __shared__ double sx[RB], sy[RB];
  sx[threadIdx.x] = v.x;
  sy[threadIdx.x] = v.y;
  __syncthreads();
  for (int s = RB / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sx[threadIdx.x] += sx[threadIdx.x + s];
      sy[threadIdx.x] += sy[threadIdx.x + s];
    }
    __syncthreads();
  }
  double2 r = make_double2(sx[0], sy[0]);
  __syncthreads();
  return r;
}

// partial[v][blk] = sum over the block's slice of conj(x) * y   (y == nullptr: |x|^2)
// x, y of vector v start at v * xs, v * ys (xs = ys = N for packed batches).
__global__ void __launch_bounds__(RB) dot_partial_s(const double2* __restrict__ x, long long xs,
                                                    const double2* __restrict__ y, long long ys,
                                                    long long N, double2* __restrict__ partial) {
  const int v = blockIdx.y;
  const double2* xv = x + (size_t)v * xs;
  const double2* yv = y ? y + (size_t)v * ys : nullptr;
  double2 acc = make_double2(0, 0);
  for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < N; i += (long long)gridDim.x * RB) {
    double2 a = xv[i];
    if (yv) {
      double2 b = yv[i];
      acc.x += a.x * b.x + a.y * b.y;
      acc.y += a.x * b.y - a.y * b.x;
    } else {
      acc.x += a.x * a.x + a.y * a.y;
    }
  }
  double2 s = block_sum2(acc);
  if (threadIdx.x == 0) partial[(size_t)v * gridDim.x + blockIdx.x] = s;
}

// sum of partial[v][0..nblk) in a fixed order
__device__ double2 sum_partials(const double2* partial, int v, int nblk) {
  double2 acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < nblk; i += RB) acc = cadd(acc, partial[(size_t)v * nblk + i]);
  return block_sum2(acc);
}

// ---------------------------------------------------------------------------
// Haydock
// ---------------------------------------------------------------------------
// b_0 = |b|; active = (b_0 > 0 and finite)
__global__ void __launch_bounds__(RB) hay_init_finalize(const double2* partial, int nblk, double* bco,
                                                        int n_steps, int* active, int* status) {
  const int v = blockIdx.x;
  double2 s = sum_partials(partial, v, nblk);
  if (threadIdx.x == 0) {
    double b0 = sqrt(s.x);
    bco[(size_t)v * (n_steps + 1)] = b0;
    int ok = isfinite(b0) && b0 > 0;
    active[v] = ok;
    if (!isfinite(b0)) atomicOr(status, ST_NAN);
  }
}

// y[v] = x[v] / bco[v][col]   (only active vectors)
__global__ void hay_scale(const double2* __restrict__ x, double2* __restrict__ y, long long N,
                          const double* __restrict__ bco, int col, int stride, const int* __restrict__ active) {
  const int v = blockIdx.y;
  if (!active[v]) return;
  const double inv = 1.0 / bco[(size_t)v * stride + col];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double2 a = x[(size_t)v * N + i];
    y[(size_t)v * N + i] = make_double2(a.x * inv, a.y * inv);
  }
}

// a[v][i] = Re <v_i | w>
__global__ void __launch_bounds__(RB) hay_a_finalize(const double2* partial, int nblk, double* a,
                                                     int n_steps, int i, const int* active, int* status) {
  const int v = blockIdx.x;
  double2 s = sum_partials(partial, v, nblk);
  if (threadIdx.x == 0 && active[v]) {
    a[(size_t)v * n_steps + i] = s.x;
    if (!isfinite(s.x)) atomicOr(status, ST_NAN);
  }
}

// w -= a_i v_i + b_i v_{i-1};  partial |w|^2
__global__ void __launch_bounds__(RB) hay_update(double2* __restrict__ w, const double2* __restrict__ vc,
                                                 const double2* __restrict__ vp, long long N,
                                                 const double* __restrict__ a, const double* __restrict__ bco,
                                                 int n_steps, int i, const int* __restrict__ active,
                                                 double2* __restrict__ partial) {
  const int v = blockIdx.y;
  double2 acc = make_double2(0, 0);
  if (active[v]) {
    const double ai = a[(size_t)v * n_steps + i];
    const double bi = i >= 1 ? bco[(size_t)v * (n_steps + 1) + i] : 0.0;
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < N; e += (long long)gridDim.x * RB) {
      size_t o = (size_t)v * N + e;
      double2 ww = w[o], c = vc[o];
      ww.x -= ai * c.x;
      ww.y -= ai * c.y;
      if (i >= 1) {
        double2 p = vp[o];
        ww.x -= bi * p.x;
        ww.y -= bi * p.y;
      }
      w[o] = ww;
      acc.x += ww.x * ww.x + ww.y * ww.y;
    }
  }
  double2 s = block_sum2(acc);
  if (threadIdx.x == 0) partial[(size_t)v * gridDim.x + blockIdx.x] = s;
}

// b_{i+1} = |w|; breakdown test; steps_done = i + 1
__global__ void __launch_bounds__(RB) hay_b_finalize(const double2* partial, int nblk, const double* a,
                                                     double* bco, int n_steps, int i, int* active,
                                                     int* steps, int* status) {
  const int v = blockIdx.x;
  double2 s = sum_partials(partial, v, nblk);
  if (threadIdx.x == 0 && active[v]) {
    double bn = sqrt(s.x);
    double ai = a[(size_t)v * n_steps + i];
    bco[(size_t)v * (n_steps + 1) + i + 1] = bn;
    steps[v] = i + 1;
    if (!isfinite(bn) || !isfinite(ai)) {
      active[v] = 0;
      atomicOr(status, ST_NAN);
    } else if (bn <= 1e-12 * fmax(1.0, fabs(ai))) {
      active[v] = 0;
      atomicOr(status, ST_BREAKDOWN);
    }
  }
}

// coef[v][j] = sum of partials (grid (nj, nv)); optionally accumulated into hacc
__global__ void __launch_bounds__(RB) gs_dot_finalize(const double2* partial, int nblk, double2* coef,
                                                      int coef_stride, double2* hacc, int hacc_stride) {
  const int j = blockIdx.x, v = blockIdx.y;
  double2 acc = make_double2(0, 0);
  const double2* p = partial + ((size_t)v * gridDim.x + j) * nblk;
  for (int i = threadIdx.x; i < nblk; i += RB) acc = cadd(acc, p[i]);
  double2 s = block_sum2(acc);
  if (threadIdx.x == 0) {
    coef[(size_t)v * coef_stride + j] = s;
    if (hacc) {
      double2 o = hacc[(size_t)v * hacc_stride + j];
      hacc[(size_t)v * hacc_stride + j] = cadd(o, s);
    }
  }
}

// w[v] -= sum_j coef[v][j] basis[v][j]   (only where mask[v] != 0, mask may be null)
__global__ void gs_subtract(const double2* __restrict__ basis, long long bstride, double2* __restrict__ w,
                            long long N, const double2* __restrict__ coef, int coef_stride, int nj,
                            const int* __restrict__ mask) {
  const int v = blockIdx.y;
  if (mask && !mask[v]) return;
  const double2* bv = basis + (size_t)v * bstride;
  const double2* cv = coef + (size_t)v * coef_stride;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    double2 acc = w[(size_t)v * N + e];
    for (int j = 0; j < nj; ++j) {
      double2 c = cv[j], b = bv[(size_t)j * N + e];
      acc.x -= c.x * b.x - c.y * b.y;
      acc.y -= c.x * b.y + c.y * b.x;
    }
    w[(size_t)v * N + e] = acc;
  }
}

__global__ void copy_vecs(const double2* __restrict__ src, double2* __restrict__ dst, long long N,
                          long long dst_stride) {
  const int v = blockIdx.y;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x)
    dst[(size_t)v * dst_stride + e] = src[(size_t)v * N + e];
}

template <typename T>
bse_status dalloc(bse_handle* h, T** p, size_t bytes, const char* what) {
  if (cudaMalloc((void**)p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return bse_fail(h, BSE_ERR_OOM, std::string("cudaMalloc failed for ") + what);
  }
  return BSE_OK;
}

struct Freer {
  std::vector<void*> ptrs;
  ~Freer() {
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
  template <typename T> void add(T* p) { ptrs.push_back((void*)p); }
};

#define TRY(x)                   \
  do {                           \
    bse_status _s = (x);         \
    if (_s != BSE_OK) return _s; \
  } while (0)

// grid-stride launch shape for elementwise kernels over N per vector
inline dim3 ew_grid(long long N, int nv) {
  long long b = (N + 255) / 256;
  if (b > 1184) b = 1184;
  return dim3((unsigned)b, (unsigned)nv);
}

bse_status apply_chunked(bse_handle* h, const double2* in, double2* out, int n_vec) {
  for (int v0 = 0; v0 < n_vec; v0 += h->max_vec) {
    int nv = n_vec - v0 < h->max_vec ? n_vec - v0 : h->max_vec;
    TRY(bse_apply_device(h, in + (size_t)v0 * h->N, out + (size_t)v0 * h->N, nv));
  }
  return BSE_OK;
}

// CGS2: for pass in 0,1: coef = basis^H w; w -= basis coef; hacc += coef.
// Gram-Schmidt projections <basis_j|w> for JB basis vectors at a time: w is
// read once per group of JB (not once per basis vector).  partial[v][j][blk].
constexpr int GS_JB = 8;
constexpr int GS_BLK = 64;   // blocks per vector of the multi-dot: long loops, few partials to reduce
__global__ void __launch_bounds__(RB) gs_dot_multi(const double2* __restrict__ basis, long long bstride,
                                                   const double2* __restrict__ w, long long N, int nj,
                                                   double2* __restrict__ partial, const int* __restrict__ mask) {
  const int v = blockIdx.y;
  const bool on = !mask || mask[v];
  const double2* bv = basis + (size_t)v * bstride;
  const double2* wv = w + (size_t)v * N;
  __shared__ double2 sred[RB / 32][GS_JB];
  for (int j0 = 0; j0 < nj; j0 += GS_JB) {
    double2 acc[GS_JB];
#pragma unroll
    for (int q = 0; q < GS_JB; ++q) acc[q] = make_double2(0, 0);
    if (on) {
      for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < N; e += (long long)gridDim.x * RB) {
        const double2 b = wv[e];
#pragma unroll
        for (int q = 0; q < GS_JB; ++q) {
          if (j0 + q < nj) {
            const double2 a = bv[(size_t)(j0 + q) * N + e];
            acc[q].x += a.x * b.x + a.y * b.y;
            acc[q].y += a.x * b.y - a.y * b.x;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < GS_JB; ++q) {
      for (int off = 16; off > 0; off >>= 1) {
        acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, off);
        acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, off);
      }
      if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5][q] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < GS_JB && j0 + threadIdx.x < nj) {
      double2 s = make_double2(0, 0);
      for (int wq = 0; wq < RB / 32; ++wq) s = cadd(s, sred[wq][threadIdx.x]);
      partial[((size_t)v * nj + j0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

bse_status cgs2(bse_handle* h, const double2* basis, long long bstride, double2* w, int nv, int nj,
                double2* partial, double2* coef, int coef_stride, double2* hacc, int hacc_stride,
                const int* mask) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  for (int pass = 0; pass < 2; ++pass) {
    BSE_PROF(h, BSE_K_RECURSION, gs_dot_multi<<<dim3(GS_BLK, nv), RB, 0, st>>>(basis, bstride, w, N, nj, partial, mask));
    BSE_PROF(h, BSE_K_RECURSION, gs_dot_finalize<<<dim3(nj, nv), RB, 0, st>>>(partial, GS_BLK, coef, coef_stride, hacc, hacc_stride));
    BSE_PROF(h, BSE_K_RECURSION, gs_subtract<<<ew_grid(N, nv), 256, 0, st>>>(basis, bstride, w, N, coef, coef_stride, nj, mask));
  }
  return BSE_OK;
}

// DGKS test after one classical Gram-Schmidt pass: with s_after = |w|^2 (from
// partial sums) and s_proj = sum_j |h_j|^2 of the coefficients just removed,
// |w_before|^2 = s_after + s_proj, and a second pass is needed where more than
// half of |w|^2 was removed (|w_after| < |w_before| / sqrt 2, i.e. s_after < s_proj).
__global__ void __launch_bounds__(RB) gs_dgks_mask(const double2* __restrict__ partial, int nblk,
                                                   const double2* __restrict__ coef, int coef_stride, int nj,
                                                   const int* __restrict__ mask, int* __restrict__ mask2) {
  const int v = blockIdx.x;
  const double2 s = sum_partials(partial, v, nblk);
  if (threadIdx.x == 0) {
    double proj = 0.0;
    for (int j = 0; j < nj; ++j) {
      const double2 c = coef[(size_t)v * coef_stride + j];
      proj += c.x * c.x + c.y * c.y;
    }
    const int on = mask ? mask[v] : 1;
    mask2[v] = on && !(s.x >= proj);   // NaN also takes the second pass
  }
}

// Classical Gram-Schmidt with the DGKS criterion: one pass, and a second only
// for the systems whose first pass cancelled more than half of |w|^2.
bse_status cgs_dgks(bse_handle* h, const double2* basis, long long bstride, double2* w, int nv, int nj,
                    double2* partial, double2* coef, int coef_stride, double2* hacc, int hacc_stride,
                    const int* mask, int* mask2) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  BSE_PROF(h, BSE_K_RECURSION, gs_dot_multi<<<dim3(GS_BLK, nv), RB, 0, st>>>(basis, bstride, w, N, nj, partial, mask));
  BSE_PROF(h, BSE_K_RECURSION, gs_dot_finalize<<<dim3(nj, nv), RB, 0, st>>>(partial, GS_BLK, coef, coef_stride, hacc, hacc_stride));
  BSE_PROF(h, BSE_K_RECURSION, gs_subtract<<<ew_grid(N, nv), 256, 0, st>>>(basis, bstride, w, N, coef, coef_stride, nj, mask));
  const int nbn = norm_blocks(N, nv);
  BSE_PROF(h, BSE_K_RECURSION, dot_partial_s<<<dim3(nbn, nv), RB, 0, st>>>(w, N, nullptr, 0, N, partial));
  BSE_PROF(h, BSE_K_RECURSION, gs_dgks_mask<<<nv, RB, 0, st>>>(partial, nbn, coef, coef_stride, nj, mask, mask2));
  BSE_PROF(h, BSE_K_RECURSION, gs_dot_multi<<<dim3(GS_BLK, nv), RB, 0, st>>>(basis, bstride, w, N, nj, partial, mask2));
  BSE_PROF(h, BSE_K_RECURSION, gs_dot_finalize<<<dim3(nj, nv), RB, 0, st>>>(partial, GS_BLK, coef, coef_stride, hacc, hacc_stride));
  BSE_PROF(h, BSE_K_RECURSION, gs_subtract<<<ew_grid(N, nv), 256, 0, st>>>(basis, bstride, w, N, coef, coef_stride, nj, mask2));
  return BSE_OK;
}

// ---------------------------------------------------------------------------
// continued fraction  (Eqs. 1-2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 csqrt_(double2 a) {
  double r = hypot(a.x, a.y);
  double re = sqrt(fmax(0.5 * (r + a.x), 0.0));
  double im = sqrt(fmax(0.5 * (r - a.x), 0.0));
  return make_double2(re, a.y < 0 ? -im : im);
}

__global__ void cf_kernel(const double* __restrict__ a, const double* __restrict__ bco,
                          const int* __restrict__ steps, int n_stride, const double* __restrict__ omega,
                          int n_omega, double gamma, int terminator, double* __restrict__ sigma) {
  const int v = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_omega) return;
  const double* av = a + (size_t)v * n_stride;
  const double* bv = bco + (size_t)v * (n_stride + 1);
  const int n = min(steps[v], n_stride);   // a row holds n_stride coefficients
  if (n <= 0) {
    sigma[(size_t)v * n_omega + j] = 0.0;
    return;
  }
  const double2 z = make_double2(omega[j], gamma);
  double2 t = make_double2(0, 0);
  if (terminator && bv[n] > 0) {
    const double binf = bv[n], b2 = binf * binf;
    double2 zz = make_double2(z.x - av[n - 1], z.y);
    double2 disc = make_double2(zz.x * zz.x - zz.y * zz.y - 4 * b2, 2 * zz.x * zz.y);
    double2 r = csqrt_(disc);
    double2 g1 = make_double2((zz.x - r.x) / (2 * b2), (zz.y - r.y) / (2 * b2));
    double2 g2 = make_double2((zz.x + r.x) / (2 * b2), (zz.y + r.y) / (2 * b2));
    double2 g = g1.y <= 0 ? g1 : g2;
    t = make_double2(b2 * g.x, b2 * g.y);
  }
  double2 d = make_double2(z.x - av[n - 1] - t.x, z.y - t.y);
  for (int i = n - 2; i >= 0; --i) {
    double bb = bv[i + 1] * bv[i + 1];
    double2 q = cdiv(make_double2(bb, 0), d);
    d = make_double2(z.x - av[i] - q.x, z.y - q.y);
  }
  double2 g = cdiv(make_double2(1, 0), d);
  sigma[(size_t)v * n_omega + j] = -(bv[0] * bv[0]) / M_PI * g.y;
}

// ---------------------------------------------------------------------------
// GMRES helpers.  Hessenberg per system stored column-major: Hs[v][j][i] =
// H(i, j), (m+1) rows per column, so the Gram-Schmidt coefficients of column j
// accumulate into a contiguous slice.
// ---------------------------------------------------------------------------
// r = b - (W - z x) = b - W + z x   (W = H x); r written to V_0 of each system
__global__ void gm_residual(const double2* __restrict__ b, const double2* __restrict__ W,
                            const double2* __restrict__ x, const double2* __restrict__ z,
                            double2* __restrict__ V, long long vstride, long long N, int first) {
  const int v = blockIdx.y;
  const double2 zv = z[v];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    size_t o = (size_t)v * N + e;
    double2 bb = b[e];
    if (first) {
      V[(size_t)v * vstride + e] = bb;
    } else {
      double2 xx = x[o], ww = W[o];
      V[(size_t)v * vstride + e] =
          make_double2(bb.x - ww.x + zv.x * xx.x - zv.y * xx.y, bb.y - ww.y + zv.x * xx.y + zv.y * xx.x);
    }
  }
}

// beta = |r|, rel = beta/|b|; active = rel > rtol && iters < max_iter; g = [beta, 0...]
__global__ void __launch_bounds__(RB) gm_beta(const double2* partial, int nblk, double bnorm, double rtol,
                                              int max_iter, const int* iters, double* beta, double* rel,
                                              int* active, double2* g, int m) {
  const int v = blockIdx.x;
  double2 s = sum_partials(partial, v, nblk);
  if (threadIdx.x == 0) {
    double bt = sqrt(s.x);
    beta[v] = bt;
    rel[v] = bt / bnorm;
    active[v] = (bt / bnorm > rtol) && (iters[v] < max_iter) && isfinite(bt);
    for (int i = 0; i <= m; ++i) g[(size_t)v * (m + 1) + i] = make_double2(i == 0 ? bt : 0.0, 0.0);
  }
}

// compact form for the still-active systems: slot s holds system idx[s]
// T[s] = P V_j[idx[s]]
__global__ void gm_precond_c(const double2* __restrict__ V, long long vstride, double2* __restrict__ T, long long N,
                             const double* __restrict__ d, const double2* __restrict__ z, int jacobi,
                             const int* __restrict__ idx) {
  const int s = blockIdx.y, v = idx[s];
  const double2 zv = z[v];
  const double2* vv = V + (size_t)v * vstride;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    double2 a = vv[e];
    if (jacobi) a = cdiv(a, make_double2(d[e] - zv.x, -zv.y));
    T[(size_t)s * N + e] = a;
  }
}

// W[idx[s]] = Wc[s] - z[idx[s]] T[s]
__global__ void gm_scatter_shift(const double2* __restrict__ Wc, const double2* __restrict__ T,
                                 const double2* __restrict__ z, double2* __restrict__ W, long long N,
                                 const int* __restrict__ idx) {
  const int s = blockIdx.y, v = idx[s];
  const double2 zv = z[v];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    const double2 t = T[(size_t)s * N + e], w = Wc[(size_t)s * N + e];
    W[(size_t)v * N + e] = make_double2(w.x - (zv.x * t.x - zv.y * t.y), w.y - (zv.x * t.y + zv.y * t.x));
  }
}

#define HS(H, i, j) (H)[(size_t)(j) * (m + 1) + (i)]

// H(j+1, j) = |w|; Givens update of column j; estimated residual; iteration count.
__global__ void __launch_bounds__(RB) gm_givens(const double2* partial, int nblk, double2* Hs, double* cs,
                                                double2* sn, double2* g, double* hnorm, int m, int j,
                                                double bnorm, double rtol, int max_iter, int* active,
                                                int* iters, int* jdone, double* est) {
  const int v = blockIdx.x;
  double2 s = sum_partials(partial, v, nblk);
  if (threadIdx.x != 0 || !active[v]) return;
  double hn = sqrt(s.x);
  hnorm[v] = hn;
  double2* H = Hs + (size_t)v * (m + 1) * m;
  double* c = cs + (size_t)v * m;
  double2* sv = sn + (size_t)v * m;
  double2* gv = g + (size_t)v * (m + 1);
  HS(H, j + 1, j) = make_double2(hn, 0);
  for (int i = 0; i < j; ++i) {
    double2 h0 = HS(H, i, j), h1 = HS(H, i + 1, j);
    double2 si = sv[i];
    // t1 = c h0 + s h1 ; t2 = -conj(s) h0 + c h1
    double2 t1 = make_double2(c[i] * h0.x + si.x * h1.x - si.y * h1.y, c[i] * h0.y + si.x * h1.y + si.y * h1.x);
    double2 t2 = make_double2(-(si.x * h0.x + si.y * h0.y) + c[i] * h1.x, -(si.x * h0.y - si.y * h0.x) + c[i] * h1.y);
    HS(H, i, j) = t1;
    HS(H, i + 1, j) = t2;
  }
  double2 aa = HS(H, j, j), bb = HS(H, j + 1, j);
  double na_ = hypot(aa.x, aa.y), nb_ = hypot(bb.x, bb.y);
  double rr = hypot(na_, nb_);
  if (na_ == 0.0) {
    c[j] = 0.0;
    sv[j] = make_double2(1, 0);
    HS(H, j, j) = bb;
  } else {
    double2 ph = make_double2(aa.x / na_, aa.y / na_);
    c[j] = na_ / rr;
    sv[j] = make_double2((ph.x * bb.x + ph.y * bb.y) / rr, (ph.y * bb.x - ph.x * bb.y) / rr);  // ph conj(bb)/rr
    HS(H, j, j) = make_double2(ph.x * rr, ph.y * rr);
  }
  HS(H, j + 1, j) = make_double2(0, 0);
  double2 gj = gv[j], sj = sv[j];
  gv[j + 1] = make_double2(-(sj.x * gj.x + sj.y * gj.y), -(sj.x * gj.y - sj.y * gj.x));  // -conj(s) g_j
  gv[j] = make_double2(c[j] * gj.x, c[j] * gj.y);
  iters[v] += 1;
  jdone[v] = j + 1;
  double e = hypot(gv[j + 1].x, gv[j + 1].y) / bnorm;
  est[v] = e;
  if (e <= rtol || iters[v] >= max_iter || hn == 0.0 || !isfinite(e)) active[v] = 0;
}

// V_{j+1} = w / |w| for systems still active after column j
__global__ void gm_next(const double2* w, long long wstride, double2* V, long long vstride, long long N,
                        const double* __restrict__ hnorm, const int* __restrict__ mask) {
  const int v = blockIdx.y;
  if (!mask[v] || !(hnorm[v] > 0)) return;
  const double inv = 1.0 / hnorm[v];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    double2 a = w[(size_t)v * wstride + e];
    V[(size_t)v * vstride + e] = make_double2(a.x * inv, a.y * inv);
  }
}

// back substitution y = R^{-1} g over the system's own jdone columns
__global__ void gm_solve(const double2* Hs, const double2* g, double2* y, const int* jdone, int m, int nz) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nz) return;
  const double2* H = Hs + (size_t)v * (m + 1) * m;
  const double2* gv = g + (size_t)v * (m + 1);
  double2* yv = y + (size_t)v * m;
  const int nj = jdone[v];
  for (int i = nj - 1; i >= 0; --i) {
    double2 acc = gv[i];
    for (int k = i + 1; k < nj; ++k) {
      double2 hk = HS(H, i, k), yk = yv[k];
      acc.x -= hk.x * yk.x - hk.y * yk.y;
      acc.y -= hk.x * yk.y + hk.y * yk.x;
    }
    yv[i] = cdiv(acc, HS(H, i, i));
  }
  for (int i = nj; i < m; ++i) yv[i] = make_double2(0, 0);
}

// x += P (V y)
__global__ void gm_update_x(const double2* __restrict__ V, long long vstride, const double2* __restrict__ y,
                            const int* __restrict__ jdone, int m, double2* __restrict__ x, long long N,
                            const double* __restrict__ d, const double2* __restrict__ z, int jacobi) {
  const int v = blockIdx.y;
  const int nj = jdone[v];
  if (nj <= 0) return;
  const double2* vv = V + (size_t)v * vstride;
  const double2* yv = y + (size_t)v * m;
  const double2 zv = z[v];
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0, 0);
    for (int j = 0; j < nj; ++j) {
      double2 a = vv[(size_t)j * N + e], c = yv[j];
      acc.x += c.x * a.x - c.y * a.y;
      acc.y += c.x * a.y + c.y * a.x;
    }
    if (jacobi == 2) {   // learned preconditioner: keep V y, P is applied afterwards
      x[(size_t)v * N + e] = acc;
      continue;
    }
    if (jacobi) acc = cdiv(acc, make_double2(d[e] - zv.x, -zv.y));
    double2 o = x[(size_t)v * N + e];
    x[(size_t)v * N + e] = make_double2(o.x + acc.x, o.y + acc.y);
  }
}

}  // namespace

// learned preconditioner (k_mlp.cu)
bse_status bse_mlp_factors(bse_handle* h, bse_mlp* m, const double2* z_host, int n_z, float2* p, float2* u, float2* v);
bse_status bse_mlp_apply(bse_handle* h, const float2* p, const float2* u, const float2* v, const double2* x,
                         long long xstride, int ns, const int* idx, double2* y, long long ystride, int add,
                         double2* part, long long fstride);
size_t bse_mlp_apply_scratch(int ns);

// ---------------------------------------------------------------------------
namespace {
// w -= a_i v_i + b_i v_{i-1}; partial |w|^2; the last block (counter) computes
// b_{i+1} = |w| for every vector in block order, tests breakdown, resets counter.
__global__ void __launch_bounds__(RB) hay_update_fin(double2* __restrict__ w, const double2* __restrict__ vc,
                                                     const double2* __restrict__ vp, long long N,
                                                     const double* __restrict__ a, double* __restrict__ bco,
                                                     int n_steps, int i, int* __restrict__ active,
                                                     double2* __restrict__ partial, unsigned* counter, int* steps,
                                                     int* status) {
  const int v = blockIdx.y;
  double acc = 0;
  if (active[v]) {
    const double ai = a[(size_t)v * n_steps + i];
    const double bi = i >= 1 ? bco[(size_t)v * (n_steps + 1) + i] : 0.0;
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < N; e += (long long)gridDim.x * RB) {
      const size_t o = (size_t)v * N + e;
      double2 ww = w[o];
      const double2 c = vc[o];
      ww.x -= ai * c.x;
      ww.y -= ai * c.y;
      if (i >= 1) {
        const double2 p = vp[o];
        ww.x -= bi * p.x;
        ww.y -= bi * p.y;
      }
      w[o] = ww;
      acc += ww.x * ww.x + ww.y * ww.y;
    }
  }
  const double2 s = block_sum2(make_double2(acc, 0.0));
  __shared__ int last;
  if (threadIdx.x == 0) {
    partial[(size_t)v * gridDim.x + blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int vv = 0; vv < (int)gridDim.y; ++vv) {
    const double2 t = sum_partials(partial, vv, gridDim.x);
    if (threadIdx.x == 0 && active[vv]) {
      const double bn = sqrt(t.x);
      const double ai = a[(size_t)vv * n_steps + i];
      bco[(size_t)vv * (n_steps + 1) + i + 1] = bn;
      steps[vv] = i + 1;
      if (!isfinite(bn) || !isfinite(ai)) {
        active[vv] = 0;
        atomicOr(status, ST_NAN);
      } else if (bn <= 1e-12 * fmax(1.0, fabs(ai))) {
        active[vv] = 0;
        atomicOr(status, ST_BREAKDOWN);
      }
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}
}  // namespace

namespace {
// Deterministic block-wide sum of part[0..n).x; every block of a grid gets the
// same value (fixed element-to-thread map and order).  All threads return it.
__device__ double block_sum_x_k(const double2* __restrict__ part, int n) {
  __shared__ double ws[RB / 32];
  __shared__ double tot;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += RB) acc += part[i].x;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < RB / 32; ++w) s += ws[w];
    tot = s;
  }
  __syncthreads();
  const double r = tot;
  __syncthreads();
  return r;
}

// Haydock update with deferred reductions (no atomics, no last block): every
// block reduces the epilogue's partials of <v_i|H v_i> to a_i itself (block 0
// records it), applies w -= a_i v_i + b_i v_{i-1}, and writes its partial of
// |w|^2, which the next step's operand pass (or hay_norm_final) reduces.
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// With op.hi set the update also writes the next step's band->grid operand
// from w_{i+1} (unnormalised): bf16 hi/lo rows 2c (Re: psi_r, -psi_i) and 2c+1
// (Im: psi_i, psi_r) at columns 2n, 2n+1, and the FP32 copy of w_{i+1}; the
// next step's epilogue applies 1/b_{i+1}.
__global__ void __launch_bounds__(RB) hay_update_deferred(double2* __restrict__ w, const double2* __restrict__ vc,
                                                          const double2* __restrict__ vp, long long N,
                                                          const double2* __restrict__ fpart, int nfb,
                                                          double* __restrict__ a, const double* __restrict__ bco,
                                                          int n_steps, int i, const int* __restrict__ active,
                                                          double2* __restrict__ partial, int* status,
                                                          bse_operand_out op) {
  const int v = blockIdx.y;
  if (!active[v]) {
    if (threadIdx.x == 0) partial[(size_t)v * gridDim.x + blockIdx.x] = make_double2(0.0, 0.0);
    return;
  }
  const double ai = block_sum_x_k(fpart + (size_t)v * nfb, nfb);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a[(size_t)v * n_steps + i] = ai;
    if (!isfinite(ai)) atomicOr(status, ST_NAN);
  }
  const double bi = i >= 1 ? bco[(size_t)v * (n_steps + 1) + i] : 0.0;
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < N; e += (long long)gridDim.x * RB) {
    const size_t o = (size_t)v * N + e;
    double2 ww = w[o];
    const double2 c = vc[o];
    // explicit FMAs: the fused epilogue update computes the same bits
    ww.x = fma(-ai, c.x, ww.x);
    ww.y = fma(-ai, c.y, ww.y);
    if (i >= 1) {
      const double2 p = vp[o];
      ww.x = fma(-bi, p.x, ww.x);
      ww.y = fma(-bi, p.y, ww.y);
    }
    w[o] = ww;
    acc = fma(ww.x, ww.x, fma(ww.y, ww.y, acc));
    if (op.hi) {
      const float re = (float)ww.x, im = (float)ww.y;
      op.psi_f[o] = make_float2(re, im);
      const int n = (int)(e % op.nb);
      const long long ak = e / op.nb;
      const int k = (int)(ak % op.nk);
      const int cc = v * op.na + (int)(ak / op.nk);
      __nv_bfloat16 h0, l0, h1, l1, h2, l2;
      split_bf16(re, h0, l0);
      split_bf16(-im, h1, l1);
      split_bf16(im, h2, l2);
      const size_t o0 = ((size_t)k * op.nnmax + 2 * cc) * op.kp + 2 * n;
      const size_t o1 = o0 + op.kp;
      *reinterpret_cast<__nv_bfloat162*>(op.hi + o0) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162*>(op.lo + o0) = __halves2bfloat162(l0, l1);
      *reinterpret_cast<__nv_bfloat162*>(op.hi + o1) = __halves2bfloat162(h2, h0);
      *reinterpret_cast<__nv_bfloat162*>(op.lo + o1) = __halves2bfloat162(l2, l0);
    }
  }
  __shared__ double ws[RB / 32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < RB / 32; ++k) s += ws[k];
    partial[(size_t)v * gridDim.x + blockIdx.x] = make_double2(s, 0.0);
  }
}

// b_col = |w| from the update's partials after the last step (one block per
// vector): records b, the step count and the breakdown test.
__global__ void __launch_bounds__(RB) hay_norm_final(const double2* __restrict__ partial, int nhp,
                                                     const double* __restrict__ a, double* __restrict__ bco,
                                                     int n_steps, int col, int* active, int* steps, int* status) {
  const int v = blockIdx.x;
  const double s = block_sum_x_k(partial + (size_t)v * nhp, nhp);
  if (threadIdx.x != 0 || !active[v]) return;
  const double bn = sqrt(s);
  const double ai = a[(size_t)v * n_steps + col - 1];
  bco[(size_t)v * (n_steps + 1) + col] = bn;
  steps[v] = col;
  if (!isfinite(bn) || !isfinite(ai)) {
    active[v] = 0;
    atomicOr(status, ST_NAN);
  } else if (bn <= 1e-12 * fmax(1.0, fabs(ai))) {
    active[v] = 0;
    atomicOr(status, ST_BREAKDOWN);
  }
}
}  // namespace

namespace {
// Grow-only Haydock workspace of a handle: three vectors, partial sums, flags.
constexpr int HPART = UBLK > BSE_FINAL_BLOCKS ? UBLK : BSE_FINAL_BLOCKS;   // |w|^2 partials per vector

size_t hay_ws_bytes(long long N, int n_vec) {
  return 3 * (size_t)n_vec * N * sizeof(double2) + (size_t)n_vec * HPART * sizeof(double2) +
         (size_t)n_vec * BSE_FINAL_BLOCKS * sizeof(double2) + 256 + (size_t)n_vec * sizeof(int) + 256;
}

bse_status hay_reserve(bse_handle* h, int n_vec) {
  const size_t need = hay_ws_bytes(h->N, n_vec);
  if (h->ws_cap >= need) return BSE_OK;
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_cap = 0;
  TRY(dalloc(h, (char**)&h->ws, need, "haydock workspace"));
  h->ws_cap = need;
  return BSE_OK;
}

// Enqueue one Haydock run on the handle's stream (no host synchronisation).
// Buffers that must outlive the launches are registered in `fr`; the device
// status word is returned through status_out.  With allow_graph the step loop
// is captured into a CUDA graph of its own.
bse_status hay_enqueue(bse_handle* h, const double2* b, int n_vec, int n_steps, int reorth, double* a_d,
                       double* b_d, int* steps_d, Freer& fr, int** status_out, bool allow_graph) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  double2 *v3 = nullptr, *partial = nullptr, *basis = nullptr, *coef = nullptr, *fpart = nullptr;
  int *active = nullptr, *status = nullptr;
  unsigned* counters = nullptr;
  {
    TRY(hay_reserve(h, n_vec));
    const size_t bv = 3 * (size_t)n_vec * N * sizeof(double2);
    const size_t bp = (size_t)n_vec * HPART * sizeof(double2);
    const size_t bf = (size_t)n_vec * BSE_FINAL_BLOCKS * sizeof(double2);
    char* p = (char*)h->ws;
    v3 = (double2*)p;
    partial = (double2*)(p + bv);
    fpart = (double2*)(p + bv + bp);
    status = (int*)(p + bv + bp + bf);
    counters = (unsigned*)(p + bv + bp + bf + 64);
    active = (int*)(p + bv + bp + bf + 256);
  }
  double2* hpart = partial;   // partials of the Haydock reductions
  // a_i from the fused H psi epilogue when the form supports it and one pass covers all vectors
  const bool fuse_a = bse_apply_fuses_dot(h) && n_vec <= h->max_vec;
  const bool fuse_b = !reorth;
  // deferred form (tensor-core path, no re-orthogonalisation): a_i and b_{i+1}
  // are reduced by their consumers (the update kernel, the next operand pass),
  // and v_{i+1} = w / b_{i+1} is applied in place by the next operand pass
  const bool lazy_scale = fuse_a && fuse_b && n_vec <= 64;
  // ... and for N_alpha in {1, 6} the update writes the next operand itself
  // (the operand pass disappears from steps >= 1)
  const bool fused_op = lazy_scale && (h->na == 1 || h->na == 6);
  const bse_operand_out opd = fused_op ? bse_tc_operand(h) : bse_operand_out();
  const int ublk = (int)std::min<long long>(UBLK, (N + RB - 1) / RB);
  const int nfb = fuse_a ? bse_tc_final_blocks(h) : 0;
  // ... and, for one vector of a site running alone, the update itself runs
  // inside the epilogue's grid after a bounded grid barrier (one launch less
  // per step); its |w|^2 partials are then one per epilogue block
  const bool fused_upd = fused_op && allow_graph && n_vec == 1 && bse_tc_fused_update_ok(h, n_vec);
  // the separate deferred update runs on the epilogue's grid as well, so that
  // both forms partition the vector and order every sum alike (a many-site
  // run, which keeps the separate kernel, equals a single-site run bit for bit)
  const int dblk = lazy_scale ? nfb : ublk;
  const int nnorm = dblk;
  if (reorth) {
    // Gram-Schmidt partials need one row per basis vector
    TRY(dalloc(h, &partial, (size_t)n_vec * NBLK * (n_steps + 1) * sizeof(double2), "gs partials"));
    fr.add(partial);
    TRY(dalloc(h, &basis, (size_t)n_vec * (n_steps + 1) * N * sizeof(double2), "re-orthogonalisation basis"));
    fr.add(basis);
    TRY(dalloc(h, &coef, (size_t)n_vec * (n_steps + 1) * sizeof(double2), "gs coefficients"));
    fr.add(coef);
  }
  cudaMemsetAsync(a_d, 0, (size_t)n_vec * n_steps * sizeof(double), st);
  cudaMemsetAsync(b_d, 0, (size_t)n_vec * (n_steps + 1) * sizeof(double), st);
  cudaMemsetAsync(steps_d, 0, n_vec * sizeof(int), st);
  cudaMemsetAsync(status, 0, 256, st);   // status word and the two last-block counters
  double2* buf[3] = {v3, v3 + (size_t)n_vec * N, v3 + 2 * (size_t)n_vec * N};
  double2 *vp = buf[0], *vc = buf[1], *w = buf[2];
  const dim3 eg = ew_grid(N, n_vec);
  // v_0 = b / |b|
  BSE_PROF(h, BSE_K_RECURSION, dot_partial_s<<<dim3(NBLK, n_vec), RB, 0, st>>>(b, N, nullptr, 0, N, hpart));
  BSE_PROF(h, BSE_K_RECURSION, hay_init_finalize<<<n_vec, RB, 0, st>>>(hpart, NBLK, b_d, n_steps, active, status));
  BSE_PROF(h, BSE_K_RECURSION, hay_scale<<<eg, 256, 0, st>>>(b, vc, N, b_d, 0, n_steps + 1, active));
  if (reorth) {
    BSE_PROF(h, BSE_K_RECURSION, copy_vecs<<<eg, 256, 0, st>>>(vc, basis, N, (long long)(n_steps + 1) * N));
  }
  // The step loop is recorded into one CUDA graph and launched once (launch
  // gaps between the ~10 kernels of a step otherwise cost ~8 % of the step);
  // without a capturable stream it runs eagerly.  Profiling events become
  // event-record nodes of the graph.
  const bool want_graph = allow_graph && h->stream != nullptr && !getenv("BSE_NO_GRAPH");
  // A call that repeats the previous one (same buffers, sizes and tiles; no
  // per-call re-orthogonalisation buffers, no profiling events) relaunches
  // its instantiated graph instead of capturing the loop again.
  int t_split = 0, t_stages = 0;
  bse_tc_tiles(h, &t_split, &t_stages);
  const unsigned long long key[12] = {(unsigned long long)(uintptr_t)b, (unsigned long long)(uintptr_t)a_d,
                                      (unsigned long long)(uintptr_t)b_d, (unsigned long long)(uintptr_t)steps_d,
                                      (unsigned long long)(uintptr_t)h->ws, (unsigned long long)n_vec,
                                      (unsigned long long)n_steps, (unsigned long long)t_split,
                                      (unsigned long long)t_stages, h->tc_wait_ns,
                                      (unsigned long long)(uintptr_t)st, 1ull};
  const bool cacheable = want_graph && !reorth && !h->prof;
  if (cacheable && h->hay_exec && std::equal(key, key + 12, h->hay_key)) {
    TRY(bse_cuda_check(h, cudaGraphLaunch(h->hay_exec, st), "haydock graph launch"));
    h->launches += h->hay_exec_launches;
    *status_out = status;
    return bse_cuda_check(h, cudaGetLastError(), "haydock kernels");
  }
  bse_drop_graph(h);
  const long long launches0 = h->launches;
  bool capturing = false;
  if (want_graph) {
    capturing = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (!capturing) cudaGetLastError();
  }
  double2* const vp0 = vp;
  double2* const vc0 = vc;
  double2* const w0 = w;
  bse_status loop_status = BSE_OK;
  const size_t ev_mark = h->ev_used;   // profiling events of a refused capture are recorded again
  for (int pass = 0; pass < 2; ++pass) {
  h->ev_used = ev_mark;
  vp = vp0;
  vc = vc0;
  w = w0;
  loop_status = BSE_OK;
  for (int i = 0; i < n_steps && loop_status == BSE_OK; ++i) {
    if (fuse_a) {
      bse_dotfuse f;
      f.partial = fpart;
      f.counter = counters;
      f.a = a_d;
      f.a_stride = n_steps;
      f.i = i;
      f.active = active;
      f.status = status;
      if (lazy_scale) {
        f.deferred = true;
        if (i >= 1) {
          f.norm_part = hpart;
          f.norm_n = nnorm;
          f.bco = b_d;
          f.active_rw = active;
          f.steps = steps_d;
          f.operand_ready = fused_op;
        }
        if (fused_upd) {
          f.fused_update = true;
          f.vprev = vp;
          f.upart = hpart;
          f.barrier = counters + 2;
          f.op = i + 1 < n_steps ? opd : bse_operand_out();
        }
      }
      loop_status = bse_apply_device(h, vc, w, n_vec, &f);     // w = H v_i, a_i = Re <v_i|w>
      if (loop_status != BSE_OK) break;
    } else {
      loop_status = apply_chunked(h, vc, w, n_vec);            // w = H v_i
      if (loop_status != BSE_OK) break;
      BSE_PROF(h, BSE_K_RECURSION, dot_partial_s<<<dim3(NBLK, n_vec), RB, 0, st>>>(vc, N, w, N, N, hpart));
      BSE_PROF(h, BSE_K_RECURSION, hay_a_finalize<<<n_vec, RB, 0, st>>>(hpart, NBLK, a_d, n_steps, i, active, status));
    }
    if (fused_upd) {
      // the epilogue already applied the update
    } else if (lazy_scale) {
      BSE_PROF(h, BSE_K_RECURSION,
               hay_update_deferred<<<dim3(dblk, n_vec), RB, 0, st>>>(
                   w, vc, vp, N, fpart, nfb, a_d, b_d, n_steps, i, active, hpart, status,
                   i + 1 < n_steps ? opd : bse_operand_out()));
    } else if (fuse_b) {
      BSE_PROF(h, BSE_K_RECURSION,
               hay_update_fin<<<dim3(ublk, n_vec), RB, 0, st>>>(
                   w, vc, vp, N, a_d, b_d, n_steps, i, active, hpart,
                                                                 counters + 1, steps_d, status));
    } else {
      BSE_PROF(h, BSE_K_RECURSION, hay_update<<<dim3(NBLK, n_vec), RB, 0, st>>>(w, vc, vp, N, a_d, b_d, n_steps, i, active, hpart));
      loop_status = cgs2(h, basis, (long long)(n_steps + 1) * N, w, n_vec, i + 1, partial, coef, n_steps + 1,
                         nullptr, 0, active);
      if (loop_status != BSE_OK) break;
      BSE_PROF(h, BSE_K_RECURSION, dot_partial_s<<<dim3(NBLK, n_vec), RB, 0, st>>>(w, N, nullptr, 0, N, hpart));
      BSE_PROF(h, BSE_K_RECURSION, hay_b_finalize<<<n_vec, RB, 0, st>>>(hpart, NBLK, a_d, b_d, n_steps, i, active, steps_d, status));
    }
    if (!lazy_scale) {
      BSE_PROF(h, BSE_K_RECURSION, hay_scale<<<eg, 256, 0, st>>>(w, w, N, b_d, i + 1, n_steps + 1, active));   // v_{i+1}
    }
    if (reorth && i + 1 <= n_steps) {
      BSE_PROF(h, BSE_K_RECURSION, copy_vecs<<<eg, 256, 0, st>>>(w, basis + (size_t)(i + 1) * N, N, (long long)(n_steps + 1) * N));
    }
    double2* t = vp;
    vp = vc;
    vc = w;
    w = t;
  }
  if (lazy_scale && loop_status == BSE_OK && n_steps >= 1) {
    BSE_PROF(h, BSE_K_RECURSION,
             hay_norm_final<<<n_vec, RB, 0, st>>>(hpart, nnorm, a_d, b_d, n_steps, n_steps, active, steps_d, status));
  }
  if (!capturing) break;
  // end the capture on every path; launch the graph, or re-run eagerly
  cudaGraph_t graph = nullptr;
  cudaError_t ge = cudaStreamEndCapture(st, &graph);
  capturing = false;
  cudaGraphExec_t exec = nullptr;
  if (ge == cudaSuccess && loop_status == BSE_OK) ge = cudaGraphInstantiate(&exec, graph, 0);
  if (ge == cudaSuccess && loop_status == BSE_OK) ge = cudaGraphLaunch(exec, st);
  if (graph) cudaGraphDestroy(graph);
  if (ge == cudaSuccess && loop_status == BSE_OK && cacheable) {
    h->hay_exec = exec;   // kept for a repeat of this call
    h->hay_exec_launches = h->launches - launches0;
    std::copy(key, key + 12, h->hay_key);
    exec = nullptr;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (ge == cudaSuccess && loop_status == BSE_OK) break;
  cudaGetLastError();   // capture refused: run the same launches eagerly
  }
  *status_out = status;
  TRY(loop_status);
  return bse_cuda_check(h, cudaGetLastError(), "haydock kernels");
}

// wait for the run and map its device status word
bse_status hay_finish(bse_handle* h, const int* status) {
  int hs = 0;
  TRY(bse_cuda_check(h, cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status copy"));
  TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "haydock sync"));
  if (hs & ST_TIMEOUT) return bse_fail(h, BSE_ERR_TIMEOUT, "Haydock grid barrier timed out");
  if (hs & ST_NAN) return bse_fail(h, BSE_ERR_NAN, "non-finite Haydock coefficient");
  if (hs & ST_BREAKDOWN) return BSE_ERR_BREAKDOWN;
  return BSE_OK;
}
}  // namespace

bse_status bse_haydock_device(bse_handle* h, const double2* b, int n_vec, int n_steps, int reorth, double* a_d,
                              double* b_d, int* steps_d) {
  Freer fr;
  int* status = nullptr;
  TRY(hay_enqueue(h, b, n_vec, n_steps, reorth, a_d, b_d, steps_d, fr, &status, true));
  return hay_finish(h, status);
}

// Several sites (one handle each, each on its own stream) recorded into ONE
// CUDA graph: a master stream forks to every site stream, each site's whole
// Haydock run is captured there, and the streams join back.  One graph launch
// then runs every site, the kernels of different sites overlapping on the GPU.
// Falls back to one site after another when a stream cannot be captured.
bse_status bse_haydock_batch_device(bse_handle* const* hs, const double2* const* bs, int n_sites, int n_vec,
                                    int n_steps, double* const* a_d, double* const* b_d, int* const* steps_d,
                                    bse_status* site_status) {
  std::vector<Freer> frs(n_sites);
  std::vector<int*> status(n_sites, nullptr);
  bool capturable = true;
  for (int s = 0; s < n_sites; ++s) capturable = capturable && hs[s]->stream != nullptr && !hs[s]->prof;
  for (int s = 0; s < n_sites && capturable; ++s)
    for (int t = s + 1; t < n_sites; ++t) capturable = capturable && hs[s]->stream != hs[t]->stream;
  for (int s = 0; s < n_sites; ++s) TRY(hay_reserve(hs[s], n_vec));   // no allocation while capturing
  cudaStream_t master = nullptr;
  std::vector<cudaEvent_t> ev(n_sites + 1, nullptr);
  bool graph_done = false;
  if (capturable && !getenv("BSE_NO_GRAPH") && cudaStreamCreateWithFlags(&master, cudaStreamNonBlocking) == cudaSuccess) {
    bool ok = true;
    for (auto& e : ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (ok && cudaStreamBeginCapture(master, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      cudaEventRecord(ev[n_sites], master);
      bse_status es = BSE_OK;
      for (int s = 0; s < n_sites && es == BSE_OK; ++s) {
        cudaStreamWaitEvent(hs[s]->stream, ev[n_sites], 0);
        // sites overlap on the GPU: no kernel whose CTAs wait on one another
        hs[s]->concurrent = true;
        es = hay_enqueue(hs[s], bs[s], n_vec, n_steps, 0, a_d[s], b_d[s], steps_d[s], frs[s], &status[s], false);
        hs[s]->concurrent = false;
        cudaEventRecord(ev[s], hs[s]->stream);
        cudaStreamWaitEvent(master, ev[s], 0);
      }
      cudaGraph_t graph = nullptr;
      cudaError_t ge = cudaStreamEndCapture(master, &graph);
      cudaGraphExec_t exec = nullptr;
      if (ge == cudaSuccess && es == BSE_OK) ge = cudaGraphInstantiate(&exec, graph, 0);
      if (ge == cudaSuccess && es == BSE_OK) ge = cudaGraphLaunch(exec, master);
      if (ge == cudaSuccess && es == BSE_OK) ge = cudaStreamSynchronize(master);
      graph_done = ge == cudaSuccess && es == BSE_OK;
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
  }
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (master) cudaStreamDestroy(master);
  if (!graph_done) {   // one site after another, each with its own captured loop
    for (int s = 0; s < n_sites; ++s) {
      site_status[s] = hay_enqueue(hs[s], bs[s], n_vec, n_steps, 0, a_d[s], b_d[s], steps_d[s], frs[s], &status[s],
                                   true);
    }
  }
  bse_status worst = BSE_OK;
  for (int s = 0; s < n_sites; ++s) {
    if (!graph_done && site_status[s] != BSE_OK) {
      worst = site_status[s];
      continue;
    }
    site_status[s] = hay_finish(hs[s], status[s]);
    if (site_status[s] != BSE_OK && site_status[s] != BSE_ERR_BREAKDOWN) worst = site_status[s];
  }
  return worst;
}

bse_status bse_cf_device(const double* a, const double* bcoef, const int* steps, int n_vec, int n_stride,
                         const double* omega, int n_omega, double gamma, int terminator, double* sigma,
                         cudaStream_t st) {
  dim3 g((unsigned)((n_omega + 127) / 128), (unsigned)n_vec);
  cf_kernel<<<g, 128, 0, st>>>(a, bcoef, steps, n_stride, omega, n_omega, gamma, terminator, sigma);
  return cudaGetLastError() == cudaSuccess ? BSE_OK : BSE_ERR_CUDA;
}

bse_status bse_gmres_device(bse_handle* h, const double2* b, const double2* z, int n_z, double rtol,
                            int restart, int max_iter, int precond, double2* x, int* iters_d,
                            double* rel_d) {
  cudaStream_t st = h->stream;
  const long long N = h->N;
  const int m = restart;
  const int jac = (precond & 0xff) == BSE_PRECOND_JACOBI;
  const bool mlp = (precond & 0xff) == BSE_PRECOND_MLP;
  if (mlp && !h->mlp) return bse_fail(h, BSE_ERR_INVALID_ARG, "gmres: no preconditioner network attached");
  float2 *pc_p = nullptr, *pc_u = nullptr, *pc_v = nullptr;
  double2* pc_part = nullptr;
  Freer frm;
  if (mlp) {
    // per-shift factors of P = diag(p) + U V^H / N from the network (one forward pass per shift)
    std::vector<double2> zh(n_z);
    TRY(bse_cuda_check(h, cudaMemcpyAsync(zh.data(), z, n_z * sizeof(double2), cudaMemcpyDefault, h->stream), "z copy"));
    TRY(bse_cuda_check(h, cudaStreamSynchronize(h->stream), "z sync"));
    const size_t n = (size_t)h->N;
    TRY(dalloc(h, &pc_p, (size_t)n_z * n * sizeof(float2), "precond p")); frm.add(pc_p);
    TRY(dalloc(h, &pc_u, (size_t)n_z * n * 8 * sizeof(float2), "precond U")); frm.add(pc_u);
    TRY(dalloc(h, &pc_v, (size_t)n_z * n * 8 * sizeof(float2), "precond V")); frm.add(pc_v);
    TRY(dalloc(h, &pc_part, bse_mlp_apply_scratch(n_z), "precond scratch")); frm.add(pc_part);
    TRY(bse_mlp_factors(h, h->mlp, zh.data(), n_z, pc_p, pc_u, pc_v));
  }
  Freer fr;
  double2 *V, *T, *W, *partial, *Hs, *sn, *g, *y, *coef;
  double *cs, *beta, *hnorm, *est;
  int *active, *jdone, *mask;
  const long long vstride = (long long)(m + 1) * N;
  TRY(dalloc(h, &V, (size_t)n_z * vstride * sizeof(double2), "krylov basis")); fr.add(V);
  TRY(dalloc(h, &T, (size_t)n_z * N * sizeof(double2), "gmres T")); fr.add(T);
  TRY(dalloc(h, &W, (size_t)n_z * N * sizeof(double2), "gmres W")); fr.add(W);
  TRY(dalloc(h, &partial, (size_t)n_z * NBLK * (m + 1) * sizeof(double2), "partials")); fr.add(partial);
  TRY(dalloc(h, &Hs, (size_t)n_z * (m + 1) * m * sizeof(double2), "hessenberg")); fr.add(Hs);
  TRY(dalloc(h, &sn, (size_t)n_z * m * sizeof(double2), "givens s")); fr.add(sn);
  TRY(dalloc(h, &g, (size_t)n_z * (m + 1) * sizeof(double2), "givens g")); fr.add(g);
  TRY(dalloc(h, &y, (size_t)n_z * m * sizeof(double2), "y")); fr.add(y);
  TRY(dalloc(h, &coef, (size_t)n_z * (m + 1) * sizeof(double2), "coef")); fr.add(coef);
  TRY(dalloc(h, &cs, (size_t)n_z * m * sizeof(double), "givens c")); fr.add(cs);
  TRY(dalloc(h, &beta, (size_t)n_z * sizeof(double), "beta")); fr.add(beta);
  TRY(dalloc(h, &hnorm, (size_t)n_z * sizeof(double), "hnorm")); fr.add(hnorm);
  TRY(dalloc(h, &est, (size_t)n_z * sizeof(double), "est")); fr.add(est);
  TRY(dalloc(h, &active, (size_t)n_z * sizeof(int), "active")); fr.add(active);
  TRY(dalloc(h, &jdone, (size_t)n_z * sizeof(int), "jdone")); fr.add(jdone);
  TRY(dalloc(h, &mask, (size_t)n_z * sizeof(int), "mask")); fr.add(mask);
  int* mask2;
  TRY(dalloc(h, &mask2, (size_t)n_z * sizeof(int), "reorthogonalisation mask")); fr.add(mask2);
  double2* Wc;
  int* didx;
  TRY(dalloc(h, &Wc, (size_t)n_z * N * sizeof(double2), "gmres packed H T")); fr.add(Wc);
  TRY(dalloc(h, &didx, (size_t)n_z * sizeof(int), "active index")); fr.add(didx);
  std::vector<int> hidx(n_z);

  double bnorm = 0;
  {
    BSE_PROF(h, BSE_K_RECURSION, dot_partial_s<<<dim3(NBLK, 1), RB, 0, st>>>(b, N, nullptr, 0, N, partial));
    std::vector<double2> hp(NBLK);
    TRY(bse_cuda_check(h, cudaMemcpyAsync(hp.data(), partial, NBLK * sizeof(double2), cudaMemcpyDeviceToHost, st), "bnorm"));
    TRY(bse_cuda_check(h, cudaStreamSynchronize(st), "bnorm sync"));
    for (int i = 0; i < NBLK; ++i) bnorm += hp[i].x;
    bnorm = sqrt(bnorm);
  }
  if (!(bnorm > 0) || !isfinite(bnorm)) return bse_fail(h, BSE_ERR_INVALID_ARG, "b must be nonzero and finite");
  const int nbn = norm_blocks(N, n_z);   // blocks per system of the residual and Arnoldi norms
  const bool x0 = (precond & BSE_GMRES_X0) != 0;   // x holds the initial guess
  if (!x0) cudaMemsetAsync(x, 0, (size_t)n_z * N * sizeof(double2), st);
  cudaMemsetAsync(iters_d, 0, n_z * sizeof(int), st);
  const dim3 eg = ew_grid(N, n_z);
  std::vector<int> hact(n_z);
  for (int cycle = 0;; ++cycle) {
    // true residual r = b - (H - z) x into V_0, |r|, activity
    const bool zero_x = cycle == 0 && !x0;
    if (!zero_x) TRY(apply_chunked(h, x, W, n_z));
    BSE_PROF(h, BSE_K_RECURSION, gm_residual<<<eg, 256, 0, st>>>(b, W, x, z, V, vstride, N, zero_x));
    BSE_PROF(h, BSE_K_RECURSION, dot_partial_s<<<dim3(nbn, n_z), RB, 0, st>>>(V, vstride, nullptr, 0, N, partial));
    BSE_PROF(h, BSE_K_RECURSION, gm_beta<<<n_z, RB, 0, st>>>(partial, nbn, bnorm, rtol, max_iter, iters_d, beta, rel_d, active, g, m));
    TRY(bse_cuda_check(h, cudaMemcpyAsync(hact.data(), active, n_z * sizeof(int), cudaMemcpyDeviceToHost, st), "active copy"));
    TRY(bse_cuda_check(h, cudaStreamSynchronize(st), "gmres sync"));
    int nact = 0;
    for (int v = 0; v < n_z; ++v) nact += hact[v];
    if (nact == 0) break;
    cudaMemsetAsync(jdone, 0, n_z * sizeof(int), st);
    cudaMemsetAsync(Hs, 0, (size_t)n_z * (m + 1) * m * sizeof(double2), st);
    cudaMemsetAsync(hnorm, 0, n_z * sizeof(double), st);
    // V_0 = r / beta (in place)
    BSE_PROF(h, BSE_K_RECURSION, gm_next<<<eg, 256, 0, st>>>(V, vstride, V, vstride, N, beta, active));
    for (int j = 0; j < m; ++j) {
      cudaMemcpyAsync(mask, active, n_z * sizeof(int), cudaMemcpyDeviceToDevice, st);
      // H is applied to the still-active systems only, packed into nact slots
      int ns = 0;
      for (int v = 0; v < n_z; ++v)
        if (hact[v]) hidx[ns++] = v;
      TRY(bse_cuda_check(h, cudaMemcpyAsync(didx, hidx.data(), ns * sizeof(int), cudaMemcpyHostToDevice, st), "idx"));
      const dim3 ec(eg.x, (unsigned)ns);
      if (mlp) {
        TRY(bse_mlp_apply(h, pc_p, pc_u, pc_v, V + (size_t)j * N, vstride, ns, didx, T, N, 0, pc_part, 1));
      } else {
        BSE_PROF(h, BSE_K_RECURSION, gm_precond_c<<<ec, 256, 0, st>>>(V + (size_t)j * N, vstride, T, N, h->jdiag, z, jac, didx));
      }
      TRY(apply_chunked(h, T, Wc, ns));
      BSE_PROF(h, BSE_K_RECURSION, gm_scatter_shift<<<ec, 256, 0, st>>>(Wc, T, z, W, N, didx));
      // Arnoldi: classical Gram-Schmidt, repeated where the DGKS test asks for it
      TRY(cgs_dgks(h, V, vstride, W, n_z, j + 1, partial, coef, m + 1, Hs + (size_t)j * (m + 1),
                   (m + 1) * m, mask, mask2));
      BSE_PROF(h, BSE_K_RECURSION, dot_partial_s<<<dim3(nbn, n_z), RB, 0, st>>>(W, N, nullptr, 0, N, partial));
      BSE_PROF(h, BSE_K_RECURSION, gm_givens<<<n_z, RB, 0, st>>>(partial, nbn, Hs, cs, sn, g, hnorm, m, j, bnorm, rtol, max_iter,
                                   active, iters_d, jdone, est));
      if (j + 1 < m) {
        BSE_PROF(h, BSE_K_RECURSION, gm_next<<<eg, 256, 0, st>>>(W, N, V + (size_t)(j + 1) * N, vstride, N, hnorm, active));
      }
      TRY(bse_cuda_check(h, cudaMemcpyAsync(hact.data(), active, n_z * sizeof(int), cudaMemcpyDeviceToHost, st), "active copy"));
      TRY(bse_cuda_check(h, cudaStreamSynchronize(st), "gmres sync"));
      nact = 0;
      for (int v = 0; v < n_z; ++v) nact += hact[v];
      if (nact == 0) break;
    }
    BSE_PROF(h, BSE_K_RECURSION, gm_solve<<<(n_z + 127) / 128, 128, 0, st>>>(Hs, g, y, jdone, m, n_z));
    if (mlp) {
      // x += P (V y): V y into W (zero for systems without new columns), then P
      cudaMemsetAsync(W, 0, (size_t)n_z * N * sizeof(double2), st);
      BSE_PROF(h, BSE_K_RECURSION, gm_update_x<<<eg, 256, 0, st>>>(V, vstride, y, jdone, m, W, N, h->jdiag, z, 2));
      TRY(bse_mlp_apply(h, pc_p, pc_u, pc_v, W, N, n_z, nullptr, x, N, 1, pc_part, 1));
    } else {
      BSE_PROF(h, BSE_K_RECURSION, gm_update_x<<<eg, 256, 0, st>>>(V, vstride, y, jdone, m, x, N, h->jdiag, z, jac));
    }
  }
  TRY(bse_cuda_check(h, cudaGetLastError(), "gmres kernels"));
  std::vector<int> hit(n_z);
  std::vector<double> hrel(n_z);
  TRY(bse_cuda_check(h, cudaMemcpyAsync(hit.data(), iters_d, n_z * sizeof(int), cudaMemcpyDeviceToHost, st), "iters"));
  TRY(bse_cuda_check(h, cudaMemcpyAsync(hrel.data(), rel_d, n_z * sizeof(double), cudaMemcpyDeviceToHost, st), "rel"));
  TRY(bse_cuda_check(h, cudaStreamSynchronize(st), "gmres end"));
  for (int v = 0; v < n_z; ++v)
    if (!(hrel[v] <= rtol)) return BSE_ERR_NOT_CONVERGED;
  return BSE_OK;
}
