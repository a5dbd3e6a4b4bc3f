// Split-bf16 tensor-core form of Algorithm 1 (Sec. 3.2.1) on sm_103a.
//
// Both band<->grid contractions are real GEMMs on the re/im-interleaved
// Bloch functions U~ (U = e^{ik.x} u):
//   band->grid:  Phi_k[x][j]  = sum_q U~_k[x][q] Bpsi_k[j][q]
//       q = 2n + u (u = re/im part of U), j = 2c + s (s = re/im part of phi_c),
//       Bpsi holds (psi_r, -psi_i) for s = 0 and (psi_i, psi_r) for s = 1.
//   grid->band:  D_k[q][j] = sum_x U~_k[x][q] Phi'_k[x][j]
//       psi'_{c,n} = (D[2n][2c] + D[2n+1][2c+1]) + i (D[2n][2c+1] - D[2n+1][2c]).
// Every operand is split v = hi + lo into two bf16 numbers and each product
// is formed as hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory.
//
// tc_gemm is a persistent warp-specialised kernel: warp 0 streams 128 x 64
// operand tiles with TMA (128-byte swizzle) into a ring of shared-memory
// stages, warp 1 issues tcgen05.mma (M = 128, N = 16..256, K = 16) from one
// thread into double-buffered TMEM accumulators, warps 2-5 drain TMEM with
// tcgen05.ld and write the results.  Every mbarrier wait is bounded in time;
// on timeout the kernel records an error word, drains its own copies and
// frees its TMEM before returning.
#include "bse_internal.cuh"
#include "tc_ptx.cuh"
#include "k_onepass.cuh"

#include <cuda.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>

namespace {

constexpr int TC_M = 128;
constexpr int TC_KB = 64;                  // bf16 per K block = one 128-byte swizzle row
constexpr int TC_THREADS = 192;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s
constexpr int SMEM_BUDGET = 224 * 1024;


// ---------------------------------------------------------------------------
// persistent split-bf16 GEMM
// ---------------------------------------------------------------------------
struct TcParams {
  int mode;            // 0: band->grid (phi out), 1: grid->band (split-K partials out)
  int ntiles;          // work units = batch * mtiles * nsplit * ntn
  int mtiles, nsplit;
  int kb_per_split, kb_total;
  int nn;              // MMA N of one tile (multiple of 16, <= 256)
  int ntn;             // N tiles (B rows nt*nn .. nt*nn + nn - 1, two rows per complex column)
  int mt0;             // first M tile (band->grid over one x-slab)
  int kb_base;         // first K block and ...
  int split_base;      // ... first partial-sum slot (grid->band over one x-slab)
  int stages;
  uint32_t tmem_cols;
  float2* out;
  int nk, nx, nb, nc;
  int* err;
  unsigned long long wait_ns;   // limit of each pipeline wait (the drain after an abort keeps WAIT_NS)
  uint32_t lbo, sbo;   // mode 2: MN-major descriptor offsets of the A operand (bytes)
};

struct Tile {
  int batch, mt, split, nt, kb0, nkb;
};

// N tile fastest, so that consecutive CTAs share the A tile (u_nk) in L2
__device__ __forceinline__ Tile decode(const TcParams& p, int t) {
  Tile r;
  r.nt = t % p.ntn;
  t /= p.ntn;
  r.split = t % p.nsplit;
  int rest = t / p.nsplit;
  r.mt = p.mt0 + rest % p.mtiles;
  r.batch = rest / p.mtiles;
  r.kb0 = p.kb_base + r.split * p.kb_per_split;
  int left = p.kb_base + p.kb_total - r.kb0;
  r.nkb = left < p.kb_per_split ? left : p.kb_per_split;
  if (r.nkb < 0) r.nkb = 0;
  return r;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm(const __grid_constant__ CUtensorMap ma_hi, const __grid_constant__ CUtensorMap ma_lo,
            const __grid_constant__ CUtensorMap mb_hi, const __grid_constant__ CUtensorMap mb_lo, const TcParams p) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  const uint32_t a_bytes = TC_M * 128;
  const uint32_t b_bytes = (uint32_t)p.nn * 128;
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
  unsigned long long* bars = (unsigned long long*)(sm + (size_t)S * stage_bytes);
  // bars: full[S], empty[S], tfull[2], tempty[2], fin
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * S + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int* consumed = (int*)(tmem_slot + 2);
  int* issued = (int*)(tmem_slot + 3);
  const uint32_t sbase = smem_u32(sm);
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[S + s]); };
  auto tfull = [&](int a) { return smem_u32(&bars[2 * S + a]); };
  auto tempty = [&](int a) { return smem_u32(&bars[2 * S + 2 + a]); };
  const uint32_t fin = smem_u32(&bars[2 * S + 4]);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull(a), 1);
      mbar_init(tempty(a), 4);
    }
    mbar_init(fin, 1);
    *abort_flag = 0;
    *consumed = 0;
    *issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), p.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&ma_hi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&ma_lo) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&mb_hi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&mb_lo) : "memory");
    int it = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
      Tile tl = decode(p, t);
      for (int kb = 0; kb < tl.nkb; ++kb, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!mbar_wait(empty(s), ph ^ 1u, abort_flag, p.wait_ns)) {
          ok = false;
          break;
        }
        const uint32_t st = sbase + (uint32_t)s * stage_bytes;
        mbar_expect_tx(full(s), stage_bytes);
        if (p.mode == 0) {
          // row-major operands [batch][rows][K]: K block = 64 consecutive elements of each row
          const int kc = (tl.kb0 + kb) * TC_KB;
          tma_load_3d(st, &ma_hi, full(s), kc, tl.mt * TC_M, tl.batch);
          tma_load_3d(st + a_bytes, &ma_lo, full(s), kc, tl.mt * TC_M, tl.batch);
          tma_load_3d(st + 2 * a_bytes, &mb_hi, full(s), kc, tl.nt * p.nn, tl.batch);
          tma_load_3d(st + 2 * a_bytes + b_bytes, &mb_lo, full(s), kc, tl.nt * p.nn, tl.batch);
        } else if (p.mode == 2) {
          // grid->band from the row-major U~ [k][x][q]: rows x = 64 kt .. 64 kt + 63
          // of q 0..63 and 64..127 of the M tile, an MN-major A operand
          const int kt = tl.kb0 + kb;
          const int q0 = tl.mt * TC_M;
          tma_load_3d(st, &ma_hi, full(s), q0, kt * TC_KB, tl.batch);
          tma_load_3d(st + a_bytes / 2, &ma_hi, full(s), q0 + TC_KB, kt * TC_KB, tl.batch);
          tma_load_3d(st + a_bytes, &ma_lo, full(s), q0, kt * TC_KB, tl.batch);
          tma_load_3d(st + a_bytes + a_bytes / 2, &ma_lo, full(s), q0 + TC_KB, kt * TC_KB, tl.batch);
          tma_load_4d(st + 2 * a_bytes, &mb_hi, full(s), 0, tl.nt * p.nn, kt, tl.batch);
          tma_load_4d(st + 2 * a_bytes + b_bytes, &mb_lo, full(s), 0, tl.nt * p.nn, kt, tl.batch);
        } else {
          // K-tiled operands [batch][K/64][rows][64]: one contiguous block per K block
          const int kt = tl.kb0 + kb;
          tma_load_4d(st, &ma_hi, full(s), 0, tl.mt * TC_M, kt, tl.batch);
          tma_load_4d(st + a_bytes, &ma_lo, full(s), 0, tl.mt * TC_M, kt, tl.batch);
          tma_load_4d(st + 2 * a_bytes, &mb_hi, full(s), 0, tl.nt * p.nn, kt, tl.batch);
          tma_load_4d(st + 2 * a_bytes + b_bytes, &mb_lo, full(s), 0, tl.nt * p.nn, kt, tl.batch);
        }
        *(volatile int*)issued = it + 1;
      }
    }
    if (!ok) {
      atomicExch(p.err, 1);
      *abort_flag = 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = idesc_bf16(TC_M, p.nn) | (p.mode == 2 ? IDESC_A_MN : 0u);
    int it = 0, local = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x, ++local) {
      Tile tl = decode(p, t);
      const int acc = local & 1;
      const uint32_t aph = (uint32_t)(local >> 1) & 1u;
      if (!mbar_wait(tempty(acc), aph ^ 1u, abort_flag, p.wait_ns)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem_base + (uint32_t)(acc * p.nn);
      for (int kb = 0; kb < tl.nkb; ++kb, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!mbar_wait(full(s), ph, abort_flag, p.wait_ns)) {
          ok = false;
          break;
        }
        *(volatile int*)consumed = it + 1;
        tc_fence_after();
        const uint32_t st = sbase + (uint32_t)s * stage_bytes;
#pragma unroll
        for (int ks = 0; ks < TC_KB / 16; ++ks) {
          // K-major A: 16 K elements = 32 bytes along the row; MN-major A (mode 2):
          // 16 rows of K = 2048 bytes
          const unsigned long long a_hi =
              p.mode == 2 ? sdesc_mn_sw128(st + ks * 2048, p.lbo, p.sbo) : sdesc_sw128(st + ks * 32);
          const unsigned long long a_lo = p.mode == 2 ? sdesc_mn_sw128(st + a_bytes + ks * 2048, p.lbo, p.sbo)
                                                      : sdesc_sw128(st + a_bytes + ks * 32);
          const unsigned long long b_hi = sdesc_sw128(st + 2 * a_bytes + ks * 32);
          const unsigned long long b_lo = sdesc_sw128(st + 2 * a_bytes + b_bytes + ks * 32);
          mma_bf16(d, a_hi, b_hi, idesc, (kb | ks) != 0);
          mma_bf16(d, a_hi, b_lo, idesc, 1);
          mma_bf16(d, a_lo, b_hi, idesc, 1);
        }
        mma_commit(empty(s));
      }
      if (!ok) break;
      mma_commit(tfull(acc));
    }
    if (!ok) {
      atomicExch(p.err, 1);
      *abort_flag = 1;
    }
    // all issued MMAs retire before the teardown frees TMEM
    mma_commit(fin);
    if (!mbar_wait(fin, 0, abort_flag, WAIT_NS)) {
      // abort raised elsewhere: still give the last MMAs a bounded grace period
      const unsigned long long t0 = gtime();
      while (!mbar_try(fin, 0) && gtime() - t0 < WAIT_NS) {
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue (128 threads, one TMEM lane each) ----------------
    const int q = warp & 3;
    const int row_in_tile = q * 32 + lane;
    int local = 0;
    for (int t = blockIdx.x; t < p.ntiles; t += gridDim.x, ++local) {
      Tile tl = decode(p, t);
      const int acc = local & 1;
      const uint32_t aph = (uint32_t)(local >> 1) & 1u;
      // the lanes agree on the outcome before the warp-wide tensor-memory load
      if (!__all_sync(0xffffffffu, mbar_wait(tfull(acc), aph, abort_flag, p.wait_ns))) {
        if (lane == 0) {
          atomicExch(p.err, 1);
          *abort_flag = 1;
        }
        break;
      }
      tc_fence_after();
      const int row = tl.mt * TC_M + row_in_tile;
      const int cbase = tl.nt * (p.nn >> 1);   // first complex column of this N tile
      for (int c16 = 0; c16 < p.nn / 16; ++c16) {
        float v[16];
        tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * p.nn + c16 * 16), v);
        if (p.mode == 0) {
          // phi[k][c][x], x = row
          if (row < p.nx) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int c = cbase + c16 * 8 + i;
              if (c < p.nc) p.out[((size_t)tl.batch * p.nc + c) * p.nx + row] = make_float2(v[2 * i], v[2 * i + 1]);
            }
          }
        } else {
          float pv[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) pv[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
          const int n = row >> 1;
          if ((lane & 1) == 0 && n < p.nb) {
            // partials [split][k][c][n]
            float2* o = p.out + ((size_t)(p.split_base + tl.split) * p.nk + tl.batch) * p.nc * p.nb + n;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int c = cbase + c16 * 8 + i;
              if (c < p.nc) o[(size_t)c * p.nb] = make_float2(v[2 * i] + pv[2 * i + 1], v[2 * i + 1] - pv[2 * i]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(acc));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag) {
    // drain TMA copies that were issued but never consumed
    for (int it = *consumed; it < *issued; ++it) {
      const unsigned long long t0 = gtime();
      while (!mbar_try(full(it % S), (uint32_t)(it / S) & 1u) && gtime() - t0 < WAIT_NS) {
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, p.tmem_cols);
  }
}

// ---------------------------------------------------------------------------
// operand preparation and the FP32 k-transform
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split2(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Deterministic block-wide sum of part[0..n).x (fixed element-to-thread map and
// order, so every block of a grid obtains the same value); all threads return it.
__device__ double block_sum_x(const double2* __restrict__ part, int n) {
  __shared__ double ws[32];
  __shared__ double tot;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i].x;
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    tot = s;
  }
  __syncthreads();
  const double r = tot;
  __syncthreads();
  return r;
}

// Bpsi_k[j][q] (hi, lo): j = 2c + s, q = 2n + u, one thread per psi element
// (c, k, n).  Row j = 2c gives Re phi = Ur psi_r - Ui psi_i (q = 2n: psi_r,
// q = 2n+1: -psi_i), row 2c+1 gives Im phi = Ur psi_i + Ui psi_r.  Entries with
// q >= 2Nb stay zero (the buffer is zeroed once and never written there); rows
// j >= 2Nc only feed output columns that are not stored.  psi_f receives psi
// rounded to FP32 for the FP32 terms of the epilogue and the short range.
// With f.norm_part set (lazy Haydock normalisation, step i = f.i): every block
// reduces |w_i|^2 of each vector from the update's partials (same order in
// every block), block 0 records b_i = |w_i|, the step count and the breakdown
// test, and psi is divided by b_i in place for vectors that stay active.
constexpr int PREP_MAXV = 64;
__global__ void __launch_bounds__(256) prep_bpsi(double2* __restrict__ psi, __nv_bfloat16* __restrict__ hi,
                                                 __nv_bfloat16* __restrict__ lo, float2* __restrict__ psi_f, int nk,
                                                 int nb, int nc, int kp, int nnmax, int na, bse_dotfuse f) {
  __shared__ double sinv[PREP_MAXV];   // 1/b_i per vector, 0 = leave unscaled
  const int nvec = nc / na;
  if (f.norm_part) {
    for (int v = 0; v < nvec; ++v) {
      const double s = block_sum_x(f.norm_part + (size_t)v * f.norm_n, f.norm_n);
      if (threadIdx.x == 0) {
        double inv = 0.0;
        if (f.active_rw[v]) {
          const double bn = sqrt(s);
          const double ai = f.a[(size_t)v * f.a_stride + f.i - 1];
          int st = 0;
          if (!isfinite(bn) || !isfinite(ai)) st = 2;
          else if (bn <= 1e-12 * fmax(1.0, fabs(ai))) st = 1;
          if (blockIdx.x == 0) {
            f.bco[(size_t)v * (f.a_stride + 1) + f.i] = bn;
            f.steps[v] = f.i;
            if (st) {
              f.active_rw[v] = 0;
              atomicOr(f.status, st);
            }
          }
          if (!st) inv = 1.0 / bn;
        }
        sinv[v] = inv;
      }
    }
    __syncthreads();
  }
  const size_t total = (size_t)nc * nk * nb;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(e % nb);
    const size_t ck = e / nb;
    const int k = (int)(ck % nk), c = (int)(ck / nk);
    double2 ps = psi[e];
    if (f.norm_part) {
      const double inv = sinv[c / na];
      if (inv != 0.0) {
        ps = make_double2(ps.x * inv, ps.y * inv);
        psi[e] = ps;
      }
    }
    const float re = (float)ps.x, im = (float)ps.y;
    psi_f[e] = make_float2(re, im);
    __nv_bfloat16 h0, l0, h1, l1, h2, l2;
    split2(re, h0, l0);
    split2(-im, h1, l1);
    split2(im, h2, l2);
    const size_t o0 = ((size_t)k * nnmax + 2 * c) * kp + 2 * n;
    const size_t o1 = o0 + kp;
    *reinterpret_cast<__nv_bfloat162*>(hi + o0) = __halves2bfloat162(h0, h1);
    *reinterpret_cast<__nv_bfloat162*>(lo + o0) = __halves2bfloat162(l0, l1);
    *reinterpret_cast<__nv_bfloat162*>(hi + o1) = __halves2bfloat162(h2, h0);
    *reinterpret_cast<__nv_bfloat162*>(lo + o1) = __halves2bfloat162(l2, l0);
  }
}

// Block-level <psi|H psi> partial + last-block reduction shared by both epilogues.
__device__ void fused_dot_tail(const bse_dotfuse& f, double dre, double dim) {
  __shared__ double sre[8], sim[8];
  __shared__ int last;
  const int nw = blockDim.x >> 5;   // warps per block (<= 8)
  for (int off = 16; off > 0; off >>= 1) {
    dre += __shfl_xor_sync(0xffffffffu, dre, off);
    dim += __shfl_xor_sync(0xffffffffu, dim, off);
  }
  if ((threadIdx.x & 31) == 0) {
    sre[threadIdx.x >> 5] = dre;
    sim[threadIdx.x >> 5] = dim;
  }
  __syncthreads();
  const int v = blockIdx.y;
  if (threadIdx.x == 0) {
    double r = 0, im = 0;
    for (int w = 0; w < nw; ++w) {
      r += sre[w];
      im += sim[w];
    }
    f.partial[(size_t)v * gridDim.x + blockIdx.x] = make_double2(r, im);
    if (!f.deferred) {
      __threadfence();
      const unsigned prev = atomicAdd(f.counter, 1u);
      last = prev == gridDim.x * gridDim.y - 1;
    }
  }
  if (f.deferred) return;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int vv = 0; vv < (int)gridDim.y; ++vv) {
    double r = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) r += f.partial[(size_t)vv * gridDim.x + b].x;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sre[threadIdx.x >> 5] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int w = 0; w < nw; ++w) s += sre[w];
      if (f.active[vv]) {
        f.a[(size_t)vv * f.a_stride + f.i] = s;
        if (!isfinite(s)) atomicOr(f.status, 2);
      }
    }
  }
  if (threadIdx.x == 0) *f.counter = 0u;
}

// Grid-wide barrier of a resident grid (every block calls it once per use):
// arrivals are counted in bar[0], the last block resets them and advances the
// generation bar[1], which the others wait for -- at most 1 s of %globaltimer,
// after which the block records BSE_ST_TIMEOUT and reports failure.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g0 = atomicOr(bar + 1, 0u);
    __threadfence();
    int good = 1;
    if (atomicAdd(bar, 1u) == nblocks - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = gtime();
      while (atomicOr(bar + 1, 0u) == g0) {
        if (gtime() - t0 > 1000000000ull) {
          good = 0;
          atomicOr(status, BSE_ST_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ void split_pair(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Haydock update of vector v = blockIdx.y inside the epilogue's grid, after
// the barrier: a_i from every block's <psi|H psi> partial (same order in every
// block), w = H v_i - a_i v_i - b_i v_{i-1} over the vector (grid-stride), the
// block's |w|^2 partial and the next step's band->grid operand from w.
// act / bi: the vector's state as this block found it in the lazy
// normalisation (every block computes the same values).
__device__ void fused_update_phase(const bse_dotfuse& f, double2* __restrict__ w, const double2* __restrict__ vc,
                                   long long n_per_vec, bool act, double bi) {
  const int v = blockIdx.y;
  if (!act) {
    if (threadIdx.x == 0) f.upart[(size_t)v * gridDim.x + blockIdx.x] = make_double2(0.0, 0.0);
    return;
  }
  __shared__ double ws_[8];
  __shared__ double ai_s;
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += __ldcg(&f.partial[(size_t)v * gridDim.x + b].x);
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) ws_[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws_[k];
    ai_s = t;
    if (blockIdx.x == 0) {
      f.a[(size_t)v * f.a_stride + f.i] = t;
      if (!isfinite(t)) atomicOr(f.status, 2);
    }
  }
  __syncthreads();
  const double ai = ai_s;
  const bse_operand_out& op = f.op;
  double acc = 0.0;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n_per_vec;
       e += (long long)gridDim.x * blockDim.x) {
    const size_t o = (size_t)v * n_per_vec + e;
    double2 ww = __ldcg(&w[o]);
    const double2 c = __ldcg(&vc[o]);
    // the same FMAs as the separate update kernel (bit-identical results)
    ww.x = fma(-ai, c.x, ww.x);
    ww.y = fma(-ai, c.y, ww.y);
    if (f.i >= 1) {
      const double2 p = f.vprev[o];
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
      split_pair(re, h0, l0);
      split_pair(-im, h1, l1);
      split_pair(im, h2, l2);
      const size_t o0 = ((size_t)k * op.nnmax + 2 * cc) * op.kp + 2 * n;
      const size_t o1 = o0 + op.kp;
      *reinterpret_cast<__nv_bfloat162*>(op.hi + o0) = __halves2bfloat162(h0, h1);
      *reinterpret_cast<__nv_bfloat162*>(op.lo + o0) = __halves2bfloat162(l0, l1);
      *reinterpret_cast<__nv_bfloat162*>(op.hi + o1) = __halves2bfloat162(h2, h0);
      *reinterpret_cast<__nv_bfloat162*>(op.lo + o1) = __halves2bfloat162(l2, l0);
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) ws_[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws_[k];
    f.upart[(size_t)v * gridDim.x + blockIdx.x] = make_double2(t, 0.0);
  }
}

// Epilogue with NA core states per thread: one thread per (k, n) of vector
// v = blockIdx.y computes all NA outputs, so A[:, kn] and psi[v][:][kn] are
// read once; c' and chi are staged in shared memory as FP32.
// out[c][k][n] = sum_split part + E psi - chi psi + short-range out for NA
// core states, G of them per thread (NA / G threads per (k, n): more loads in
// flight for this latency-bound pass); the projectors are read in FP32.
template <int NA, int G, bool FUSED>
__global__ void __launch_bounds__(256, 4) g2b_final_na(const float2* __restrict__ part, int nsplit,
                                                    double2* __restrict__ psi,
                                                    const float2* __restrict__ psi_f, double2* __restrict__ out,
                                                    const double* __restrict__ e_nk, const double2* __restrict__ chi,
                                                    const float2* __restrict__ a_proj,
                                                    const double2* __restrict__ srcp, int nk, int nb, int np, int nc,
                                                    bse_dotfuse f) {
  constexpr int NG = NA / G;
  constexpr int PU = 12;   // projector loads in flight per thread
  __shared__ float2 cps[NA * BSE_MAX_PROJ];
  __shared__ float2 chs[NA * NA];
  const size_t nkb = (size_t)nk * nb;
  const int v = blockIdx.y;
  for (int i = threadIdx.x; i < NA * np; i += blockDim.x) {
    const double2 q = srcp[(size_t)v * NA * np + i];
    cps[i] = make_float2((float)q.x, (float)q.y);
  }
  for (int i = threadIdx.x; i < NA * NA; i += blockDim.x) chs[i] = make_float2((float)chi[i].x, (float)chi[i].y);
  __syncthreads();
  // lazy normalisation (operand written by the previous update from w_i): every
  // block reduces |w_i|^2 in the same order; block 0 records b_i, the step count
  // and the breakdown test; the linear terms are scaled by 1/b_i and psi is
  // normalised in place (each element by the one thread that owns it)
  const bool lazy = f.operand_ready && f.norm_part;
  double inv = 1.0;
  bool vec_active = true;   // (fused update) this vector goes on after this step's normalisation
  double b_i = 0.0;         // (fused update) b_i = |w_i| as this block computed it
  if (FUSED && !lazy) vec_active = f.active[v] != 0;
  if (lazy) {
    const double s = block_sum_x(f.norm_part + (size_t)v * f.norm_n, f.norm_n);
    __shared__ double sinv, sbn;
    if (threadIdx.x == 0) {
      double iv = 0.0;
      sbn = 0.0;
      if (f.active_rw[v]) {
        const double bn = sqrt(s);
        sbn = bn;
        const double ai = f.a[(size_t)v * f.a_stride + f.i - 1];
        int st = 0;
        if (!isfinite(bn) || !isfinite(ai)) st = 2;
        else if (bn <= 1e-12 * fmax(1.0, fabs(ai))) st = 1;
        if (blockIdx.x == 0) {
          f.bco[(size_t)v * (f.a_stride + 1) + f.i] = bn;
          f.steps[v] = f.i;
          if (st) {
            f.active_rw[v] = 0;
            atomicOr(f.status, st);
          }
        }
        if (!st) iv = 1.0 / bn;
      }
      sinv = iv;
    }
    __syncthreads();
    inv = sinv;
    b_i = sbn;
    vec_active = inv != 0.0;
  }
  const float finv = (float)inv;
  double dre = 0.0;
  const size_t total = nkb * NG;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t kn = e / NG;
    const int a0 = (int)(e % NG) * G;
    const int k = (int)(kn / nb), n = (int)(kn % nb);
    float2 pf[NA];
#pragma unroll
    for (int b = 0; b < NA; ++b) pf[b] = psi_f[(size_t)(v * NA + b) * nkb + kn];
    float2 acc[G];
#pragma unroll
    for (int g = 0; g < G; ++g) acc[g] = make_float2(0.f, 0.f);
    for (int p0 = 0; p0 < np; p0 += PU) {
      float2 ap[PU];
#pragma unroll
      for (int u = 0; u < PU; ++u)
        ap[u] = p0 + u < np ? a_proj[(size_t)(p0 + u) * nkb + kn] : make_float2(0.f, 0.f);
#pragma unroll
      for (int u = 0; u < PU; ++u) {
        if (p0 + u < np) {
#pragma unroll
          for (int g = 0; g < G; ++g) {
            const float2 q = cps[(a0 + g) * np + p0 + u];
            acc[g].x += ap[u].x * q.x + ap[u].y * q.y;   // conj(A) c'
            acc[g].y += ap[u].x * q.y - ap[u].y * q.x;
          }
        }
      }
    }
    const double e_kn = e_nk[kn];
#pragma unroll
    for (int g = 0; g < G; ++g) {
      const int a = a0 + g;
      float rx = acc[g].x, ry = acc[g].y;
#pragma unroll
      for (int b = 0; b < NA; ++b) {
        const float2 ch = chs[a * NA + b];
        rx -= ch.x * pf[b].x - ch.y * pf[b].y;
        ry -= ch.x * pf[b].y + ch.y * pf[b].x;
      }
      const int c = v * NA + a;
      // split-K partials (FP32 tensor-core accumulators) summed in FP32 with
      // the FP32 short-range and spin-orbit terms; E psi and the sum in FP64
      for (int sp = 0; sp < nsplit; ++sp) {
        const float2 t = part[(((size_t)sp * nk + k) * nc + c) * nb + n];
        rx += t.x;
        ry += t.y;
      }
      double2 ps = psi[(size_t)c * nkb + kn];
      if (lazy) {
        rx *= finv;
        ry *= finv;
        ps = make_double2(ps.x * inv, ps.y * inv);
        if (inv != 0.0) psi[(size_t)c * nkb + kn] = ps;
      }
      const double2 val = make_double2((double)rx + e_kn * ps.x, (double)ry + e_kn * ps.y);
      out[(size_t)c * nkb + kn] = val;
      dre += ps.x * val.x + ps.y * val.y;   // Re <psi|H psi>: the only part the recursion uses
    }
  }
  if (f.partial) fused_dot_tail(f, dre, 0.0);
  if constexpr (FUSED) {
    if (!grid_barrier(f.barrier, gridDim.x * gridDim.y, f.status)) return;
    fused_update_phase(f, out, psi, (long long)NA * (long long)nkb, vec_active, b_i);
  }
}

// out[c][k][n] = sum_split part + E psi - chi psi + short-range out.  Grid
// (blocks per vector, n_vec); with f.partial set, also a[v][i] = Re <psi_v|out_v>.
__global__ void __launch_bounds__(256) g2b_final(const float2* __restrict__ part, int nsplit,
                                                 const double2* __restrict__ psi, double2* __restrict__ out,
                                                 const double* __restrict__ e_nk, const double2* __restrict__ chi,
                                                 const double2* __restrict__ a_proj, const double2* __restrict__ srcp,
                                                 int nk, int nb, int na, int np, int nc, bse_dotfuse f) {
  const size_t nkb = (size_t)nk * nb;
  const int v = blockIdx.y;
  double dre = 0.0, dim = 0.0;
  for (size_t e_ = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e_ < (size_t)na * nkb;
       e_ += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(e_ / nkb);
    const size_t kn = e_ % nkb;
    const int c = v * na + a;
    const int k = (int)(kn / nb), n = (int)(kn % nb);
    double2 lr = make_double2(0, 0);
    for (int sp = 0; sp < nsplit; ++sp) {
      const float2 t = part[(((size_t)sp * nk + k) * nc + c) * nb + n];
      lr.x += t.x;
      lr.y += t.y;
    }
    const double2 ps = psi[((size_t)c * nk + k) * nb + n];
    const double e = e_nk[kn];
    // -chi psi and the short-range projection out in FP32; E psi and the sum in FP64
    float rx = 0.f, ry = 0.f;
    for (int b = 0; b < na; ++b) {
      const double2 chd = chi[a * na + b];
      const double2 pbd = psi[((size_t)(v * na + b) * nk + k) * nb + n];
      const float2 ch = make_float2((float)chd.x, (float)chd.y), pb = make_float2((float)pbd.x, (float)pbd.y);
      rx -= ch.x * pb.x - ch.y * pb.y;
      ry -= ch.x * pb.y + ch.y * pb.x;
    }
    if (np > 0) {
      const double2* cp = srcp + (size_t)v * na * np + (size_t)a * np;
      for (int p = 0; p < np; ++p) {
        const double2 apd = a_proj[(size_t)p * nkb + kn];
        const double2 qd = cp[p];
        const float2 ap = make_float2((float)apd.x, (float)apd.y), qq = make_float2((float)qd.x, (float)qd.y);
        rx += ap.x * qq.x + ap.y * qq.y;
        ry += ap.x * qq.y - ap.y * qq.x;
      }
    }
    const double2 val = make_double2(lr.x + (double)rx + e * ps.x, lr.y + (double)ry + e * ps.y);
    out[((size_t)c * nk + k) * nb + n] = val;
    dre += ps.x * val.x + ps.y * val.y;
    dim += ps.x * val.y - ps.y * val.x;
  }
  if (f.partial) fused_dot_tail(f, dre, dim);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// 3-D bf16 map {inner, rows, batch} with row stride `inner_stride` elements and
// batch stride `batch_stride` elements; box {64, box_rows, 1}, 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t inner, uint64_t rows, uint64_t batch, uint64_t inner_stride,
              uint64_t batch_stride, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {inner, rows, batch};
  cuuint64_t strides[2] = {inner_stride * 2, batch_stride * 2};
  cuuint32_t box[3] = {(cuuint32_t)TC_KB, box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 4-D bf16 map of a K-tiled array [batch][ktiles][rows][64] (row stride 64
// elements, tile stride rows_stride*64, batch stride ktiles*rows_stride*64);
// box {64, box_rows, 1, 1} = one contiguous block, 128-byte swizzle.
bool make_map_tiled(CUtensorMap* m, const void* base, uint64_t rows, uint64_t rows_stride, uint64_t ktiles,
                    uint64_t batch, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[4] = {(cuuint64_t)TC_KB, rows, ktiles, batch};
  cuuint64_t strides[3] = {(cuuint64_t)TC_KB * 2, rows_stride * TC_KB * 2, ktiles * rows_stride * TC_KB * 2};
  cuuint32_t box[4] = {(cuuint32_t)TC_KB, box_rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

struct TcState {
  int kp = 0, nnmax = 0, smax = 0, sms = 0;
  int stages = 0;       // pipeline stages (0: chosen by rule per tile width)
  int part_cap = 0;     // split-K factor the partial buffer is sized for
  int* err = nullptr;   // device error word
  unsigned* sync = nullptr;   // one-pass step: per-slab counters, abort and done words
  uint32_t lbo = 8192, sbo = 1024;   // MN-major descriptors: q blocks 8 KB apart, 8-row groups 1 KB apart
  // a2: U~ row-major, box 64 x 128 rows (band->grid A); a2m: the same array,
  // box 64 x 64 rows (grid->band A read MN-major); a6: the K-tiled transposed copy
  CUtensorMap a2_hi, a2_lo, a2m_hi, a2m_lo, a6_hi, a6_lo;
};

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// error word (offset 0) and, from offset 256, the one-pass step's counters
size_t tc_word_bytes(const bse_handle* h) {
  const size_t nslab = (size_t)(h->nx + TC_M - 1) / TC_M;
  return 256 + ((2 * nslab + 3) * sizeof(unsigned) + 255) / 256 * 256;
}

// MMA N of one tile for `rows` B rows (two per complex column): one tile up
// to 256 rows (the tcgen05 maximum, two accumulators filling TMEM's 512
// columns); wider operands in 256-row tiles (the last one partly out of the
// tensor, zero-filled by TMA, its columns not stored)
inline int tile_n(int rows) { return rows <= 256 ? rows : 256; }

// most pipeline stages that fit shared memory for MMA width nn (at most 8)
int fit_stages(int nn) {
  const int stage = 2 * TC_M * 128 + 2 * nn * 128;
  int s = (SMEM_BUDGET - 1024 - 256) / stage;
  return s > 8 ? 8 : s;
}

int pick_stages(int nn, int tuned) {
  int s = fit_stages(nn);
  if (tuned > 0) return tuned < s ? tuned : s;
  // rule: narrow (HBM-bound) tiles get four stages (~150 KB), which keep ~25 MB
  // in flight over the GPU and leave shared memory for the short-range kernels
  // of the side stream to run on the same SMs during the GEMM
  if (nn <= 32 && s > 4) s = 4;
  return s;
}

bse_status launch_gemm(bse_handle* h, TcState* ts, int mode, const CUtensorMap& a_hi, const CUtensorMap& a_lo,
                       const CUtensorMap& b_hi, const CUtensorMap& b_lo, TcParams p, int kind, cudaStream_t st) {
  p.stages = pick_stages(p.nn, ts->stages);
  if (p.stages < 2) return bse_fail(h, BSE_ERR_UNSUPPORTED, "tensor-core tile does not fit shared memory");
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * p.nn)) cols <<= 1;
  p.tmem_cols = cols;
  p.err = ts->err;
  p.wait_ns = h->tc_wait_ns;
  p.lbo = ts->lbo;
  p.sbo = ts->sbo;
  const size_t smem = 1024 + (size_t)p.stages * (2 * TC_M * 128 + 2 * p.nn * 128) + 256;
  cudaFuncSetAttribute(tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int grid = p.ntiles < ts->sms ? p.ntiles : ts->sms;
  if (grid < 1) return BSE_OK;
  BSE_PROF(h, kind, tc_gemm<<<grid, TC_THREADS, smem, st>>>(a_hi, a_lo, b_hi, b_lo, p));
  (void)mode;
  return bse_cuda_check(h, cudaGetLastError(), "tc_gemm launch");
}

}  // namespace

bse_status bse_tc_prepare(bse_handle* h) {
  TcState* ts = new (std::nothrow) TcState();
  if (!ts) return bse_fail(h, BSE_ERR_OOM, "tc state");
  h->tmap_host = ts;
  if (!encode_fn()) return bse_fail(h, BSE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  cudaDeviceGetAttribute(&ts->sms, cudaDevAttrMultiProcessorCount, h->dev);
  ts->kp = round_up(2 * h->nb, 8);
  ts->nnmax = round_up(2 * h->na * h->max_vec, 16);
  // split-K of grid->band: aim for >= 8 work units per SM, >= 8 K blocks per unit
  const int kbt = (h->nx + TC_KB - 1) / TC_KB;
  const int units = h->nk * ((2 * h->nb + TC_M - 1) / TC_M);
  int sp = 1;
  while (units * sp < 8 * ts->sms && kbt / (sp * 2) >= 8) sp *= 2;
  ts->smax = sp;
  ts->part_cap = sp;
  const size_t nbp = (size_t)h->nk * ts->nnmax * ts->kp;
  const size_t x64 = (size_t)(h->nx + TC_KB - 1) / TC_KB;
  const size_t nbf = (size_t)h->nk * x64 * ts->nnmax * TC_KB;   // K-tiled [k][x/64][row][64]
  {
    bse_status s = bse_handle_malloc(h, (void**)&h->bpsi, 2 * nbp * sizeof(__nv_bfloat16), "band->grid operand");
    if (s == BSE_OK)
      s = bse_handle_malloc(h, (void**)&h->psi_f, (size_t)h->max_vec * h->na * h->nk * h->nb * sizeof(float2),
                            "FP32 psi");
    if (s == BSE_OK) s = bse_handle_malloc(h, (void**)&h->bphi, 2 * nbf * sizeof(__nv_bfloat16), "grid->band operand");
    if (s == BSE_OK)
      s = bse_handle_malloc(h, (void**)&h->part,
                            (size_t)ts->smax * h->nk * h->nb * h->na * h->max_vec * sizeof(float2), "split-K partials");
    if (s == BSE_OK) s = bse_handle_malloc(h, (void**)&h->tmap, tc_word_bytes(h), "tensor-core error and sync words");
    if (s != BSE_OK) return s;
  }
  ts->err = (int*)h->tmap;
  ts->sync = (unsigned*)((char*)h->tmap + 256);
  cudaMemsetAsync(h->tmap, 0, tc_word_bytes(h), h->stream);
  cudaMemsetAsync(h->bphi, 0, 2 * nbf * sizeof(__nv_bfloat16), h->stream);
  cudaMemsetAsync(h->bpsi, 0, 2 * nbp * sizeof(__nv_bfloat16), h->stream);
  const int kp = ts->kp;
  bool ok = make_map(&ts->a2_hi, h->u_hi, kp, h->nx, h->nk, kp, (uint64_t)h->nx * kp, TC_M) &&
            make_map(&ts->a2_lo, h->u_lo, kp, h->nx, h->nk, kp, (uint64_t)h->nx * kp, TC_M) &&
            make_map(&ts->a2m_hi, h->u_hi, kp, h->nx, h->nk, kp, (uint64_t)h->nx * kp, TC_KB) &&
            make_map(&ts->a2m_lo, h->u_lo, kp, h->nx, h->nk, kp, (uint64_t)h->nx * kp, TC_KB) &&
            make_map_tiled(&ts->a6_hi, h->ut_hi, 2 * h->nb, 2 * h->nb, x64, h->nk, TC_M) &&
            make_map_tiled(&ts->a6_lo, h->ut_lo, 2 * h->nb, 2 * h->nb, x64, h->nk, TC_M);
  if (!ok) return bse_fail(h, BSE_ERR_CUDA, "tensor map encoding failed");
  return bse_cuda_check(h, cudaStreamSynchronize(h->stream), "tc prepare");
}

int bse_tc_kp(const bse_handle* h) { return h->tmap_host ? ((const TcState*)h->tmap_host)->kp : 0; }

void bse_tc_free(bse_handle* h) {
  delete (TcState*)h->tmap_host;
  h->tmap_host = nullptr;
}

bse_status bse_tc_prep(bse_handle* h, const double2* psi, int n_vec, const bse_dotfuse* fuse) {
  TcState* ts = (TcState*)h->tmap_host;
  const int nc = n_vec * h->na;
  const size_t nbp = (size_t)h->nk * ts->nnmax * ts->kp;
  const size_t total = (size_t)nc * h->nk * h->nb;
  // with the lazy normalisation each block first reduces the update's |w|^2
  // partials in FP64 (slow pipe), so two blocks per SM; without it (plain
  // H psi, GMRES's wide passes) enough blocks to keep loads in flight
  const bool lazy = fuse && fuse->norm_part;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)(lazy ? 2 : 16) * ts->sms);
  bse_dotfuse f = lazy ? *fuse : bse_dotfuse();
  if (f.norm_part && n_vec > PREP_MAXV) return bse_fail(h, BSE_ERR_UNSUPPORTED, "lazy normalisation: too many vectors");
  BSE_PROF(h, BSE_K_PREP,
           prep_bpsi<<<blocks, 256, 0, h->stream>>>(const_cast<double2*>(psi), h->bpsi, h->bpsi + nbp, h->psi_f,
                                                    h->nk, h->nb, nc, ts->kp, ts->nnmax, h->na, f));
  return bse_cuda_check(h, cudaGetLastError(), "prep_bpsi launch");
}

namespace {
// band->grid over the M tiles [mt_b, mt_e) (x rows mt*128 ..), on stream st
bse_status b2g_range(bse_handle* h, int n_vec, int mt_b, int mt_e, cudaStream_t st) {
  TcState* ts = (TcState*)h->tmap_host;
  const int nc = n_vec * h->na;
  const int rows = round_up(2 * nc, 16);
  const int nn = tile_n(rows);
  const size_t nbp = (size_t)h->nk * ts->nnmax * ts->kp;
  __nv_bfloat16* bh = h->bpsi;
  __nv_bfloat16* bl = h->bpsi + nbp;
  CUtensorMap b_hi, b_lo;
  if (!make_map(&b_hi, bh, ts->kp, rows, h->nk, ts->kp, (uint64_t)ts->nnmax * ts->kp, nn) ||
      !make_map(&b_lo, bl, ts->kp, rows, h->nk, ts->kp, (uint64_t)ts->nnmax * ts->kp, nn))
    return bse_fail(h, BSE_ERR_CUDA, "tensor map encoding failed");
  TcParams p{};
  p.mode = 0;
  p.mt0 = mt_b;
  p.mtiles = mt_e - mt_b;
  p.nsplit = 1;
  p.kb_total = (ts->kp + TC_KB - 1) / TC_KB;
  p.kb_per_split = p.kb_total;
  p.ntn = (rows + nn - 1) / nn;
  p.ntiles = h->nk * p.mtiles * p.ntn;
  p.nn = nn;
  p.out = (float2*)h->phi;
  p.nk = h->nk;
  p.nx = h->nx;
  p.nb = h->nb;
  p.nc = nc;
  return launch_gemm(h, ts, 0, ts->a2_hi, ts->a2_lo, b_hi, b_lo, p, BSE_K_BAND_TO_GRID, st);
}

// grid->band over the K blocks [kb_b, kb_e) (x = kb*64 ..), split into at
// most `want` parts written to partial slots split_base..; *nsplit_out
// receives the number of slots written.  On stream st.
bse_status g2b_range(bse_handle* h, int n_vec, int kb_b, int kb_e, int split_base, int want, int* nsplit_out,
                     cudaStream_t st) {
  TcState* ts = (TcState*)h->tmap_host;
  const int nc = n_vec * h->na;
  const int rows = round_up(2 * nc, 16);
  const int nn = tile_n(rows);
  const size_t x64 = (size_t)(h->nx + TC_KB - 1) / TC_KB;
  const size_t nbf = (size_t)h->nk * x64 * ts->nnmax * TC_KB;
  CUtensorMap b_hi, b_lo;
  if (!make_map_tiled(&b_hi, h->bphi, rows, ts->nnmax, x64, h->nk, nn) ||
      !make_map_tiled(&b_lo, h->bphi + nbf, rows, ts->nnmax, x64, h->nk, nn))
    return bse_fail(h, BSE_ERR_CUDA, "tensor map encoding failed");
  TcParams p{};
  p.mode = h->sched == BSE_SCHED_TWO_PASS_ROWMAJOR ? 2 : 1;
  p.mtiles = (2 * h->nb + TC_M - 1) / TC_M;
  p.kb_base = kb_b;
  p.kb_total = kb_e - kb_b;
  p.nsplit = want < p.kb_total ? want : p.kb_total;
  if (p.nsplit < 1) p.nsplit = 1;
  p.kb_per_split = (p.kb_total + p.nsplit - 1) / p.nsplit;
  p.nsplit = (p.kb_total + p.kb_per_split - 1) / p.kb_per_split;   // no empty split
  p.split_base = split_base;
  p.ntn = (rows + nn - 1) / nn;
  p.ntiles = h->nk * p.mtiles * p.nsplit * p.ntn;
  p.nn = nn;
  p.out = (float2*)h->part;
  p.nk = h->nk;
  p.nx = h->nx;
  p.nb = h->nb;
  p.nc = nc;
  *nsplit_out = p.nsplit;
  if (p.mode == 2) return launch_gemm(h, ts, 2, ts->a2m_hi, ts->a2m_lo, b_hi, b_lo, p, BSE_K_GRID_TO_BAND, st);
  return launch_gemm(h, ts, 1, ts->a6_hi, ts->a6_lo, b_hi, b_lo, p, BSE_K_GRID_TO_BAND, st);
}

}  // namespace

bse_status bse_tc_band_to_grid(bse_handle* h, int n_vec) {
  TcState* ts = (TcState*)h->tmap_host;
  (void)ts;
  return b2g_range(h, n_vec, 0, (h->nx + TC_M - 1) / TC_M, h->stream);
}

bse_status bse_kconv_bf16(bse_handle* h, int n_vec) {
  TcState* ts = (TcState*)h->tmap_host;
  const size_t nbf = (size_t)h->nk * ((h->nx + TC_KB - 1) / TC_KB) * ts->nnmax * TC_KB;
  return bse_kconv_split(h, n_vec, h->bphi, h->bphi + nbf, ts->nnmax, 0, h->nx, h->stream);
}

namespace {
// grid->band epilogue: sums the nsplit split-K partials, adds E psi - chi psi
// and the short-range projection out (and the Haydock hooks of `fuse`)
bse_status g2b_epilogue(bse_handle* h, const double2* psi, double2* hpsi, int n_vec, const bse_dotfuse* fuse,
                        bool wait_side, int nsplit) {
  const int nc = n_vec * h->na;
  struct {
    int nsplit;
  } p{nsplit};
  if (wait_side) cudaStreamWaitEvent(h->stream, h->ev_join, 0);   // short-range c' ready
  const int blocks = bse_tc_final_blocks(h);
  bse_dotfuse f = fuse ? *fuse : bse_dotfuse();
  auto final_grid = [&](int) { return dim3((unsigned)blocks, (unsigned)n_vec); };
  const double2* srp = h->sr_cp;
  const float2* apf = h->a_proj_f;
#define G2B_NA(NA_, FUSED_)                                                                                      \
  BSE_PROF(h, BSE_K_PREP,                                                                                         \
           (g2b_final_na<NA_, 1, FUSED_><<<final_grid(NA_), 256, 0, h->stream>>>(                                 \
               (const float2*)h->part, p.nsplit, const_cast<double2*>(psi), h->psi_f, hpsi, h->e_nk, h->chi, apf, \
               srp, h->nk, h->nb, h->np, nc, f)))
  if (h->na == 6 && f.fused_update) {
    G2B_NA(6, true);
  } else if (h->na == 6) {
    G2B_NA(6, false);
  } else if (h->na == 1 && f.fused_update) {
    G2B_NA(1, true);
  } else if (h->na == 1) {
    G2B_NA(1, false);
  } else {
    if (f.fused_update) return bse_fail(h, BSE_ERR_UNSUPPORTED, "fused Haydock update needs 1 or 6 core states");
    BSE_PROF(h, BSE_K_PREP,
             g2b_final<<<dim3((unsigned)blocks, (unsigned)n_vec), 256, 0, h->stream>>>(
                 (const float2*)h->part, p.nsplit, psi, hpsi, h->e_nk, h->chi, h->a_proj, h->sr_cp, h->nk, h->nb,
                 h->na, h->np, nc, f));
  }
#undef G2B_NA
  return bse_cuda_check(h, cudaGetLastError(), "g2b_final launch");
}
}  // namespace

bse_status bse_tc_grid_to_band(bse_handle* h, const double2* psi, double2* hpsi, int n_vec,
                               const bse_dotfuse* fuse, bool wait_side) {
  TcState* ts = (TcState*)h->tmap_host;
  int ns = 1;
  bse_status s = g2b_range(h, n_vec, 0, (h->nx + TC_KB - 1) / TC_KB, 0, ts->smax, &ns, h->stream);
  if (s != BSE_OK) return s;
  return g2b_epilogue(h, psi, hpsi, n_vec, fuse, wait_side, ns);
}

// One-pass step (k_onepass.cu) for one pass over n_vec vectors: band->grid,
// k-transform and grid->band slab by slab in one persistent kernel, then the
// grid->band epilogue on its single partial-sum slot.
bse_status bse_tc_apply_onepass(bse_handle* h, const double2* psi, double2* hpsi, int n_vec,
                                const bse_dotfuse* fuse, bool wait_side) {
  TcState* ts = (TcState*)h->tmap_host;
  const int rows = 16;
  const size_t nbp = (size_t)h->nk * ts->nnmax * ts->kp;
  const uint64_t x64 = (uint64_t)(h->nx + TC_KB - 1) / TC_KB;
  const size_t nbf = (size_t)h->nk * x64 * ts->nnmax * TC_KB;
  CUtensorMap maps[8];
  maps[0] = ts->a2_hi;
  maps[1] = ts->a2_lo;
  maps[2] = ts->a2m_hi;
  maps[3] = ts->a2m_lo;
  if (!make_map(&maps[4], h->bpsi, ts->kp, rows, h->nk, ts->kp, (uint64_t)ts->nnmax * ts->kp, rows) ||
      !make_map(&maps[5], h->bpsi + nbp, ts->kp, rows, h->nk, ts->kp, (uint64_t)ts->nnmax * ts->kp, rows) ||
      !make_map_tiled(&maps[6], h->bphi, rows, ts->nnmax, x64, h->nk, rows) ||
      !make_map_tiled(&maps[7], h->bphi + nbf, rows, ts->nnmax, x64, h->nk, rows))
    return bse_fail(h, BSE_ERR_CUDA, "tensor map encoding failed");
  OnePassParams p{};
  p.nk = h->nk;
  p.nx = h->nx;
  p.nb = h->nb;
  p.nc = n_vec * h->na;
  p.nslab = (h->nx + TC_M - 1) / TC_M;
  p.kb_b2g = (ts->kp + TC_KB - 1) / TC_KB;
  p.lag = h->op_lag;
  p.stages = h->op_stages;
  p.tmem_cols = 128;
  p.nnmax = ts->nnmax;
  p.lbo = (int)ts->lbo;
  p.sbo = (int)ts->sbo;
  p.l2hint = h->op_l2hint;
  p.phi = (float2*)h->phi;
  p.part = (float2*)h->part;
  p.bphi_hi = h->bphi;
  p.bphi_lo = h->bphi + nbf;
  p.w = (const float*)h->w;
  p.sync = ts->sync;
  p.err = ts->err;
  p.wait_ns = h->tc_wait_ns;
  // as few k per CTA as the SMs allow, the same number on every CTA (the slab
  // counters pace every CTA to the busiest); SMs left over run the
  // short-range kernels of the side stream
  const int kpc = (h->nk + ts->sms - 1) / ts->sms;
  const int grid = (h->nk + kpc - 1) / kpc;
  cudaError_t e = cudaSuccess;
  BSE_PROF(h, BSE_K_ONE_PASS, e = bse_onepass_launch(h->nk3[0], grid, maps, p, h->stream));
  if (e != cudaSuccess) return bse_cuda_check(h, e, "one-pass launch");
  return g2b_epilogue(h, psi, hpsi, n_vec, fuse, wait_side, 1);
}

namespace {
// largest n_vec the one-pass step takes on this handle (0: none)
int onepass_max_vec(const bse_handle* h, int stages) {
  const TcState* ts = (const TcState*)h->tmap_host;
  if (!ts || h->prec != BSE_PREC_SPLIT_BF16 || h->na > 8) return 0;
  if (2 * h->nb > TC_M || ts->kp > 2 * TC_KB || h->nx % 8 != 0 || !bse_kconv_takes_slabs(h)) return 0;
  const int grid = std::min(ts->sms, h->nk);
  if (grid < 1 || (h->nk + grid - 1) / grid > OP_MAX_KPC) return 0;
  if (bse_onepass_smem(h->nk3[0], stages) > 227 * 1024) return 0;
  if (bse_onepass_max_blocks_per_sm(h->nk3[0], stages) < 1) return 0;
  return std::min(8 / h->na, h->max_vec);
}
}  // namespace

// Schedule of the split-bf16 step (see bse_set_schedule in bse.h).
extern "C" bse_status bse_set_schedule(bse_handle* h, int schedule, int lag, int stages, int flags) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (schedule < BSE_SCHED_TWO_PASS || schedule > BSE_SCHED_ONE_PASS || lag < 0 || lag > 3 || stages < 0 ||
      stages == 1 || stages > 5 || flags < 0 || flags > 1)
    return bse_fail(h, BSE_ERR_INVALID_ARG,
                    "set_schedule: need schedule 0..2, lag 0..3, stages 0 or 2..5, flags 0 or 1");
  if (h->prec != BSE_PREC_SPLIT_BF16 || !h->tmap_host) return BSE_OK;
  if (lag == 0) lag = 2;
  if (stages == 0) stages = 5;
  if (schedule == BSE_SCHED_ONE_PASS && onepass_max_vec(h, stages) < 1)
    return bse_fail(h, BSE_ERR_UNSUPPORTED,
                    "set_schedule: the one-pass step needs 2 Nb <= 128, N_alpha <= 8, a 4^3 or 8^3 k mesh, a "
                    "grid of a multiple of 8 points and at most 4 k points per SM");
  const bse_status ss = bse_cuda_check(h, cudaStreamSynchronize(h->stream), "set_schedule sync");
  if (ss != BSE_OK) return ss;
  h->sched = schedule;
  h->op_lag = lag;
  h->op_stages = stages;
  h->op_l2hint = flags & BSE_SCHED_L2_HINT ? 1 : 0;
  h->op_max_vec = schedule == BSE_SCHED_ONE_PASS ? onepass_max_vec(h, stages) : 0;
  bse_drop_graph(h);
  return BSE_OK;
}

extern "C" int bse_schedule(const bse_handle* h) { return h ? h->sched : -1; }

// The step in x-slabs: band->grid of every slab on the handle's stream, and
// for each slab, once its band->grid is done, the k-transform and grid->band
// of that slab on a second stream -- so a slab's k-transform runs beside the
// next slab's contractions -- then the epilogue over every slab's partials.
bse_status bse_tc_apply_slabbed(bse_handle* h, const double2* psi, double2* hpsi, int n_vec,
                                const bse_dotfuse* fuse, bool wait_side) {
  TcState* ts = (TcState*)h->tmap_host;
  const int S = h->slabs;
  const int mt = (h->nx + TC_M - 1) / TC_M;
  const int kbt = (h->nx + TC_KB - 1) / TC_KB;
  const size_t nbf = (size_t)h->nk * kbt * ts->nnmax * TC_KB;
  const int sps = ts->smax / S > 1 ? ts->smax / S : 1;   // split-K parts per slab
  bse_status s = BSE_OK;
  for (int i = 0; i < S && s == BSE_OK; ++i) {
    s = b2g_range(h, n_vec, mt * i / S, mt * (i + 1) / S, h->stream);
    cudaEventRecord(h->ev_slab[i], h->stream);
  }
  if (s != BSE_OK) return s;
  int base = 0;
  h->cur = h->side2;
  for (int i = 0; i < S && s == BSE_OK; ++i) {
    const int m0 = mt * i / S, m1 = mt * (i + 1) / S;
    const int x0 = m0 * TC_M, x1 = m1 * TC_M < h->nx ? m1 * TC_M : h->nx;
    cudaStreamWaitEvent(h->side2, h->ev_slab[i], 0);
    s = bse_kconv_split(h, n_vec, h->bphi, h->bphi + nbf, ts->nnmax, x0, x1, h->side2);
    if (s != BSE_OK) break;
    int ns = 0;
    const int kb1 = (x1 + TC_KB - 1) / TC_KB;
    s = g2b_range(h, n_vec, x0 / TC_KB, kb1, base, sps, &ns, h->side2);
    base += ns;
  }
  h->cur = nullptr;
  cudaEventRecord(h->ev_side2, h->side2);
  cudaStreamWaitEvent(h->stream, h->ev_side2, 0);
  if (s != BSE_OK) return s;
  return g2b_epilogue(h, psi, hpsi, n_vec, fuse, wait_side, base);
}

void bse_tc_tiles(const bse_handle* h, int* split, int* stages) {
  const TcState* ts = (const TcState*)h->tmap_host;
  *split = ts ? ts->smax : 0;
  *stages = ts ? ts->stages : 0;
}

bool bse_tc_fused_update_ok(const bse_handle* h, int n_vec) {
  const TcState* ts = (const TcState*)h->tmap_host;
  if (!ts || h->prec != BSE_PREC_SPLIT_BF16 || (h->na != 1 && h->na != 6)) return false;
  int per_sm = 0;
  const cudaError_t e = h->na == 6
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, g2b_final_na<6, 1, true>, 256, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, g2b_final_na<1, 1, true>, 256, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (long long)per_sm * ts->sms >= (long long)bse_tc_final_blocks(h) * n_vec;
}

bse_operand_out bse_tc_operand(const bse_handle* h) {
  bse_operand_out o;
  const TcState* ts = (const TcState*)h->tmap_host;
  if (!ts || h->prec != BSE_PREC_SPLIT_BF16) return o;
  const size_t nbp = (size_t)h->nk * ts->nnmax * ts->kp;
  o.hi = h->bpsi;
  o.lo = h->bpsi + nbp;
  o.psi_f = h->psi_f;
  o.nk = h->nk;
  o.nb = h->nb;
  o.na = h->na;
  o.kp = ts->kp;
  o.nnmax = ts->nnmax;
  return o;
}

int bse_tc_final_blocks(const bse_handle* h) {
  const size_t nkb = (size_t)h->nk * h->nb;
  // one thread per (k, n, alpha) of a vector up to four blocks per SM,
  // grid-stride beyond: every block's <psi|H psi> partial is reduced again by
  // each block of the Haydock update (FP64, a slow pipe on this part), so the
  // count is capped; four per SM measured 28 us against 33 us at two per SM
  // on the L2,3 workload
  const size_t threads = nkb * (size_t)h->na;
  size_t bk = (threads + 255) / 256;
  const TcState* ts = (const TcState*)h->tmap_host;
  const size_t cap = ts && ts->sms > 0 ? (size_t)4 * ts->sms : 608;
  if (bk > cap) bk = cap;
  if (bk > BSE_FINAL_BLOCKS) bk = BSE_FINAL_BLOCKS;
  return (int)bk;
}

namespace {
// partial-sum buffer for `need` split-K slots (outside any stream capture)
bse_status ensure_part_cap(bse_handle* h, TcState* ts, int need) {
  if (need <= ts->part_cap) return BSE_OK;
  float2* np = nullptr;
  if (cudaMalloc((void**)&np, (size_t)need * h->nk * h->nb * h->na * h->max_vec * sizeof(float2)) != cudaSuccess) {
    cudaGetLastError();
    return bse_fail(h, BSE_ERR_OOM, "partial-sum buffer");
  }
  cudaFree(h->part);
  h->part = (float*)np;
  ts->part_cap = need;
  return BSE_OK;
}

// slab count 1, 2 or 4 (streams and events created on first use)
bse_status apply_slabs(bse_handle* h, TcState* ts, int slabs) {
  if (slabs > 1) {
    if (!h->side2) {
      if (cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&h->ev_side2, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return bse_fail(h, BSE_ERR_CUDA, "slab stream creation failed");
      }
      for (auto& e : h->ev_slab)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
          cudaGetLastError();
          return bse_fail(h, BSE_ERR_CUDA, "slab event creation failed");
        }
    }
    const int sps = ts->smax / slabs > 1 ? ts->smax / slabs : 1;
    const bse_status s = ensure_part_cap(h, ts, slabs * sps);
    if (s != BSE_OK) return s;
  }
  h->slabs = slabs;
  bse_drop_graph(h);
  return BSE_OK;
}

bool slabs_allowed(const bse_handle* h, int slabs) {
  return slabs == 1 || (bse_kconv_takes_slabs(h) && (h->nx + TC_M - 1) / TC_M >= slabs);
}
}  // namespace

// Number of x-slabs of the tensor-core step (see bse_set_slabs in bse.h).
extern "C" bse_status bse_set_slabs(bse_handle* h, int slabs) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (slabs != 1 && slabs != 2 && slabs != 4) return bse_fail(h, BSE_ERR_INVALID_ARG, "set_slabs: slabs must be 1, 2 or 4");
  if (h->prec != BSE_PREC_SPLIT_BF16 || !h->tmap_host) return BSE_OK;
  if (!slabs_allowed(h, slabs))
    return bse_fail(h, BSE_ERR_UNSUPPORTED, "set_slabs: needs a 4^3 or 8^3 k mesh, an even grid and one 128-row tile per slab");
  const bse_status ss = bse_cuda_check(h, cudaStreamSynchronize(h->stream), "set_slabs sync");
  if (ss != BSE_OK) return ss;
  return apply_slabs(h, (TcState*)h->tmap_host, slabs);
}

extern "C" int bse_slabs(const bse_handle* h) { return h ? h->slabs : 0; }

// Limit of every pipeline wait of the tensor-core kernel (see bse_set_wait_limit in bse.h).
extern "C" bse_status bse_set_wait_limit(bse_handle* h, double seconds) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (!(seconds >= 1e-6 && seconds <= 60.0))
    return bse_fail(h, BSE_ERR_INVALID_ARG, "set_wait_limit: need 1e-6 <= seconds <= 60");
  const bse_status ss = bse_cuda_check(h, cudaStreamSynchronize(h->stream), "set_wait_limit sync");
  if (ss != BSE_OK) return ss;
  h->tc_wait_ns = (unsigned long long)(seconds * 1e9);
  bse_drop_graph(h);
  return BSE_OK;
}

// Fixed tile parameters (see bse_set_tiles in bse.h).
extern "C" bse_status bse_set_tiles(bse_handle* h, int split_k, int stages) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (split_k < 0 || split_k > 16 || stages < 0 || stages == 1 || stages > 8)
    return bse_fail(h, BSE_ERR_INVALID_ARG, "set_tiles: need 0 <= split_k <= 16 and stages 0 or 2..8");
  if (h->prec != BSE_PREC_SPLIT_BF16 || !h->tmap_host) return BSE_OK;
  TcState* ts = (TcState*)h->tmap_host;
  {
    const bse_status ss = bse_cuda_check(h, cudaStreamSynchronize(h->stream), "set_tiles sync");
    if (ss != BSE_OK) return ss;
  }
  if (split_k == 0) {   // back to the rule of bse_setup
    const int kbt = (h->nx + TC_KB - 1) / TC_KB;
    const int units = h->nk * ((2 * h->nb + TC_M - 1) / TC_M);
    int sp = 1;
    while (units * sp < 8 * ts->sms && kbt / (sp * 2) >= 8) sp *= 2;
    split_k = sp;
  }
  if (split_k > ts->part_cap) {
    float2* np = nullptr;
    if (cudaMalloc((void**)&np, (size_t)split_k * h->nk * h->nb * h->na * h->max_vec * sizeof(float2)) !=
        cudaSuccess) {
      cudaGetLastError();
      return bse_fail(h, BSE_ERR_OOM, "set_tiles: partial-sum buffer");
    }
    cudaFree(h->part);
    h->part = (float*)np;
    ts->part_cap = split_k;
  }
  ts->smax = split_k;
  ts->stages = stages;
  bse_drop_graph(h);
  return apply_slabs(h, ts, h->slabs);   // the slabs' partial slots for the new split
}

// Timed search over the tensor-core tile parameters of one handle (see
// bse_autotune in bse.h).
extern "C" bse_status bse_autotune(bse_handle* h, int n_vec, int reps, int* split_out, int* stages_out) {
  if (!h) return BSE_ERR_INVALID_ARG;
  if (n_vec < 1 || n_vec > h->max_vec || reps < 1)
    return bse_fail(h, BSE_ERR_INVALID_ARG, "autotune: need 1 <= n_vec <= max_vec and reps >= 1");
  if (h->prec != BSE_PREC_SPLIT_BF16 || !h->tmap_host) {
    if (split_out) *split_out = 0;
    if (stages_out) *stages_out = 0;
    return BSE_OK;
  }
  TcState* ts = (TcState*)h->tmap_host;
  cudaStream_t st = h->stream;
  {
    const bse_status ss = bse_cuda_check(h, cudaStreamSynchronize(st), "autotune sync");
    if (ss != BSE_OK) return ss;
  }
  const int kbt = (h->nx + TC_KB - 1) / TC_KB;
  std::vector<int> splits;
  for (int s = 1; s <= 16 && s <= kbt; s *= 2) splits.push_back(s);
  const int nn = tile_n(round_up(2 * n_vec * h->na, 16));
  const int fit = fit_stages(nn);
  std::vector<int> stages;
  for (int s : {3, 4, 6, 8})
    if (s <= fit) stages.push_back(s);
  if (stages.empty()) stages.push_back(fit);
  if (splits.back() > ts->part_cap) {   // partial sums for the largest split-K factor tried
    float2* np = nullptr;
    if (cudaMalloc((void**)&np, (size_t)splits.back() * h->nk * h->nb * h->na * h->max_vec * sizeof(float2)) !=
        cudaSuccess) {
      cudaGetLastError();
      return bse_fail(h, BSE_ERR_OOM, "autotune: partial-sum buffer");
    }
    cudaFree(h->part);
    h->part = (float*)np;
    ts->part_cap = splits.back();
  }
  double2 *psi = nullptr, *hpsi = nullptr;
  const size_t bytes = (size_t)n_vec * h->N * sizeof(double2);
  if (cudaMalloc((void**)&psi, bytes) != cudaSuccess || cudaMalloc((void**)&hpsi, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(psi);
    return bse_fail(h, BSE_ERR_OOM, "autotune: test vectors");
  }
  cudaMemsetAsync(psi, 0x3f, bytes, st);   // finite test values (~4.8e-4); the timing does not depend on them
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int keep_split = ts->smax, keep_stages = ts->stages, keep_slabs = h->slabs;
  int best_split = keep_split, best_stages = keep_stages, best_slabs = keep_slabs;
  float best = 3.4e38f;
  bse_status s = BSE_OK;
  std::vector<int> slab_set;
  for (int sl : {1, 2})
    if (slabs_allowed(h, sl)) slab_set.push_back(sl);
  for (int sl : slab_set)
  for (int sp : splits) {
    if (s != BSE_OK) break;
    for (int sg : stages) {
      ts->smax = sp;
      ts->stages = sg;
      s = apply_slabs(h, ts, sl);
      if (s != BSE_OK) break;
      s = bse_apply_device(h, psi, hpsi, n_vec);   // warm-up
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && s == BSE_OK; ++r) s = bse_apply_device(h, psi, hpsi, n_vec);
      cudaEventRecord(e1, st);
      if (s == BSE_OK) s = bse_cuda_check(h, cudaEventSynchronize(e1), "autotune timing");
      if (s != BSE_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        best_split = sp;
        best_stages = sg;
        best_slabs = sl;
      }
    }
    if (s != BSE_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(psi);
  cudaFree(hpsi);
  if (s == BSE_OK) s = bse_tc_status(h);
  if (s != BSE_OK) {
    ts->smax = keep_split;
    ts->stages = keep_stages;
    apply_slabs(h, ts, keep_slabs);
    return s;
  }
  ts->smax = best_split;
  ts->stages = best_stages;
  s = apply_slabs(h, ts, best_slabs);
  if (s != BSE_OK) return s;
  if (split_out) *split_out = best_split;
  if (stages_out) *stages_out = best_stages;
  return BSE_OK;
}

bse_status bse_tc_status(bse_handle* h) {
  if (h->prec != BSE_PREC_SPLIT_BF16 || !h->tmap_host) return BSE_OK;
  TcState* ts = (TcState*)h->tmap_host;
  int e = 0;
  if (cudaMemcpy(&e, ts->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bse_cuda_check(h, cudaGetLastError(), "tc status");
  if (e) {
    // reported once: clear the word so that later calls on the handle start clean
    if (cudaMemset(ts->err, 0, sizeof(int)) != cudaSuccess) return bse_cuda_check(h, cudaGetLastError(), "tc status reset");
    return bse_fail(h, BSE_ERR_TIMEOUT, "tensor-core pipeline wait timed out");
  }
  return BSE_OK;
}
