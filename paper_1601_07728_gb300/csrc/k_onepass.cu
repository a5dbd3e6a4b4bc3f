// One-pass split-bf16 step of Algorithm 1 (Sec. 3.2.1): band->grid
// contraction, k->R sum, x W(x, R), R->k sum and grid->band contraction in one
// persistent kernel, slab by slab over the real-space grid, so that U~ = e^{ik.x}u
// can stream from HBM once per H psi instead of once per contraction.
//
// The grid is cut into slabs of 128 points.  For slab s:
//   band->grid  Phi_k[x][j] = sum_q U~_k[x][q] Bpsi_k[j][q]     for every k, x in s
//   k-transform Phi'(x, k) = (1/Nk) sum_R e^{-ik.R} W(x,R) sum_k' e^{ik'.R} Phi(x, k')
//   grid->band  D_k[q][j] += sum_{x in s} U~_k[x][q] Phi'_k[x][j]
// (the complex-as-real forms of tc_gemm, same operand splits hi*hi + hi*lo +
// lo*hi, FP32 accumulation in tensor memory; grid->band reads the row-major
// U~ tile as an MN-major operand).  The k-transform of a grid point needs the
// band->grid results of every k, so each slab passes through every CTA twice:
// CTA b owns k = b, b + G, ... (at most 4) and does their band->grid tiles of
// slab s, a share of the slab's k-transform units (8 grid points x one column
// each, on all k), and, once every unit of slab s is done on every CTA, the
// grid->band tiles of slab s for its k, reading the slab's U~ tiles again
// (from L2 while the slabs between the two reads fit there).  The producer
// issues those grid->band tiles between the band->grid tiles of later slabs
// as soon as the slab is ready, and holds at most lag + 1 slabs between their
// two reads; a record per pipeline stage tells the MMA issuer which tile it
// holds.  The grid->band accumulators D_k stay in tensor memory across all
// slabs, so the result needs no split-K partial sums.
//
// Warp roles (480 threads): warp 0 issues TMA copies into a ring of 36 KB
// stages, warp 1 issues tcgen05.mma from one thread, warps 2-5 drain the
// band->grid accumulators into Phi (FP32, global) and at the end D_k into the
// result, warps 6-13 run the k-transform units in a 32 KB shared tile, warp 14
// polls the per-slab k-transform counters and hands readiness to the producer
// through shared memory.  Cross-CTA order: per slab, a band->grid counter
// (each epilogue warp adds its tiles after one fence) and a k-transform
// counter (one per unit, after a barrier and one fence); consumers read them
// with acquire loads.  Every wait is bounded in time; a wait that gives up
// raises a grid-wide abort word and the error word, and every role then
// stops, drains its own copies and MMAs, and frees tensor memory.  The last
// CTA to finish resets the counters for the next launch.  The kernel needs all
// CTAs resident at once (one per SM, checked by the host).
#include "bse_internal.cuh"
#include "dft_dev.cuh"
#include "tc_ptx.cuh"

#include "k_onepass.cuh"

namespace {

constexpr int OP_M = 128;          // grid points per slab = rows of a band->grid tile
constexpr int OP_KB = 64;          // K elements per stage (one 128-byte swizzle row)
constexpr int OP_NN = 16;          // MMA N: 2 rows per complex column, up to 8 columns
constexpr uint32_t A_BYTES = OP_M * 128;            // one bf16 plane of the U~ tile of a stage
constexpr uint32_t B_BYTES = OP_NN * 128;           // one bf16 plane of the B tile
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr uint32_t MN_BOX = 64 * 128;               // grid->band A box: 64 x rows of 64 q
constexpr int KC_XW = 8;           // grid points per k-transform unit
constexpr int KC_THREADS = 256;
constexpr int OP_THREADS = 192 + KC_THREADS + 32;   // + the counter poller warp
constexpr unsigned long long DRAIN_NS = 2000000000ull;
// stage records (producer -> MMA issuer): tile kind, k index (bits 4-6),
// first stage of a tile (zeroes the accumulator), last stage of a
// band->grid tile (hands the accumulator to the epilogue)
constexpr int REC_B2G = 1, REC_G2B = 2, REC_FIRST = 4, REC_LAST = 8;

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat16 lo_half, __nv_bfloat16 hi_half) {
  const __nv_bfloat162 v = __halves2bfloat162(lo_half, hi_half);
  return *reinterpret_cast<const uint32_t*>(&v);
}

// grid-wide abort word and error word after a failed wait
__device__ __forceinline__ void op_raise(const OnePassParams& p, volatile int* labort) {
  atomicExch(p.err, 1);
  atomicExch(p.sync + 2 * p.nslab + 1, 1u);
  *labort = 1;
}

// bounded wait until *c >= target; false on timeout or abort (local or
// grid-wide).  Polls back off, so that the waiters of every CTA do not crowd
// the counter's L2 line while the other CTAs update it.
__device__ bool op_wait_count(const OnePassParams& p, const unsigned* c, unsigned target, volatile int* labort) {
  if (ld_acquire_gpu(c) >= target) return true;
  const volatile unsigned* gab = p.sync + 2 * p.nslab + 1;
  const unsigned long long t0 = gtime();
  while (true) {
    __nanosleep(128);
    if (ld_acquire_gpu(c) >= target) return true;
    if (*gab || *labort) return false;
    if (gtime() - t0 > p.wait_ns) return false;
  }
}

// bounded mbarrier wait that also gives up on the grid-wide abort word (read
// from global memory only every 64 polls)
__device__ bool op_mbar_wait(const OnePassParams& p, uint32_t a, uint32_t parity, volatile int* labort) {
  if (mbar_try(a, parity)) return true;
  const volatile unsigned* gab = p.sync + 2 * p.nslab + 1;
  const unsigned long long t0 = gtime();
  for (unsigned n = 1;; ++n) {
    if (mbar_try(a, parity)) return true;
    if (*labort) return false;
    if ((n & 63) == 0 && (*gab || gtime() - t0 > p.wait_ns)) return false;
  }
}

// bounded wait until the shared word at addr exceeds v (CTA-scope acquire)
__device__ bool op_wait_flag(const OnePassParams& p, uint32_t addr, int v, volatile int* labort) {
  if (ld_acquire_cta_shared(addr) > v) return true;
  const volatile unsigned* gab = p.sync + 2 * p.nslab + 1;
  const unsigned long long t0 = gtime();
  for (unsigned n = 1;; ++n) {
    if (ld_acquire_cta_shared(addr) > v) return true;
    if (*labort) return false;
    if ((n & 63) == 0 && (*gab || gtime() - t0 > p.wait_ns)) return false;
  }
}

__device__ __forceinline__ int slab_points(const OnePassParams& p, int s) {
  const int r = p.nx - s * OP_M;
  return r < OP_M ? r : OP_M;
}
// k-transform units of slab s (8 grid points x one column each)
__device__ __forceinline__ int slab_units(const OnePassParams& p, int s) {
  return ((slab_points(p, s) + KC_XW - 1) / KC_XW) * p.nc;
}

// One k-transform unit: column c, the 8 grid points of block xb (xb*8 ..
// xb*8 + 7), every k.  Its band->grid results are contiguous (unit-major
// Phi, written so by the epilogue) and arrive in the shared tile by one bulk
// copy; thread tid = (pencil group g, x pair xp) then owns one pencil per
// pass: forward along axes 2, 1, 0, W(x, R)/Nk, inverse along axes 0, 1, 2.
// The four threads of a pencil group hold the 8 grid points of a row of the
// K-tiled grid->band operand between them; a 4 x 4 lane transpose gives each
// of them 16 contiguous bytes (8 points of one bf16 plane of re or im) per k.
template <int N>
__device__ __forceinline__ bool kc_unit(const OnePassParams& p, float4* S, uint32_t kc_bar, uint32_t phase, int c,
                                        int xb, int tid, volatile int* labort, volatile int* kc_fail,
                                        volatile int* kc_copies) {
  constexpr int NK = N * N * N, NP = N * N;
  constexpr int XP = KC_XW / 2;
  constexpr int NG = KC_THREADS / XP;
  static_assert(NP <= NG && XP == 4, "one pencil per thread and pass; four x pairs per unit");
  const int xp = tid & (XP - 1), g = tid / XP;
  const int xbase = xb * KC_XW;
  const int x = xbase + 2 * xp;
  const bool act = g < NP;
  // W(x, R)/Nk of pass C, loaded while the tile arrives
  float2 wr[N];
  {
    const float inv = 1.f / (float)NK;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      wr[j] = act ? __ldg(reinterpret_cast<const float2*>(p.w + (size_t)(j * NP + g) * p.nx + x))
                  : make_float2(0.f, 0.f);
      wr[j].x *= inv;
      wr[j].y *= inv;
    }
  }
  if (tid == 0) {
    // Phi of the unit, [k][8 points], written by other CTAs (made visible by
    // the acquire of the band->grid counter): read through the async proxy
    fence_proxy_async_global();
    kc_copies[0] += 1;   // issued (the abort drain waits for copies not seen to land)
    mbar_expect_tx(kc_bar, NK * KC_XW * 8);
    bulk_load(smem_u32(S), p.phi + ((size_t)xb * p.nc + c) * NK * KC_XW, NK * KC_XW * 8, kc_bar);
  }
  // every thread of the unit takes the same branch: a failed wait is agreed on
  // through shared memory (set once, never cleared: the role then ends)
  if (!op_mbar_wait(p, kc_bar, phase, labort)) *kc_fail = 1;
  named_bar_sync(1, KC_THREADS);
  if (*kc_fail) return false;
  if (tid == 0) kc_copies[1] = kc_copies[0];   // landed
  float2 tw[N];   // the radix-2/4/8 butterflies take no twiddle table
#pragma unroll
  for (int j = 0; j < N; ++j) tw[j] = make_float2(0.f, 0.f);
  // pass A: forward along axis 2 (k = g N + j)
  if (act) {
    float2 va[N], vb[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float4 q = S[(g * N + j) * XP + xp];
      va[j] = make_float2(q.x, q.y);
      vb[j] = make_float2(q.z, q.w);
    }
    dftN<float, N, +1>(va, tw);
    dftN<float, N, +1>(vb, tw);
#pragma unroll
    for (int j = 0; j < N; ++j) S[(g * N + j) * XP + xp] = make_float4(va[j].x, va[j].y, vb[j].x, vb[j].y);
  }
  named_bar_sync(1, KC_THREADS);
  // pass B: forward along axis 1; pencil g = (m0, m2)
  if (act) {
    const int kb = (g / N) * NP + (g % N);
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
  named_bar_sync(1, KC_THREADS);
  // pass C: forward along axis 0, x W(x, R)/Nk, inverse along axis 0; pencil g = (m1, m2)
  if (act) {
    float2 va[N], vb[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float4 q = S[(j * NP + g) * XP + xp];
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
    for (int j = 0; j < N; ++j) S[(j * NP + g) * XP + xp] = make_float4(va[j].x, va[j].y, vb[j].x, vb[j].y);
  }
  named_bar_sync(1, KC_THREADS);
  // pass D: inverse along axis 1
  if (act) {
    const int kb = (g / N) * NP + (g % N);
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
  named_bar_sync(1, KC_THREADS);
  // pass E: inverse along axis 2, bf16 hi/lo split, and the store to the
  // K-tiled planes [k][x/64][row][64] (rows 2c = re, 2c + 1 = im)
  if (act) {
    float2 va[N], vb[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float4 q = S[(g * N + j) * XP + xp];
      va[j] = make_float2(q.x, q.y);
      vb[j] = make_float2(q.z, q.w);
    }
    dftN<float, N, -1>(va, tw);
    dftN<float, N, -1>(vb, tw);
    const size_t x64 = (size_t)((p.nx + 63) >> 6);
#pragma unroll
    for (int j = 0; j < N; ++j) {
      // this thread's two points as bf16 pairs: kind 0 = re hi, 1 = re lo, 2 = im hi, 3 = im lo
      __nv_bfloat16 h0, l0, h1, l1, h2, l2, h3, l3;
      split_bf(va[j].x, h0, l0);
      split_bf(vb[j].x, h1, l1);
      split_bf(va[j].y, h2, l2);
      split_bf(vb[j].y, h3, l3);
      uint32_t w[4];
      w[0] = bf2_bits(h0, h1);
      w[1] = bf2_bits(l0, l1);
      w[2] = bf2_bits(h2, h3);
      w[3] = bf2_bits(l2, l3);
      // lane xp keeps kind xp of all four x pairs: out[m] = kind xp of x pair m
      uint32_t out[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int send = (xp + r) & 3, from = (xp - r) & 3;
        const uint32_t v = send == 0 ? w[0] : send == 1 ? w[1] : send == 2 ? w[2] : w[3];
        // whole warps are active here (pencil groups fill warps), each lane
        // reading from its own group of four
        const uint32_t got = __shfl_sync(0xffffffffu, v, (threadIdx.x & 28) | from);
        out[0] = from == 0 ? got : out[0];
        out[1] = from == 1 ? got : out[1];
        out[2] = from == 2 ? got : out[2];
        out[3] = from == 3 ? got : out[3];
      }
      if (xbase < p.nx) {
        const int k = g * N + j;
        const size_t o = (((size_t)k * x64 + (xbase >> 6)) * p.nnmax + 2 * c + (xp >> 1)) * 64 + (xbase & 63);
        __nv_bfloat16* dst = (xp & 1) ? p.bphi_lo : p.bphi_hi;
        *reinterpret_cast<uint4*>(dst + o) = make_uint4(out[0], out[1], out[2], out[3]);
      }
    }
  }
  return true;
}

template <int N>
__global__ void __launch_bounds__(OP_THREADS, 1)
    tc_onepass(const __grid_constant__ CUtensorMap ua_hi, const __grid_constant__ CUtensorMap ua_lo,
               const __grid_constant__ CUtensorMap um_hi, const __grid_constant__ CUtensorMap um_lo,
               const __grid_constant__ CUtensorMap bp_hi, const __grid_constant__ CUtensorMap bp_lo,
               const __grid_constant__ CUtensorMap bf_hi, const __grid_constant__ CUtensorMap bf_lo,
               const OnePassParams p) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int S = p.stages;
  float4* kc_tile = (float4*)(sm + (size_t)S * STAGE_BYTES);
  unsigned long long* bars = (unsigned long long*)(sm + (size_t)S * STAGE_BYTES + (size_t)N * N * N * KC_XW * 8);
  // bars: full[S], empty[S], tfull[2], tempty[2], gfin, kc (k-transform tile copy)
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * S + 6);
  volatile int* labort = (volatile int*)(tmem_slot + 1);
  int* consumed = (int*)(tmem_slot + 2);
  int* issued = (int*)(tmem_slot + 3);
  volatile int* rec = (volatile int*)(tmem_slot + 4);   // [S] tile record of each stage
  // slabs whose k-transform is complete on every CTA (set by the poller warp)
  int* kc_ready = (int*)(tmem_slot + 4 + OP_MAX_STAGES);
  const uint32_t kc_ready_a = smem_u32(kc_ready);
  volatile int* kc_fail = (volatile int*)(kc_ready + 1);   // a k-transform tile copy gave up
  volatile int* kc_copies = (volatile int*)(kc_ready + 2);  // tile copies issued, seen landed
  const uint32_t sbase = smem_u32(sm);
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[S + s]); };
  auto tfull = [&](int a) { return smem_u32(&bars[2 * S + a]); };
  auto tempty = [&](int a) { return smem_u32(&bars[2 * S + 2 + a]); };
  const uint32_t gfin = smem_u32(&bars[2 * S + 4]);
  const uint32_t kc_bar = smem_u32(&bars[2 * S + 5]);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;
  unsigned* b2g_cnt = p.sync;              // [nslab]
  unsigned* kc_cnt = p.sync + p.nslab;     // [nslab]

  // the k of this CTA
  int myk[OP_MAX_KPC];
  int nmy = 0;
  for (int k = blockIdx.x; k < p.nk && nmy < OP_MAX_KPC; k += G) myk[nmy++] = k;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull(a), 1);
      mbar_init(tempty(a), 4);
    }
    mbar_init(gfin, 1);
    mbar_init(kc_bar, 1);
    *labort = 0;
    *consumed = 0;
    *issued = 0;
    *kc_ready = 0;
    *kc_fail = 0;
    kc_copies[0] = 0;
    kc_copies[1] = 0;
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
  int total_stages = p.nslab * nmy * p.kb_b2g;
  for (int sl = 0; sl < p.nslab; ++sl) total_stages += nmy * ((slab_points(p, sl) + OP_KB - 1) / OP_KB);

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&ua_hi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&ua_lo) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&um_hi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&um_lo) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&bp_hi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&bp_lo) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&bf_hi) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&bf_lo) : "memory");
    // U~ is read twice per slab: keep it in L2 after the first (band->grid)
    // read, let it go after the second
    const unsigned long long keep = p.l2hint ? l2_policy_evict_last() : 0ull;
    const unsigned long long drop = p.l2hint ? l2_policy_evict_first() : 0ull;
    int it = 0;
    bool ok = true;
    // band->grid tile of (slab t, k = myk[i]): U~ rows of the slab, K blocks of q
    auto issue_b2g = [&](int t, int i) {
      for (int kb = 0; kb < p.kb_b2g; ++kb, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!op_mbar_wait(p, empty(s), ph ^ 1u, labort)) return false;
        const uint32_t st = sbase + (uint32_t)s * STAGE_BYTES;
        rec[s] = REC_B2G | (i << 4) | (kb == 0 ? REC_FIRST : 0) | (kb == p.kb_b2g - 1 ? REC_LAST : 0);
        mbar_expect_tx(full(s), STAGE_BYTES);
        if (p.l2hint) {
          tma_load_3d_hint(st, &ua_hi, full(s), kb * OP_KB, t * OP_M, myk[i], keep);
          tma_load_3d_hint(st + A_BYTES, &ua_lo, full(s), kb * OP_KB, t * OP_M, myk[i], keep);
        } else {
          tma_load_3d(st, &ua_hi, full(s), kb * OP_KB, t * OP_M, myk[i]);
          tma_load_3d(st + A_BYTES, &ua_lo, full(s), kb * OP_KB, t * OP_M, myk[i]);
        }
        tma_load_3d(st + 2 * A_BYTES, &bp_hi, full(s), kb * OP_KB, 0, myk[i]);
        tma_load_3d(st + 2 * A_BYTES + B_BYTES, &bp_lo, full(s), kb * OP_KB, 0, myk[i]);
        *(volatile int*)issued = it + 1;
      }
      return true;
    };
    // grid->band tile of (slab sl, k = myk[i]): the same U~ rows as MN-major A, K blocks of x
    auto issue_g2b = [&](int sl, int i) {
      const int kbs = (slab_points(p, sl) + OP_KB - 1) / OP_KB;
      for (int kb = 0; kb < kbs; ++kb, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!op_mbar_wait(p, empty(s), ph ^ 1u, labort)) return false;
        const uint32_t st = sbase + (uint32_t)s * STAGE_BYTES;
        const int xr = sl * OP_M + kb * OP_KB;
        rec[s] = REC_G2B | (i << 4) | (sl == 0 && kb == 0 ? REC_FIRST : 0);
        mbar_expect_tx(full(s), STAGE_BYTES);
        // A: U~ rows xr .. xr+63, q 0..63 and 64..127 (two MN-major blocks)
        if (p.l2hint) {
          tma_load_3d_hint(st, &um_hi, full(s), 0, xr, myk[i], drop);
          tma_load_3d_hint(st + MN_BOX, &um_hi, full(s), OP_KB, xr, myk[i], drop);
          tma_load_3d_hint(st + A_BYTES, &um_lo, full(s), 0, xr, myk[i], drop);
          tma_load_3d_hint(st + A_BYTES + MN_BOX, &um_lo, full(s), OP_KB, xr, myk[i], drop);
        } else {
          tma_load_3d(st, &um_hi, full(s), 0, xr, myk[i]);
          tma_load_3d(st + MN_BOX, &um_hi, full(s), OP_KB, xr, myk[i]);
          tma_load_3d(st + A_BYTES, &um_lo, full(s), 0, xr, myk[i]);
          tma_load_3d(st + A_BYTES + MN_BOX, &um_lo, full(s), OP_KB, xr, myk[i]);
        }
        // B: Phi' K tile xr/64 of k
        tma_load_4d(st + 2 * A_BYTES, &bf_hi, full(s), 0, 0, xr / OP_KB, myk[i]);
        tma_load_4d(st + 2 * A_BYTES + B_BYTES, &bf_lo, full(s), 0, 0, xr / OP_KB, myk[i]);
        *(volatile int*)issued = it + 1;
      }
      return true;
    };
    // Grid->band tiles of slab gs are issued, one per band->grid tile, as soon
    // as the k-transform of slab gs is complete on every CTA (polled), so that
    // the slab's U~ is read again while still in L2 and HBM reads of later
    // slabs stay in flight meanwhile; before the band->grid tiles of slab t
    // the producer waits for slab t - lag if it is still pending, which bounds
    // the slabs of U~ between the two reads.  Each stage's record tells the
    // MMA issuer which tile it holds.
    int gs = 0, gi = 0;   // next grid->band tile: slab gs, k index gi
    bool gready = false;  // slab gs's k-transform is complete
    auto g2b_poll = [&](int t_issued) {
      // slab gs can be complete only once its band->grid tiles were issued
      if (!gready && gs < p.nslab && gs < t_issued && ld_acquire_cta_shared(kc_ready_a) > gs) {
        fence_proxy_async_global();
        gready = true;
      }
      return gready;
    };
    auto g2b_next = [&]() {
      if (!issue_g2b(gs, gi)) return false;
      if (++gi == nmy) {
        gi = 0;
        ++gs;
        gready = false;
      }
      return true;
    };
    for (int t = 0; t < p.nslab && ok; ++t) {
      // bound on the slabs between their two reads: at most lag + 1 once the
      // band->grid tiles of slab t are issued
      while (ok && gs < t - p.lag) {
        if (!gready) {
          if (!op_wait_flag(p, kc_ready_a, gs, labort)) {
            ok = false;
            break;
          }
          fence_proxy_async_global();
          gready = true;
        }
        if (!g2b_next()) ok = false;
      }
      for (int i = 0; i < nmy && ok; ++i) {
        if (!issue_b2g(t, i)) {
          ok = false;
          break;
        }
        if (g2b_poll(t) && !g2b_next()) ok = false;
      }
    }
    // the remaining grid->band tiles
    while (ok && gs < p.nslab) {
      if (!gready) {
        if (!op_wait_flag(p, kc_ready_a, gs, labort)) {
          ok = false;
          break;
        }
        fence_proxy_async_global();
        gready = true;
      }
      if (!g2b_next()) ok = false;
    }
    if (!ok) op_raise(p, labort);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t id_b2g = idesc_bf16(OP_M, OP_NN);
    const uint32_t id_g2b = idesc_bf16(OP_M, OP_NN) | IDESC_A_MN;
    int local = 0;
    bool ok = true;
    int acc = 0;
    // every stage the producer fills, in its order; the record says which tile
    for (int it = 0; it < total_stages && ok; ++it) {
      const int s = it % S;
      const uint32_t ph = (uint32_t)(it / S) & 1u;
      if (!op_mbar_wait(p, full(s), ph, labort)) {
        ok = false;
        break;
      }
      const int r = rec[s];
      const int i = (r >> 4) & 7;
      const uint32_t st = sbase + (uint32_t)s * STAGE_BYTES;
      if (r & REC_B2G) {
        if (r & REC_FIRST) {
          acc = local & 1;
          const uint32_t aph = (uint32_t)(local >> 1) & 1u;
          ++local;
          if (!op_mbar_wait(p, tempty(acc), aph ^ 1u, labort)) {
            ok = false;
            break;
          }
        }
        *(volatile int*)consumed = it + 1;
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(acc * OP_NN);
#pragma unroll
        for (int ks = 0; ks < OP_KB / 16; ++ks) {
          const unsigned long long a_hi = sdesc_sw128(st + ks * 32);
          const unsigned long long a_lo = sdesc_sw128(st + A_BYTES + ks * 32);
          const unsigned long long b_hi = sdesc_sw128(st + 2 * A_BYTES + ks * 32);
          const unsigned long long b_lo = sdesc_sw128(st + 2 * A_BYTES + B_BYTES + ks * 32);
          mma_bf16(d, a_hi, b_hi, id_b2g, !((r & REC_FIRST) && ks == 0));
          mma_bf16(d, a_hi, b_lo, id_b2g, 1);
          mma_bf16(d, a_lo, b_hi, id_b2g, 1);
        }
        mma_commit(empty(s));
        if (r & REC_LAST) mma_commit(tfull(acc));
      } else {
        *(volatile int*)consumed = it + 1;
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(2 * OP_NN + i * OP_NN);
#pragma unroll
        for (int ks = 0; ks < OP_KB / 16; ++ks) {
          // 16 grid points (two 8-row groups) per MMA: rows advance 2048 bytes
          const unsigned long long a_hi = sdesc_mn_sw128(st + ks * 2048, p.lbo, p.sbo);
          const unsigned long long a_lo = sdesc_mn_sw128(st + A_BYTES + ks * 2048, p.lbo, p.sbo);
          const unsigned long long b_hi = sdesc_sw128(st + 2 * A_BYTES + ks * 32);
          const unsigned long long b_lo = sdesc_sw128(st + 2 * A_BYTES + B_BYTES + ks * 32);
          mma_bf16(d, a_hi, b_hi, id_g2b, !((r & REC_FIRST) && ks == 0));
          mma_bf16(d, a_hi, b_lo, id_g2b, 1);
          mma_bf16(d, a_lo, b_hi, id_g2b, 1);
        }
        mma_commit(empty(s));
      }
    }
    if (!ok) op_raise(p, labort);
    // every issued MMA retires before the accumulators are read or freed
    mma_commit(gfin);
    if (!mbar_wait(gfin, 0, labort, DRAIN_NS)) {
      const unsigned long long t0 = gtime();
      while (!mbar_try(gfin, 0) && gtime() - t0 < DRAIN_NS) {
      }
    }
  } else if (warp >= 2 && warp < 6) {
    // ---------------- epilogue (128 threads, one TMEM lane each) ----------------
    const int q = warp & 3;
    const int row_in_tile = q * 32 + lane;
    int local = 0;
    bool ok = true;
    for (int t = 0; t < p.nslab && ok; ++t) {
      for (int i = 0; i < nmy; ++i, ++local) {
        const int acc = local & 1;
        const uint32_t aph = (uint32_t)(local >> 1) & 1u;
        // the lanes agree on the outcome before the warp-wide tensor-memory load
        if (!__all_sync(0xffffffffu, op_mbar_wait(p, tfull(acc), aph, labort))) {
          if (lane == 0) op_raise(p, labort);
          ok = false;
          break;
        }
        tc_fence_after();
        float v[16];
        tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * OP_NN), v);
        const int x = t * OP_M + row_in_tile;
        if (x < p.nx) {
          // unit-major Phi [x/8][c][k][x%8]: a k-transform unit's input is contiguous
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (c < p.nc)
              p.phi[(((size_t)(x >> 3) * p.nc + c) * p.nk + myk[i]) * KC_XW + (x & 7)] = make_float2(v[2 * c], v[2 * c + 1]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty(acc));
      }
      // release this warp's rows of Phi of slab t (every k of this CTA) to the
      // k-transform units of every CTA: one fence after the warp's stores
      __syncwarp();
      if (ok && lane == 0) {
        __threadfence();
        atomicAdd(b2g_cnt + t, (unsigned)nmy);
      }
    }
    // grid->band result: D_k[q][j] -> part[k][c][n] (the split-K slot 0 layout)
    if (ok && __all_sync(0xffffffffu, op_mbar_wait(p, gfin, 0, labort))) {
      tc_fence_after();
      for (int i = 0; i < nmy; ++i) {
        float v[16], pv[16];
        tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(2 * OP_NN + i * OP_NN), v);
#pragma unroll
        for (int e = 0; e < 16; ++e) pv[e] = __shfl_xor_sync(0xffffffffu, v[e], 1);
        const int n = row_in_tile >> 1;
        if ((lane & 1) == 0 && n < p.nb) {
          float2* o = p.part + (size_t)myk[i] * p.nc * p.nb + n;
#pragma unroll
          for (int c = 0; c < 8; ++c)
            if (c < p.nc) o[(size_t)c * p.nb] = make_float2(v[2 * c] + pv[2 * c + 1], v[2 * c + 1] - pv[2 * c]);
        }
      }
    }
  } else if (warp == 6 + KC_THREADS / 32) {
    // ---------------- counter poller ----------------
    // watches the k-transform counters of every slab and hands the result to
    // the producer through shared memory, so the producer's issue loop never
    // waits on an L2 round trip
    if (lane == 0) {
      for (int sl = 0; sl < p.nslab; ++sl) {
        if (!op_wait_count(p, kc_cnt + sl, (unsigned)slab_units(p, sl), labort)) {
          op_raise(p, labort);
          break;
        }
        st_release_cta_shared(kc_ready_a, sl + 1);
      }
    }
  } else if (warp >= 6) {
    // ---------------- k-transform units ----------------
    const int tid = threadIdx.x - 192;
    __shared__ int kc_go;
    unsigned kc_phase = 0;   // completed copies into the k-transform tile
    const int nu_full = (OP_M / KC_XW) * p.nc;
    for (int s = 0; s < p.nslab; ++s) {
      const int nu = slab_units(p, s);
      // units u of slab s with (s * nu_full + u) % G == blockIdx.x
      const int first = (int)(((long long)blockIdx.x - (long long)s * nu_full) % G + G) % G;
      if (first >= nu) continue;
      if (tid == 0) kc_go = op_wait_count(p, b2g_cnt + s, (unsigned)(p.nk * 4), labort) ? 1 : 0;
      named_bar_sync(1, KC_THREADS);
      if (!kc_go) {
        if (tid == 0) op_raise(p, labort);
        break;
      }
      bool unit_ok = true;
      for (int u = first; u < nu && unit_ok; u += G, ++kc_phase) {
        unit_ok = kc_unit<N>(p, kc_tile, kc_bar, kc_phase & 1u, u % p.nc, s * (OP_M / KC_XW) + u / p.nc, tid, labort,
                             kc_fail, kc_copies);
        if (!unit_ok) break;
        // the unit's Phi' stores precede the barrier; one fence by the thread
        // that publishes the unit
        named_bar_sync(1, KC_THREADS);
        if (tid == 0) {
          __threadfence();
          atomicAdd(kc_cnt + s, 1u);
        }
      }
      if (!unit_ok) {
        if (tid == 0) op_raise(p, labort);
        break;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (threadIdx.x == 0 && *labort) {
    // drain TMA copies that were issued but never consumed
    for (int it = *consumed; it < *issued; ++it) {
      const unsigned long long t0 = gtime();
      while (!mbar_try(full(it % S), (uint32_t)(it / S) & 1u) && gtime() - t0 < DRAIN_NS) {
      }
    }
    // and a k-transform tile copy whose wait gave up (phase = copies issued - 1)
    if (kc_copies[0] > kc_copies[1]) {
      const unsigned long long t0 = gtime();
      while (!mbar_try(kc_bar, (uint32_t)(kc_copies[0] - 1) & 1u) && gtime() - t0 < DRAIN_NS) {
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, p.tmem_cols);
  }
  // the last CTA to finish resets the slab counters and the abort word
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(p.sync + 2 * p.nslab + 2, 1u);
    if (done == (unsigned)G - 1) {
      for (int i = 0; i < 2 * p.nslab + 2; ++i) p.sync[i] = 0u;
      __threadfence();
      p.sync[2 * p.nslab + 2] = 0u;
    }
  }
}

}  // namespace

size_t bse_onepass_smem(int n_mesh, int stages) {
  return 1024 + (size_t)stages * STAGE_BYTES + (size_t)n_mesh * n_mesh * n_mesh * KC_XW * 8 + 512;
}

int bse_onepass_threads() { return OP_THREADS; }

cudaError_t bse_onepass_launch(int n_mesh, int grid, const CUtensorMap* maps, const OnePassParams& p,
                               cudaStream_t st) {
  const size_t smem = bse_onepass_smem(n_mesh, p.stages);
  if (n_mesh == 8) {
    cudaFuncSetAttribute(tc_onepass<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_onepass<8><<<grid, OP_THREADS, smem, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], maps[6],
                                                   maps[7], p);
  } else if (n_mesh == 4) {
    cudaFuncSetAttribute(tc_onepass<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    tc_onepass<4><<<grid, OP_THREADS, smem, st>>>(maps[0], maps[1], maps[2], maps[3], maps[4], maps[5], maps[6],
                                                   maps[7], p);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int bse_onepass_max_blocks_per_sm(int n_mesh, int stages) {
  int per_sm = 0;
  const size_t smem = bse_onepass_smem(n_mesh, stages);
  cudaError_t e;
  if (n_mesh == 8) {
    cudaFuncSetAttribute(tc_onepass<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_onepass<8>, OP_THREADS, smem);
  } else {
    cudaFuncSetAttribute(tc_onepass<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc_onepass<4>, OP_THREADS, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm;
}
