// Host interface of the one-pass tensor-core step (k_onepass.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>

#define OP_MAX_KPC 4   // k points per CTA (grid->band accumulators held in tensor memory)
#define OP_MAX_STAGES 5

struct OnePassParams {
  int nk, nx, nb, nc;          // k points, grid points, bands, columns (n_vec * N_alpha <= 8)
  int nslab;                   // ceil(nx / 128)
  int kb_b2g;                  // K blocks of 64 of the band->grid contraction (ceil(Kp / 64) <= 2)
  int lag;                     // grid->band of slab s is issued after band->grid of slab s + lag
  int stages;                  // pipeline stages of 36 KB
  unsigned tmem_cols;
  int nnmax;                   // row stride of the grid->band operand planes
  int lbo, sbo;                // MN-major descriptor offsets of the grid->band A operand (bytes)
  int l2hint;                  // keep U~ in L2 between its two reads (TMA cache policies)
  float2* phi;                 // band->grid result (FP32), unit-major [nx/8][nc][nk][8]
  float2* part;                // [nk][nc][nb] grid->band result
  __nv_bfloat16* bphi_hi;      // grid->band operand planes [nk][ceil(nx/64)][nnmax][64]
  __nv_bfloat16* bphi_lo;
  const float* w;              // W(x, R) [nk][nx], FP32
  unsigned* sync;              // [2 nslab + 3]: band->grid and k-transform counters per slab, abort, done
  int* err;                    // device error word
  unsigned long long wait_ns;  // limit of each wait
};

size_t bse_onepass_smem(int n_mesh, int stages);
int bse_onepass_threads();
int bse_onepass_max_blocks_per_sm(int n_mesh, int stages);
// maps: U~ hi/lo (box 64 x 128 rows), U~ hi/lo (box 64 x 64 rows), Bpsi hi/lo, Phi' hi/lo
cudaError_t bse_onepass_launch(int n_mesh, int grid, const CUtensorMap* maps, const OnePassParams& p,
                               cudaStream_t st);
