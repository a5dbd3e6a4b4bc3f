// Internal declarations shared by the CUDA translation units of libbse.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/bse.h"

#define BSE_MAX_ALPHA 16
#define BSE_MAX_NK_AXIS 16
#define BSE_MAX_PROJ 64
#define BSE_FINAL_BLOCKS 1024  // blocks per vector of the fused grid->band epilogue

// ---------------------------------------------------------------------------
// complex helpers (interleaved re, im)
// ---------------------------------------------------------------------------
template <typename T> struct cvec;
template <> struct cvec<double> { typedef double2 type; };
template <> struct cvec<float> { typedef float2 type; };

template <typename C> __host__ __device__ __forceinline__ C cmake(double re, double im);
template <> __host__ __device__ __forceinline__ double2 cmake<double2>(double re, double im) { return make_double2(re, im); }
template <> __host__ __device__ __forceinline__ float2 cmake<float2>(double re, double im) { return make_float2((float)re, (float)im); }

// acc += a * b
template <typename C> __device__ __forceinline__ void cmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __device__ __forceinline__ void cmac_conj(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// ---------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------
struct bse_handle {
  int dev = 0;
  cudaStream_t stream = nullptr;
  int na = 0, nb = 0, np = 0, prec = 0, max_vec = 1;
  int nk3[3] = {1, 1, 1}, nx3[3] = {1, 1, 1};
  int nk = 0, nx = 0;
  long long N = 0;
  double kshift[3] = {0, 0, 0};

  // FP64 system data (every precision)
  double* e_nk = nullptr;     // [Nk][Nb]
  double2* chi = nullptr;     // [Na][Na]
  double2* a_proj = nullptr;  // [Np][Nk*Nb]
  float2* a_proj_f = nullptr; // FP32 copy for the reduced-precision forms
  double2* m_sr = nullptr;    // [Na*Np][Na*Np]
  double* jdiag = nullptr;    // [Na][Nk][Nb]
  double* twiddle = nullptr;  // [3][16][2] e^{+2 pi i j / nk_d}, j < nk_d

  // band<->grid operands
  void* u = nullptr;          // FP64: double2 [Nk][Nx][Nb]; FP32: float2; phase folded
  void* w = nullptr;          // [Nk][Nx] double (FP64) or float
  __nv_bfloat16* u_hi = nullptr;   // SPLIT_BF16: [Nk][Nx][Kp] (re, im interleaved, Kp = 2Nb padded to 8)
  __nv_bfloat16* u_lo = nullptr;
  __nv_bfloat16* ut_hi = nullptr;  // SPLIT_BF16: K-tiled transposed copy [Nk][ceil(Nx/64)][2Nb][64]
  __nv_bfloat16* ut_lo = nullptr;

  // scratch sized for max_vec columns
  void* phi = nullptr;        // [Nk][Nx][Nc] complex (double2 for FP64, float2 otherwise)
  double2* sr_c = nullptr;    // [max_vec][Na*Np]
  double2* sr_cp = nullptr;   // [max_vec][Na*Np]
  double2* sr_part = nullptr; // [ceil(Nk*Nb/64)][max_vec*Na][Np] split-K partial projections
  __nv_bfloat16* bpsi = nullptr;    // SPLIT_BF16: [Nk][2][Nrow][2Nb] B operand of band->grid
  float2* psi_f = nullptr;          // SPLIT_BF16: FP32 copy of the operand psi [max_vec][N] (operand pass)
  __nv_bfloat16* bphi = nullptr;    // SPLIT_BF16: hi/lo K-tiled [Nk][ceil(Nx/64)][Nrow][64] B operand of grid->band
  float* part = nullptr;            // SPLIT_BF16: split-K partial tiles
  void* tmap = nullptr;             // SPLIT_BF16: tensor maps (device copy)
  void* tmap_host = nullptr;

  // learned GMRES preconditioner attached by the caller (not owned), and the
  // per-(k,n) local-basis weight |A_{:,nk}| it uses as a feature
  bse_mlp* mlp = nullptr;
  float* mlp_anorm = nullptr;

  // side stream for the short-range term (overlaps the band->grid pass)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // x-slabs of the tensor-core step (bse_set_slabs): the k-transform and
  // grid->band of each slab run on side2 after the slab's band->grid
  int slabs = 1;
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_slab[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t ev_side2 = nullptr;
  cudaStream_t cur = nullptr;   // stream the next profiled launch goes to

  // schedule of the split-bf16 step (bse_set_schedule): two passes over U with
  // the transposed copy, two passes reading U row-major for both, or one pass
  int sched = 0;
  int op_lag = 2, op_stages = 5, op_l2hint = 1;
  int op_max_vec = 0;          // one pass: largest n_vec it takes (0: none)
  bool concurrent = false;     // kernels of other handles may run beside this one's (many-site graph)

  // grow-only device workspace of the Haydock driver (kept between calls)
  void* ws = nullptr;
  size_t ws_cap = 0;

  // reusable device staging for host arguments of bse_apply_h
  void* io_in = nullptr;
  void* io_out = nullptr;
  size_t io_cap = 0;

  // profiling hook: event pairs around launches
  bool prof = false;
  std::vector<cudaEvent_t> ev;     // 2 per launch
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  long long prof_count[BSE_K_COUNT] = {0};
  double prof_ms[BSE_K_COUNT] = {0};

  // limit of each wait of the tensor-core pipeline (bse_set_wait_limit)
  unsigned long long tc_wait_ns = 2000000000ull;

  // the last Haydock call's step-loop graph, relaunched when a call repeats it
  // (same buffers, sizes, tiles and limits); hay_key identifies the call
  cudaGraphExec_t hay_exec = nullptr;
  long long hay_exec_launches = 0;   // kernels per launch of the graph
  unsigned long long hay_key[12] = {0};

  // device memory allocated for the handle by bse_setup, and the cap on it
  // (BSE_DEVICE_BYTES_LIMIT in the environment at set-up; 0 = none)
  size_t dev_bytes = 0;
  size_t dev_cap = 0;

  long long launches = 0;
  std::string err;
};

// cudaMalloc for a handle's set-up buffers, counted against h->dev_cap
// (BSE_ERR_OOM beyond it, or when the device is out of memory)
bse_status bse_handle_malloc(bse_handle* h, void** p, size_t bytes, const char* what);

// drop the cached Haydock graph (tiles, limits or buffers changed)
void bse_drop_graph(bse_handle* h);

// bracket a launch with profiling events (no-op unless enabled)
void bse_prof_begin(bse_handle* h, int kind);
void bse_prof_end(bse_handle* h);

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
bool bse_is_device_ptr(const void* p);
bse_status bse_fail(bse_handle* h, bse_status s, const std::string& msg);
bse_status bse_cuda_check(bse_handle* h, cudaError_t e, const char* what);

#define BSE_LAUNCHED(h) ((h)->launches++)
#define BSE_PROF(h, kind, ...)   \
  do {                           \
    bse_prof_begin((h), (kind)); \
    __VA_ARGS__;                 \
    bse_prof_end(h);             \
    BSE_LAUNCHED(h);             \
  } while (0)

// setup kernels (k_setup.cu)
bse_status bse_setup_device(bse_handle* h, const bse_system_desc* d);

// Where a Haydock update writes the next step's band->grid operand (bf16
// hi/lo [Nk][Nrow][K_p]) and FP32 psi; hi == nullptr: not written.
struct bse_operand_out {
  __nv_bfloat16* hi = nullptr;
  __nv_bfloat16* lo = nullptr;
  float2* psi_f = nullptr;
  int nk = 0, nb = 0, na = 0, kp = 0, nnmax = 0;
};

// Haydock hook fused into the last kernel of H psi: a[v][i] = Re <psi_v | H psi_v>
// from per-block partial sums; the last block to finish (counter) reduces them
// in a fixed order and resets the counter.
struct bse_dotfuse {
  double2* partial = nullptr;   // [n_vec][nblk]
  unsigned* counter = nullptr;
  double* a = nullptr;          // a[v * a_stride + i]
  int a_stride = 0, i = 0;
  const int* active = nullptr;
  int* status = nullptr;        // bit 0: breakdown, bit 1: non-finite value
  // deferred mode: the epilogue only writes its per-block partials of
  // <psi|H psi>; the Haydock update kernel reduces them (in every block, in a
  // fixed order) instead of a last-block reduction here
  bool deferred = false;
  // lazy normalisation (deferred mode, step i >= 1): psi holds w_i
  // unnormalised; the operand pass reduces norm_part [n_vec][norm_n] to
  // b_i = |w_i|, records b_i (bco[v * (a_stride + 1) + i]), the step count and
  // the breakdown test, and divides psi by b_i in place
  const double2* norm_part = nullptr;
  int norm_n = 0;
  double* bco = nullptr;
  int* active_rw = nullptr;
  int* steps = nullptr;
  // operand_ready (tensor-core form, N_alpha in {1, 6}): the previous Haydock
  // update already wrote the band->grid operand and the FP32 copy of psi = w_i
  // unnormalised, so the operand pass is skipped and the grid->band epilogue
  // does the lazy normalisation (every term it adds is linear in psi)
  bool operand_ready = false;
  // fused update (tensor-core form, N_alpha in {1, 6}, whole grid resident):
  // after its dot partials the epilogue meets every other block at a bounded
  // grid barrier, reduces a_i itself and applies w = H v_i - a_i v_i - b_i
  // v_{i-1} in place of the separate Haydock update kernel, writing the |w|^2
  // partials (upart [n_vec][gridDim.x]) and the next operand (op)
  bool fused_update = false;
  const double2* vprev = nullptr;   // v_{i-1}
  double2* upart = nullptr;
  unsigned* barrier = nullptr;      // {arrivals, generation}; arrivals zero between uses
  bse_operand_out op;
};
// status bit of a grid barrier that gave up (BSE_ERR_TIMEOUT)
#define BSE_ST_TIMEOUT 4

// A[p][k][n] = dv sum_x conj(f_p(x)) e^{ik.x} u_nk(x) on device arrays (k_local.cu)
bse_status bse_local_projection_device(const double2* u, const int* nk, const int* nx, int nb, const double* kshift,
                                       const double2* f, int np, double dv, double2* a, cudaStream_t st);
// screening: G_j = psi diag(1/(mu + i t_j - eps)) psi^H for all j, chi0 from them (k_screen.cu)
bse_status bse_screening_device(const double2* psi, const double* eps, int nr, int nkk, double mu, const double* t,
                                const double* w, int nt, double2* G, double2* chi, cudaStream_t st);
// the tensor-core form's operand buffers of a handle (k_tc.cu)
bse_operand_out bse_tc_operand(const bse_handle* h);

// H psi on device pointers (k_apply.cu); psi/hpsi [n_vec][N] double2, n_vec <= max_vec.
// With fuse != nullptr the tensor-core form also produces a_i (returns
// BSE_ERR_UNSUPPORTED from other forms, whose callers compute it separately).
bse_status bse_apply_device(bse_handle* h, const double2* psi, double2* hpsi, int n_vec,
                            const bse_dotfuse* fuse = nullptr);
bool bse_apply_fuses_dot(const bse_handle* h);

// tensor-core band<->grid path (k_tc.cu)
bse_status bse_tc_prepare(bse_handle* h);
// B operand of band->grid from psi (and, with fuse->norm_part set, the lazy normalisation of psi)
bse_status bse_tc_prep(bse_handle* h, const double2* psi, int n_vec, const bse_dotfuse* fuse);
// blocks per vector of the grid->band epilogue (the number of <psi|H psi> partials it writes)
int bse_tc_final_blocks(const bse_handle* h);
// true if the fused epilogue + Haydock update can run for n_vec vectors (the
// whole grid of the epilogue is resident at once, so its barrier completes)
bool bse_tc_fused_update_ok(const bse_handle* h, int n_vec);
// current tile parameters of the tensor-core form (0, 0 for other forms)
void bse_tc_tiles(const bse_handle* h, int* split, int* stages);
bse_status bse_tc_band_to_grid(bse_handle* h, int n_vec);
bse_status bse_tc_grid_to_band(bse_handle* h, const double2* psi, double2* hpsi, int n_vec,
                               const bse_dotfuse* fuse, bool wait_side);
// band->grid, k-transform and grid->band in h->slabs x-slabs (two streams), then the epilogue
bse_status bse_tc_apply_slabbed(bse_handle* h, const double2* psi, double2* hpsi, int n_vec,
                                const bse_dotfuse* fuse, bool wait_side);
bse_status bse_kconv_bf16(bse_handle* h, int n_vec);
// k-transform x W (k_kconv.cu): in place on phi[k][c][x], or into bf16 hi/lo planes
bse_status bse_kconv_inplace(bse_handle* h, int n_vec);
bse_status bse_kconv_split(bse_handle* h, int n_vec, __nv_bfloat16* hi, __nv_bfloat16* lo, int nnmax, int x0, int x1,
                           cudaStream_t st);
// one-pass step: band->grid, k-transform and grid->band slab by slab in one kernel, then the epilogue
bse_status bse_tc_apply_onepass(bse_handle* h, const double2* psi, double2* hpsi, int n_vec,
                                const bse_dotfuse* fuse, bool wait_side);
// true if the k-transform can run on part of the grid (x-slabs)
bool bse_kconv_takes_slabs(const bse_handle* h);
bse_status bse_tc_status(bse_handle* h);   // device error word of the tensor-core pipeline
void bse_tc_free(bse_handle* h);

// Krylov drivers (k_krylov.cu)
bse_status bse_haydock_device(bse_handle* h, const double2* b, int n_vec, int n_steps, int reorth,
                              double* a, double* bcoef, int* steps_done);
bse_status bse_haydock_batch_device(bse_handle* const* hs, const double2* const* bs, int n_sites, int n_vec,
                                    int n_steps, double* const* a_d, double* const* b_d, int* const* steps_d,
                                    bse_status* site_status);
bse_status bse_gmres_device(bse_handle* h, const double2* b, const double2* z, int n_z, double rtol,
                            int restart, int max_iter, int precond, double2* x, int* iters,
                            double* rel_resid);
bse_status bse_cf_device(const double* a, const double* bcoef, const int* steps, int n_vec,
                         int n_stride, const double* omega, int n_omega, double gamma,
                         int terminator, double* sigma, cudaStream_t st);
