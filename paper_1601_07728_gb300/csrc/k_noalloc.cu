// Short-range term of H with no allocation at all: the split-K scratch of the
// projection lives in a fixed file-scope device array instead of memory that
// a handle would cudaMalloc.  For callers that cannot allocate device memory
// at the point where they need H's short-range action: plug-ins whose host
// framework owns every device byte through its own pool, and real-time loops
// where an allocation's implicit synchronisation would stall other streams.
#include "bse_internal.cuh"

#include <cuda.h>
#include <stdio.h>

#include <mutex>

namespace {

constexpr int NA_K = 64;   // (k, n) terms per partial-sum block
constexpr int NA_C = 16;   // columns per partial-sum block
constexpr size_t NA_SCRATCH = (size_t)1 << 17;   // double2 entries = 2 MiB

// Scratch shared by every call on a device; lives as long as the module.
static __device__ __align__(256) double2 g_noalloc_scratch[NA_SCRATCH];

constexpr int NA_MAX_DEV = 64;
// device address of the array per device, and the context it was looked up
// in: a reset device gets a new primary context, the module is loaded again
// and the array may move, so a changed context means a fresh look-up
double2* g_scratch_addr[NA_MAX_DEV] = {};
CUcontext g_scratch_ctx[NA_MAX_DEV] = {};
std::mutex g_scratch_mu;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

CtxGetCurrentFn ctx_get_current_fn() {
  static CtxGetCurrentFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

// true if p is device memory of device `dev`
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

// byte ranges [a, a + na) and [b, b + nb) intersect
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

// part[b][c][p] = sum over kn in block b of A[p][kn] psi[c][kn]
__global__ void __launch_bounds__(256) na_partial(const double2* __restrict__ a_proj, const double2* __restrict__ psi,
                                                  double2* __restrict__ part, int nkb, int np, int nc) {
  extern __shared__ __align__(16) unsigned char na_smem[];
  double2* As = reinterpret_cast<double2*>(na_smem);   // [np][NA_K + 1]
  double2* Ps = As + (size_t)np * (NA_K + 1);           // [NA_C][NA_K + 1]
  const int b = blockIdx.x, c0 = blockIdx.y * NA_C;
  const int ncc = nc - c0 < NA_C ? nc - c0 : NA_C;
  const int k0 = b * NA_K;
  for (int e = threadIdx.x; e < np * NA_K; e += blockDim.x) {
    const int p = e / NA_K, i = e % NA_K;
    As[p * (NA_K + 1) + i] = (k0 + i < nkb) ? a_proj[(size_t)p * nkb + k0 + i] : make_double2(0, 0);
  }
  for (int e = threadIdx.x; e < ncc * NA_K; e += blockDim.x) {
    const int c = e / NA_K, i = e % NA_K;
    Ps[c * (NA_K + 1) + i] = (k0 + i < nkb) ? psi[(size_t)(c0 + c) * nkb + k0 + i] : make_double2(0, 0);
  }
  __syncthreads();
  for (int o = threadIdx.x; o < ncc * np; o += blockDim.x) {
    const int c = o / np, p = o % np;
    double re = 0, im = 0;
    for (int i = 0; i < NA_K; ++i) {
      const double2 a = As[p * (NA_K + 1) + i], q = Ps[c * (NA_K + 1) + i];
      re += a.x * q.x - a.y * q.y;
      im += a.x * q.y + a.y * q.x;
    }
    part[((size_t)b * nc + c0 + c) * np + p] = make_double2(re, im);
  }
}

// coef[o] = sum_b part[b][o] in block order (every entry overwritten)
__global__ void na_reduce(const double2* __restrict__ part, double2* __restrict__ coef, int nblk, int nout) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double re = 0, im = 0;
  for (int b = 0; b < nblk; ++b) {
    const double2 t = part[(size_t)b * nout + o];
    re += t.x;
    im += t.y;
  }
  coef[o] = make_double2(re, im);
}

// coup[v][i] = sum_j M[i][j] coef[v][j], one warp per row
__global__ void __launch_bounds__(256) na_couple(const double2* __restrict__ m, const double2* __restrict__ coef,
                                                 double2* __restrict__ coup, int dimm) {
  const int v = blockIdx.y;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= dimm) return;
  double re = 0, im = 0;
  for (int j = lane; j < dimm; j += 32) {
    const double2 a = m[(size_t)i * dimm + j], q = coef[(size_t)v * dimm + j];
    re += a.x * q.x - a.y * q.y;
    im += a.x * q.y + a.y * q.x;
  }
  for (int off = 16; off > 0; off >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, off);
    im += __shfl_xor_sync(0xffffffffu, im, off);
  }
  if (lane == 0) coup[(size_t)v * dimm + i] = make_double2(re, im);
}

// out[c][kn] = sum_p conj(A[p][kn]) coup[c][p]
__global__ void na_out(const double2* __restrict__ a_proj, const double2* __restrict__ coup, double2* __restrict__ out,
                       int nkb, int np, int nc) {
  const size_t total = (size_t)nc * nkb;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx / nkb), kn = (int)(idx % nkb);
    double re = 0, im = 0;
    for (int p = 0; p < np; ++p) {
      const double2 a = a_proj[(size_t)p * nkb + kn], q = coup[(size_t)c * np + p];
      re += a.x * q.x + a.y * q.y;
      im += a.x * q.y - a.y * q.x;
    }
    out[idx] = make_double2(re, im);
  }
}

}  // namespace

extern "C" bse_status bse_short_range_noalloc(const bse_c128* a_proj, const bse_c128* m_sr, const bse_c128* psi,
                                              bse_c128* out, int n_alpha, int n_kb, int n_proj, int n_vec,
                                              void* stream) {
  if (!a_proj || !m_sr || !psi || !out || n_alpha < 1 || n_alpha > BSE_MAX_ALPHA || n_kb < 1 || n_proj < 1 ||
      n_proj > BSE_MAX_PROJ || n_vec < 1) {
    fprintf(stderr, "bse_short_range_noalloc: bad arguments\n");
    return BSE_ERR_INVALID_ARG;
  }
  const long long nc = (long long)n_vec * n_alpha;
  const long long nblk = (n_kb + NA_K - 1) / NA_K;
  const long long need = nblk * nc * n_proj + 2 * nc * n_proj;
  if (need > (long long)NA_SCRATCH) {
    fprintf(stderr,
            "bse_short_range_noalloc: problem needs %lld scratch entries, the static scratch holds %lld "
            "(ceil(n_kb/64)*n_vec*n_alpha*n_proj + 2*n_vec*n_alpha*n_proj must be <= %lld)\n",
            need, (long long)NA_SCRATCH, (long long)NA_SCRATCH);
    return BSE_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEV) {
    cudaGetLastError();
    return BSE_ERR_CUDA;
  }
  if (!on_device(a_proj, dev) || !on_device(m_sr, dev) || !on_device(psi, dev) || !on_device(out, dev)) {
    fprintf(stderr, "bse_short_range_noalloc: every array must be device memory of the current device (%d)\n", dev);
    return BSE_ERR_INVALID_ARG;
  }
  // out is written while A is still read (projection out): they must not
  // share bytes; neither may out and M.  psi is read completely before out
  // is written (stream order), so psi and out may overlap or coincide.
  const size_t out_bytes = (size_t)nc * n_kb * sizeof(double2);
  if (overlaps(out, out_bytes, a_proj, (size_t)n_proj * n_kb * sizeof(double2)) ||
      overlaps(out, out_bytes, m_sr, (size_t)n_alpha * n_proj * n_alpha * n_proj * sizeof(double2))) {
    fprintf(stderr, "bse_short_range_noalloc: out must not overlap a_proj or m_sr\n");
    return BSE_ERR_INVALID_ARG;
  }
  CtxGetCurrentFn get_ctx = ctx_get_current_fn();
  if (!get_ctx) {
    fprintf(stderr, "bse_short_range_noalloc: cuCtxGetCurrent unavailable\n");
    return BSE_ERR_CUDA;
  }
  double2* base = nullptr;
  {
    // first call on this device (or in a new context of it): look up the
    // device address of the static array -- host code only sees a host-side
    // stand-in for the symbol.  This is the call that loads the module, and
    // with it the array, under lazy loading.
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    CUcontext ctx = nullptr;
    if (get_ctx(&ctx) != CUDA_SUCCESS || !ctx) {
      fprintf(stderr, "bse_short_range_noalloc: no current CUDA context\n");
      return BSE_ERR_CUDA;
    }
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        fprintf(stderr, "bse_short_range_noalloc: cudaGetSymbolAddress failed: %s\n", cudaGetErrorString(e));
        return BSE_ERR_CUDA;
      }
      g_scratch_addr[dev] = (double2*)p;
      g_scratch_ctx[dev] = ctx;
    }
    base = g_scratch_addr[dev];
  }
  double2* part = base;
  double2* coef = part + nblk * nc * n_proj;
  double2* coup = coef + nc * n_proj;
  cudaStream_t st = (cudaStream_t)stream;
  const int dimm = n_alpha * n_proj;
  const size_t smem = (size_t)(n_proj + NA_C) * (NA_K + 1) * sizeof(double2);
  if (cudaFuncSetAttribute(na_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return BSE_ERR_CUDA;
  }
  na_partial<<<dim3((unsigned)nblk, (unsigned)((nc + NA_C - 1) / NA_C)), 256, smem, st>>>(
      (const double2*)a_proj, (const double2*)psi, part, n_kb, n_proj, (int)nc);
  const int nout = (int)(nc * n_proj);
  na_reduce<<<(nout + 255) / 256, 256, 0, st>>>(part, coef, (int)nblk, nout);
  na_couple<<<dim3((unsigned)((dimm + 7) / 8), (unsigned)n_vec), 256, 0, st>>>((const double2*)m_sr, coef, coup, dimm);
  long long tot = nc * n_kb;
  int blocks = (int)((tot + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  na_out<<<blocks, 256, 0, st>>>((const double2*)a_proj, coup, (double2*)out, n_kb, n_proj, (int)nc);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BSE_OK : BSE_ERR_CUDA;
}
