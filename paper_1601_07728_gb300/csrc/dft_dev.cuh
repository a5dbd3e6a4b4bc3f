// Device helpers of the k-mesh Fourier sums of Algorithm 1 (Sec. 3.2.1):
// complex arithmetic on float2 / double2, the in-register 1-D DFT of a
// pencil of N <= 8 points (radix-2/4/8 butterflies for N = 2, 4, 8, explicit
// sums otherwise) and the bf16 hi/lo split of an FP32 value.  Shared by the
// stand-alone k-transform kernels and the one-pass tensor-core step.
#pragma once

#include <cuda_bf16.h>

namespace {

template <typename T> struct CT;
template <> struct CT<float> { typedef float2 t; };
template <> struct CT<double> { typedef double2 t; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C o; o.x = a.x + b.x; o.y = a.y + b.y; return o; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C o; o.x = a.x - b.x; o.y = a.y - b.y; return o; }
// a * (SIGN i)
template <int SIGN, typename C> __device__ __forceinline__ C cmuli(C a) { C o; o.x = -SIGN * a.y; o.y = SIGN * a.x; return o; }
// a * b
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  C o;
  o.x = a.x * b.x - a.y * b.y;
  o.y = a.x * b.y + a.y * b.x;
  return o;
}

// v_q <- sum_j e^{SIGN 2 pi i j q / N} v_j ; tw[j] = e^{+2 pi i j / N}
template <typename T, int N, int SIGN>
__device__ __forceinline__ void dftN(typename CT<T>::t* v, const typename CT<T>::t* tw) {
  typedef typename CT<T>::t C;
  if constexpr (N == 1) {
    return;
  } else if constexpr (N == 2) {
    C a = cadd(v[0], v[1]), b = csub(v[0], v[1]);
    v[0] = a;
    v[1] = b;
  } else if constexpr (N == 4) {
    C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]), a2 = cadd(v[1], v[3]), a3 = cmuli<SIGN>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
  } else if constexpr (N == 8) {
    const T r = (T)0.70710678118654752440;
    C a0 = cadd(v[0], v[4]), a1 = csub(v[0], v[4]), a2 = cadd(v[2], v[6]), a3 = csub(v[2], v[6]);
    C a4 = cadd(v[1], v[5]), a5 = csub(v[1], v[5]), a6 = cadd(v[3], v[7]), a7 = csub(v[3], v[7]);
    C e0 = cadd(a0, a2), e2 = csub(a0, a2), e1 = cadd(a1, cmuli<SIGN>(a3)), e3 = csub(a1, cmuli<SIGN>(a3));
    C o0 = cadd(a4, a6), o2 = csub(a4, a6), o1 = cadd(a5, cmuli<SIGN>(a7)), o3 = csub(a5, cmuli<SIGN>(a7));
    C t1, t3;
    t1.x = r * (o1.x - SIGN * o1.y);
    t1.y = r * (o1.y + SIGN * o1.x);
    C t2 = cmuli<SIGN>(o2);
    t3.x = r * (-o3.x - SIGN * o3.y);
    t3.y = r * (-o3.y + SIGN * o3.x);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, t1);
    v[5] = csub(e1, t1);
    v[2] = cadd(e2, t2);
    v[6] = csub(e2, t2);
    v[3] = cadd(e3, t3);
    v[7] = csub(e3, t3);
  } else {
    C out[N];
#pragma unroll
    for (int q = 0; q < N; ++q) {
      C acc;
      acc.x = 0;
      acc.y = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        C t = tw[(j * q) % N];
        if (SIGN < 0) t.y = -t.y;
        C p = cmulc(t, v[j]);
        acc.x += p.x;
        acc.y += p.y;
      }
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = out[q];
  }
}

__device__ __forceinline__ void split_bf(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

}  // namespace
