// Shared device helpers of libmpsvqe: complex arithmetic on float2/double2,
// warp reductions and the device-side data layouts of a state.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

namespace mpsv {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using type = float2; };
template <> struct CplxOf<double> { using type = double2; };
template <typename R> using cplx = typename CplxOf<R>::type;

template <typename R> __host__ __device__ __forceinline__ cplx<R> cmk(R re, R im) {
  cplx<R> z;
  z.x = re;
  z.y = im;
  return z;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) {
  a.x -= b.x;
  a.y -= b.y;
  return a;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
  C r;
  r.x = a.x * b.x + a.y * b.y;
  r.y = a.x * b.y - a.y * b.x;
  return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) {
  a.y = -a.y;
  return a;
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
  a.x *= s;
  a.y *= s;
  return a;
}
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
template <typename Cto, typename Cfrom> __device__ __forceinline__ Cto ccast(Cfrom z) {
  Cto r;
  r.x = static_cast<decltype(r.x)>(z.x);
  r.y = static_cast<decltype(r.y)>(z.y);
  return r;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// A gate as the kernels read it: row-major 4x4 (two-qubit) or 2x2 in the
// first four entries (one-qubit), FP64 complex.
struct DevGate {
  int q;
  int arity;
  int pad0, pad1;
  double2 u[16];
};

// A template gate: u = exp(i phi) mp + exp(-i phi) mm, phi = coeff * theta[param].
struct DevTmplGate {
  int q;
  int arity;
  int param;
  int pad;
  double coeff;
  double pad2;
  double2 mp[16];
  double2 mm[16];
};

// Per-state statistics the kernels accumulate on the device.
struct DevReport {
  double discarded_weight;
  double min_kept_sv;
  double inv_norm;  // 1 / ||kept s|| of the last two-qubit gate (read by the G3 kernel)
  int max_chi;
  int degenerate_cuts;
  int not_converged;
  int max_sweeps;
  long long two_qubit_gates;
  double svd_flops;
  int tc_error;  // a tensor-core kernel ran out of its bounded wait
  int pad;
};

// Parameters of the truncation SVD.
struct SvdParams {
  int chi_max;
  int max_sweeps;
  double trunc_rel;
  double tol;  // <= 0: default
};

}  // namespace mpsv
