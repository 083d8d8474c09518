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
  long long sweeps_fp32, sweeps_fp64;  // Jacobi sweeps run, summed over SVDs
  double phase_cycles[4];              // cluster SVD phases (CTA 0 clock): load, FP32 sweeps, V / A rebuild, FP64 sweeps + output
};

// Parameters of the truncation SVD.
struct SvdParams {
  int chi_max;
  int max_sweeps;
  double trunc_rel;
  double tol;  // <= 0: default
  int mixed;   // FP64 SVD of a complex64 state: FP32 sweeps, then FP64 ones (cluster kernel)
};


// Rotation of a column pair of the one-sided Jacobi SVD from its Gram entries
// alpha = a_i^H a_i, beta = a_j^H a_j, g = gr + i gi = a_i^H a_j (Algorithm 1
// of the paper, with the phase of g moved onto column j): the new columns are
// a_i' = c a_i - conj(s e^{i phi}) a_j and a_j' = c a_j + s e^{i phi} a_i.
// Returns false when the pair is left alone: already orthogonal to tol, a
// column at the rounding floor, or both columns with squared norm <= tau2.
// With tau2 = eps_rel^2 ||A||_F^2 / n^2 (n columns) the columns below it
// hold at most eps_rel^2 ||A||_F^2 / n <= (eps_rel s_1)^2 together, so
// whatever their mutual angles, their singular values fall below the
// truncation threshold eps_rel s_1; they only have to be orthogonalised
// against the larger columns, which stay exact.
template <typename S>
__device__ __forceinline__ bool jacobi_rotation(S alpha, S beta, S gr, S gi, S tol, S floor, S tiny, S tau2, S& c,
                                                cplx<S>& sph) {
  if (!(max(alpha, beta) > tau2)) return false;
  const S mag = sqrt(gr * gr + gi * gi);
  if (!(mag > tiny) || !(mag > tol * sqrt(alpha * beta)) || !(min(alpha, beta) > floor)) return false;
  const S zeta = (beta - alpha) / (S(2) * mag);
  const S t = (zeta >= S(0) ? S(1) : S(-1)) / (fabs(zeta) + sqrt(S(1) + zeta * zeta));
  c = S(1) / sqrt(S(1) + t * t);
  const S s = t * c;
  sph = cmk<S>(s * gr / mag, s * gi / mag);  // s e^{i phi}
  return true;
}

// FP64 form.  FP64 square roots and divisions cost dozens of instructions on
// an SM with two FP64 FMA units, so the angle is found in FP32 on Gram
// entries scaled by a power of two near |g|, and (c, s e^{i phi}) is then
// brought to unit norm in FP64 by c^2 + |s|^2 = 1 + d -> scale by
// 1 - d/2 + 3 d^2 / 8, the first terms of the binomial series of
// (1 + d)^(-1/2) (|d| ~ 1e-7, so the dropped O(d^3) term leaves the
// rotation unitary to FP64 rounding).  The angle itself is only FP32-accurate, which costs at most
// an extra sweep: a pair left with |g| ~ 1e-7 |g| is rotated again.
template <>
__device__ __forceinline__ bool jacobi_rotation<double>(double alpha, double beta, double gr, double gi, double tol,
                                                        double floor, double tiny, double tau2, double& c,
                                                        cplx<double>& sph) {
  if (!(max(alpha, beta) > tau2)) return false;
  const double mag2 = gr * gr + gi * gi;
  if (!(mag2 > tiny) || !(mag2 > tol * tol * alpha * beta) || !(min(alpha, beta) > floor)) return false;
  // 2^-h with 2^(2h) ~ mag2 (mag2 is a normal double here)
  const long long e2 = ((__double_as_longlong(mag2) >> 52) & 0x7ff) - 1023;
  const long long h = e2 >> 1;
  const double scl = __longlong_as_double((1023 - h) << 52);
  const float xr = float(gr * scl), xi = float(gi * scl);
  const float magf = sqrtf(xr * xr + xi * xi);
  const float zeta = float((beta - alpha) * scl) / (2.f * magf);
  if (!(fabsf(zeta) < 3e38f)) return false;
  const float t = fabsf(zeta) > 1e15f ? 0.5f / zeta
                                       : (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float cf = rsqrtf(1.f + t * t);
  const float sf = t * cf / magf;
  const double cd = cf, sr = double(sf) * double(xr), si = double(sf) * double(xi);
  const double d = fma(cd, cd, fma(sr, sr, fma(si, si, -1.0)));
  const double f = fma(d, fma(0.375, d, -0.5), 1.0);
  c = cd * f;
  sph = cmk<double>(sr * f, si * f);
  return true;
}

}  // namespace mpsv
