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
  int not_converged;  // SVDs that reached the sweep cap
  int tc_error;       // a tensor-core kernel ran out of its bounded wait (read with not_converged in one copy)
  int max_sweeps;
  int pad;
  long long two_qubit_gates;
  double svd_flops;
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
// Returns false when the pair is left alone: already orthogonal to tol, or a
// column at the rounding floor.
template <typename S>
__device__ __forceinline__ bool jacobi_rotation(S alpha, S beta, S gr, S gi, S tol, S floor, S tiny, S& c,
                                                cplx<S>& sph) {
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
                                                        double floor, double tiny, double& c, cplx<double>& sph) {
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

// The pair rules of the truncation SVD (tail columns).  Jacobi only has to
// make the columns that the truncation keeps orthogonal to each other and to
// all others; the columns it discards may stay mixed among themselves as long
// as none of their singular values could reach the cut.  At the start of a
// sweep, from the squared column norms nrm2[0..n): the kept set K is what the
// truncation would keep now (nrm2 > trunc_rel^2 max nrm2, the chi_max largest
// by rank when more pass), D the rest, and the cut is trunc_rel^2 max nrm2 (or
// the smallest kept nrm2 under a chi_max cut).  The class of column c goes to
// cls[c]:
//  * kTailSkip when sum_D nrm2 <= cut / 4: every singular value of the D
//    block is then at most half of every kept column's norm, so once K is
//    orthogonal to itself and to D, K holds the leading singular vectors
//    whatever D looks like (and the discarded weight is sum_D nrm2); pairs of
//    two such columns are not rotated.  The factor 1/4 also bounds how much
//    rotating a kept column against one D column disturbs its orthogonality
//    to the others, so the kept columns converge quickly (a bare per-column
//    threshold did not: a column just above it never converged against mixed
//    columns just below it).
//  * kTailLoose otherwise, for the deep tail T: the D columns with nrm2 <=
//    t_d, where t_d <= cut / 4 is the largest such norm below a gap, i.e.
//    the next larger nrm2 of any column is at least 4 t_d.  Pairs of two of
//    them are rotated only while |g| > loose_tol sqrt(b_ii b_jj), loose_tol =
//    min(2 / n, cut / (16 sum_T nrm2)), returned in *loose.  By Gershgorin on
//    their Gram matrix the singular values of T then stay below
//    (cut / 4)(1 + n loose_tol) < cut.  Every other column has nrm2 >= 4
//    t_d, so its rotations against T have small angles (|s| <= 4|g| / (3
//    nrm2)) and disturb its orthogonality to the rest of T by at most
//    loose_tol sum_T nrm2 / nrm2 <= 1/4 of what it was: it still converges.
//    (Without the gap a degenerate pair of columns straddling the threshold
//    rotated by large angles and carried the loose couplings of its deep
//    member into its tight one, and with 2 / n alone columns just above the
//    threshold crawled against many mixed columns just below it.)
//  * 0 for every other column (the normal stopping rule).
// Every thread of the block calls it; blocks with the same nrm2 and size
// compute the same classes.
constexpr int kTailLoose = 1, kTailSkip = 2;

__device__ __forceinline__ void truncation_tail(const double* nrm2, int n, double trunc_rel, int chi_max, int* cls,
                                                double* loose) {
  __shared__ double s_red[33];
  __shared__ int s_cnt;
  __shared__ double s_cut;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  // largest squared norm
  double mx = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) mx = fmax(mx, nrm2[c]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) s_red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v = fmax(v, s_red[w]);
    s_red[32] = v;
    s_cnt = 0;
  }
  __syncthreads();
  const double thr = trunc_rel * trunc_rel * s_red[32];
  int cnt = 0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) cnt += nrm2[c] > thr;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) atomicAdd(&s_cnt, cnt);
  __syncthreads();
  const bool by_rank = s_cnt > chi_max;
  if (threadIdx.x == 0) s_cut = thr;
  __syncthreads();
  // kept flags (1 = kept) into cls[] first
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    if (by_rank) {
      const double v = nrm2[c];
      int rk = 0;
      for (int h = 0; h < n; ++h) rk += (nrm2[h] > v) || (nrm2[h] == v && h < c);
      cls[c] = rk < chi_max;
      if (rk == chi_max - 1) s_cut = v;
    } else {
      cls[c] = nrm2[c] > thr;
    }
  }
  __syncthreads();
  // weight of D, summed in a fixed order
  double part = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    if (!cls[c]) part += nrm2[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  __syncthreads();
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += s_red[w];
    s_red[32] = v;
  }
  __syncthreads();
  const double cut = s_cut;
  const bool skip = s_red[32] <= 0.25 * cut;
  // deep-tail threshold t_d: the largest candidate norm (a discarded column
  // with nrm2 <= cut / 4) whose next larger norm among all columns is at
  // least 4 times it
  double td = -1.0;
  if (!skip)
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const double v = nrm2[c];
      if (cls[c] || !(v <= 0.25 * cut)) continue;
      double nxt = INFINITY;
      for (int h = 0; h < n; ++h)
        if (nrm2[h] > v) nxt = fmin(nxt, nrm2[h]);
      if (nxt >= 4.0 * v) td = fmax(td, v);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) td = fmax(td, __shfl_xor_sync(0xffffffffu, td, o));
  __syncthreads();
  if (lane == 0) s_red[warp] = td;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = -1.0;
    for (int w = 0; w < nw; ++w) v = fmax(v, s_red[w]);
    s_red[32] = v;
  }
  __syncthreads();
  td = s_red[32];
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    cls[c] = cls[c] ? 0 : (skip ? kTailSkip : (nrm2[c] <= td ? kTailLoose : 0));
  __syncthreads();
  // weight of the deep tail T, summed in a fixed order, for the loose tolerance
  part = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x)
    if (cls[c] == kTailLoose) part += nrm2[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  __syncthreads();
  if (lane == 0) s_red[warp] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < nw; ++w) v += s_red[w];
    const double l = 2.0 / n;
    *loose = v > 0.0 ? fmin(l, cut / (16.0 * v)) : l;
  }
  __syncthreads();
}

// The stopping tolerance of a pair from the classes of its columns (see
// truncation_tail): a negative value means the pair is not rotated.
template <typename S>
__device__ __forceinline__ S pair_tol(int ci, int cj, S tol, S loose) {
  const int c = min(ci, cj);
  return c == kTailSkip ? S(-1) : (c == kTailLoose ? max(tol, loose) : tol);
}

}  // namespace mpsv
