// Gate-application kernels of the MPS simulator (arXiv:2303.03681, Methods,
// "MPS algorithm for quantum circuit simulation").
//
// Bond dimensions live in device memory (chi[b], b = 0..n); every kernel
// reads the dimensions it needs, so a whole gate sequence is issued without a
// host round trip and can be captured in a CUDA graph.  Grids are sized for
// the bond capacities; blocks past the actual dimensions return at once.
//
// A two-qubit gate on sites (q, q+1) runs three kernels:
//   theta_kernel  C[(a_l,i),(j,a_r)] = sum Q[ij,i'j'] B_q[a_l,i',a_m] B_{q+1}[a_m,j',a_r]
//                 and A = lam_q[a_l] C (Eq. tildeC) in the SVD's column-major layout;
//   svd_truncate_kernel  one-sided Jacobi SVD of A (Algorithm 1), truncation,
//                 B~_{q+1} = V (first k rows), lam_{q+1} = s[:k] / ||s[:k]||;
//   g3_kernel     B~_q = C V^dagger / ||s[:k]|| (Eq. Bl with the unscaled C).
#pragma once

#include "common.cuh"
#include "dfloat.cuh"

namespace mpsv {

constexpr int kTile = 16;

// Tile elements and accumulators of the CUDA-core complex contractions
// (theta, G3, the environments).  Complex64 states multiply-add in FP32.
// Complex128 states hold their shared-memory tiles as double-float values
// (converted once per tile load) and accumulate with exact heads plus FP32
// error terms (CAcc) on the FP32 pipes: this part executes FP64 at 2 FMA
// per clock per SM against 128 FP32, and a double-float multiply-add costs
// 12 FP32 operations per real product (relative error about K 2^-47 of the
// sum of |terms| for K products, 1e-12 at K = 128).
template <typename R> struct Mac;
template <> struct Mac<float> {
  using Elem = float2;
  struct Acc {
    float2 v = make_float2(0.f, 0.f);
  };
  static __device__ __forceinline__ Elem load(float2 x) { return x; }
  static __device__ __forceinline__ Elem zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void fma(Acc& a, Elem x, Elem y) { cfma(a.v, x, y); }    // += x y
  static __device__ __forceinline__ void fmac(Acc& a, Elem x, Elem y) { cfmac(a.v, x, y); }  // += conj(x) y
  static __device__ __forceinline__ float2 value(const Acc& a) { return a.v; }
};
template <> struct Mac<double> {
  using Elem = float4;
  using Acc = CAcc;
  static __device__ __forceinline__ Elem load(double2 x) { return cff_from_double2(x); }
  static __device__ __forceinline__ Elem zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void fma(Acc& a, Elem x, Elem y) { a.fma(x, y); }
  static __device__ __forceinline__ void fmac(Acc& a, Elem x, Elem y) { a.fmac(x, y); }
  static __device__ __forceinline__ double2 value(const Acc& a) { return a.value(); }
};

// ---------------------------------------------------------------------------
// reset to a computational basis state (chi = 1 everywhere)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void reset_kernel(cplx<R>* __restrict__ B, const size_t* __restrict__ site_off,
                             double* __restrict__ lam, const size_t* __restrict__ lam_off,
                             int* __restrict__ chi, const uint8_t* __restrict__ bits, int n,
                             DevReport* __restrict__ rep) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    cplx<R>* b = B + site_off[t];
    int bit = bits ? (bits[t] & 1) : 0;
    b[0] = cmk<R>(bit ? R(0) : R(1), R(0));
    b[1] = cmk<R>(bit ? R(1) : R(0), R(0));
  }
  if (t <= n) {
    chi[t] = 1;
    lam[lam_off[t]] = 1.0;
  }
  if (t == 0) {
    rep->discarded_weight = 0.0;
    rep->min_kept_sv = 1.0;
    rep->inv_norm = 1.0;
    rep->max_chi = 1;
    rep->degenerate_cuts = 0;
    rep->not_converged = 0;
    rep->max_sweeps = 0;
    rep->two_qubit_gates = 0;
    rep->svd_flops = 0.0;
    rep->tc_error = 0;
    rep->sweeps_fp32 = rep->sweeps_fp64 = 0;
    for (int i = 0; i < 4; ++i) rep->phase_cycles[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// theta = B_q B_{q+1}; gate; lam scaling (G1 + G2)
// ---------------------------------------------------------------------------
template <typename R, typename S>
__global__ void __launch_bounds__(kTile* kTile)
    theta_kernel(const cplx<R>* __restrict__ Bl, const cplx<R>* __restrict__ Br,
                 const DevGate* __restrict__ gate, const double* __restrict__ lam_l,
                 const int* __restrict__ chi, int q, cplx<R>* __restrict__ Cm, cplx<S>* __restrict__ A) {
  using C = cplx<R>;
  using MT = Mac<R>;
  using E = typename MT::Elem;
  const int chi_l = chi[q], chi_m = chi[q + 1], chi_r = chi[q + 2];
  const int al0 = blockIdx.y * kTile, ar0 = blockIdx.x * kTile;
  if (al0 >= chi_l || ar0 >= chi_r) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  __shared__ E sL[2][kTile][kTile + 1];
  __shared__ E sR[2][kTile][kTile + 1];
  typename MT::Acc acc[2][2];
  const C zero = cmk<R>(0, 0);
  for (int m0 = 0; m0 < chi_m; m0 += kTile) {
    {
      const int al = al0 + ty, mm = m0 + tx;
      const bool ok = al < chi_l && mm < chi_m;
      sL[0][ty][tx] = ok ? MT::load(Bl[(size_t)(al * 2 + 0) * chi_m + mm]) : MT::zero();
      sL[1][ty][tx] = ok ? MT::load(Bl[(size_t)(al * 2 + 1) * chi_m + mm]) : MT::zero();
    }
    {
      const int mm = m0 + ty, ar = ar0 + tx;
      const bool ok = mm < chi_m && ar < chi_r;
      sR[0][ty][tx] = ok ? MT::load(Br[(size_t)(mm * 2 + 0) * chi_r + ar]) : MT::zero();
      sR[1][ty][tx] = ok ? MT::load(Br[(size_t)(mm * 2 + 1) * chi_r + ar]) : MT::zero();
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kTile; ++kk) {
      const E l0 = sL[0][ty][kk], l1 = sL[1][ty][kk];
      const E r0 = sR[0][kk][tx], r1 = sR[1][kk][tx];
      MT::fma(acc[0][0], l0, r0);
      MT::fma(acc[0][1], l0, r1);
      MT::fma(acc[1][0], l1, r0);
      MT::fma(acc[1][1], l1, r1);
    }
    __syncthreads();
  }
  const int al = al0 + ty, ar = ar0 + tx;
  if (al >= chi_l || ar >= chi_r) return;
  const int m = 2 * chi_l, n = 2 * chi_r;
  const double lam = lam_l[al];
  C th[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) th[i][j] = MT::value(acc[i][j]);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      C out = zero;
#pragma unroll
      for (int ip = 0; ip < 2; ++ip)
#pragma unroll
        for (int jp = 0; jp < 2; ++jp) cfma(out, ccast<C>(gate->u[(2 * i + j) * 4 + 2 * ip + jp]), th[ip][jp]);
      const int row = 2 * al + i, col = j * chi_r + ar;
      Cm[(size_t)row * n + col] = out;
      if (A) {
        cplx<S> o = ccast<cplx<S>>(out);
        A[(size_t)col * m + row] = cmk<S>(S(lam) * o.x, S(lam) * o.y);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// one-sided Jacobi SVD + truncation (S1 + S2), one CTA per matrix
// ---------------------------------------------------------------------------

// Round-robin (circle method) schedule: in round r of nn-1 rounds, pair k.
__device__ __forceinline__ void rr_pair(int r, int k, int nn, int& i, int& j) {
  const int mod = nn - 1;
  int a, b;
  if (k == 0) {
    a = mod;
    b = r;
  } else {
    a = (r + k) % mod;
    b = (r - k + mod) % mod;
  }
  i = min(a, b);
  j = max(a, b);
}

template <typename S> struct SvdEps;
template <> struct SvdEps<double> {
  static __device__ double unit() { return 1.1102230246251565e-16; }
  static __device__ double tiny() { return 1e-290; }
};
template <> struct SvdEps<float> {
  static __device__ float unit() { return 5.9604645e-08f; }
  static __device__ float tiny() { return 1e-35f; }
};

// Jacobi sweeps on A (m x n, column-major) accumulating V (n x n, column-major).
// Returns the number of sweeps used (max_sweeps + 1 if not converged).
// Columns whose squared norm is at most `floor` (the rounding level of A)
// are left alone: rotating two of them only reshuffles rounding noise, and a
// rotation against a larger column would move it by less than that noise.
// Pairs of two columns the truncation discards follow the tail rules
// (truncation_tail, pair_tol); nrm2 and tail are n-entry shared-memory scratch.
template <typename S>
__device__ int jacobi_sweeps(cplx<S>* A, cplx<S>* V, int m, int n, int max_sweeps, S tol, S floor, double trunc_rel,
                             int chi_max, double* nrm2, int* tail, int* s_flag) {
  using C = cplx<S>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nn = n + (n & 1);
  const int pairs = nn / 2;
  const S tiny = SvdEps<S>::tiny();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    for (int j = warp; j < n; j += nwarps) {
      double acc = 0.0;
      for (int row = lane; row < m; row += 32) {
        const C x = A[(size_t)j * m + row];
        acc += double(x.x) * x.x + double(x.y) * x.y;
      }
      acc = warp_sum(acc);
      if (lane == 0) nrm2[j] = acc;
    }
    __syncthreads();
    __shared__ double s_loose;
    truncation_tail(nrm2, n, trunc_rel, chi_max, tail, &s_loose);
    const S loose = S(s_loose);
    if (threadIdx.x == 0) *s_flag = 0;
    __syncthreads();
    bool rotated = false;
    for (int r = 0; r < nn - 1; ++r) {
      for (int k = warp; k < pairs; k += nwarps) {
        int i, j;
        rr_pair(r, k, nn, i, j);
        if (j >= n) continue;
        const S tl = pair_tol(tail[i], tail[j], tol, loose);
        if (tl < S(0)) continue;
        C* ai = A + (size_t)i * m;
        C* aj = A + (size_t)j * m;
        S alpha = 0, beta = 0;
        C gam = cmk<S>(0, 0);
        for (int row = lane; row < m; row += 32) {
          const C x = ai[row], y = aj[row];
          alpha = fma(x.x, x.x, fma(x.y, x.y, alpha));
          beta = fma(y.x, y.x, fma(y.y, y.y, beta));
          cfmac(gam, x, y);
        }
        alpha = warp_sum(alpha);
        beta = warp_sum(beta);
        gam.x = warp_sum(gam.x);
        gam.y = warp_sum(gam.y);
        S c;
        C sph;  // s e^{i phi}
        if (!jacobi_rotation<S>(alpha, beta, gam.x, gam.y, tl, floor, tiny, c, sph)) continue;
        rotated = true;
        for (int row = lane; row < m; row += 32) {
          const C x = ai[row], y = aj[row];
          C ni = cmk<S>(c * x.x, c * x.y);
          ni = csub(ni, cmulc(sph, y));  // - s e^{-i phi} y
          C nj = cmk<S>(c * y.x, c * y.y);
          nj = cadd(nj, cmul(sph, x));
          ai[row] = ni;
          aj[row] = nj;
        }
        C* vi = V + (size_t)i * n;
        C* vj = V + (size_t)j * n;
        for (int row = lane; row < n; row += 32) {
          const C x = vi[row], y = vj[row];
          C ni = cmk<S>(c * x.x, c * x.y);
          ni = csub(ni, cmulc(sph, y));
          C nj = cmk<S>(c * y.x, c * y.y);
          nj = cadd(nj, cmul(sph, x));
          vi[row] = ni;
          vj[row] = nj;
        }
      }
      __syncthreads();
    }
    if (lane == 0 && rotated) *s_flag = 1;
    __syncthreads();
    const int any = *s_flag;
    __syncthreads();
    if (!any) return sweep + 1;
  }
  return max_sweeps + 1;
}

// Dynamic shared memory: [A m*n | V n*n] (when use_smem) then sig[n] (double), perm[n] (int).
template <typename S, typename R>
__global__ void __launch_bounds__(1024, 1)
    svd_truncate_kernel(cplx<S>* __restrict__ Ag, cplx<S>* __restrict__ Vg, int use_smem, int* __restrict__ chi,
                        int q, SvdParams p, cplx<R>* __restrict__ Bnext, double* __restrict__ lam_next,
                        DevReport* __restrict__ rep) {
  using C = cplx<S>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  __shared__ int s_k;
  __shared__ double s_nrm;
  const int chi_l = chi[q], chi_r = chi[q + 2];
  const int m = 2 * chi_l, n = 2 * chi_r;
  C* A = Ag;
  C* V = Vg;
  unsigned char* tail = smem_raw;
  if (use_smem) {
    A = reinterpret_cast<C*>(smem_raw);
    V = A + (size_t)m * n;
    tail = reinterpret_cast<unsigned char*>(V + (size_t)n * n);
    for (size_t t = threadIdx.x; t < (size_t)m * n; t += blockDim.x) A[t] = Ag[t];
  }
  double* sig = reinterpret_cast<double*>(tail);
  int* perm = reinterpret_cast<int*>(sig + n);
  for (size_t t = threadIdx.x; t < (size_t)n * n; t += blockDim.x) {
    const size_t col = t / n, row = t % n;
    V[t] = cmk<S>(col == row ? S(1) : S(0), S(0));
  }
  __syncthreads();

  // rotate while |b_ij| > tol sqrt(b_ii b_jj), tol = 4 sqrt(max(m, n)) u
  const S tol = p.tol > 0 ? S(p.tol) : S(4.0 * sqrt(double(max(m, n)))) * SvdEps<S>::unit();
  // ||A||_F^2 sets the noise floor of a column
  {
    double part = 0.0;
    for (size_t t = threadIdx.x; t < (size_t)m * n; t += blockDim.x) {
      const double x = A[t].x, y = A[t].y;
      part += x * x + y * y;
    }
    part = warp_sum(part);
    if (threadIdx.x == 0) s_nrm = 0.0;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_nrm, part);
    __syncthreads();
  }
  const double fro2 = s_nrm;
  const S floor = S(16.0 * double(SvdEps<S>::unit()) * double(SvdEps<S>::unit()) * fro2);
  __syncthreads();
  const int sweeps = jacobi_sweeps<S>(A, V, m, n, p.max_sweeps, tol, floor, p.trunc_rel, p.chi_max, sig, perm, &s_flag);

  // sigma_j = ||A_j|| (Algorithm 1: column norms)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int j = warp; j < n; j += nwarps) {
    double acc = 0.0;
    const C* aj = A + (size_t)j * m;
    for (int row = lane; row < m; row += 32) {
      const double x = aj[row].x, y = aj[row].y;
      acc += x * x + y * y;
    }
    acc = warp_sum(acc);
    if (lane == 0) sig[j] = sqrt(acc);
  }
  __syncthreads();
  // descending order, ties by index (deterministic)
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double sj = sig[j];
    int rank = 0;
    for (int i = 0; i < n; ++i) {
      const double si = sig[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    perm[rank] = j;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int a = 0; a < n; ++a) total += sig[perm[a]] * sig[perm[a]];
    const double smax = sig[perm[0]];
    int cnt = 0;
    for (int a = 0; a < n; ++a) {
      const double s = sig[perm[a]];
      if (p.trunc_rel > 0.0 ? (s > p.trunc_rel * smax) : (s > 0.0)) ++cnt;
    }
    int k = min(cnt, min(p.chi_max, min(m, n)));
    if (k < 1) k = 1;
    double kept = 0.0;
    for (int a = 0; a < k; ++a) kept += sig[perm[a]] * sig[perm[a]];
    double nrm = sqrt(kept);
    if (!(nrm > 0.0)) nrm = 1.0;
    s_k = k;
    s_nrm = nrm;
    rep->discarded_weight += total > 0.0 ? 1.0 - kept / total : 0.0;
    const double smin = sig[perm[k - 1]] / nrm;
    if (smin < rep->min_kept_sv) rep->min_kept_sv = smin;
    if (k > rep->max_chi) rep->max_chi = k;
    if (k < n && k == p.chi_max) {
      const double a0 = sig[perm[k - 1]], a1 = sig[perm[k]];
      if (a1 > 0.0 && fabs(a0 - a1) <= 1e-10 * a0) rep->degenerate_cuts += 1;
    }
    if (sweeps > p.max_sweeps) rep->not_converged += 1;
    if (sweeps > rep->max_sweeps) rep->max_sweeps = sweeps;
    rep->two_qubit_gates += 1;
    // per sweep and column pair: three dot products over m rows (16 m flops)
    // and one rotation of the A and V columns (12 (m + n) flops)
    rep->svd_flops += (double)min(sweeps, p.max_sweeps) * 0.5 * n * (n - 1) * (16.0 * m + 12.0 * (m + n));
    (sizeof(S) == 8 ? rep->sweeps_fp64 : rep->sweeps_fp32) += min(sweeps, p.max_sweeps);
    rep->inv_norm = 1.0 / nrm;
    chi[q + 1] = k;
  }
  __syncthreads();
  const int k = s_k;
  const double inv = 1.0 / s_nrm;
  for (int a = threadIdx.x; a < k; a += blockDim.x) lam_next[a] = sig[perm[a]] * inv;
  // B~_{q+1}[a, c] = conj(V[c, perm[a]])   (V = W, right singular vectors)
  for (size_t t = threadIdx.x; t < (size_t)k * n; t += blockDim.x) {
    const int a = (int)(t / n), c = (int)(t % n);
    const C v = V[(size_t)perm[a] * n + c];
    Bnext[t] = ccast<cplx<R>>(cconj(v));
  }
}

// ---------------------------------------------------------------------------
// B~_q = C B~_{q+1}^dagger / ||s[:k]||  (G3, Eq. Bl)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kTile* kTile)
    g3_kernel(const cplx<R>* __restrict__ Cm, const cplx<R>* __restrict__ Bn, const int* __restrict__ chi, int q,
              const DevReport* __restrict__ rep, cplx<R>* __restrict__ Bout) {
  using C = cplx<R>;
  using MT = Mac<R>;
  using E = typename MT::Elem;
  const int chi_l = chi[q], k = chi[q + 1], chi_r = chi[q + 2];
  const int m = 2 * chi_l, n = 2 * chi_r;
  const int r0 = blockIdx.y * kTile, a0 = blockIdx.x * kTile;
  if (r0 >= m || a0 >= k) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  __shared__ E sA[kTile][kTile + 1];
  __shared__ E sB[kTile][kTile + 1];  // conj(B~_{q+1})
  typename MT::Acc acc;
  for (int c0 = 0; c0 < n; c0 += kTile) {
    const int c = c0 + tx;
    sA[ty][tx] = (r0 + ty < m && c < n) ? MT::load(Cm[(size_t)(r0 + ty) * n + c]) : MT::zero();
    sB[ty][tx] = (a0 + ty < k && c < n) ? MT::load(cconj(Bn[(size_t)(a0 + ty) * n + c])) : MT::zero();
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kTile; ++kk) MT::fma(acc, sA[ty][kk], sB[tx][kk]);
    __syncthreads();
  }
  const int r = r0 + ty, a = a0 + tx;
  if (r < m && a < k) {
    const R inv = R(rep->inv_norm);
    const C v = MT::value(acc);
    Bout[(size_t)r * k + a] = cmk<R>(v.x * inv, v.y * inv);
  }
}

// ---------------------------------------------------------------------------
// one-qubit gate (exact, keeps the canonical form)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void gate1_kernel(cplx<R>* __restrict__ B, const DevGate* __restrict__ gate, const int* __restrict__ chi,
                             int q) {
  using C = cplx<R>;
  const int chi_l = chi[q], chi_r = chi[q + 1];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= chi_l * chi_r) return;
  const int al = t / chi_r, ar = t % chi_r;
  C* p0 = B + (size_t)(al * 2 + 0) * chi_r + ar;
  C* p1 = B + (size_t)(al * 2 + 1) * chi_r + ar;
  const C b0 = *p0, b1 = *p1;
  C n0 = cmk<R>(0, 0), n1 = cmk<R>(0, 0);
  cfma(n0, ccast<C>(gate->u[0]), b0);
  cfma(n0, ccast<C>(gate->u[1]), b1);
  cfma(n1, ccast<C>(gate->u[2]), b0);
  cfma(n1, ccast<C>(gate->u[3]), b1);
  *p0 = n0;
  *p1 = n1;
}

// ---------------------------------------------------------------------------
// bind template angles: u = exp(i phi) M+ + exp(-i phi) M-
// ---------------------------------------------------------------------------
static __global__ void bind_kernel(const DevTmplGate* __restrict__ tmpl, int n_gates, const double* __restrict__ theta,
                                   DevGate* __restrict__ out) {
  const int g = blockIdx.x;
  if (g >= n_gates) return;
  const DevTmplGate& t = tmpl[g];
  const double phi = t.param >= 0 ? t.coeff * theta[t.param] : 0.0;
  double s, c;
  sincos(phi, &s, &c);
  const int e = threadIdx.x;
  if (e < 16) {
    const double2 a = t.mp[e], b = t.mm[e];
    // (c + i s) a + (c - i s) b
    double2 u;
    u.x = c * (a.x + b.x) - s * (a.y - b.y);
    u.y = c * (a.y + b.y) + s * (a.x - b.x);
    out[g].u[e] = u;
  }
  if (e == 0) {
    out[g].q = t.q;
    out[g].arity = t.arity;
  }
}

}  // namespace mpsv
