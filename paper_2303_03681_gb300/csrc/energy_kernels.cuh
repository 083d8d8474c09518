// Pauli-sum energy kernels (arXiv:2303.03681, Eqs. expec1/expec2).
//
// <P> for a string with first non-identity site m and last n is
//   Tr( T_{P_n} ... T_{P_m}( diag(lam_m^2) ) ),
//   T_P(L)[b, d] = sum_{a, c, i} conj(B[a, i, b]) L[a, c] P[i, pi(i)] B[c, pi(i), d],
// where pi(i) is the column of the single nonzero entry of row i of the
// Pauli matrix.  Strings are arranged in a prefix trie; the environment L of
// a trie node is computed once and shared by every string through it.  Site
// j (level j) runs:
//   env_m_kernel      M^b_p = L_p B_j[:, b, :] for each parent entry p
//                     (L_p = diag(lam_j^2) for strings starting at j),
//   env_child_kernel  L_c = sum_i ph_i B_j[:, i, :]^H M^{pi(i)}_p for each
//                     node c that has children,
//   env_leaf_kernel   <P> = Re sum_i ph_i <B_j[:, i, :], M^{pi(i)}_p> for a
//                     string ending at j whose node has no children,
//   env_trace_kernel  <P> = Re Tr L_c for a string ending at a node with children;
// energy_reduce_kernel sums c_k <P_k> in FP64 in a fixed order.
#pragma once

#include "common.cuh"
#include "gate_kernels.cuh"  // kTile, Mac

namespace mpsv {

// (pi(0), pi(1), phase_0, phase_1) of I, X, Y, Z.
struct PauliRow {
  int p0, p1;
  double2 ph0, ph1;
};
__device__ __forceinline__ PauliRow pauli_row(int op) {
  PauliRow r;
  switch (op) {
    case 1:  // X
      r.p0 = 1; r.p1 = 0; r.ph0 = make_double2(1, 0); r.ph1 = make_double2(1, 0); break;
    case 2:  // Y = [[0,-i],[i,0]]
      r.p0 = 1; r.p1 = 0; r.ph0 = make_double2(0, -1); r.ph1 = make_double2(0, 1); break;
    case 3:  // Z
      r.p0 = 0; r.p1 = 1; r.ph0 = make_double2(1, 0); r.ph1 = make_double2(-1, 0); break;
    default:  // I
      r.p0 = 0; r.p1 = 1; r.ph0 = make_double2(1, 0); r.ph1 = make_double2(1, 0); break;
  }
  return r;
}

struct EnvLevel {
  const int* parent_src;  // per parent entry: slot in the previous environment buffer, -1 = diag(lam^2)
  const int2* child;      // per materialised node: (parent entry, op)
  const int4* leaf;       // per string ending at a leaf node: (parent entry, op, term, 0)
  const int2* trace;      // per string ending at a materialised node: (slot, term)
  int n_parents, n_children, n_leaves, n_traces;
  int site;
  int cap_l, cap_r;  // bond dimensions left / right of the site at launch (grid extents and slot strides)
};

// M_p[a][b][d] = sum_c L_p[a][c] B[c][b][d]   (b = 0, 1): row-major chi_l x 2 chi_r,
// i.e. M_p = L_p B with B viewed as chi_l x 2 chi_r; slot stride of M: 2 cap_l cap_r
template <typename R>
__global__ void __launch_bounds__(kTile* kTile)
    env_m_kernel(const cplx<R>* __restrict__ Lprev, const cplx<R>* __restrict__ B, const double* __restrict__ lam,
                 const int* __restrict__ chi, EnvLevel lv, cplx<R>* __restrict__ M) {
  using C = cplx<R>;
  const int chi_l = chi[lv.site], chi_r = chi[lv.site + 1];
  const int tiles_c = (lv.cap_r + kTile - 1) / kTile, tiles_r = (lv.cap_l + kTile - 1) / kTile;
  const int per = tiles_c * tiles_r;
  const int p = blockIdx.x / per, tile = blockIdx.x % per;
  const int a0 = (tile / tiles_c) * kTile, d0 = (tile % tiles_c) * kTile;
  if (p >= lv.n_parents || a0 >= chi_l || d0 >= chi_r) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int src = lv.parent_src[p];
  C* out = M + (size_t)p * 2 * lv.cap_l * lv.cap_r;
  const int a = a0 + ty, d = d0 + tx;
  const C zero = cmk<R>(0, 0);
  if (src < 0) {
    if (a < chi_l && d < chi_r) {
      const R w = R(lam[a] * lam[a]);
      const C b0 = B[(size_t)(a * 2 + 0) * chi_r + d], b1 = B[(size_t)(a * 2 + 1) * chi_r + d];
      out[(size_t)a * 2 * chi_r + d] = cscale(b0, w);
      out[(size_t)a * 2 * chi_r + chi_r + d] = cscale(b1, w);
    }
    return;
  }
  using MT = Mac<R>;
  using E = typename MT::Elem;
  const C* L = Lprev + (size_t)src * lv.cap_l * lv.cap_l;
  __shared__ E sL[kTile][kTile + 1];
  __shared__ E sB[2][kTile][kTile + 1];
  typename MT::Acc acc0, acc1;
  for (int c0 = 0; c0 < chi_l; c0 += kTile) {
    sL[ty][tx] = (a < chi_l && c0 + tx < chi_l) ? MT::load(L[(size_t)a * chi_l + c0 + tx]) : MT::zero();
    const int c = c0 + ty;
    const bool ok = c < chi_l && d < chi_r;
    sB[0][ty][tx] = ok ? MT::load(B[(size_t)(c * 2 + 0) * chi_r + d]) : MT::zero();
    sB[1][ty][tx] = ok ? MT::load(B[(size_t)(c * 2 + 1) * chi_r + d]) : MT::zero();
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kTile; ++kk) {
      const E l = sL[ty][kk];
      MT::fma(acc0, l, sB[0][kk][tx]);
      MT::fma(acc1, l, sB[1][kk][tx]);
    }
    __syncthreads();
  }
  if (a < chi_l && d < chi_r) {
    out[(size_t)a * 2 * chi_r + d] = MT::value(acc0);
    out[(size_t)a * 2 * chi_r + chi_r + d] = MT::value(acc1);
  }
}

// L_c[b][d] = sum_i ph_i sum_a conj(B[a][i][b]) M^{pi(i)}_p[a][d]
template <typename R>
__global__ void __launch_bounds__(kTile* kTile)
    env_child_kernel(const cplx<R>* __restrict__ M, const cplx<R>* __restrict__ B, const int* __restrict__ chi,
                     EnvLevel lv, cplx<R>* __restrict__ Lcur) {
  using C = cplx<R>;
  const int chi_l = chi[lv.site], chi_r = chi[lv.site + 1];
  const int tiles = (lv.cap_r + kTile - 1) / kTile;
  const int per = tiles * tiles;
  const int cidx = blockIdx.x / per, tile = blockIdx.x % per;
  const int b0 = (tile / tiles) * kTile, d0 = (tile % tiles) * kTile;
  if (cidx >= lv.n_children || b0 >= chi_r || d0 >= chi_r) return;
  const int2 cd = lv.child[cidx];
  const PauliRow pr = pauli_row(cd.y);
  const C* Mp = M + (size_t)cd.x * 2 * lv.cap_l * lv.cap_r;
  const C* M0 = Mp + (size_t)pr.p0 * chi_r;  // partner of row i = 0 (row stride 2 chi_r)
  const C* M1 = Mp + (size_t)pr.p1 * chi_r;  // partner of row i = 1
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int b = b0 + ty, d = d0 + tx;
  using MT = Mac<R>;
  using E = typename MT::Elem;
  __shared__ E sB[2][kTile][kTile + 1];  // [i][a][b]
  __shared__ E sM[2][kTile][kTile + 1];  // [i][a][d]
  typename MT::Acc acc0, acc1;
  for (int a0 = 0; a0 < chi_l; a0 += kTile) {
    const int a = a0 + ty;
    const int bb = b0 + tx;
    const bool okb = a < chi_l && bb < chi_r;
    sB[0][ty][tx] = okb ? MT::load(B[(size_t)(a * 2 + 0) * chi_r + bb]) : MT::zero();
    sB[1][ty][tx] = okb ? MT::load(B[(size_t)(a * 2 + 1) * chi_r + bb]) : MT::zero();
    const bool okm = a < chi_l && d < chi_r;
    sM[0][ty][tx] = okm ? MT::load(M0[(size_t)a * 2 * chi_r + d]) : MT::zero();
    sM[1][ty][tx] = okm ? MT::load(M1[(size_t)a * 2 * chi_r + d]) : MT::zero();
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kTile; ++kk) {
      MT::fmac(acc0, sB[0][kk][ty], sM[0][kk][tx]);
      MT::fmac(acc1, sB[1][kk][ty], sM[1][kk][tx]);
    }
    __syncthreads();
  }
  if (b < chi_r && d < chi_r) {
    C out = cmul(ccast<C>(pr.ph0), MT::value(acc0));
    out = cadd(out, cmul(ccast<C>(pr.ph1), MT::value(acc1)));
    Lcur[(size_t)cidx * lv.cap_r * lv.cap_r + (size_t)b * chi_r + d] = out;
  }
}

// One warp per leaf: Re sum_i ph_i sum_{a,b} conj(B[a][i][b]) M^{pi(i)}[a][b], FP64 accumulation.
template <typename R>
__global__ void env_leaf_kernel(const cplx<R>* __restrict__ M, const cplx<R>* __restrict__ B,
                                const int* __restrict__ chi, EnvLevel lv, double* __restrict__ vals) {
  using C = cplx<R>;
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= lv.n_leaves) return;
  const int chi_l = chi[lv.site], chi_r = chi[lv.site + 1];
  const int4 lf = lv.leaf[w];
  const PauliRow pr = pauli_row(lf.y);
  const C* Mp = M + (size_t)lf.x * 2 * lv.cap_l * lv.cap_r;
  const C* Mi0 = Mp + (size_t)pr.p0 * chi_r;  // row stride 2 chi_r
  const C* Mi1 = Mp + (size_t)pr.p1 * chi_r;
  double2 s0 = make_double2(0, 0), s1 = make_double2(0, 0);
  const int tot = chi_l * chi_r;
  for (int t = lane; t < tot; t += 32) {
    const int a = t / chi_r, b = t % chi_r;
    const C x0 = B[(size_t)(a * 2 + 0) * chi_r + b], x1 = B[(size_t)(a * 2 + 1) * chi_r + b];
    const C y0 = Mi0[(size_t)a * 2 * chi_r + b], y1 = Mi1[(size_t)a * 2 * chi_r + b];
    const double2 p0 = ccast<double2>(cmulc(x0, y0)), p1 = ccast<double2>(cmulc(x1, y1));
    s0.x += p0.x; s0.y += p0.y;
    s1.x += p1.x; s1.y += p1.y;
  }
  s0.x = warp_sum(s0.x); s0.y = warp_sum(s0.y);
  s1.x = warp_sum(s1.x); s1.y = warp_sum(s1.y);
  if (lane == 0) {
    const double re = (pr.ph0.x * s0.x - pr.ph0.y * s0.y) + (pr.ph1.x * s1.x - pr.ph1.y * s1.y);
    vals[lf.z] = re;
  }
}

// One warp per string ending at a materialised node: Re Tr L.
template <typename R>
__global__ void env_trace_kernel(const cplx<R>* __restrict__ Lcur, const int* __restrict__ chi, EnvLevel lv,
                                 double* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= lv.n_traces) return;
  const int chi_r = chi[lv.site + 1];
  const int2 tr = lv.trace[w];
  const cplx<R>* L = Lcur + (size_t)tr.x * lv.cap_r * lv.cap_r;
  double s = 0.0;
  for (int b = lane; b < chi_r; b += 32) s += (double)L[(size_t)b * chi_r + b].x;
  s = warp_sum(s);
  if (lane == 0) vals[tr.y] = s;
}

// E = constant + sum_k c_k vals[k] (terms with an empty support keep vals = 1).
// One block of 1024 threads; fixed summation order.
// A set *err (a tensor-core contraction gave up waiting) turns the energy into NaN.
static __global__ void energy_reduce_kernel(const double* __restrict__ vals, const double* __restrict__ coeffs,
                                            long long n_terms, double constant, const int* __restrict__ err,
                                            double* __restrict__ out) {
  __shared__ double part[32];
  double s = 0.0;
  for (long long k = threadIdx.x; k < n_terms; k += blockDim.x) s += coeffs[k] * vals[k];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) *out = (err && *err) ? __longlong_as_double(0x7ff8000000000000ll) : constant + v;
  }
}

static __global__ void fill_kernel(double* __restrict__ p, long long n, double v) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) p[t] = v;
}

// Linear observables of the per-string values (reduced density matrices):
// out[r] = sum_{e in [row_ptr[r], row_ptr[r+1])} w[e] * vals[cols[e]], complex
// weights, FP64.  One warp per row; lane l takes the entries l, l + 32, ...
// and the lanes are summed in a fixed tree, so the result does not depend on
// the launch.  blockDim.x must be a multiple of 32 (whole warps leave
// together, so the shuffles see full warps).
static __global__ void observables_kernel(const double* __restrict__ vals, const long long* __restrict__ row_ptr,
                                          const int* __restrict__ cols, const double2* __restrict__ w,
                                          long long n_rows, double2* __restrict__ out) {
  const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= n_rows) return;
  double re = 0.0, im = 0.0;
  const long long end = row_ptr[r + 1];
  for (long long e = row_ptr[r] + lane; e < end; e += 32) {
    const double v = vals[cols[e]];
    const double2 c = w[e];
    re = fma(c.x, v, re);
    im = fma(c.y, v, im);
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) out[r] = make_double2(re, im);
}

// ---------------------------------------------------------------------------
// tensor-core forms (complex64 states): the same products as env_m_kernel and
// env_child_kernel, as problems of tc::cgemm_kernel
// ---------------------------------------------------------------------------

// M_p = L_src B_j for the parents whose environment is a stored matrix;
// list[z] = (parent entry p, environment slot src).
struct EnvMProb {
  const int2* list;
  const float2* Lprev;
  const float2* B;
  float2* M;
  int chi_l, chi_r;
  __device__ __forceinline__ void dims(int, int& m, int& n, int& k) const {
    m = chi_l;
    n = 2 * chi_r;
    k = chi_l;
  }
  __device__ __forceinline__ float2 a(int z, int row, int kk) const {
    return Lprev[(size_t)list[z].y * chi_l * chi_l + (size_t)row * chi_l + kk];
  }
  __device__ __forceinline__ float2 b(int, int kk, int col) const { return B[(size_t)kk * 2 * chi_r + col]; }
  __device__ __forceinline__ void store(int z, int row, int col, float2 v) const {
    M[(size_t)list[z].x * 2 * chi_l * chi_r + (size_t)row * 2 * chi_r + col] = v;
  }
};

// L_c[b][d] = sum_{i, a} ph_i conj(B[a][i][b]) M_p[a][pi(i)][d]; K runs over (i, a).
struct EnvChildProb {
  const int2* child;  // (parent entry, op)
  const float2* B;
  const float2* M;
  float2* Lcur;
  int chi_l, chi_r;
  __device__ __forceinline__ void dims(int, int& m, int& n, int& k) const {
    m = chi_r;
    n = chi_r;
    k = 2 * chi_l;
  }
  __device__ __forceinline__ float2 a(int z, int row, int kk) const {
    const int i = kk >= chi_l ? 1 : 0, aa = kk - i * chi_l;
    const PauliRow pr = pauli_row(child[z].y);
    const double2 ph = i ? pr.ph1 : pr.ph0;
    const float2 x = B[(size_t)(aa * 2 + i) * chi_r + row];  // conj(x) * ph
    return make_float2(float(ph.x) * x.x + float(ph.y) * x.y, float(ph.y) * x.x - float(ph.x) * x.y);
  }
  __device__ __forceinline__ float2 b(int z, int kk, int col) const {
    const int i = kk >= chi_l ? 1 : 0, aa = kk - i * chi_l;
    const int2 cd = child[z];
    const PauliRow pr = pauli_row(cd.y);
    const int pi = i ? pr.p1 : pr.p0;
    return M[(size_t)cd.x * 2 * chi_l * chi_r + (size_t)aa * 2 * chi_r + (size_t)pi * chi_r + col];
  }
  __device__ __forceinline__ void store(int z, int row, int col, float2 v) const {
    Lcur[(size_t)z * chi_r * chi_r + (size_t)row * chi_r + col] = v;
  }
};

// M_p = diag(lam^2) B for the parents that start strings at this site; list[z] = entry p.
template <typename R>
__global__ void env_m_diag_kernel(const int* __restrict__ list, int n, const cplx<R>* __restrict__ B,
                                  const double* __restrict__ lam, int chi_l, int chi_r, cplx<R>* __restrict__ M) {
  const size_t per = (size_t)chi_l * 2 * chi_r;
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * n) return;
  const int z = (int)(t / per);
  const size_t e = t % per;
  const int a = (int)(e / (2 * chi_r));
  const R w = R(lam[a] * lam[a]);
  M[(size_t)list[z] * per + e] = cscale(B[e], w);
}

}  // namespace mpsv
