// One-sided Jacobi SVD on a thread-block cluster (Algorithm 1 of the paper's
// "SVD and one-side jacobi" subsection, parallelised over up to 16 SMs).
//
// The kernel orthogonalises the n = 2 chi_r columns of A = C~ (m = 2 chi_l
// rows, read from the row-major theta C as A[r, c] = lam_q[r / 2] C[r, c])
// and accumulates the same rotations into V (Algorithm 1: A = A J, V = V J).
// Each column is stored as the stacked vector [A(:, c); V(:, c)] of length
// m + n, so one rotation updates both.  When the columns are orthogonal,
// A = U Sigma and V holds the right singular vectors W; the kept rows of
// B~_{q+1} = W^H are conjugated columns of V, unitary to rounding for any
// singular value (normalising columns of A instead would amplify the
// rounding error of small columns by s_1 / s_j).
//
// Parallel order.  The n columns are split into 2P blocks of b columns
// (zero-padded).  CTA p of the P-CTA cluster holds the blocks at positions p
// and 2P-1-p of a circle-method round robin over the 2P blocks: in each of
// the 2P-1 rounds of a sweep every CTA orthogonalises all column pairs
// between its two blocks (and, in the first round, also the pairs inside
// each block), then every block except the one at position 0 advances one
// position.  Blocks move through distributed shared memory into ping-pong
// buffers, so one cluster barrier per round orders the hand-over.  When the
// stacked columns do not fit the shared memory they stay in a global
// workspace, and a round only renames the positions.
//
// FP64 accuracy at FP32 speed.  This part runs FP64 at 2 FMA/clk/SM, so an
// all-FP64 Jacobi of a 100-column theta takes tens of milliseconds.  The
// mixed form runs the sweeps in FP32 to FP32 convergence (V32 accumulated as
// usual), re-orthonormalises V32 in FP64 with two pairwise first-order
// passes v_i <- v_i - 1/2 sum_j (v_j^H v_i) v_j (the symmetric update
// V (I - E / 2), E = V^H V - I, which leaves ||E||^2), rebuilds A = C~ V in
// FP64 from the theta, converts the stacked columns to double-float
// (dfloat.cuh) and finishes with double-float sweeps on the FP32 units,
// which start near convergence and converge quadratically.  The singular
// values, the truncation and B~_{q+1} then come from columns accurate to
// about 2^-46 (the all-FP64 form, svd_fp64 = 2, sweeps in FP64 throughout).
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"

namespace mpsv {

namespace cg = cooperative_groups;

// Position (0 .. 2P-1) -> (CTA rank, slot 0 = top / 1 = bottom).
__device__ __forceinline__ void pos_owner(int pos, int P, int& rank, int& slot) {
  if (pos < P) {
    rank = pos;
    slot = 0;
  } else {
    rank = 2 * P - 1 - pos;
    slot = 1;
  }
}

// Stacked-column elements a lane keeps in registers in the cross rounds
// (columns up to 32 * kClusterRegs = 512 entries long).
constexpr int kClusterRegs = 16;

template <typename S>
__device__ __forceinline__ void warp_sum4(S& a, S& b, S& c, S& d) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
}

// One warp rotates two stacked columns [A; V] held in shared memory; the Gram
// entries use the first m (A) rows.
template <typename S>
__device__ __forceinline__ int jacobi_pair_smem(cplx<S>* ai, cplx<S>* aj, int m, int len, int lane, S tol, S floor,
                                                S tiny) {
  using C = cplx<S>;
  S alpha = 0, beta = 0, gr = 0, gi = 0;
  for (int r = lane; r < m; r += 32) {
    const C x = ai[r], y = aj[r];
    alpha = fma(x.x, x.x, fma(x.y, x.y, alpha));
    beta = fma(y.x, y.x, fma(y.y, y.y, beta));
    gr = fma(x.x, y.x, fma(x.y, y.y, gr));
    gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
  }
  warp_sum4(alpha, beta, gr, gi);
  S c;
  C sph;
  if (!jacobi_rotation(alpha, beta, gr, gi, tol, floor, tiny, c, sph)) return 0;
  for (int r = lane; r < len; r += 32) {
    const C x = ai[r], y = aj[r];
    ai[r] = csub(cmk<S>(c * x.x, c * x.y), cmulc(sph, y));
    aj[r] = cadd(cmk<S>(c * y.x, c * y.y), cmul(sph, x));
  }
  return 1;
}

// Same with the first column in registers: x[i] is row lane + 32 i.
template <typename S>
__device__ __forceinline__ int jacobi_pair_reg(cplx<S> (&x)[kClusterRegs], cplx<S>* aj, int m, int len, int lane,
                                               S tol, S floor, S tiny) {
  using C = cplx<S>;
  S alpha = 0, beta = 0, gr = 0, gi = 0;
#pragma unroll
  for (int i = 0; i < kClusterRegs; ++i) {
    const int r = lane + 32 * i;
    if (r < m) {
      const C xv = x[i], y = aj[r];
      alpha = fma(xv.x, xv.x, fma(xv.y, xv.y, alpha));
      beta = fma(y.x, y.x, fma(y.y, y.y, beta));
      gr = fma(xv.x, y.x, fma(xv.y, y.y, gr));
      gi = fma(xv.x, y.y, fma(-xv.y, y.x, gi));
    }
  }
  warp_sum4(alpha, beta, gr, gi);
  S c;
  C sph;
  if (!jacobi_rotation(alpha, beta, gr, gi, tol, floor, tiny, c, sph)) return 0;
#pragma unroll
  for (int i = 0; i < kClusterRegs; ++i) {
    const int r = lane + 32 * i;
    if (r < len) {
      const C xv = x[i], y = aj[r];
      x[i] = csub(cmk<S>(c * xv.x, c * xv.y), cmulc(sph, y));
      aj[r] = cadd(cmk<S>(c * y.x, c * y.y), cmul(sph, xv));
    }
  }
  return 1;
}



// Double-float forms of the two pair steps (FP64-accurate sweeps; the columns
// hold float4 = (re_h, re_l, im_h, im_l)).  The Gram entries accumulate per
// lane as exact heads plus FP32 error terms (GramAcc) and in double-float
// across the warp; the rotation (an FP32 angle
// brought to unit norm in double-float, ff_angle) is applied in
// double-float.
__device__ __forceinline__ void ff_warp_sum4(ff& a, ff& b, ff& c, ff& d) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = ff_add(a, ff_shfl_xor(a, o));
    b = ff_add(b, ff_shfl_xor(b, o));
    c = ff_add(c, ff_shfl_xor(c, o));
    d = ff_add(d, ff_shfl_xor(d, o));
  }
}

__device__ __forceinline__ void ff_gram_row(const float4& x, const float4& y, GramAcc& alpha, GramAcc& beta,
                                            GramAcc& gr, GramAcc& gi) {
  const ff xr = re_of(x), xi = im_of(x), yr = re_of(y), yi = im_of(y);
  alpha.add(xr, xr);
  alpha.add(xi, xi);
  beta.add(yr, yr);
  beta.add(yi, yi);
  gr.add(xr, yr);
  gr.add(xi, yi);
  gi.add(xr, yi);
  gi.add(ff_neg(xi), yr);
}

// x' = c x - conj(s) y, y' = c y + s x with s = sr + i si
__device__ __forceinline__ void ff_rotate(float4& x, float4& y, ff c, ff sr, ff si) {
  const ff xr = re_of(x), xi = im_of(x), yr = re_of(y), yi = im_of(y);
  const ff nxr = ff_sub(ff_mul(c, xr), ff_add(ff_mul(sr, yr), ff_mul(si, yi)));
  const ff nxi = ff_sub(ff_mul(c, xi), ff_sub(ff_mul(sr, yi), ff_mul(si, yr)));
  const ff nyr = ff_add(ff_mul(c, yr), ff_sub(ff_mul(sr, xr), ff_mul(si, xi)));
  const ff nyi = ff_add(ff_mul(c, yi), ff_add(ff_mul(sr, xi), ff_mul(si, xr)));
  x = cff(nxr, nxi);
  y = cff(nyr, nyi);
}

// 2^-e for the exponent e of a positive normal float x (x 2^-e in [1, 2)).
__device__ __forceinline__ float pow2_inv_exponent(float x) {
  const int e = ((__float_as_int(x) >> 23) & 0xff) - 127;
  return __int_as_float((127 - e) << 23);
}

// The rotation of a pair from its double-float Gram entries, on the FP32
// pipes only (this part runs FP64 at 2 FMA/clk/SM, and an FP64 angle for
// every pair of 16 warps cost more than the rest of the pair step).  The
// stopping test and the angle use FP32 values of the heads, scaled by a
// power of two so that max(b_ii, b_jj) lies in [1, 2) (|g| is taken as a
// scaled hypot, so no square underflows); b_jj - b_ii is formed in
// double-float first, so the angle of a nearly degenerate pair is not
// rounding noise.  The FP32 angle gives (c, s e^{i phi}) with c^2 + |s|^2 =
// 1 + d, |d| ~ 2^-24; d is evaluated to ~2^-47 with exact products and sums
// (two_prod, two_sum) and the rotation is scaled by f = 1 - d/2 + 3d^2/8
// (the binomial series of (1 + d)^(-1/2)), which makes it unitary to
// double-float rounding.  The angle itself is FP32-accurate: a pair left
// with |g| ~ 1e-7 of its old value is rotated again in the next sweep.
__device__ __forceinline__ bool ff_angle(ff alpha, ff beta, ff gr, ff gi, float tol, float floor, ff& c, ff& sr,
                                         ff& si) {
  const float a = alpha.h, b = beta.h;
  if (!(fminf(a, b) > floor)) return false;
  const float scl = pow2_inv_exponent(fmaxf(a, b));
  const float xr = gr.h * scl, xi = gi.h * scl;  // |x| <= sqrt(a b) scl < 2
  const float ax = fabsf(xr), ay = fabsf(xi);
  const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
  if (!(mx > 0.f)) return false;
  const float rr = mn / mx;
  const float mag = mx * sqrtf(fmaf(rr, rr, 1.f));
  if (!(mag > tol * sqrtf(a * scl) * sqrtf(b * scl))) return false;
  const ff dba = ff_sub(beta, alpha);
  const float zeta = (dba.h * scl) / (2.f * mag);
  if (!(fabsf(zeta) < 3e38f)) return false;
  const float t = fabsf(zeta) > 1e15f ? 0.5f / zeta
                                       : copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
  const float cf = rsqrtf(fmaf(t, t, 1.f));
  const float sf = t * cf / mag;
  // s e^{i phi} = sf (xr + i xi), exact as double-float
  const ff s_r = two_prod(sf, xr), s_i = two_prod(sf, xi);
  // d = c^2 + |s|^2 - 1 with exact products and sums of the heads (cf^2
  // can round just below 1/2, so even cf^2 - 1 goes through two_sum)
  const ff c2 = two_prod(cf, cf), r2 = two_prod(s_r.h, s_r.h), i2 = two_prod(s_i.h, s_i.h);
  const ff u0 = two_sum(c2.h, -1.f);
  const ff u1 = two_sum(u0.h, r2.h);
  const ff u2 = two_sum(u1.h, i2.h);
  const float tail = __fadd_rn(__fadd_rn(__fadd_rn(u0.l, u1.l), u2.l), __fadd_rn(c2.l, __fadd_rn(r2.l, i2.l)));
  const float cross = 2.f * __fmaf_rn(s_r.h, s_r.l, __fmul_rn(s_i.h, s_i.l));
  const float d = __fadd_rn(u2.h, __fadd_rn(tail, cross));
  const float fl = __fmaf_rn(0.375f * d, d, -0.5f * d);  // f = 1 + fl
  c = quick_two_sum(cf, __fmul_rn(cf, fl));
  sr = quick_two_sum(s_r.h, __fmaf_rn(s_r.h, fl, s_r.l));
  si = quick_two_sum(s_i.h, __fmaf_rn(s_i.h, fl, s_i.l));
  return true;
}

__device__ __forceinline__ int ff_pair_smem(float4* ai, float4* aj, int m, int len, int lane, double tol, double floor,
                                            double tiny) {
  GramAcc ga, gb, gc, gd;
  for (int r = lane; r < m; r += 32) ff_gram_row(ai[r], aj[r], ga, gb, gc, gd);
  ff alpha = ga.value(), beta = gb.value(), gr = gc.value(), gi = gd.value();
  ff_warp_sum4(alpha, beta, gr, gi);
  ff c, sr, si;
  if (!ff_angle(alpha, beta, gr, gi, float(tol), float(floor), c, sr, si)) return 0;
  for (int r = lane; r < len; r += 32) {
    float4 x = ai[r], y = aj[r];
    ff_rotate(x, y, c, sr, si);
    ai[r] = x;
    aj[r] = y;
  }
  return 1;
}

__device__ __forceinline__ int ff_pair_reg(float4 (&x)[kClusterRegs], float4* aj, int m, int len, int lane,
                                           double tol, double floor, double tiny) {
  GramAcc ga, gb, gc, gd;
#pragma unroll
  for (int i = 0; i < kClusterRegs; ++i) {
    const int r = lane + 32 * i;
    if (r < m) ff_gram_row(x[i], aj[r], ga, gb, gc, gd);
  }
  ff alpha = ga.value(), beta = gb.value(), gr = gc.value(), gi = gd.value();
  ff_warp_sum4(alpha, beta, gr, gi);
  ff c, sr, si;
  if (!ff_angle(alpha, beta, gr, gi, float(tol), float(floor), c, sr, si)) return 0;
#pragma unroll
  for (int i = 0; i < kClusterRegs; ++i) {
    const int r = lane + 32 * i;
    if (r < len) {
      float4 y = aj[r];
      ff_rotate(x[i], y, c, sr, si);
      aj[r] = y;
    }
  }
  return 1;
}

// |z|^2 of a stored column entry in double (complex S or double-float)
template <bool kDF, typename C>
__device__ __forceinline__ double entry_nrm2(const C* col, int r) {
  if constexpr (kDF) {
    const double2 z = cff_to_double2(reinterpret_cast<const float4*>(col)[r]);
    return z.x * z.x + z.y * z.y;
  } else {
    return double(col[r].x) * col[r].x + double(col[r].y) * col[r].y;
  }
}

// Symmetric first-order orthonormalisation of the V parts (rows m .. len) of
// two stacked columns: with e = v_i^H v_j, v_i -= conj(e)/2 v_j and
// v_j -= e/2 v_i (from the old values).
template <typename S>
__device__ __forceinline__ void orth_pair(cplx<S>* vi, cplx<S>* vj, int m, int len, int lane) {
  S gr = 0, gi = 0;
  for (int r = m + lane; r < len; r += 32) {
    const cplx<S> x = vi[r], y = vj[r];
    gr = fma(x.x, y.x, fma(x.y, y.y, gr));
    gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
  }
  gr = S(0.5) * warp_sum(gr);
  gi = S(0.5) * warp_sum(gi);
  for (int r = m + lane; r < len; r += 32) {
    const cplx<S> x = vi[r], y = vj[r];
    vi[r] = cmk<S>(x.x - fma(gr, y.x, gi * y.y), x.y - fma(gr, y.y, -gi * y.x));
    vj[r] = cmk<S>(y.x - fma(gr, x.x, -gi * x.y), y.y - fma(gr, x.y, gi * x.x));
  }
}

// Cluster-uniform sizes of one SVD.
struct ClusterGeom {
  int Pl, me;   // CTAs launched, this CTA's rank
  int P, b;     // CTAs taking part, columns per block
  int m, ncols, len, ncols_pad;
  int nw, nt, wl, wp;
  bool member;  // me < P
};

// Column id (0 .. ncols_pad-1) of column c of the block in slot `slot` of
// CTA `me` in round `rnd` of a sweep: the block at position pos >= 1 has
// moved rnd places along the circle 1 .. 2P-1 since the sweep began, when
// position p held block p; position 0 keeps block 0.
__device__ __forceinline__ int col_id(const ClusterGeom& g, int slot, int c, int rnd) {
  const int pos = slot == 0 ? g.me : 2 * g.P - 1 - g.me;
  const int M = 2 * g.P - 1;
  const int blk = pos == 0 ? 0 : 1 + ((pos - 1 - rnd) % M + M) % M;
  return blk * g.b + c;
}

// Stacked columns of one precision: shared-memory ping-pong slots
// [pp][slot][c][len], or 2P global blocks [block][c][len] that stay put while
// the round robin renames positions.
// The layout is a template parameter so that the shared-memory form's
// pointers stay shared-memory pointers for the compiler (shared loads and
// stores rather than generic ones).
template <typename T, bool kGlobal>
struct ColStore {
  cplx<T>* base;  // shared-memory slots, or the global blocks
  int b, len, P, me;
  __device__ cplx<T>* col(int pp, int slot, int c, int rnd) const {
    if constexpr (!kGlobal) {
      return base + ((size_t)(pp * 2 + slot) * b + c) * len;
    } else {
      const int pos = slot == 0 ? me : 2 * P - 1 - me;
      const int M = 2 * P - 1;
      const int blk = pos == 0 ? 0 : 1 + ((pos - 1 - rnd) % M + M) % M;
      return base + ((size_t)blk * b + c) * len;
    }
  }
};

// Sweeps of the circle-method round robin.  kOp 0: Jacobi rotations until a
// sweep rotates no pair (or max_sweeps); kOp 1: max_sweeps orthonormalisation
// sweeps.  Every CTA of the cluster calls it (non-members only keep the
// cluster barriers in step).  Returns the sweeps run.
//
// Tail rule (kOp 0): at the start of each sweep every CTA learns the squared
// norms of all columns (nrm2, through distributed shared memory) and marks
// the columns the truncation discards (truncation_tail, into tail[]); a pair
// of two marked columns is not rotated.
//
// Clean pairs (kOp 0): a pair whose two columns have not changed since the
// pair was last tested at the tight tolerance, and found orthogonal, is
// orthogonal still; it is not tested again.  Byte flags per column id, kept
// identical in every member CTA: dirty[] (rotated in this sweep; a rotation
// sets both columns' flags in every member CTA through distributed shared
// memory, visible by the next round's cluster barrier), dirty_prev[] (rotated
// in the previous sweep) and tight_prev[] (tail class 0 in the previous
// sweep).  A pair is clean when both columns are tight now and were in the
// previous sweep, and neither was rotated in the previous sweep or so far in
// this one.  The first sweep tests every pair.
//
// kDF: the columns hold double-float values (float4, see dfloat.cuh) and the
// rotations run in double-float; T is double then.
template <typename T, int kOp, bool kGlobal, bool kDF = false>
__device__ __forceinline__ int cluster_sweeps(const ClusterGeom& g, const ColStore<T, kGlobal>& cs, int& cur, int max_sweeps, T tol, T floor,
                              T tiny, double trunc_rel, int chi_max, double* nrm2, int* tail, unsigned char* flags,
                              bool& converged, const cg::cluster_group& cluster, int* s_flag_in, int* s_any) {
  using C = cplx<T>;
  using E = std::conditional_t<kDF, float4, C>;  // a stored entry
  static_assert(!kDF || (sizeof(float4) == sizeof(C) && kOp == 0), "double-float columns replace complex128 ones");
  // In the cross rounds, when every warp has one top-slot column, warp w
  // keeps it in registers for the b rotations it takes part in; only the
  // bottom-slot columns are re-read, so one barrier per sub-round orders
  // their hand-off.
  const bool cache_x = kOp == 0 && g.len <= 32 * kClusterRegs && g.b <= g.nw;
  __shared__ double s_loose;
  T loose = T(0);  // the tail rule's loose tolerance of the sweep (pair_tol)
  const bool active = g.member && g.wp < g.b;
  unsigned char* dirty = flags;
  unsigned char* dirty_prev = flags + g.ncols_pad;
  unsigned char* tight_prev = flags + 2 * g.ncols_pad;
  if (kOp == 0) {
    for (int id = threadIdx.x; id < g.ncols_pad; id += g.nt) {
      dirty[id] = 0;
      dirty_prev[id] = 1;
      tight_prev[id] = 0;
    }
    __syncthreads();
  }
  // a pair (column ids i, j) that needs no test (see above)
  auto clean = [&](int i, int j) -> bool {
    return tail[i] == 0 && tail[j] == 0 && tight_prev[i] && tight_prev[j] && !(dirty_prev[i] | dirty_prev[j] |
                                                                               dirty[i] | dirty[j]);
  };
  // both columns rotated: flag them in every member CTA (lane 0 of the warp)
  auto mark = [&](int i, int j) {
    if (g.wl != 0) return;
    for (int r2 = 0; r2 < g.P; ++r2) {
      unsigned char* d = r2 == g.me ? dirty : cluster.map_shared_rank(dirty, r2);
      d[i] = 1;
      d[j] = 1;
    }
  };
  int sweep = 0;
  converged = false;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    if (kOp == 0) {
      // squared norms of this CTA's columns (positions hold their own blocks
      // at the start of a sweep) to every member CTA
      for (int c = g.wp; g.member && c < 2 * g.b; c += g.nw) {
        const C* a = cs.col(cur, c / g.b, c % g.b, 0);
        double acc = 0.0;
        for (int r = g.wl; r < g.m; r += 32) acc += entry_nrm2<kDF>(a, r);
        acc = warp_sum(acc);
        if (g.wl == 0) {
          const int id = col_id(g, c / g.b, c % g.b, 0);
          for (int r2 = 0; r2 < g.P; ++r2) *cluster.map_shared_rank(nrm2 + id, r2) = acc;
        }
      }
      cluster.sync();
      if (g.member) {
        truncation_tail(nrm2, g.ncols_pad, trunc_rel, chi_max, tail, &s_loose);
        loose = T(s_loose);
      }
    }
    for (int rnd = 0; rnd < 2 * g.P - 1; ++rnd) {
      if (!g.member) {
        // not taking part: only the cluster barrier below
      } else if (rnd == 0) {
        // every pair among the CTA's 2b columns: round robin over 2b players
        const int mod = 2 * g.b - 1;
        for (int sr = 0; sr < 2 * g.b - 1; ++sr) {
          for (int pw = g.wp; pw < g.b; pw += g.nw) {
            int a0, a1;
            if (pw == 0) {
              a0 = mod;
              a1 = sr;
            } else {
              a0 = (sr + pw) % mod;
              a1 = (sr - pw + mod) % mod;
            }
            C* x = cs.col(cur, a0 / g.b, a0 % g.b, rnd);
            C* y = cs.col(cur, a1 / g.b, a1 % g.b, rnd);
            if (kOp == 0) {
              const int i0 = col_id(g, a0 / g.b, a0 % g.b, rnd), i1 = col_id(g, a1 / g.b, a1 % g.b, rnd);
              const T tl = pair_tol(tail[i0], tail[i1], tol, loose);
              if (tl >= T(0) && !clean(i0, i1)) {
                int r;
                if constexpr (kDF)
                  r = ff_pair_smem(reinterpret_cast<float4*>(x), reinterpret_cast<float4*>(y), g.m, g.len, g.wl, tl,
                                   floor, tiny);
                else
                  r = jacobi_pair_smem<T>(x, y, g.m, g.len, g.wl, tl, floor, tiny);
                if (r) mark(i0, i1);
                rotated |= r;
              }
            } else
              orth_pair<T>(x, y, g.m, g.len, g.wl);
          }
          __syncthreads();
        }
      } else {
        E xr[kClusterRegs];
        E* xcol = reinterpret_cast<E*>(cs.col(cur, 0, active ? g.wp : 0, rnd));
        if (active && cache_x) {
#pragma unroll
          for (int i = 0; i < kClusterRegs; ++i) {
            const int r = g.wl + 32 * i;
            if constexpr (kDF)
              xr[i] = r < g.len ? xcol[r] : make_float4(0.f, 0.f, 0.f, 0.f);
            else
              xr[i] = r < g.len ? xcol[r] : cmk<T>(0, 0);
          }
        }
        for (int sr = 0; sr < g.b; ++sr) {
          if (cache_x) {
            if (active) {
              const int i0 = col_id(g, 0, g.wp, rnd), i1 = col_id(g, 1, (g.wp + sr) % g.b, rnd);
              const T tl = pair_tol(tail[i0], tail[i1], tol, loose);
              if (tl >= T(0) && !clean(i0, i1)) {
                int r;
                if constexpr (kDF)
                  r = ff_pair_reg(xr, reinterpret_cast<float4*>(cs.col(cur, 1, (g.wp + sr) % g.b, rnd)), g.m, g.len,
                                  g.wl, tl, floor, tiny);
                else
                  r = jacobi_pair_reg<T>(xr, cs.col(cur, 1, (g.wp + sr) % g.b, rnd), g.m, g.len, g.wl, tl, floor,
                                         tiny);
                if (r) mark(i0, i1);
                rotated |= r;
              }
            }
          } else {
            for (int pw = g.wp; pw < g.b; pw += g.nw) {
              C* x = cs.col(cur, 0, pw, rnd);
              C* y = cs.col(cur, 1, (pw + sr) % g.b, rnd);
              if (kOp == 0) {
                const int i0 = col_id(g, 0, pw, rnd), i1 = col_id(g, 1, (pw + sr) % g.b, rnd);
                const T tl = pair_tol(tail[i0], tail[i1], tol, loose);
                if (tl >= T(0) && !clean(i0, i1)) {
                  int r;
                  if constexpr (kDF)
                    r = ff_pair_smem(reinterpret_cast<float4*>(x), reinterpret_cast<float4*>(y), g.m, g.len, g.wl,
                                     tl, floor, tiny);
                  else
                    r = jacobi_pair_smem<T>(x, y, g.m, g.len, g.wl, tl, floor, tiny);
                  if (r) mark(i0, i1);
                  rotated |= r;
                }
              } else
                orth_pair<T>(x, y, g.m, g.len, g.wl);
            }
          }
          __syncthreads();
        }
        if (active && cache_x) {
#pragma unroll
          for (int i = 0; i < kClusterRegs; ++i) {
            const int r = g.wl + 32 * i;
            if (r < g.len) xcol[r] = xr[i];
          }
        }
        __syncthreads();
      }
      if (g.P == 1) continue;  // a single CTA keeps its blocks (and needs no cluster barrier)
      if constexpr (!kGlobal) {
        // hand the blocks on: position pos -> pos + 1 (pos >= 1), 2P-1 -> 1
        const int nxt = cur ^ 1;
        const size_t units = (size_t)g.b * g.len * sizeof(C) / sizeof(uint4);
        for (int slot = 0; slot < 2 && g.member; ++slot) {
          const int pos = slot == 0 ? g.me : 2 * g.P - 1 - g.me;
          const int npos = pos == 0 ? 0 : (pos == 2 * g.P - 1 ? 1 : pos + 1);
          int drank, dslot;
          pos_owner(npos, g.P, drank, dslot);
          const uint4* src = reinterpret_cast<const uint4*>(cs.col(cur, slot, 0, 0));
          uint4* dst = reinterpret_cast<uint4*>(cluster.map_shared_rank(cs.col(nxt, dslot, 0, 0), drank));
          for (size_t t = threadIdx.x; t < units; t += g.nt) dst[t] = src[t];
        }
        cluster.sync();
        cur = nxt;
      } else {
        cluster.sync();  // global columns: this round's writes before the next round's reads
      }
    }
    if (kOp == 1) continue;
    // ---- convergence: every CTA tells every CTA whether it rotated
    if (threadIdx.x == 0) *s_any = 0;
    __syncthreads();
    if (rotated) *s_any = 1;
    __syncthreads();
    if (threadIdx.x < g.Pl) {
      int* dst = cluster.map_shared_rank(s_flag_in, (int)threadIdx.x);
      dst[g.me] = *s_any;
    }
    cluster.sync();
    int any = 0;
    for (int r2 = 0; r2 < g.Pl; ++r2) any |= s_flag_in[r2];
    cluster.sync();  // all reads done before the next sweep's writes
    // roll the clean-pair flags (no CTA writes dirty[] again before the next
    // sweep's norm exchange barrier)
    for (int id = threadIdx.x; g.member && id < g.ncols_pad; id += g.nt) {
      dirty_prev[id] = dirty[id];
      dirty[id] = 0;
      tight_prev[id] = tail[id] == 0;
    }
    __syncthreads();
    if (!any) {
      converged = true;
      ++sweep;
      break;
    }
  }
  return sweep;
}

// Threads per CTA of the cluster SVD: FP64 columns need more registers per
// thread (the cached column alone is 64), so FP64 CTAs stop at 8 warps and a
// warp takes several pairs in turn when a block has more than 8 columns.
template <typename S> constexpr int kClusterMaxThreads = sizeof(S) == 8 ? 256 : 512;

template <typename S>
struct ClusterSvdSmem {
  // layout of the dynamic shared memory (offsets in bytes); len = m + n
  size_t buf, red, sig, rank, flags;
  size_t total;
  __host__ __device__ static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ ClusterSvdSmem(int b, int len, int ncols_pad, int nthreads) {
    buf = 0;
    size_t slots = 2ull * 2 * b * len * sizeof(cplx<S>);  // ping-pong x {top, bottom}
    red = align16(buf + slots);
    sig = align16(red + 4ull * (nthreads / 32 + 1) * sizeof(S) * 2);
    rank = align16(sig + (size_t)ncols_pad * sizeof(double));
    flags = align16(rank + (size_t)ncols_pad * sizeof(int));  // three byte flags per column
    total = align16(flags + 3 * (size_t)ncols_pad) + 64;
  }
};

// Elements of cplx<S> the global workspace needs for a theta of capacity
// mcap x ncap: the stacked columns (at most 2 P - 1 padding columns, P <= 16)
// in S, plus an FP32 copy for the mixed form.
__host__ __device__ inline size_t cluster_svd_workspace(size_t mcap, size_t ncap, size_t s_bytes) {
  const size_t e = (ncap + 32) * (mcap + ncap);
  return s_bytes == 8 ? e + (e + 1) / 2 : e;
}

// Everything after the geometry: the column layout (shared or global) is a
// compile-time choice so that shared-memory accesses compile as such.
// kDF: the FP64-accurate sweeps of the mixed form run in double-float (the
// rebuilt FP64 columns are converted in place; see dfloat.cuh).
template <typename S, typename R, bool kGlobal, bool kDF>
__device__ __forceinline__ void svd_cluster_body(const ClusterGeom& g, const cg::cluster_group& cluster,
                                                 const cplx<R>* __restrict__ Cm, const double* __restrict__ lam_l,
                                                 int* __restrict__ chi, int q, const SvdParams& p,
                                                 cplx<R>* __restrict__ Bnext, double* __restrict__ lam_next,
                                                 DevReport* __restrict__ rep, cplx<S>* __restrict__ gbuf,
                                                 unsigned char* smem, int* s_flag_in, double* s_fro, int& s_k,
                                                 double& s_nrm, int* s_any, long long t_start) {
  using C = cplx<S>;
  long long t_load = 0, t_lo = 0, t_fix = 0;
  const bool mixed = sizeof(S) == 8 && p.mixed;
  const int m = g.m, ncols = g.ncols, len = g.len, b = g.b, P = g.P, me = g.me, nt = g.nt;
  const ClusterSvdSmem<S> L(b, kGlobal ? 0 : len, g.ncols_pad, nt);
  double* sig = reinterpret_cast<double*>(smem + L.sig);
  int* rnk = reinterpret_cast<int*>(smem + L.rank);
  const ColStore<S, kGlobal> cs{kGlobal ? gbuf : reinterpret_cast<C*>(smem + L.buf), b, len, P, me};
  // FP32 columns of the mixed form: in shared memory both FP32 ping-pong
  // buffers fit in the first S ping-pong buffer; in global memory they follow
  // the S blocks.
  const ColStore<float, kGlobal> cs32{kGlobal ? reinterpret_cast<cplx<float>*>(gbuf + (size_t)g.ncols_pad * len)
                                               : reinterpret_cast<cplx<float>*>(smem + L.buf),
                                      b, len, P, me};

  // ---- load: position pos holds the initial block pos (columns pos*b ..)
  for (int slot = 0; slot < 2 && g.member; ++slot) {
    const int pos = slot == 0 ? me : 2 * P - 1 - me;
    for (size_t t = threadIdx.x; t < (size_t)b * len; t += nt) {
      const int c = (int)(t / len), r = (int)(t % len);
      const int col = pos * b + c;
      double vr = 0.0, vi = 0.0;
      if (col < ncols) {
        if (r < m) {
          const cplx<R> x = Cm[(size_t)r * ncols + col];
          const double w = lam_l[r >> 1];
          vr = w * double(x.x);
          vi = w * double(x.y);
        } else if (r - m == col) {
          vr = 1.0;
        }
      }
      if (mixed)
        cs32.col(0, slot, c, 0)[r] = cmk<float>(float(vr), float(vi));
      else
        cs.col(0, slot, c, 0)[r] = cmk<S>(S(vr), S(vi));
    }
  }
  // ||A||_F^2 from the theta: each CTA's share goes to every CTA, summed in rank order
  double part = 0.0;
  for (size_t t = threadIdx.x; g.member && t < (size_t)2 * b * m; t += nt) {
    const int c = (int)(t / m), r = (int)(t % m);
    const int pos = c < b ? me : 2 * P - 1 - me;
    const int col = pos * b + c % b;
    if (col >= ncols) continue;
    const cplx<R> x = Cm[(size_t)r * ncols + col];
    const double w = lam_l[r >> 1];
    part += w * w * (double(x.x) * x.x + double(x.y) * x.y);
  }
  part = warp_sum(part);
  if (threadIdx.x == 0) s_nrm = 0.0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_nrm, part);
  __syncthreads();
  if (threadIdx.x < g.Pl) *cluster.map_shared_rank(&s_fro[me], (int)threadIdx.x) = s_nrm;
  cluster.sync();
  double fro2 = 0.0;
  for (int r2 = 0; r2 < g.Pl; ++r2) fro2 += s_fro[r2];

  // Stopping rule and rounding floor: rotate while |b_ij| > tol sqrt(b_ii b_jj)
  // with tol = 4 sqrt(max(m, n)) u (a few times the rounding error of a dot
  // product); columns with squared norm below (4 u ||A||_F)^2 are rounding
  // noise and left alone.
  const double tol_scale = 4.0 * sqrt(double(max(m, ncols)));
  // the tail rule's per-sweep scratch: squared norms and tail flags of all
  // columns (the singular values and ranks use the same arrays afterwards)
  double* nrm2 = sig;
  int* tail = rnk;
  unsigned char* flags = smem + L.flags;
  int cur = 0, used = 0, used32 = 0;
  bool converged = false;
  t_load = clock64();
  t_lo = t_fix = t_load;
  if (mixed) {
    const float u32 = 5.9604645e-08f;
    int cur32 = 0;
    bool conv32 = false;
    used32 = cluster_sweeps<float, 0, kGlobal>(g, cs32, cur32, p.max_sweeps, float(tol_scale) * u32,
                                               float(16.0 * double(u32) * double(u32) * fro2), 1e-35f, p.trunc_rel,
                                               p.chi_max, nrm2, tail, flags, conv32, cluster, s_flag_in, s_any);
    used = used32;
    t_lo = clock64();
    // FP64 columns: V promoted (A follows from the theta below)
    cur = kGlobal ? 0 : 1;
    for (int slot = 0; slot < 2 && g.member; ++slot)
      for (size_t t = threadIdx.x; t < (size_t)b * ncols; t += nt) {
        const int c = (int)(t / ncols), r = m + (int)(t % ncols);
        const cplx<float> v = cs32.col(cur32, slot, c, 0)[r];
        cs.col(cur, slot, c, 0)[r] = cmk<S>(S(v.x), S(v.y));
      }
    // every CTA has read its FP32 columns before the first hand-over may
    // overwrite them (in shared memory they share a buffer with FP64 ones)
    cluster.sync();
    // two first-order passes: E ~ 1e-6 -> E^2 -> E^4 (one pass left V
    // unitary only to ~1e-10 after long FP32 phases)
    for (int pass = 0; pass < 2; ++pass) {
      bool dummy;
      cluster_sweeps<S, 1, kGlobal>(g, cs, cur, 1, S(0), S(0), S(0), 0.0, 0, nrm2, tail, flags, dummy, cluster,
                                    s_flag_in, s_any);
      // the diagonal of the first-order step: |v|^2 -> 1
      for (int c = g.wp; g.member && c < 2 * b; c += g.nw) {
        C* v = cs.col(cur, c / b, c % b, 0);
        S n2 = 0;
        for (int r = m + g.wl; r < len; r += 32) n2 = fma(v[r].x, v[r].x, fma(v[r].y, v[r].y, n2));
        n2 = warp_sum(n2);
        const S f = S(1.5) - S(0.5) * n2;
        if (n2 > S(0))
          for (int r = m + g.wl; r < len; r += 32) v[r] = cmk<S>(f * v[r].x, f * v[r].y);
      }
      __syncthreads();
    }
    // A = C~ V in FP64 for this CTA's columns
    for (size_t t = threadIdx.x; g.member && t < (size_t)2 * b * m; t += nt) {
      const int c = (int)(t / m), r = (int)(t % m);
      C* x = cs.col(cur, c / b, c % b, 0);
      const cplx<R>* crow = Cm + (size_t)r * ncols;
      S ar = 0, ai = 0;
      for (int k = 0; k < ncols; ++k) {
        const cplx<R> cv = crow[k];
        const C v = x[m + k];
        ar = fma(S(cv.x), v.x, fma(-S(cv.y), v.y, ar));
        ai = fma(S(cv.x), v.y, fma(S(cv.y), v.x, ai));
      }
      const S w = S(lam_l[r >> 1]);
      x[r] = cmk<S>(w * ar, w * ai);
    }
    __syncthreads();
    if constexpr (kDF) {
      // the stacked FP64 columns of this CTA to double-float, in place
      for (size_t t = threadIdx.x; g.member && t < (size_t)2 * b * len; t += nt) {
        C* col = cs.col(cur, (int)(t / ((size_t)b * len)), (int)((t / len) % b), 0);
        const int r = (int)(t % len);
        const double2 z = make_double2(double(col[r].x), double(col[r].y));
        reinterpret_cast<float4*>(col)[r] = cff_from_double2(z);
      }
      __syncthreads();
    }
    t_fix = clock64();
  }
  // unit roundoff of the last sweeps: FP64, double-float (about 48 bits with
  // the sloppy additions of dfloat.cuh: 2^-46 to be safe) or FP32
  const S eps_u = kDF ? S(1.4210854715202004e-14) : (sizeof(S) == 8 ? S(1.1102230246251565e-16) : S(5.9604645e-08f));
  const S tol = p.tol > 0 ? S(p.tol) : S(tol_scale) * eps_u;
  const S floor = S(16.0 * double(eps_u) * double(eps_u) * fro2);
  const S tiny = sizeof(S) == 8 ? S(1e-290) : S(1e-35f);
  used += cluster_sweeps<S, 0, kGlobal, kDF>(g, cs, cur, p.max_sweeps, tol, floor, tiny, p.trunc_rel, p.chi_max, nrm2, tail,
                                        flags, converged, cluster, s_flag_in, s_any);
  const int sweep = used;

  // ---- singular values: norms of the A parts, shared with every CTA
  const int lane = g.wl, warp = g.wp;
  const int ncols_pad = g.ncols_pad;
  for (int c = warp; g.member && c < 2 * b; c += g.nw) {
    const C* a = cs.col(cur, c / b, c % b, 0);
    double acc = 0.0;
    for (int r = lane; r < m; r += 32) acc += entry_nrm2<kDF>(a, r);
    acc = warp_sum(acc);
    if (lane == 0) {
      const double sv = sqrt(acc);
      const int gc = me * 2 * b + c;
      for (int r2 = 0; r2 < P; ++r2) *cluster.map_shared_rank(sig + gc, r2) = sv;
    }
  }
  cluster.sync();
  if (!g.member) {
    cluster.sync();  // pairs with the final barrier of the members
    return;
  }
  // ranks (descending, ties by index), the same in every CTA
  for (int gc = threadIdx.x; gc < ncols_pad; gc += nt) {
    const double sg = sig[gc];
    int rk = 0;
    for (int h = 0; h < ncols_pad; ++h) {
      const double sh = sig[h];
      rk += (sh > sg) || (sh == sg && h < gc);
    }
    rnk[gc] = rk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0, smax = 0.0;
    for (int gc = 0; gc < ncols_pad; ++gc) {
      total += sig[gc] * sig[gc];
      smax = fmax(smax, sig[gc]);
    }
    int cnt = 0;
    for (int gc = 0; gc < ncols_pad; ++gc)
      if (p.trunc_rel > 0.0 ? (sig[gc] > p.trunc_rel * smax) : (sig[gc] > 0.0)) ++cnt;
    int k = min(cnt, min(p.chi_max, min(m, ncols)));
    if (k < 1) k = 1;
    double kept = 0.0, smin = 0.0, s_next = 0.0;
    for (int gc = 0; gc < ncols_pad; ++gc) {
      if (rnk[gc] < k) kept += sig[gc] * sig[gc];
      if (rnk[gc] == k - 1) smin = sig[gc];
      if (rnk[gc] == k) s_next = sig[gc];
    }
    double nrm = sqrt(kept);
    if (!(nrm > 0.0)) nrm = 1.0;
    s_k = k;
    s_nrm = nrm;
    if (me == 0) {
      rep->discarded_weight += total > 0.0 ? 1.0 - kept / total : 0.0;
      if (smin / nrm < rep->min_kept_sv) rep->min_kept_sv = smin / nrm;
      if (k > rep->max_chi) rep->max_chi = k;
      if (k < ncols && k == p.chi_max && s_next > 0.0 && fabs(smin - s_next) <= 1e-10 * smin)
        rep->degenerate_cuts += 1;
      if (!converged) rep->not_converged += 1;
      const int used_cap = converged ? sweep : p.max_sweeps + 1;
      if (used_cap > rep->max_sweeps) rep->max_sweeps = used_cap;
      rep->two_qubit_gates += 1;
      // per sweep and column pair: three dot products over m rows (16 m flops)
      // and one rotation of the stacked columns (12 (m + n) flops)
      rep->svd_flops += (double)sweep * 0.5 * ncols * (ncols - 1) * (16.0 * m + 12.0 * len);
      rep->inv_norm = 1.0 / nrm;
      rep->sweeps_fp32 += used32;
      (sizeof(S) == 8 ? rep->sweeps_fp64 : rep->sweeps_fp32) += sweep - used32;
      const long long t_end = clock64();
      rep->phase_cycles[0] += double(t_load - t_start);
      rep->phase_cycles[1] += double(t_lo - t_load);
      rep->phase_cycles[2] += double(t_fix - t_lo);
      rep->phase_cycles[3] += double(t_end - t_fix);
      chi[q + 1] = k;
    }
  }
  __syncthreads();
  const int k = s_k;
  const double inv = 1.0 / s_nrm;
  if (me == 0)
    for (int gc = threadIdx.x; gc < ncols_pad; gc += nt)
      if (rnk[gc] < k) lam_next[rnk[gc]] = sig[gc] * inv;
  // B~_{q+1}[a, :] = conj(V[:, gc]) for the column gc of rank a < k
  for (int c = warp; c < 2 * b; c += g.nw) {
    const int gc = me * 2 * b + c;
    const int a = rnk[gc];
    if (a >= k) continue;
    const C* v = cs.col(cur, c / b, c % b, 0) + m;
    for (int r = lane; r < ncols; r += 32) {
      if constexpr (kDF)
        Bnext[(size_t)a * ncols + r] =
            ccast<cplx<R>>(cconj(cff_to_double2(reinterpret_cast<const float4*>(v)[r])));
      else
        Bnext[(size_t)a * ncols + r] = ccast<cplx<R>>(cconj(v[r]));
    }
  }
  cluster.sync();  // no CTA leaves while its shared memory may still be read
}


template <typename S, typename R>
__global__ void __launch_bounds__(kClusterMaxThreads<S>, 1)
    svd_cluster_kernel(const cplx<R>* __restrict__ Cm, const double* __restrict__ lam_l, int* __restrict__ chi, int q,
                       SvdParams p, cplx<R>* __restrict__ Bnext, double* __restrict__ lam_next,
                       DevReport* __restrict__ rep, cplx<S>* __restrict__ gbuf, unsigned smem_bytes) {
  using C = cplx<S>;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag_in[16];
  __shared__ double s_fro[16];
  __shared__ int s_k;
  __shared__ double s_nrm;
  __shared__ int s_any;

  const long long t_start = clock64();
  ClusterGeom g;
  g.Pl = (int)cluster.num_blocks();  // CTAs launched (sized for the bond capacities)
  g.me = (int)cluster.block_rank();
  const int chi_l = chi[q], chi_r = chi[q + 2];
  g.m = 2 * chi_l;      // rows of A
  g.ncols = 2 * chi_r;  // columns of A = rows of V
  g.len = g.m + g.ncols;
  g.nw = (int)(blockDim.x >> 5);
  g.nt = blockDim.x;
  g.wl = threadIdx.x & 31;
  g.wp = threadIdx.x >> 5;
  // CTAs that take part, from the actual bond dimensions: complex64 pair
  // steps are latency-bound, so as few CTAs as the warps allow (fewer rounds
  // and cluster barriers); FP64 ones are bound by the FP64 units, so one pair
  // per warp on as many CTAs as there are.  The others (rank >= P) only keep
  // the cluster barriers in step.
  const int per = sizeof(S) == 8 ? 1 : g.nw;
  g.P = min(g.Pl, max(1, (g.ncols + 2 * per - 1) / (2 * per)));
  // Without a global workspace the columns must fit the launch's shared
  // memory: fewer CTAs mean wider blocks (an FP32 theta of 96 columns takes 3
  // CTAs of 16 columns where the capacity plan sized 4 of 12), so spread them
  // over more of the launched CTAs until they fit.  The plan guarantees that
  // all Pl CTAs fit the capacity, hence the actual sizes.
  while (gbuf == nullptr && g.P < g.Pl) {
    const int bb = (g.ncols + 2 * g.P - 1) / (2 * g.P);
    if (ClusterSvdSmem<S>(bb, g.len, 2 * g.P * bb, g.nt).total <= smem_bytes) break;
    ++g.P;
  }
  g.member = g.me < g.P;
  g.b = (g.ncols + 2 * g.P - 1) / (2 * g.P);  // a warp takes pairs w, w + nw, ...
  g.ncols_pad = 2 * g.P * g.b;

  // Shared memory when the stacked columns fit the launch's allocation, else the global workspace.
  const bool fits = ClusterSvdSmem<S>(g.b, g.len, g.ncols_pad, g.nt).total <= smem_bytes;
  if (!fits && gbuf == nullptr) {
    // unreachable for launches sized by the host plan; leave without touching
    // the state (every CTA returns before any cluster barrier) and report it
    // as a sweep-cap hit so that the caller sees MPS_ENOTCONV
    if (g.me == 0 && threadIdx.x == 0) atomicAdd(&rep->not_converged, 1);
    return;
  }
  const bool in_smem = fits;
  // the mixed form's FP64-accurate sweeps run in double-float
  if constexpr (sizeof(S) == 8) {
    if (p.mixed) {
      if (in_smem)
        svd_cluster_body<S, R, false, true>(g, cluster, Cm, lam_l, chi, q, p, Bnext, lam_next, rep, gbuf, smem,
                                            s_flag_in, s_fro, s_k, s_nrm, &s_any, t_start);
      else
        svd_cluster_body<S, R, true, true>(g, cluster, Cm, lam_l, chi, q, p, Bnext, lam_next, rep, gbuf, smem,
                                           s_flag_in, s_fro, s_k, s_nrm, &s_any, t_start);
      return;
    }
  }
  if (in_smem)
    svd_cluster_body<S, R, false, false>(g, cluster, Cm, lam_l, chi, q, p, Bnext, lam_next, rep, gbuf, smem, s_flag_in,
                                         s_fro, s_k, s_nrm, &s_any, t_start);
  else
    svd_cluster_body<S, R, true, false>(g, cluster, Cm, lam_l, chi, q, p, Bnext, lam_next, rep, gbuf, smem, s_flag_in,
                                        s_fro, s_k, s_nrm, &s_any, t_start);
}

}  // namespace mpsv
