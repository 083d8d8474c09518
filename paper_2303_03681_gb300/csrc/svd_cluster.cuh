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
// buffers, so one cluster barrier per round orders the hand-over.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

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

// Rotation of a column pair from its Gram entries (Algorithm 1 with the phase
// of b_ij moved onto column j); returns false when the pair is left alone.
template <typename S>
__device__ __forceinline__ bool jacobi_rotation(S alpha, S beta, S gr, S gi, S tol, S floor, S tiny, S& c, cplx<S>& sph) {
  const S mag = sqrt(gr * gr + gi * gi);
  if (!(mag > tiny) || !(mag > tol * sqrt(alpha * beta)) || !(min(alpha, beta) > floor)) return false;
  const S zeta = (beta - alpha) / (S(2) * mag);
  const S t = (zeta >= S(0) ? S(1) : S(-1)) / (fabs(zeta) + sqrt(S(1) + zeta * zeta));
  c = S(1) / sqrt(S(1) + t * t);
  const S s = t * c;
  sph = cmk<S>(s * gr / mag, s * gi / mag);  // s e^{i phi}
  return true;
}

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

template <typename S>
struct ClusterSvdSmem {
  // layout of the dynamic shared memory (offsets in bytes); len = m + n
  size_t buf, red, sig, rank;
  size_t total;
  __host__ __device__ static size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
  __host__ __device__ ClusterSvdSmem(int b, int len, int ncols_pad, int nthreads) {
    buf = 0;
    size_t slots = 2ull * 2 * b * len * sizeof(cplx<S>);  // ping-pong x {top, bottom}
    red = align16(buf + slots);
    sig = align16(red + 4ull * (nthreads / 32 + 1) * sizeof(S) * 2);
    rank = align16(sig + (size_t)ncols_pad * sizeof(double));
    total = align16(rank + (size_t)ncols_pad * sizeof(int)) + 64;
  }
};

template <typename S, typename R>
__global__ void __launch_bounds__(512, 1)
    svd_cluster_kernel(const cplx<R>* __restrict__ Cm, const double* __restrict__ lam_l, int* __restrict__ chi, int q,
                       SvdParams p, cplx<R>* __restrict__ Bnext, double* __restrict__ lam_next,
                       DevReport* __restrict__ rep) {
  using C = cplx<S>;
  cg::cluster_group cluster = cg::this_cluster();
  const int P = (int)cluster.num_blocks();
  const int me = (int)cluster.block_rank();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_flag_in[16];
  __shared__ double s_fro[16];
  __shared__ int s_k;
  __shared__ double s_nrm;

  const int chi_l = chi[q], chi_r = chi[q + 2];
  const int m = 2 * chi_l;      // rows of A
  const int ncols = 2 * chi_r;  // columns of A = rows of V
  const int len = m + ncols;    // stacked column [A; V]
  const int b = (ncols + 2 * P - 1) / (2 * P);
  const int ncols_pad = 2 * P * b;
  const int nt = blockDim.x;
  const ClusterSvdSmem<S> L(b, len, ncols_pad, nt);
  C* bufs = reinterpret_cast<C*>(smem + L.buf);
  double* sig = reinterpret_cast<double*>(smem + L.sig);
  int* rnk = reinterpret_cast<int*>(smem + L.rank);
  const size_t slot_elems = (size_t)b * len;
  auto col_ptr = [&](int pp, int slot, int c) -> C* { return bufs + ((size_t)(pp * 2 + slot) * b + c) * len; };

  // ---- load: position pos holds the initial block pos (columns pos*b ..)
  for (int slot = 0; slot < 2; ++slot) {
    const int pos = slot == 0 ? me : 2 * P - 1 - me;
    for (size_t t = threadIdx.x; t < slot_elems; t += nt) {
      const int c = (int)(t / len), r = (int)(t % len);
      const int col = pos * b + c;
      C v = cmk<S>(0, 0);
      if (col < ncols) {
        if (r < m) {
          const cplx<R> x = Cm[(size_t)r * ncols + col];
          const S w = S(lam_l[r >> 1]);
          v = cmk<S>(w * S(x.x), w * S(x.y));
        } else if (r - m == col) {
          v = cmk<S>(1, 0);
        }
      }
      col_ptr(0, slot, c)[r] = v;
    }
  }
  __syncthreads();
  // ||A||_F^2: each CTA's share goes to every CTA, summed in rank order
  double part = 0.0;
  for (size_t t = threadIdx.x; t < 2 * slot_elems; t += nt) {
    if ((int)(t % len) >= m) continue;
    const C v = bufs[t];
    part += double(v.x) * v.x + double(v.y) * v.y;
  }
  part = warp_sum(part);
  if (threadIdx.x == 0) s_nrm = 0.0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicAdd(&s_nrm, part);
  __syncthreads();
  if (threadIdx.x < P) *cluster.map_shared_rank(&s_fro[me], (int)threadIdx.x) = s_nrm;
  cluster.sync();
  double fro2 = 0.0;
  for (int r2 = 0; r2 < P; ++r2) fro2 += s_fro[r2];

  // Stopping rule and rounding floor: rotate while |b_ij| > tol sqrt(b_ii b_jj)
  // with tol = 4 sqrt(max(m, n)) u (a few times the rounding error of a dot
  // product); columns with squared norm below (4 u ||A||_F)^2 are rounding
  // noise and left alone.
  const S eps_u = sizeof(S) == 8 ? S(1.1102230246251565e-16) : S(5.9604645e-08f);
  const S tol = p.tol > 0 ? S(p.tol) : S(4.0 * sqrt(double(max(m, ncols)))) * eps_u;
  const S floor = S(16.0 * double(eps_u) * double(eps_u) * fro2);
  const S tiny = sizeof(S) == 8 ? S(1e-290) : S(1e-35f);
  // One warp per column pair (warps past b idle in the pair loops).  In the
  // cross rounds warp w keeps its top-slot column in registers for the b
  // rotations it takes part in; only the bottom-slot columns go through
  // shared memory, so one barrier per sub-round orders their hand-off.
  const int wl = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const bool active = wp < b;
  const bool cache_x = len <= 32 * kClusterRegs;

  int sweep = 0, cur = 0;
  bool converged = false;
  for (; sweep < p.max_sweeps; ++sweep) {
    int rotated = 0;
    for (int round = 0; round < 2 * P - 1; ++round) {
      if (round == 0) {
        // every pair among the CTA's 2b columns: round robin over 2b players
        const int mod = 2 * b - 1;
        for (int sr = 0; sr < 2 * b - 1; ++sr) {
          if (active) {
            int a0, a1;
            if (wp == 0) {
              a0 = mod;
              a1 = sr;
            } else {
              a0 = (sr + wp) % mod;
              a1 = (sr - wp + mod) % mod;
            }
            rotated |= jacobi_pair_smem<S>(col_ptr(cur, a0 / b, a0 % b), col_ptr(cur, a1 / b, a1 % b), m, len, wl,
                                           tol, floor, tiny);
          }
          __syncthreads();
        }
      } else {
        C xr[kClusterRegs];
        C* xcol = col_ptr(cur, 0, active ? wp : 0);
        if (active && cache_x) {
#pragma unroll
          for (int i = 0; i < kClusterRegs; ++i) {
            const int r = wl + 32 * i;
            xr[i] = r < len ? xcol[r] : cmk<S>(0, 0);
          }
        }
        for (int sr = 0; sr < b; ++sr) {
          if (active) {
            C* aj = col_ptr(cur, 1, (wp + sr) % b);
            rotated |= cache_x ? jacobi_pair_reg<S>(xr, aj, m, len, wl, tol, floor, tiny)
                               : jacobi_pair_smem<S>(xcol, aj, m, len, wl, tol, floor, tiny);
          }
          __syncthreads();
        }
        if (active && cache_x) {
#pragma unroll
          for (int i = 0; i < kClusterRegs; ++i) {
            const int r = wl + 32 * i;
            if (r < len) xcol[r] = xr[i];
          }
        }
        __syncthreads();
      }
      // ---- hand the blocks on: position pos -> pos + 1 (pos >= 1), 2P-1 -> 1
      const int nxt = cur ^ 1;
      const size_t units = slot_elems * sizeof(C) / sizeof(uint4);
      for (int slot = 0; slot < 2; ++slot) {
        const int pos = slot == 0 ? me : 2 * P - 1 - me;
        int npos = pos == 0 ? 0 : (pos == 2 * P - 1 ? 1 : pos + 1);
        int drank, dslot;
        pos_owner(npos, P, drank, dslot);
        const uint4* src = reinterpret_cast<const uint4*>(col_ptr(cur, slot, 0));
        uint4* dst = reinterpret_cast<uint4*>(cluster.map_shared_rank(col_ptr(nxt, dslot, 0), drank));
        for (size_t t = threadIdx.x; t < units; t += nt) dst[t] = src[t];
      }
      cluster.sync();
      cur = nxt;
    }
    // ---- convergence: every CTA tells every CTA whether it rotated
    __shared__ int s_any;
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (rotated) s_any = 1;
    __syncthreads();
    if (threadIdx.x < P) {
      int* dst = cluster.map_shared_rank(s_flag_in, (int)threadIdx.x);
      dst[me] = s_any;
    }
    cluster.sync();
    int any = 0;
    for (int r2 = 0; r2 < P; ++r2) any |= s_flag_in[r2];
    cluster.sync();  // all reads done before the next sweep's writes
    if (!any) {
      converged = true;
      ++sweep;
      break;
    }
  }

  // ---- singular values: norms of the A parts, shared with every CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nt >> 5;
  for (int c = warp; c < 2 * b; c += nw) {
    const C* a = col_ptr(cur, c / b, c % b);
    double acc = 0.0;
    for (int r = lane; r < m; r += 32) acc += double(a[r].x) * a[r].x + double(a[r].y) * a[r].y;
    acc = warp_sum(acc);
    if (lane == 0) {
      const double sv = sqrt(acc);
      const int g = me * 2 * b + c;
      for (int r2 = 0; r2 < P; ++r2) *cluster.map_shared_rank(sig + g, r2) = sv;
    }
  }
  cluster.sync();
  // ranks (descending, ties by index), the same in every CTA
  for (int g = threadIdx.x; g < ncols_pad; g += nt) {
    const double sg = sig[g];
    int rk = 0;
    for (int h = 0; h < ncols_pad; ++h) {
      const double sh = sig[h];
      rk += (sh > sg) || (sh == sg && h < g);
    }
    rnk[g] = rk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0, smax = 0.0;
    for (int g = 0; g < ncols_pad; ++g) {
      total += sig[g] * sig[g];
      smax = fmax(smax, sig[g]);
    }
    int cnt = 0;
    for (int g = 0; g < ncols_pad; ++g)
      if (p.trunc_rel > 0.0 ? (sig[g] > p.trunc_rel * smax) : (sig[g] > 0.0)) ++cnt;
    int k = min(cnt, min(p.chi_max, min(m, ncols)));
    if (k < 1) k = 1;
    double kept = 0.0, smin = 0.0, s_next = 0.0;
    for (int g = 0; g < ncols_pad; ++g) {
      if (rnk[g] < k) kept += sig[g] * sig[g];
      if (rnk[g] == k - 1) smin = sig[g];
      if (rnk[g] == k) s_next = sig[g];
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
      const int used = converged ? sweep : p.max_sweeps + 1;
      if (used > rep->max_sweeps) rep->max_sweeps = used;
      rep->two_qubit_gates += 1;
      // per sweep and column pair: three dot products over m rows (16 m flops)
      // and one rotation of the stacked columns (12 (m + n) flops)
      rep->svd_flops += (double)min(used, p.max_sweeps) * 0.5 * ncols * (ncols - 1) * (16.0 * m + 12.0 * len);
      rep->inv_norm = 1.0 / nrm;
      chi[q + 1] = k;
    }
  }
  __syncthreads();
  const int k = s_k;
  const double inv = 1.0 / s_nrm;
  if (me == 0)
    for (int g = threadIdx.x; g < ncols_pad; g += nt)
      if (rnk[g] < k) lam_next[rnk[g]] = sig[g] * inv;
  // B~_{q+1}[a, :] = conj(V[:, g]) for the column g of rank a < k
  for (int c = warp; c < 2 * b; c += nw) {
    const int g = me * 2 * b + c;
    const int a = rnk[g];
    if (a >= k) continue;
    const C* v = col_ptr(cur, c / b, c % b) + m;
    for (int r = lane; r < ncols; r += 32) Bnext[(size_t)a * ncols + r] = ccast<cplx<R>>(cconj(v[r]));
  }
  cluster.sync();  // no CTA leaves while its shared memory may still be read
}

}  // namespace mpsv
