// Double-float arithmetic for the FP64-accurate Jacobi sweeps.
//
// This part executes FP64 at two fused multiply-adds per clock per SM and
// FP32 at 128: a value held as the unevaluated sum of two floats (h + l,
// |l| <= ulp(h) / 2, about 48 significant bits) and handled with the
// error-free transformations of Knuth (two-sum: the rounding error of a + b
// recovered exactly from three more additions) and of the fused multiply-add
// (two-product: a b - rn(a b) = fma(a, b, -rn(a b)) exactly) runs the sweeps
// on the FP32 pipes several times faster than FP64, at a unit roundoff of
// about 2^-46.  The exponent range is FP32's: the kernels that use it keep
// squared norms above the rounding floor, far from 1e-38.
//
// Complex double-float values are float4 (re_h, re_l, im_h, im_l): 16 bytes,
// the size of a complex128, so the stacked-column layouts are unchanged.
#pragma once

#include <cuda_runtime.h>

namespace mpsv {

struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_make(float h, float l) {
  ff r;
  r.h = h;
  r.l = l;
  return r;
}

// exact: s + e = a + b (Knuth's two-sum)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff_make(s, e);
}

// exact when |a| >= |b| or a = 0
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.h, b.h);
  s.l = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
  return quick_two_sum(s.h, s.l);
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff_make(-a.h, -a.l); }

__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

// a b with the exact product of the heads (two-product by fma)
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return quick_two_sum(p, e);
}

// acc + a b
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff acc) { return ff_add(ff_mul(a, b), acc); }

// exact: h + l = a b (the fma two-product)
__device__ __forceinline__ ff two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff_make(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return ff_make(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ ff ff_shfl_xor(ff a, int o) {
  return ff_make(__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o));
}

// complex parts of a float4 (re_h, re_l, im_h, im_l)
__device__ __forceinline__ ff re_of(const float4& z) { return ff_make(z.x, z.y); }
__device__ __forceinline__ ff im_of(const float4& z) { return ff_make(z.z, z.w); }
__device__ __forceinline__ float4 cff(ff re, ff im) { return make_float4(re.h, re.l, im.h, im.l); }

__device__ __forceinline__ float4 cff_from_double2(double2 z) {
  const ff r = ff_from_double(z.x), i = ff_from_double(z.y);
  return cff(r, i);
}

__device__ __forceinline__ double2 cff_to_double2(const float4& z) {
  return make_double2(ff_to_double(re_of(z)), ff_to_double(im_of(z)));
}

// Sums of double-float products (the per-lane Gram sums of the Jacobi SVD,
// the multiply-adds of the complex128 contractions): a running FP32 head h,
// summed exactly (two_sum), and an FP32 error term e collecting the two_sum
// errors and each product's exact error (fma) and cross terms a_h b_l +
// a_l b_h; 12 FP32 operations a product against 18 for a double-float fma.
// e holds about 2^-23 of the sum of |products|, so after K additions its
// own rounding is about K 2^-47 of that sum (1e-12 at K = 128).
struct GramAcc {
  float h = 0.f, e = 0.f;
  __device__ __forceinline__ void add(ff a, ff b) {
    const float p = __fmul_rn(a.h, b.h);
    float pe = __fmaf_rn(a.h, b.h, -p);
    pe = __fmaf_rn(a.h, b.l, pe);
    pe = __fmaf_rn(a.l, b.h, pe);
    const ff s = two_sum(h, p);
    h = s.h;
    e = __fadd_rn(e, __fadd_rn(s.l, pe));
  }
  __device__ __forceinline__ ff value() const { return quick_two_sum(h, e); }
};

// Complex multiply-adds on double-float operands into a pair of GramAcc.
struct CAcc {
  GramAcc re, im;
  // += a b
  __device__ __forceinline__ void fma(const float4& a, const float4& b) {
    const ff ar = re_of(a), ai = im_of(a), br = re_of(b), bi = im_of(b);
    re.add(ar, br);
    re.add(ff_neg(ai), bi);
    im.add(ar, bi);
    im.add(ai, br);
  }
  // += conj(a) b
  __device__ __forceinline__ void fmac(const float4& a, const float4& b) {
    const ff ar = re_of(a), ai = im_of(a), br = re_of(b), bi = im_of(b);
    re.add(ar, br);
    re.add(ai, bi);
    im.add(ar, bi);
    im.add(ff_neg(ai), br);
  }
  __device__ __forceinline__ double2 value() const {
    return make_double2(ff_to_double(re.value()), ff_to_double(im.value()));
  }
};

}  // namespace mpsv
