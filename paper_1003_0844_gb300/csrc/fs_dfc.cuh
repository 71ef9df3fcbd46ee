// Double-float complex arithmetic (the upsampler's transforms, fs_fft64.cu and
// fs_prep.cu): a value stored as float4 (re.hi, re.lo, im.hi, im.lo).
#pragma once
#include "fs_common.cuh"

namespace fs {

struct dfc {
  df32 re, im;
};
__device__ __forceinline__ dfc dfc_ld(const float4 v) { return dfc{df32{v.x, v.y}, df32{v.z, v.w}}; }
__device__ __forceinline__ float4 dfc_st(const dfc &a) { return make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo); }
__device__ __forceinline__ dfc dfc_add(const dfc &a, const dfc &b) { return dfc{df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_sub(const dfc &a, const dfc &b) { return dfc{df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_mul(const dfc &a, const dfc &b) {
  return dfc{df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// times -i (forward) or +i (inverse)
__device__ __forceinline__ dfc dfc_rot(const dfc &d, int sign) {
  return sign < 0 ? dfc{d.im, df_neg(d.re)} : dfc{df_neg(d.im), d.re};
}

}  // namespace fs
