// Exact integer BF16 slicing of FP32-pair values for tensor-core products (Ozaki-style
// error-free splitting; Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 2012), shared by the
// product kernels and the delayed-update flush.
//
// A row (or column) scaled by 2^-e so that its entries lie in (-1/2, 1/2) is cut into kOzS
// integer slices, x = 2^e sum_s a_s 2^{-8(s+1)}, |a_s| <= 129: exact in BF16, products exact,
// and sums of up to 7 * 128 products below 2^24, exact in FP32 accumulators.
#pragma once
#include <cuda_bf16.h>

#include "df.cuh"

namespace nmc {

constexpr int kOzS = 7;   // slices per operand

// 2^k from its bit pattern (exact); outside the normal exponent range, ldexpf.
__device__ __forceinline__ float pow2f(int k) {
  return (k >= -126 && k <= 127) ? __int_as_float((k + 127) << 23) : ldexpf(1.f, k);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// exponent e with |x| <= 2^e for the largest |x| given (0 -> 0)
__device__ __forceinline__ int scale_exp(float m) {
  if (!(m > 0.f)) return 0;
  int e;
  frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  return e;
}

// Cut v * 2^-e (exact power-of-two scaling of an FP32 pair) into kOzS integer slices.
__device__ __forceinline__ void slice_value(df2 v, int e, __nv_bfloat16* out, int stride) {
  const float sc = pow2f(8 - e);   // scaling by a power of two: exact
  float h = v.hi * sc, l = v.lo * sc;
  for (int s = 0; s < kOzS; ++s) {
    const float a = rintf(h);
    out[s * stride] = __float2bfloat16_rn(a);  // integer with |a| <= 256: exact
    // residual (h - a) + l as an exact pair, then scale by 2^8 for the next slice
    const float d = __fsub_rn(h, a);           // exact (|h - a| <= 1/2)
    const float t = __fadd_rn(d, l);
    const float bb = __fsub_rn(t, d);
    const float err = __fadd_rn(__fsub_rn(d, __fsub_rn(t, bb)), __fsub_rn(l, bb));
    h = t * 256.f;
    l = err * 256.f;
  }
}

// The same slices as BF16 bit patterns in registers (for fragments built without shared
// memory).
__device__ __forceinline__ void slice_bits(df2 v, int e, unsigned short (&out)[kOzS]) {
  const float sc = pow2f(8 - e);   // scaling by a power of two: exact
  float h = v.hi * sc, l = v.lo * sc;
#pragma unroll
  for (int s = 0; s < kOzS; ++s) {
    const float a = rintf(h);
    out[s] = __bfloat16_as_ushort(__float2bfloat16_rn(a));
    const float d = __fsub_rn(h, a);
    const float t = __fadd_rn(d, l);
    const float bb = __fsub_rn(t, d);
    const float err = __fadd_rn(__fsub_rn(d, __fsub_rn(t, bb)), __fsub_rn(l, bb));
    h = t * 256.f;
    l = err * 256.f;
  }
}

}  // namespace nmc
