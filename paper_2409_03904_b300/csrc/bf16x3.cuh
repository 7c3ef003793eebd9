// Exact three-term bf16 split of FP32 values for tensor-core operands
// (kind::f16 MMAs with bf16 A and B, FP32 accumulation), shared by the
// block algebra (blas_tc.cu) and the block transfers (blocking_tc.cu).
//
// v = h + m + l with h = v with its low 16 bits cleared, m the same of
// v - h, and l = v - h - m: 8 + 8 + 8 significant bits, so every term is
// exact in bf16 (its upper 16 bits).  Keeping the six products down to order
// 2^-16 (hh, hm, mh, mm, hl, lh) leaves an error below about 2^-23 of |x||y|
// per product, the size of an FP32 rounding.
#pragma once
#include <stdint.h>

namespace mrhs {

__device__ __forceinline__ void split3(float v, uint32_t& h, uint32_t& m, uint32_t& l) {
  const uint32_t vb = __float_as_uint(v);
  h = vb & 0xFFFF0000u;
  const float r = v - __uint_as_float(h);
  m = __float_as_uint(r) & 0xFFFF0000u;
  l = __float_as_uint(r - __uint_as_float(m));
}
// the bf16 (upper halves) of a and b packed, a in the low half
__device__ __forceinline__ uint32_t pack_bf16(uint32_t a, uint32_t b) {
  return __byte_perm(a, b, 0x7632);
}
__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                       uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
// eight values split and stored as three 16-byte core-matrix rows (terms h,
// m, l at base + 0, + dm, + dl)
__device__ __forceinline__ void split_store8(const float* v, uint32_t base, uint32_t dm,
                                             uint32_t dl) {
  uint32_t hh[8], mm[8], ll[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) split3(v[e], hh[e], mm[e], ll[e]);
  sts128(base, pack_bf16(hh[0], hh[1]), pack_bf16(hh[2], hh[3]), pack_bf16(hh[4], hh[5]),
         pack_bf16(hh[6], hh[7]));
  sts128(base + dm, pack_bf16(mm[0], mm[1]), pack_bf16(mm[2], mm[3]), pack_bf16(mm[4], mm[5]),
         pack_bf16(mm[6], mm[7]));
  sts128(base + dl, pack_bf16(ll[0], ll[1]), pack_bf16(ll[2], ll[3]), pack_bf16(ll[4], ll[5]),
         pack_bf16(ll[6], ll[7]));
}

}  // namespace mrhs
