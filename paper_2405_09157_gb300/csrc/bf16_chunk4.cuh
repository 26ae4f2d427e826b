// Four bfloat16 values (one 8-byte load) widened to float32: the chunk of
// the kernels that keep a float32 chunk width of 4 for bfloat16 rows (the
// reverse sweep, whose gradient rows are float4 chunks, and the batched pass,
// whose lane layouts are those of float32 rows).
#pragma once

#include "common.cuh"

namespace pdscp {

template <>
struct Chunk<__nv_bfloat16, 4> {
  static __device__ __forceinline__ void load(const __nv_bfloat16* row, int c, float* o) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(row) + c);
    o[0] = __uint_as_float(v.x << 16);  // element 2c: the low half of the first word
    o[1] = __uint_as_float(v.x & 0xffff0000u);
    o[2] = __uint_as_float(v.y << 16);
    o[3] = __uint_as_float(v.y & 0xffff0000u);
  }
};

}  // namespace pdscp
