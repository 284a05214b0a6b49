// Device helpers shared by the contraction kernels: locating a tile in a
// grouped launch and turning composite GEMM indices into element offsets.
#pragma once

#include "tn_internal.h"

namespace tn {

// Offset of composite index `idx` over legs (dims, strides), last leg fastest.
__device__ __forceinline__ int64_t leg_offset(uint32_t idx, int n, const int32_t* dims,
                                              const int64_t* strides) {
  int64_t off = 0;
  for (int q = n - 1; q >= 0; --q) {
    const uint32_t d = (uint32_t)dims[q];
    off += (int64_t)(idx % d) * strides[q];
    idx /= d;
  }
  return off;
}

// Copies the descriptor that owns global work unit `tile` (looked up in the
// unit -> descriptor map) into shared memory and returns the unit's index
// within its descriptor.
__device__ __forceinline__ int64_t fetch_desc(const ContractDesc& single, const ContractDesc* group,
                                              const int32_t* unit_desc, int64_t tile, ContractDesc* sd,
                                              int* s_idx) {
  if (threadIdx.x == 0) *s_idx = group ? unit_desc[tile] : 0;
  __syncthreads();
  const ContractDesc* src = group ? group + *s_idx : &single;
  const int nwords = (int)(sizeof(ContractDesc) / sizeof(int32_t));
  const int32_t* s = reinterpret_cast<const int32_t*>(src);
  int32_t* dst = reinterpret_cast<int32_t*>(sd);
  for (int i = threadIdx.x; i < nwords; i += blockDim.x) dst[i] = s[i];
  __syncthreads();
  return tile - sd->tile_begin;
}

struct UnitCoord {
  int64_t m0, n0, k_begin, k_end;
};

__device__ __forceinline__ UnitCoord decode_unit(const ContractDesc& d, int64_t u, int bm, int bn) {
  UnitCoord c;
  const int64_t tn = u % d.tiles_n;
  const int64_t rest = u / d.tiles_n;
  const int64_t tm = rest % d.tiles_m;
  const int64_t split = rest / d.tiles_m;
  c.m0 = tm * bm;
  c.n0 = tn * bn;
  c.k_begin = split * d.k_per_split;
  c.k_end = min(d.K, c.k_begin + d.k_per_split);
  return c;
}

// Writes (splits == 1) or accumulates (splits > 1, C pre-zeroed) four
// consecutive results; `vec` means 16-byte aligned with all four in range.
__device__ __forceinline__ void emit4(float* dst, bool vec, int64_t nrem, bool accumulate, float a,
                                      float b, float c, float e) {
  if (vec && nrem >= 4) {
    if (accumulate) atomicAdd(reinterpret_cast<float4*>(dst), make_float4(a, b, c, e));
    else *reinterpret_cast<float4*>(dst) = make_float4(a, b, c, e);
    return;
  }
  const float v[4] = {a, b, c, e};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j < nrem) {
      if (accumulate) atomicAdd(dst + j, v[j]);
      else dst[j] = v[j];
    }
  }
}

}  // namespace tn
