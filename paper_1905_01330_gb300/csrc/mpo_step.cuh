// Device code of the energy sweep's step (ii) shared by its launch forms
// (per-site kernels, the grouped batch, the persistent sweep): the exact
// power-of-two rescale and step (ii) written straight into step (iii)'s
// packed operand.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "packed.h"
#include "tn_internal.h"

namespace tn {

// e with m * 2^-e in [1/2, 1) (0 for m <= 0), clamped to the normal range.
__device__ __forceinline__ int pow2_exponent(float m) {
  if (!(m > 0.0f)) return 0;
  const int ex = (__float_as_int(m) >> 23) & 0xff;
  const int e = ex == 0 ? -126 : ex - 126;  // m * 2^-e in [1/2, 1)
  return e < -126 ? -126 : (e > 126 ? 126 : e);
}

// Step (ii) written straight into step (iii)'s packed operand (BF16 and
// BF16X3 sweeps whose extended MPO has (bond) x d <= 8 on both sides of every
// site; the layout is StepIIPack's). The float32 T2 is never written to
// memory and no pack pass reads it back. Rows past R are left as they are:
// each row of the product depends on its own row of P only, and the GEMM
// discards those rows.
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ float bf16_lo_rest(float x) {
  return x - __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void step_ii_pack(const StepIIPack& q, int64_t gtid, int64_t gstride, bool log_thread) {
  __shared__ float Ws[8][8];  // [(w, s)][(w', s')], zero past the MPO
  const int wad = q.wa * q.d, wbd = q.wb * q.d, d = q.d;
  for (int e = threadIdx.x; e < 64; e += blockDim.x) {
    const int k = e >> 3, m = e & 7;
    float v = 0.0f;
    if (k < wad && m < wbd) {
      const int w = k / d, sk = k - w * d, w2 = m / d, s2 = m - w2 * d;
      v = q.W[((w * q.wb + w2) * d + sk) * d + s2];
    }
    Ws[k][m] = v;
  }
  __syncthreads();
  int e = 0;
  if (q.maxbits) e = pow2_exponent(__uint_as_float(*q.maxbits));
  const float inv = __int_as_float((127 - e) << 23);
  if (log_thread && q.maxbits) *q.lg += (double)e * 0.69314718055994530942;
  const int32_t Da = q.Da, Db = q.Db, slabs = q.slabs;
  const float* __restrict__ T1 = q.T1;
  if ((Db & 7) == 0) {
    // a thread takes 8 consecutive b at one a': one 16-byte chunk (8 rows at
    // one shared index) per output channel (w', s'); a warp's stores fill
    // four whole 128-byte lines
    const int32_t groups = Db >> 3;
    const int64_t items = (int64_t)Da * groups;
    for (int64_t it = gtid; it < items; it += gstride) {
      const int32_t a = (int32_t)(it / groups), b0 = (int32_t)(it - (int64_t)a * groups) * 8;
      float t[8][8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k < wad) {
          const int w = k / d, sk = k - w * d;
          const float4* src = reinterpret_cast<const float4*>(T1 + ((int64_t)(w * Da + a) * d + sk) * Db + b0);
          const float4 x0 = __ldg(src), x1 = __ldg(src + 1);
          t[k][0] = x0.x; t[k][1] = x0.y; t[k][2] = x0.z; t[k][3] = x0.w;
          t[k][4] = x1.x; t[k][5] = x1.y; t[k][6] = x1.z; t[k][7] = x1.w;
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) t[k][j] = 0.0f;
        }
      }
#pragma unroll 1
      for (int m = 0; m < wbd; ++m) {
        float o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float acc = 0.0f;
#pragma unroll
          for (int k = 0; k < 8; ++k) acc = fmaf(Ws[k][m], t[k][j], acc);
          o[j] = acc * inv;
        }
        const int w2 = m / d, s2 = m - w2 * d;
        const int32_t r0 = w2 * Db + b0, kx = s2 * q.ps + a * q.pa;
        const size_t off = ((size_t)(r0 >> 7) * slabs + (kx >> 6)) * MN_BLOCK_BYTES +
                           mn_block_chunk((r0 & 127) >> 3, kx & 63);
        uint4 h;
        h.x = bf16x2_bits(o[0], o[1]);
        h.y = bf16x2_bits(o[2], o[3]);
        h.z = bf16x2_bits(o[4], o[5]);
        h.w = bf16x2_bits(o[6], o[7]);
        *reinterpret_cast<uint4*>(q.hi + off) = h;
        if (q.lo) {
          uint4 l;
          l.x = bf16x2_bits(bf16_lo_rest(o[0]), bf16_lo_rest(o[1]));
          l.y = bf16x2_bits(bf16_lo_rest(o[2]), bf16_lo_rest(o[3]));
          l.z = bf16x2_bits(bf16_lo_rest(o[4]), bf16_lo_rest(o[5]));
          l.w = bf16x2_bits(bf16_lo_rest(o[6]), bf16_lo_rest(o[7]));
          *reinterpret_cast<uint4*>(q.lo + off) = l;
        }
      }
    }
  } else {
    // small or odd bonds: a thread per column (a', b), 2-byte stores
    const int64_t items = (int64_t)Da * Db;
    for (int64_t it = gtid; it < items; it += gstride) {
      const int32_t a = (int32_t)(it / Db), b = (int32_t)(it - (int64_t)a * Db);
      float t[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        t[k] = 0.0f;
        if (k < wad) {
          const int w = k / d, sk = k - w * d;
          t[k] = __ldg(T1 + ((int64_t)(w * Da + a) * d + sk) * Db + b);
        }
      }
      for (int m = 0; m < wbd; ++m) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) acc = fmaf(Ws[k][m], t[k], acc);
        const float o = acc * inv;
        const int w2 = m / d, s2 = m - w2 * d;
        const int32_t r = w2 * Db + b, kx = s2 * q.ps + a * q.pa;
        const size_t off = ((size_t)(r >> 7) * slabs + (kx >> 6)) * MN_BLOCK_BYTES +
                           mn_block_chunk((r & 127) >> 3, kx & 63) + 2 * (r & 7);
        const __nv_bfloat16 h = __float2bfloat16_rn(o);
        *reinterpret_cast<__nv_bfloat16*>(q.hi + off) = h;
        if (q.lo) *reinterpret_cast<__nv_bfloat16*>(q.lo + off) = __float2bfloat16_rn(o - __bfloat162float(h));
      }
    }
  }
  // zeros at the shared indices past K = d Da of every block of the last slab
  const int32_t K = d * Da, kpad = slabs * 64 - K;
  if (kpad > 0) {
    const int64_t chunks = (int64_t)q.tiles * 16 * kpad;
    for (int64_t it = gtid; it < chunks; it += gstride) {
      const int32_t kk = K + (int32_t)(it % kpad);
      const int64_t rest = it / kpad;
      const int32_t mg = (int32_t)(rest & 15), tile = (int32_t)(rest >> 4);
      const size_t off = ((size_t)tile * slabs + (kk >> 6)) * MN_BLOCK_BYTES + mn_block_chunk(mg, kk & 63);
      *reinterpret_cast<uint4*>(q.hi + off) = make_uint4(0u, 0u, 0u, 0u);
      if (q.lo) *reinterpret_cast<uint4*>(q.lo + off) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

}  // namespace tn
