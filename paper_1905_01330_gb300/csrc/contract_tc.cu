// Pairwise tensordot on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C[m, n] = sum_k A(m, k) B(k, n) over the flattened shared legs
// (Sec. III.B.2 / III.B.4), float32 in and out, bf16 operands with float32
// accumulation in tensor memory (TMEM):
//   BF16   : one MMA per 16-wide k step on bf16(A), bf16(B);
//   BF16X3 : x = hi + lo (hi = bf16(x), lo = bf16(x - hi)); three MMAs per
//            k step, Ahi*Bhi + Ahi*Blo + Alo*Bhi, into the same accumulator.
//
// Roles in a 288-thread CTA computing one 128x128 output tile:
//   warps 0-7 (converters): gather 128x64 float32 slabs of A and B in place
//     through the operands' leg strides (the permutation is folded into the
//     gather: no transposed copy exists anywhere), round to bf16 (and split),
//     and store them into the 128-byte-swizzled K-major shared-memory layout
//     the MMA descriptors describe; a ring of stages is handed over with
//     mbarriers. After the k loop they drain TMEM (tcgen05.ld) and write C.
//   warp 8 (MMA): allocates TMEM, and one lane issues tcgen05.mma for each
//     stage, releasing stages with tcgen05.commit.
// Every mbarrier wait is bounded (2 s of wall time); on expiry the kernel
// records TN_ERR_TIMEOUT, stops, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "gather.cuh"
#include "ptx.cuh"

namespace tn {
namespace {

constexpr int BM = TC_BM, BN = TC_BN, BK = 64;
constexpr int NPROD = 256;             // converter threads (warps 0-7)
constexpr int NTHREADS = NPROD + 32;   // + MMA warp
constexpr int TILE_BYTES = BM * BK * 2;  // one 128x64 bf16 operand tile (16 KB)
// BF16X3 promotes the tensor-core accumulator into float32 registers every
// KC k-slabs (KC * 64 = 256 shared indices): the tensor core's float32
// accumulation truncates, and over long K that error (linear in the number
// of accumulation steps) would exceed the split's own rounding error.
constexpr int KC = 4;
template <int SPLIT>
constexpr uint32_t tmem_cols() { return SPLIT ? 2 * BN : BN; }  // f32 accumulators, 128 lanes each

template <int SPLIT>
struct TcCfg {
  static constexpr int STAGES = 3;
  static constexpr int OPS = SPLIT ? 4 : 2;  // tiles per stage: Ahi, Bhi (, Alo, Blo)
  static constexpr int STAGE_BYTES = OPS * TILE_BYTES;
};

template <int S>
struct TcAux {
  int32_t rowA[BM];
  int32_t rowB[BN];
  int32_t kA[S][BK];
  int32_t kB[S][BK];
  int32_t kcA[S][BK / 8];  // 1: the 8-wide k group is unit-stride in A
  int32_t kcB[S][BK / 8];
  uint64_t full[S];
  uint64_t empty[S];
  uint64_t accum;
  uint64_t chunk_full[2];  // BF16X3: accumulator buffer b holds a finished chunk
  uint64_t drained[2];     // BF16X3: buffer b was read back and may be overwritten
  uint32_t tmem_base;
  int32_t idx;
  ContractDesc d;
};

template <int SPLIT>
constexpr size_t tc_smem_bytes() {
  return 1024 /* alignment slack */ + (size_t)TcCfg<SPLIT>::STAGES * TcCfg<SPLIT>::STAGE_BYTES +
         sizeof(TcAux<TcCfg<SPLIT>::STAGES>);
}

// Byte offset of the 16-byte chunk (row r, k group g) in a 128B-swizzled
// K-major tile: 8-row atoms of 1024 B, rows of 128 B, chunk index XOR row%8.
__device__ __forceinline__ uint32_t sw128_chunk(int r, int g) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// Loads the 8 float32 values of one (row, k group) unit of an operand.
__device__ __forceinline__ void load_unit(const float* __restrict__ base, int32_t row_off,
                                          const int32_t* koff, int contiguous, float (&v)[8]) {
  if (row_off < 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.0f;
    return;
  }
  if (contiguous) {
    const float* p = base + (row_off + koff[0]);
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
      const float4 x = __ldg(reinterpret_cast<const float4*>(p));
      const float4 y = __ldg(reinterpret_cast<const float4*>(p) + 1);
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
      v[4] = y.x; v[5] = y.y; v[6] = y.z; v[7] = y.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __ldg(p + j);
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int32_t ko = koff[j];
    v[j] = (ko >= 0) ? __ldg(base + (row_off + ko)) : 0.0f;
  }
}

template <int SPLIT>
__device__ __forceinline__ void store_unit(uint8_t* hi_tile, uint8_t* lo_tile, int r, int g,
                                           const float (&v)[8]) {
  uint4 h;
  h.x = pack_bf16x2(v[0], v[1]);
  h.y = pack_bf16x2(v[2], v[3]);
  h.z = pack_bf16x2(v[4], v[5]);
  h.w = pack_bf16x2(v[6], v[7]);
  const uint32_t off = sw128_chunk(r, g);
  *reinterpret_cast<uint4*>(hi_tile + off) = h;
  if (SPLIT) {
    const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&h);
    uint4 l;
    l.x = pack_bf16x2(v[0] - __low2float(hb[0]), v[1] - __high2float(hb[0]));
    l.y = pack_bf16x2(v[2] - __low2float(hb[1]), v[3] - __high2float(hb[1]));
    l.z = pack_bf16x2(v[4] - __low2float(hb[2]), v[5] - __high2float(hb[2]));
    l.w = pack_bf16x2(v[6] - __low2float(hb[3]), v[7] - __high2float(hb[3]));
    *reinterpret_cast<uint4*>(lo_tile + off) = l;
  }
}

// k-group contiguity: the 8 indices k0..k0+7 are all < K and consecutive in
// memory (innermost shared leg has unit stride and the group does not wrap).
__device__ __forceinline__ int group_contiguous(const ContractDesc& d, int64_t k0, int64_t k_end,
                                                const int64_t* kstr) {
  if (d.nk == 0 || k0 + 8 > k_end) return 0;
  const int last = d.nk - 1;
  if (kstr[last] != 1) return 0;
  const int64_t dl = d.kdim[last];
  return ((k0 % dl) + 8 <= dl) ? 1 : 0;
}

template <int SPLIT>
__global__ void __launch_bounds__(NTHREADS, SPLIT ? 1 : 2)
tc_contract_kernel(const __grid_constant__ ContractDesc single, const ContractDesc* group,
                   int ndesc, int* status) {
  using Cfg = TcCfg<SPLIT>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  TcAux<S>& x = *reinterpret_cast<TcAux<S>*>(smem + (size_t)S * Cfg::STAGE_BYTES);

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      ptx::mbar_init(ptx::smem_addr(&x.full[s]), NPROD);
      ptx::mbar_init(ptx::smem_addr(&x.empty[s]), 1);
    }
    ptx::mbar_init(ptx::smem_addr(&x.accum), 1);
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&x.chunk_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&x.drained[b]), NPROD);
    }
    ptx::fence_mbar_init();
  }
  if (warp == 8) {
    ptx::tmem_alloc(ptx::smem_addr(&x.tmem_base), tmem_cols<SPLIT>());
    ptx::tmem_relinquish();
    ptx::tc_fence_before();
  }
  const int64_t tile = fetch_desc(single, group, ndesc, (int64_t)blockIdx.x, &x.d, &x.idx);
  // fetch_desc ends with __syncthreads(): barriers and the TMEM base are visible.
  ptx::tc_fence_after();
  const uint32_t tmem = x.tmem_base;
  const ContractDesc& d = x.d;
  const UnitCoord uc = decode_unit(d, tile, BM, BN);
  const int64_t m0 = uc.m0, n0 = uc.n0;
  const int64_t nkt = (uc.k_end - uc.k_begin + BK - 1) / BK;
  const uint32_t stage0 = ptx::smem_addr(smem);

  if (warp < 8) {
    // ------------------------------------------------------------ converters
    if (t < BM) {
      const int64_t m = m0 + t;
      x.rowA[t] = (m < d.M) ? (int32_t)leg_offset((uint32_t)m, d.nm, d.mdim, d.mstr) : -1;
    } else {
      const int64_t n = n0 + (t - BM);
      x.rowB[t - BM] = (n < d.N) ? (int32_t)leg_offset((uint32_t)n, d.nn, d.ndim, d.nstr) : -1;
    }
    bool ok = true;
    const int q = warp & 3, h = warp >> 2;  // TMEM lane quadrant and column half of this warp
    float acc[SPLIT ? 64 : 1];
#pragma unroll
    for (int j = 0; j < (SPLIT ? 64 : 1); ++j) acc[j] = 0.0f;
    const int64_t nchunks = (nkt + KC - 1) / KC;
    int64_t next_drain = 0;
    // BF16X3: adds finished chunk c (accumulator buffer c & 1) into acc
    auto drain = [&](int64_t c) -> bool {
      const int b = (int)(c & 1);
      const bool w = ptx::mbar_wait(ptx::smem_addr(&x.chunk_full[b]), (uint32_t)((c >> 1) & 1), status);
      if (!__all_sync(0xffffffffu, w)) return false;
      ptx::tc_fence_after();
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t r[32];
        ptx::tmem_ld_32x32b_x32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + h * 64 + half * 32), r);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[half * 32 + j] += __uint_as_float(r[j]);
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(ptx::smem_addr(&x.drained[b]));
      return true;
    };
    for (int64_t kt = 0; kt < nkt; ++kt) {
      const int s = (int)(kt % S);
      const uint32_t round = (uint32_t)(kt / S);
      bool drained_ok = true;
      if (SPLIT && (kt % KC) == 0 && kt / KC >= 2) {
        drained_ok = drain(next_drain);
        ++next_drain;
      }
      const bool waited = ptx::mbar_wait(ptx::smem_addr(&x.empty[s]), (round & 1u) ^ 1u, status) && drained_ok;
      // decode this slab's shared-index offsets (tables only; the stage itself
      // is written after the collective check below)
      if (t < 2 * BK) {
        const int j = t & (BK - 1);
        const int64_t k = uc.k_begin + kt * BK + j;
        const bool isA = t < BK;
        const int64_t* kstr = isA ? d.kstrA : d.kstrB;
        const int32_t off = (k < uc.k_end) ? (int32_t)leg_offset((uint32_t)k, d.nk, d.kdim, kstr) : -1;
        if (isA) x.kA[s][j] = off; else x.kB[s][j] = off;
        if ((j & 7) == 0) {
          const int c = group_contiguous(d, k, uc.k_end, kstr);
          if (isA) x.kcA[s][j >> 3] = c; else x.kcB[s][j >> 3] = c;
        }
      }
      // every converter reaches this barrier once per slab; a wait that
      // expired anywhere stops all of them together
      if (ptx::named_barrier_or(1, NPROD, !waited)) { ok = false; break; }

      uint8_t* st = smem + (size_t)s * Cfg::STAGE_BYTES;
      float va[4][8], vb[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int u = t + NPROD * i;
        const int r = d.a_kfast ? (u >> 3) : (u & (BM - 1));
        const int g = d.a_kfast ? (u & 7) : (u >> 7);
        load_unit(d.A, x.rowA[r], &x.kA[s][g * 8], x.kcA[s][g], va[i]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int u = t + NPROD * i;
        const int r = d.b_kfast ? (u >> 3) : (u & (BN - 1));
        const int g = d.b_kfast ? (u & 7) : (u >> 7);
        load_unit(d.B, x.rowB[r], &x.kB[s][g * 8], x.kcB[s][g], vb[i]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int u = t + NPROD * i;
        const int r = d.a_kfast ? (u >> 3) : (u & (BM - 1));
        const int g = d.a_kfast ? (u & 7) : (u >> 7);
        store_unit<SPLIT>(st, st + 2 * TILE_BYTES, r, g, va[i]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int u = t + NPROD * i;
        const int r = d.b_kfast ? (u >> 3) : (u & (BN - 1));
        const int g = d.b_kfast ? (u & 7) : (u >> 7);
        store_unit<SPLIT>(st + TILE_BYTES, st + 3 * TILE_BYTES, r, g, vb[i]);
      }
      ptx::fence_proxy_async_smem();
      ptx::mbar_arrive(ptx::smem_addr(&x.full[s]));
    }

    // -------------------------------------------------------------- epilogue
    if (SPLIT) {
      for (; ok && next_drain < nchunks; ++next_drain) ok = drain(next_drain);
    }
    const bool acc_ready = ptx::mbar_wait(ptx::smem_addr(&x.accum), 0u, status) && ok;
    if (__all_sync(0xffffffffu, acc_ready)) {  // tcgen05.ld is warp-collective
      ptx::tc_fence_after();
      const int64_t m = m0 + q * 32 + lane;
      float* __restrict__ C = d.C;
      const int64_t N = d.N;
      const bool vec = ((N & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int col = h * 64 + half * 32;
        uint32_t r[32];
        if (SPLIT) {
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(acc[half * 32 + j]);
        } else {
          ptx::tmem_ld_32x32b_x32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)col, r);
          ptx::tmem_ld_wait();
        }
        if (m < d.M) {
          float* dst = C + m * N + n0 + col;
          const int64_t nrem = N - (n0 + col);
          const bool accumulate = d.splits > 1;
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (j < nrem)
              emit4(dst + j, vec, nrem - j, accumulate, __uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                    __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
        }
      }
    }
  } else {
    // ------------------------------------------------------------ MMA warp
    constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);
    if (lane == 0) {
      for (int64_t kt = 0; kt < nkt; ++kt) {
        const int s = (int)(kt % S);
        const uint32_t round = (uint32_t)(kt / S);
        const int64_t c = kt / KC;
        const bool chunk_start = (kt % KC) == 0;
        if (SPLIT && chunk_start && c >= 2) {
          // the converters must have read this buffer's previous chunk back
          if (!ptx::mbar_wait(ptx::smem_addr(&x.drained[c & 1]), (uint32_t)(((c >> 1) - 1) & 1), status)) break;
          ptx::tc_fence_after();
        }
        if (!ptx::mbar_wait(ptx::smem_addr(&x.full[s]), round & 1u, status)) break;
        ptx::tc_fence_after();
        const uint32_t d_tmem = SPLIT ? tmem + (uint32_t)((c & 1) * BN) : tmem;
        const bool fresh = SPLIT ? chunk_start : (kt == 0);
        const uint32_t a_hi = stage0 + (uint32_t)(s * Cfg::STAGE_BYTES);
        const uint32_t b_hi = a_hi + TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t ad = ptx::sw128_kmajor_desc(a_hi + kk * 32);
          const uint64_t bd = ptx::sw128_kmajor_desc(b_hi + kk * 32);
          ptx::mma_bf16(d_tmem, ad, bd, idesc, (fresh && kk == 0) ? 0u : 1u);
          if (SPLIT) {
            const uint64_t al = ptx::sw128_kmajor_desc(a_hi + 2 * TILE_BYTES + kk * 32);
            const uint64_t bl = ptx::sw128_kmajor_desc(b_hi + 2 * TILE_BYTES + kk * 32);
            ptx::mma_bf16(d_tmem, ad, bl, idesc, 1u);
            ptx::mma_bf16(d_tmem, al, bd, idesc, 1u);
          }
        }
        ptx::mma_commit(ptx::smem_addr(&x.empty[s]));
        if (SPLIT && ((kt % KC) == KC - 1 || kt == nkt - 1)) ptx::mma_commit(ptx::smem_addr(&x.chunk_full[c & 1]));
      }
      if (nkt == 0) {
        // K = 0 never reaches the kernel (the host writes zeros); keep the
        // epilogue's wait well defined anyway.
        ptx::mbar_arrive(ptx::smem_addr(&x.accum));
      } else {
        ptx::mma_commit(ptx::smem_addr(&x.accum));
      }
    }
    __syncwarp();
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 8) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, tmem_cols<SPLIT>());
  }
}

template <int SPLIT>
int launch_tc(const ContractDesc& single, const ContractDesc* group, int ndesc, int64_t tiles,
              cudaStream_t stream) {
  const size_t smem = tc_smem_bytes<SPLIT>();
  static bool attr_set = false;  // per process; every device gets the same attribute value
  if (!attr_set) {
    if (cudaFuncSetAttribute(tc_contract_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return TN_ERR_CUDA;
    attr_set = true;
  }
  tc_contract_kernel<SPLIT><<<(unsigned)tiles, NTHREADS, smem, stream>>>(single, group, ndesc,
                                                                         status_word());
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace

int launch_contract_tc(const ContractDesc& single, const ContractDesc* group, int ndesc,
                       int64_t total_tiles, int prec, cudaStream_t stream) {
  if (total_tiles <= 0) return TN_OK;
  if (total_tiles > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (prec == TN_PREC_BF16) return launch_tc<0>(single, group, ndesc, total_tiles, stream);
  if (prec == TN_PREC_BF16X3) return launch_tc<1>(single, group, ndesc, total_tiles, stream);
  return TN_ERR_ARG;
}

}  // namespace tn
