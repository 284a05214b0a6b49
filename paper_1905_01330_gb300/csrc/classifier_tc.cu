// MPS classifier sweeps on the tcgen05 tensor cores (bf16 operands, float32
// accumulation): the BF16 path of tn_mps_classify / tn_mps_classify_backward.
//
// One step of a half-chain for a tile of 128 samples is a matrix product
//     U[b, (s, j)] = sum_k v_b[k] L[k, s, j]        (M = 128, N = 2 chi, K = chi)
// followed by v'_b[j] = Phi_0(x_b) U[b, (0, j)] + Phi_1(x_b) U[b, (1, j)] and the
// per-sample rescale (forward: divide by the largest magnitude, add its log
// to the float64 log-scale; adjoint: divide by the forward's recorded scale).
// One CTA of 128 threads owns one tile and one half-chain for all its steps:
// the vectors stay in shared memory as the MMA's A operand (bf16, 128-byte-
// swizzled K-major), each thread owns one sample (one TMEM lane, one row of
// the operand), and thread 0 issues the MMAs. The cores, packed once per call
// into the bf16 K-major image the MMA reads (`cls_pack_images`), are streamed
// into a ring of shared-memory buffers by 1-D bulk async copies a few steps
// ahead. Every mbarrier wait is bounded; a CTA that gives up records
// TN_ERR_TIMEOUT, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "classifier_tc.h"
#include "ptx.cuh"

namespace tn {
namespace {

constexpr int NT = 128;  // threads = samples per tile = TMEM lanes

__device__ __forceinline__ uint32_t sw128(int r, int g) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ----------------------------------------------------------------- packing
// Image of step t: rows n = s * chi + j (2 chi rows), K = kpad shared indices
// (kpad = max(chi, 64)), kslab-major: slab ks holds rows of 64 k (128 B),
// 128-byte swizzled, slabs 2 chi * 128 B apart. Value L[k, s, j] with
// L[k, s, j] = A[k, s, j] ("natural": k the core's left bond) or A[j, s, k].
__global__ void cls_pack_images(const __grid_constant__ ClsPackParams p) {
  const int t = blockIdx.x;  // step
  const int site = p.half == 0 ? t : p.n - 1 - t;
  const bool natural = (p.half == 0) == (p.mode == 0);
  const int Da = p.bond[site], Dc = p.bond[site + 1];
  const int Din = natural ? Da : Dc, Dout = natural ? Dc : Da;
  const float* __restrict__ A = p.core[site];
  uint8_t* img = p.images + (size_t)t * p.img_bytes;
  const int chi = p.chi, kpad = p.kpad, rows = 2 * chi;
  // one 16-byte chunk (row n, 8 consecutive k) per iteration
  const int chunks = rows * (kpad / 8);
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int n = c % rows;
    const int kg = c / rows;  // 8-group of k over all slabs
    const int s = n / chi, j = n % chi;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = kg * 8 + e;
      float x = 0.0f;
      if (k < Din && j < Dout)
        x = natural ? A[((int64_t)k * 2 + s) * Dc + j] : A[((int64_t)j * 2 + s) * Dc + k];
      v[e] = x;
    }
    uint4 h;
    h.x = pack2(v[0], v[1]);
    h.y = pack2(v[2], v[3]);
    h.z = pack2(v[4], v[5]);
    h.w = pack2(v[6], v[7]);
    const int ks = kg >> 3, g = kg & 7;
    *reinterpret_cast<uint4*>(img + (size_t)ks * rows * 128 + sw128(n, g)) = h;
  }
}

// ------------------------------------------------------------------ sweep
template <int CHI>
struct SweepCfg {
  static constexpr int KPAD = CHI < 64 ? 64 : CHI;
  static constexpr int KSLABS = KPAD / 64;
  static constexpr int N = 2 * CHI;                     // MMA N
  static constexpr int IMG = N * KPAD * 2;              // bytes of one core image
  static constexpr int VTILE = NT * KPAD * 2;           // bytes of the vector operand
  static constexpr int RING = CHI == 128 ? 2 : 4;       // core images in flight
  static constexpr int PXS = 32;                        // steps of pixels staged at once
  static constexpr uint32_t TMEM_COLS = N < 32 ? 32 : N;
};

template <int CHI>
struct SweepSmem {
  float px[SweepCfg<CHI>::PXS][NT];
  uint64_t core_full[SweepCfg<CHI>::RING];
  uint64_t acc_full;
  uint64_t final_bar;
  uint32_t tmem_base;
  int32_t abort;
};

template <int CHI>
constexpr size_t sweep_smem_bytes() {
  using C = SweepCfg<CHI>;
  return 1024 + (size_t)C::VTILE + (size_t)C::RING * C::IMG + sizeof(SweepSmem<CHI>);
}

template <int CHI>
__global__ void __launch_bounds__(NT, 1) cls_sweep_tc(const __grid_constant__ ClsTcParams p) {
  using C = SweepCfg<CHI>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* vtile = base;
  uint8_t* ring = base + C::VTILE;
  SweepSmem<CHI>& x = *reinterpret_cast<SweepSmem<CHI>*>(ring + (size_t)C::RING * C::IMG);
  const int t = threadIdx.x, warp = t >> 5;
  const int B = p.batch;
  const int b = blockIdx.x * NT + t;  // this thread's sample
  const bool live = b < B;
  const int nsteps = p.t_end - p.t_begin;
  auto step_of = [&](int q) { return p.mode == 0 ? p.t_begin + q : p.t_end - 1 - q; };

  if (t == 0) {
    for (int r = 0; r < C::RING; ++r) ptx::mbar_init(ptx::smem_addr(&x.core_full[r]), 1);
    ptx::mbar_init(ptx::smem_addr(&x.acc_full), 1);
    ptx::mbar_init(ptx::smem_addr(&x.final_bar), 1);
    x.abort = 0;
    ptx::fence_mbar_init();
    // first images of the ring
    for (int q = 0; q < C::RING && q < nsteps; ++q) {
      const uint32_t bar = ptx::smem_addr(&x.core_full[q]);
      ptx::mbar_arrive_expect_tx(bar, C::IMG);
      ptx::bulk_copy_g2s(ptx::smem_addr(ring + (size_t)q * C::IMG), p.images + (size_t)step_of(q) * C::IMG, C::IMG,
                         bar);
    }
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_addr(&x.tmem_base), C::TMEM_COLS);
    ptx::tmem_relinquish();
  }

  // the sample's vector, float32 in registers and bf16 in the operand tile
  float v[CHI];
  double lam = 0.0;
#pragma unroll
  for (int k = 0; k < CHI; ++k) v[k] = live ? p.state[(int64_t)b * CHI + k] : (k == 0 ? 1.0f : 0.0f);
  if (p.mode == 0 && live) lam = p.lam[b];
  auto write_row = [&]() {
#pragma unroll
    for (int g = 0; g < C::KPAD / 8; ++g) {
      uint4 h;
      if (g * 8 < CHI) {
        h.x = pack2(v[g * 8 + 0], v[g * 8 + 1]);
        h.y = pack2(v[g * 8 + 2], v[g * 8 + 3]);
        h.z = pack2(v[g * 8 + 4], v[g * 8 + 5]);
        h.w = pack2(v[g * 8 + 6], v[g * 8 + 7]);
      } else {
        h = make_uint4(0, 0, 0, 0);
      }
      *reinterpret_cast<uint4*>(vtile + (size_t)(g >> 3) * (NT * 128) + sw128(t, g & 7)) = h;
    }
  };
  write_row();
  ptx::fence_proxy_async_smem();
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = x.tmem_base;
  const uint32_t vaddr = ptx::smem_addr(vtile), raddr = ptx::smem_addr(ring);
  constexpr uint32_t idesc = ptx::idesc_bf16_f32(128, C::N);
  const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);

  bool ok = true;
  for (int q = 0; q < nsteps && ok; ++q) {
    const int ts = step_of(q);
    const int site = p.half == 0 ? ts : p.n - 1 - ts;
    const int r = q % C::RING;
    // stage pixels for the next PXS steps (coalesced along each sample's row)
    if (q % C::PXS == 0) {
      for (int e = t; e < C::PXS * NT; e += NT) {
        const int qq = e % C::PXS, bb = e / C::PXS;
        const int gb = blockIdx.x * NT + bb;
        float val = 0.0f;
        if (q + qq < nsteps && gb < B) {
          const int ts2 = step_of(q + qq);
          const int site2 = p.half == 0 ? ts2 : p.n - 1 - ts2;
          val = __ldg(p.pixels + (int64_t)gb * p.n + site2);
        }
        x.px[qq][bb] = val;
      }
      __syncthreads();
    }
    const float xp = x.px[q % C::PXS][t];
    const float f0 = cospif(0.5f * xp), f1 = sinpif(0.5f * xp);
    (void)site;

    // adjoint: the gradient operands of this step come from the incoming
    // vector (float32 registers) before it is overwritten
    float scl = 1.0f;
    if (p.mode == 1) {
      scl = live ? p.sc[(int64_t)ts * B + b] : 1.0f;
      if (live) {
        float* dst = p.xout + ((int64_t)(ts - p.t_begin) * B + b) * 2 * CHI;
        const float inv = 1.0f / scl;
        if (p.half == 0) {
#pragma unroll
          for (int k = 0; k < CHI; ++k) { dst[k] = f0 * v[k] * inv; dst[CHI + k] = f1 * v[k] * inv; }
        } else {
#pragma unroll
          for (int k = 0; k < CHI; ++k) { dst[2 * k] = f0 * v[k] * inv; dst[2 * k + 1] = f1 * v[k] * inv; }
        }
      }
    } else if (p.store && live && ((ts - p.store_base) % p.store_every) == 0) {
      float* dst = p.store + ((int64_t)((ts - p.store_base) / p.store_every) * B + b) * CHI;
#pragma unroll
      for (int k = 0; k < CHI; ++k) dst[k] = v[k];
    }

    if (t == 0) {
      bool w = ptx::mbar_wait(ptx::smem_addr(&x.core_full[r]), (uint32_t)((q / C::RING) & 1), p.status);
      if (w) {
        ptx::tc_fence_after();
        const uint32_t img = raddr + (uint32_t)(r * C::IMG);
#pragma unroll
        for (int ks = 0; ks < C::KSLABS; ++ks)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = ptx::sw128_kmajor_desc(vaddr + ks * (NT * 128) + kk * 32);
            const uint64_t bd = ptx::sw128_kmajor_desc(img + ks * (C::N * 128) + kk * 32);
            ptx::mma_bf16(tmem, ad, bd, idesc, (ks == 0 && kk == 0) ? 0u : 1u);
          }
        ptx::mma_commit(ptx::smem_addr(&x.acc_full));
      } else {
        x.abort = 1;
        ptx::mbar_arrive(ptx::smem_addr(&x.acc_full));
      }
    }
    __syncwarp();
    const bool waited = ptx::mbar_wait(ptx::smem_addr(&x.acc_full), (uint32_t)(q & 1), p.status);
    if (!__all_sync(0xffffffffu, waited)) {
      x.abort = 1;
    } else {
      ptx::tc_fence_after();
      // v'[j] = Phi_0 U[0, j] + Phi_1 U[1, j], 32 columns of each half at a time
#pragma unroll
      for (int c = 0; c < CHI; c += (CHI < 32 ? CHI : 32)) {
        uint32_t u0[32], u1[32];
        ptx::tmem_ld_32x32b_x32(lane_base + (uint32_t)c, u0);
        ptx::tmem_ld_32x32b_x32(lane_base + (uint32_t)(CHI + c), u1);
        ptx::tmem_ld_wait();
#pragma unroll
        for (int e = 0; e < 32; ++e)
          if (c + e < CHI) v[c + e] = f0 * __uint_as_float(u0[e]) + f1 * __uint_as_float(u1[e]);
      }
    }
    // every MMA of this step is complete: its ring slot may be refilled
    if (t == 0 && q + C::RING < nsteps && !x.abort) {
      const uint32_t bar = ptx::smem_addr(&x.core_full[r]);
      ptx::mbar_arrive_expect_tx(bar, C::IMG);
      ptx::bulk_copy_g2s(ptx::smem_addr(ring + (size_t)r * C::IMG),
                         p.images + (size_t)step_of(q + C::RING) * C::IMG, C::IMG, bar);
    }
    if (p.mode == 0) {
      float m = 0.0f;
#pragma unroll
      for (int k = 0; k < CHI; ++k) m = fmaxf(m, fabsf(v[k]));
      const float sc = m > 0.0f ? m : 1.0f;
#pragma unroll
      for (int k = 0; k < CHI; ++k) v[k] = v[k] / sc;
      lam += (double)logf(sc);  // float32 log (the FP64 pipe is narrow), float64 running sum
      if (live) p.sc[(int64_t)ts * B + b] = sc;
    } else {
#pragma unroll
      for (int k = 0; k < CHI; ++k) v[k] = v[k] / scl;
    }
    write_row();
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    ok = __syncthreads_and(!x.abort) != 0;
    ptx::tc_fence_after();
  }
  if (live) {
#pragma unroll
    for (int k = 0; k < CHI; ++k) p.state[(int64_t)b * CHI + k] = v[k];
    if (p.mode == 0) p.lam[b] = lam;
  }
  if (warp == 0) {
    if (t == 0) {
      ptx::mma_commit(ptx::smem_addr(&x.final_bar));
      ptx::mbar_wait(ptx::smem_addr(&x.final_bar), 0u, p.status);
    }
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <int CHI>
int launch_chi(const ClsTcParams& p, cudaStream_t s) {
  const size_t smem = sweep_smem_bytes<CHI>();
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(cls_sweep_tc<CHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return TN_ERR_CUDA;
    attr = true;
  }
  cls_sweep_tc<CHI><<<(p.batch + NT - 1) / NT, NT, smem, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace

size_t cls_image_bytes(int chi) {
  const int kpad = chi < 64 ? 64 : chi;
  return (size_t)(2 * chi) * kpad * 2;
}

int cls_pack(const ClsPackParams& p, int steps, cudaStream_t s) {
  if (steps <= 0) return TN_OK;
  cls_pack_images<<<steps, 256, 0, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int cls_sweep_tc_launch(int chi, const ClsTcParams& p, cudaStream_t s) {
  if (p.t_end <= p.t_begin) return TN_OK;
  if (chi == 32) return launch_chi<32>(p, s);
  if (chi == 64) return launch_chi<64>(p, s);
  if (chi == 128) return launch_chi<128>(p, s);
  return TN_ERR_UNSUPPORTED;
}

}  // namespace tn
