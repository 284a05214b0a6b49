// MPS classifier sweeps on the tcgen05 tensor cores: the BF16 and split
// BF16x3 paths of tn_mps_classify / tn_mps_classify_backward (Sec. IV.A).
//
// Forward step of a half-chain for a tile of 128 samples b, with the site's
// core seen as L[k, s, j] (k the incoming bond, j the outgoing one):
//     U[b, (s, j)] = sum_k v_b[k] L[k, s, j]             (M = 128, N = 2 chi, K = chi)
//     u_b[j] = Phi_0(x_b) U[b, (0, j)] + Phi_1(x_b) U[b, (1, j)]
// then u_b is scaled by 2^-e_b, e_b the binary exponent of max_j |u_b[j]|
// (so the largest magnitude lands in [1/2, 1)), and e_b ln 2 is added to the
// sample's log-scale. A power of two keeps the scaling exact: the scaled
// vector and its bf16 rounding are the unscaled ones with a shifted exponent.
//
// Adjoint step (walking back from the label core), with g the adjoint of the
// vector leaving the step and sc_b = 2^e_b the forward's scale:
//     x_b[(s, j)] = Phi_s(x_b) g_b[j] / sc_b
//     g'_b[k] = sum_{(s, j)} x_b[(s, j)] L[k, s, j]        (M = 128, N = chi, K = 2 chi)
//     dL[k, s, j] += sum_b v_b[k] x_b[(s, j)]              (M = 2 chi, N = chi, K = 128)
// with v_b the forward vector entering the step. The gradient product runs in
// the same CTA on the same staged x (the 128-byte-swizzled K-major x tile of
// the first product is the MN-major operand of the second) and the v tile the
// recomputing forward wrote, and is added to the step's float32 gradient with
// coalesced reductions (one 128-byte line per warp instruction).
//
// Split BF16x3 (Henry, Tang and Heinecke, ARITH 2019): every operand is
// hi = bf16(x) plus lo = bf16(x - hi) and each product is hi*hi + lo*hi +
// hi*lo in the float32 accumulator.
//
// One launch covers both half-chains (CTA = (half, tile)). A CTA has 256
// epilogue threads, two per sample (thread r owns TMEM lane r % 128 and half
// of the columns), and one producer warp that streams the packed core slabs
// (and, in the adjoint, the v tiles) into shared-memory rings with 1-D bulk
// async copies. Thread 0 issues the MMAs. Every mbarrier wait is bounded; a
// CTA that gives up records TN_ERR_TIMEOUT, lets its copies land, frees its
// TMEM and returns.
#include <cuda_bf16.h>
#include <math.h>

#include "classifier_tc.h"
#include "ptx.cuh"

namespace tn {
namespace {

constexpr int TS = CLS_TILE;         // samples per tile
constexpr int NEPI = 2 * TS;         // epilogue threads
constexpr int NTHREADS = NEPI + 32;  // + the producer warp
constexpr int PXS = 16;              // steps of pixels staged at once
constexpr int SLAB_V = TS * 128;     // one 64-column slab of a 128-row tile (bytes)
constexpr int SMEM_BUDGET = 200 * 1024;

constexpr int pow2ceil(int x) {
  int p = 32;
  while (p < x) p *= 2;
  return p;
}

template <int CHI, int SPLIT>
struct Cfg {
  static constexpr int PARTS = SPLIT ? 2 : 1;
  static constexpr int KPAD = CHI < 64 ? 64 : CHI;  // sweep vector, padded to whole slabs
  static constexpr int KSL = KPAD / 64;
  static constexpr int VT = KSL * SLAB_V;           // one part of a vector tile
  static constexpr int VTS = VT * PARTS;
  static constexpr int HC = CHI / 2;                // columns per epilogue thread
  // forward: image rows (s, j), K = k
  static constexpr int FN = 2 * CHI;
  static constexpr int FSLAB = FN * 128;
  static constexpr int FSET = FSLAB * PARTS;
  static constexpr int FRING_RAW = (SMEM_BUDGET - VTS) / FSET;
  static constexpr int FRING = FRING_RAW > 8 ? 8 : FRING_RAW;
  static constexpr uint32_t FCOLS = FN < 32 ? 32 : FN;
  // adjoint: x tile rows b, columns m = (s, j); image rows k, K = m
  static constexpr int XSL = 2 * CHI / 64;
  static constexpr int XPART = (XSL + (CHI == 32 ? 1 : 0)) * SLAB_V;  // + a zero M half at chi = 32
  static constexpr int XTS = XPART * PARTS;
  static constexpr int ASLAB = CHI * 128;
  static constexpr int ASET = ASLAB * PARTS;
  static constexpr int MH = (2 * CHI + 127) / 128;  // M halves of the gradient product
  static constexpr int ARING_RAW = (SMEM_BUDGET - XTS - 2 * VTS) / ASET;
  static constexpr int ARING = ARING_RAW > 8 ? 8 : ARING_RAW;
  static constexpr int A2OFF = CHI < 64 ? 64 : CHI;  // TMEM column of the gradient accumulator
  // two gradient accumulators when they fit (step q's is drained while step
  // q + 1's products run), else one
  static constexpr int A2BUF = A2OFF + 2 * MH * KPAD <= 512 ? 2 : 1;
  static constexpr uint32_t ACOLS = (uint32_t)pow2ceil(A2OFF + A2BUF * MH * KPAD);
};

struct __align__(8) Bars {
  uint64_t full[8];
  uint64_t empty[8];
  uint64_t vfull[2];
  uint64_t vempty[2];
  uint64_t acc_full;
  uint64_t final_bar;
  uint32_t tmem_base;
  int32_t abort;
};

struct StageTail {
  float px[PXS][TS];
  float pmax[2][TS];
  Bars bars;
};

// K-major 128-byte swizzle: byte offset of 16-byte chunk g (of 8) of row r
// inside a 64-column slab.
__device__ __forceinline__ uint32_t sw128(int r, int g) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// hi = bf16(a), lo = bf16(a - hi), two values at a time
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  hi = bf16x2_bits(h);
  lo = bf16x2_bits(__floats2bfloat162_rn(a - hf.x, b - hf.y));
}

// Writes 8 values as one 16-byte chunk of every part of a K-major tile
// (part 1 = the lo part, `part_bytes` after part 0).
template <int PARTS>
__device__ __forceinline__ void put8(uint8_t* tile, int part_bytes, uint32_t off, const float* v) {
  uint4 h, l;
  split_pair(v[0], v[1], h.x, l.x);
  split_pair(v[2], v[3], h.y, l.y);
  split_pair(v[4], v[5], h.z, l.z);
  split_pair(v[6], v[7], h.w, l.w);
  *reinterpret_cast<uint4*>(tile + off) = h;
  if (PARTS == 2) *reinterpret_cast<uint4*>(tile + part_bytes + off) = l;
}

// 2^-e and 2^e as floats (e in [-126, 126]).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Binary exponent e with m * 2^-e in [1/2, 1) (0 for m == 0), clamped so that
// 2^e and 2^-e are normal floats.
__device__ __forceinline__ int scale_exponent(float m) {
  if (!(m > 0.0f)) return 0;
  const int ex = (__float_as_int(m) >> 23) & 0xff;
  int e = ex == 0 ? -126 : ex - 126;
  return e < -126 ? -126 : (e > 126 ? 126 : e);
}

__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// 1-D bulk async copy shared -> global (bulk group of this thread).
__device__ __forceinline__ void bulk_copy_s2g(void* dst, uint32_t src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src_smem), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t* r) {
  if constexpr (N == 32) ptx::tmem_ld_32x32b_x32(taddr, r);
  else ptx::tmem_ld_32x32b_x16(taddr, r);
}

__device__ __forceinline__ void epi_barrier() { ptx::named_barrier(1, NEPI); }

// Stages pixels of steps [q0, q0 + PXS) of this tile (zeros past the end).
template <class SiteOf>
__device__ __forceinline__ void stage_pixels(float (&px)[PXS][TS], const float* pixels, int n, int B, int b0, int q0,
                                             int nsteps, SiteOf site_of) {
  for (int e = threadIdx.x; e < PXS * TS; e += NEPI) {
    const int qq = e % PXS, bb = e / PXS;
    float val = 0.0f;
    if (q0 + qq < nsteps && b0 + bb < B) val = __ldg(pixels + (int64_t)(b0 + bb) * n + site_of(q0 + qq));
    px[qq][bb] = val;
  }
}

// ------------------------------------------------------------------ packing
// Value L[k, s, j] of the core of step t: the left half reads A[k, s, j],
// the right half (swept from the chain's right end) A[j, s, k].
__global__ void cls_pack_kernel(const __grid_constant__ ClsPackParams p) {
  const int t = blockIdx.x, h = blockIdx.y;
  if (t >= p.T[h]) return;
  const int site = h == 0 ? t : p.n - 1 - t;
  const int Da = p.bond[site], Dc = p.bond[site + 1];
  const int Din = h == 0 ? Da : Dc, Dout = h == 0 ? Dc : Da;
  const float* __restrict__ A = p.core[site];
  const int chi = p.chi, parts = p.split ? 2 : 1;
  uint8_t* img = p.images[h] + (size_t)t * p.step_bytes;
  auto value = [&](int k, int s, int j) -> float {
    if (k >= Din || j >= Dout) return 0.0f;
    return h == 0 ? __ldg(A + ((int64_t)k * 2 + s) * Dc + j) : __ldg(A + ((int64_t)j * 2 + s) * Dc + k);
  };
  const int kpad = chi < 64 ? 64 : chi;
  // rows R and K extent of the image kind; a 16-byte chunk is 8 consecutive K of one row
  const int R = p.adjoint ? chi : 2 * chi;
  const int KX = p.adjoint ? 2 * chi : kpad;
  const int slab_bytes = R * 128;
  const int chunks = R * (KX / 8);
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    const int row = c % R, kg = c / R;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kk = kg * 8 + e;
      if (p.adjoint) v[e] = value(row, kk / chi, kk % chi);  // row k, K index m = (s, j)
      else v[e] = value(kk, row / chi, row % chi);            // row (s, j), K index k
    }
    const int ks = kg >> 3, g = kg & 7;
    uint8_t* dst = img + (size_t)ks * parts * slab_bytes + sw128(row, g);
    uint4 hh, ll;
    split_pair(v[0], v[1], hh.x, ll.x);
    split_pair(v[2], v[3], hh.y, ll.y);
    split_pair(v[4], v[5], hh.z, ll.z);
    split_pair(v[6], v[7], hh.w, ll.w);
    *reinterpret_cast<uint4*>(dst) = hh;
    if (p.split) *reinterpret_cast<uint4*>(dst + slab_bytes) = ll;
  }
}

// ----------------------------------------------------------------- forward
template <int CHI, int SPLIT>
constexpr size_t fwd_smem_bytes() {
  using C = Cfg<CHI, SPLIT>;
  return 1024 + (size_t)C::VTS + (size_t)C::FRING * C::FSET + sizeof(StageTail);
}

template <int CHI, int SPLIT>
__global__ void __launch_bounds__(NTHREADS, 1) cls_fwd_tc(const __grid_constant__ ClsTcParams p) {
  using C = Cfg<CHI, SPLIT>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* vt = base;
  uint8_t* ring = base + C::VTS;
  StageTail& st = *reinterpret_cast<StageTail*>(ring + (size_t)C::FRING * C::FSET);
  Bars& x = st.bars;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int h = blockIdx.x / p.ntiles, tile = blockIdx.x % p.ntiles;
  const int B = p.batch, b0 = tile * TS;
  const int t0 = p.t_begin[h];
  const int nsteps = p.t_end[h] - t0;
  const int n = p.n;
  auto site_of = [&](int q) { return p.half_site[h] + p.half_dir[h] * (t0 + q); };
  const int nslabs = nsteps * C::KSL;

  if (tid == 0) {
    for (int i = 0; i < C::FRING; ++i) {
      ptx::mbar_init(ptx::smem_addr(&x.full[i]), 1);
      ptx::mbar_init(ptx::smem_addr(&x.empty[i]), 1);
    }
    ptx::mbar_init(ptx::smem_addr(&x.acc_full), 2);  // MMA commit + the vector-image store's read
    ptx::mbar_init(ptx::smem_addr(&x.final_bar), 1);
    x.abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_addr(&x.tmem_base), C::FCOLS);
    ptx::tmem_relinquish();
  }
  // zero the vector tile (padding columns stay zero)
  for (int i = tid; i < C::VTS / 16; i += NTHREADS) reinterpret_cast<uint4*>(vt)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();

  if (warp == NEPI / 32) {
    // ---------------- producer: core slabs into the ring
    if ((tid & 31) == 0) {
      int g = 0;
      for (; g < nslabs; ++g) {
        const int slot = g % C::FRING;
        if (g >= C::FRING &&
            !ptx::mbar_wait(ptx::smem_addr(&x.empty[slot]), (uint32_t)(((g / C::FRING) - 1) & 1), p.status)) {
          x.abort = 1;
          break;
        }
        if (*(volatile int32_t*)&x.abort) break;
        const int q = g / C::KSL, ks = g % C::KSL;
        const uint32_t bar = ptx::smem_addr(&x.full[slot]);
        ptx::mbar_arrive_expect_tx(bar, C::FSET);
        ptx::bulk_copy_g2s(ptx::smem_addr(ring + (size_t)slot * C::FSET),
                           p.images[h] + ((size_t)(t0 + q) * C::KSL + ks) * C::FSET, C::FSET, bar);
      }
      // let every copy issued land before the CTA can leave
      for (int gg = g - C::FRING < 0 ? 0 : g - C::FRING; gg < g; ++gg)
        ptx::mbar_wait(ptx::smem_addr(&x.full[gg % C::FRING]), (uint32_t)((gg / C::FRING) & 1), p.status);
    }
    __syncwarp();
  } else {
    // ---------------- epilogue threads (and thread 0: the MMA issuer)
    const int r = tid & (TS - 1), hc = tid >> 7;  // sample row, column half
    const int b = b0 + r;
    const bool live = b < B;
    const int c0 = hc * C::HC;  // first column of this thread
    float v[C::HC];
#pragma unroll
    for (int k = 0; k < C::HC; ++k) v[k] = live ? p.state[h][(int64_t)b * CHI + c0 + k] : 0.0f;
    double lam0 = (live && hc == 0) ? p.lam[h][b] : 0.0;
    int lam_e = 0;
    // scale of the vector in the tile not yet applied (deferred mode)
    int e_prev = 0;
    const bool defer = p.vseg[h] == nullptr;
    auto write_vtile = [&]() {
#pragma unroll
      for (int g8 = 0; g8 < C::HC / 8; ++g8) {
        const int col = c0 + g8 * 8;
        put8<C::PARTS>(vt, C::VT, (uint32_t)((col >> 6) * SLAB_V) + sw128(r, (col >> 3) & 7), &v[g8 * 8]);
      }
    };
    write_vtile();
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    epi_barrier();
    ptx::tc_fence_after();
    const uint32_t tmem = x.tmem_base;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t vaddr = ptx::smem_addr(vt), raddr = ptx::smem_addr(ring);
    constexpr uint32_t idesc = ptx::idesc_bf16_f32(128, C::FN);
    constexpr int LDN = C::HC >= 32 ? 32 : 16;

    bool ok = true;
    int gs = 0;  // slabs consumed (thread 0)
    // thread 0: the MMAs of step qq (issued as soon as the tile holds its vector)
    auto issue = [&](int qq) {
      // the vector entering step t0 + qq, for the adjoint's gradient product
      if (p.vseg[h]) bulk_copy_s2g(p.vseg[h] + ((size_t)qq * p.ntiles + tile) * C::VTS, vaddr, C::VTS);
      bool w = true;
      for (int ks = 0; ks < C::KSL && w; ++ks, ++gs) {
        const int slot = gs % C::FRING;
        w = ptx::mbar_wait(ptx::smem_addr(&x.full[slot]), (uint32_t)((gs / C::FRING) & 1), p.status);
        if (!w) break;
        ptx::tc_fence_after();
        const uint32_t bs = raddr + (uint32_t)(slot * C::FSET);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t ao = vaddr + (uint32_t)(ks * SLAB_V + kk * 32);
          const uint64_t ah = ptx::sw128_kmajor_desc(ao), bh = ptx::sw128_kmajor_desc(bs + kk * 32);
          ptx::mma_bf16(tmem, ah, bh, idesc, (ks | kk) ? 1u : 0u);
          if (SPLIT) {
            ptx::mma_bf16(tmem, ptx::sw128_kmajor_desc(ao + C::VT), bh, idesc, 1u);
            ptx::mma_bf16(tmem, ah, ptx::sw128_kmajor_desc(bs + C::FSLAB + kk * 32), idesc, 1u);
          }
        }
        ptx::mma_commit(ptx::smem_addr(&x.empty[slot]));
      }
      if (w) ptx::mma_commit(ptx::smem_addr(&x.acc_full));
      else {
        x.abort = 1;
        ptx::mbar_arrive(ptx::smem_addr(&x.acc_full));
      }
      bulk_wait_read();
      ptx::mbar_arrive(ptx::smem_addr(&x.acc_full));
    };
    if (nsteps > 0 && tid == 0) issue(0);
    __syncwarp();
    for (int q = 0; q < nsteps && ok; ++q) {
      const int t = t0 + q;
      // pixels of the next PXS steps (the epilogue threads only)
      if (q % PXS == 0) {
        stage_pixels(st.px, p.pixels, n, B, b0, q, nsteps, site_of);
        epi_barrier();
      }
      // keep the float32 vector entering step t (v holds it times 2^e_prev)
      if (p.store[h] && live && ((t - p.store_base[h]) % p.store_every) == 0) {
        float* dst = p.store[h] + ((int64_t)((t - p.store_base[h]) / p.store_every) * B + b) * CHI + c0;
        const float ip = pow2f(-e_prev);
#pragma unroll
        for (int k = 0; k < C::HC; k += 4)
          *reinterpret_cast<float4*>(dst + k) = make_float4(v[k] * ip, v[k + 1] * ip, v[k + 2] * ip, v[k + 3] * ip);
      }
      const float xp = st.px[q % PXS][r];
      const float f0 = cospif(0.5f * xp), f1 = sinpif(0.5f * xp);
      const bool waited = ptx::mbar_wait(ptx::smem_addr(&x.acc_full), (uint32_t)(q & 1), p.status);
      if (!__all_sync(0xffffffffu, waited)) x.abort = 1;
      if (waited) {
        ptx::tc_fence_after();
        // the MMA read v_t 2^e_prev: the step's output times 2^-e_prev is u_t itself (exact)
        const float ip = pow2f(-e_prev);
        const float g0 = f0 * ip, g1 = f1 * ip;
#pragma unroll
        for (int c = 0; c < C::HC; c += LDN) {
          uint32_t u0[LDN], u1[LDN];
          tmem_ld<LDN>(lane_base + (uint32_t)(c0 + c), u0);
          tmem_ld<LDN>(lane_base + (uint32_t)(CHI + c0 + c), u1);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < LDN; ++e) v[c + e] = g0 * __uint_as_float(u0[e]) + g1 * __uint_as_float(u1[e]);
        }
      }
      // the step's scale 2^e_t from the sample's largest |u_t| over both
      // column halves. Without a vector-image store it is applied one step
      // late (the next MMA reads u_t itself, bf16(u_t) = bf16(v_{t+1}) 2^e_t),
      // so the exchange runs while that MMA does; the recomputation keeps
      // the normalised v_{t+1} in the tile it stores for the gradients.
      auto exchange = [&]() {
        float m = 0.0f;
#pragma unroll
        for (int k = 0; k < C::HC; ++k) m = fmaxf(m, fabsf(v[k]));
        st.pmax[hc][r] = m;
        ptx::named_barrier(2 + (warp & 3), 64);
        m = fmaxf(st.pmax[0][r], st.pmax[1][r]);
        const int e = scale_exponent(m);
        lam_e += e;
        if (hc == 0 && live) p.sc[h][(int64_t)t * B + b] = pow2f(e);
        return e;
      };
      if (!defer) {
        const float inv = pow2f(-exchange());
#pragma unroll
        for (int k = 0; k < C::HC; ++k) v[k] *= inv;
      }
      write_vtile();
      ptx::fence_proxy_async_smem();
      ptx::tc_fence_before();
      ok = ptx::named_barrier_or(1, NEPI, *(volatile int32_t*)&x.abort != 0) == false;
      ptx::tc_fence_after();
      if (tid == 0 && ok && q + 1 < nsteps) issue(q + 1);
      __syncwarp();
      if (defer) e_prev = exchange();
    }
    {
      const float ip = pow2f(-e_prev);
#pragma unroll
      for (int k = 0; k < C::HC; ++k) v[k] *= ip;
    }
    if (live) {
#pragma unroll
      for (int k = 0; k < C::HC; k += 4)
        *reinterpret_cast<float4*>(p.state[h] + (int64_t)b * CHI + c0 + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
      if (hc == 0) p.lam[h][b] = lam0 + (double)lam_e * 0.69314718055994530942;
    }
    if (tid == 0) {
      ptx::mma_commit(ptx::smem_addr(&x.final_bar));
      ptx::mbar_wait(ptx::smem_addr(&x.final_bar), 0u, p.status);
      bulk_wait_all();
    }
    __syncwarp();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(x.tmem_base, C::FCOLS);
  }
}

// ----------------------------------------------------------------- adjoint
template <int CHI, int SPLIT>
constexpr size_t adj_smem_bytes() {
  using C = Cfg<CHI, SPLIT>;
  return 1024 + (size_t)C::XTS + 2 * (size_t)C::VTS + (size_t)(C::ARING > 0 ? C::ARING : 0) * C::ASET +
         sizeof(StageTail);
}

template <int CHI, int SPLIT>
__global__ void __launch_bounds__(NTHREADS, 1) cls_adj_tc(const __grid_constant__ ClsTcParams p) {
  using C = Cfg<CHI, SPLIT>;
  static_assert(C::ARING >= 2, "adjoint staging does not fit in shared memory");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* xt = base;                      // x tile parts: [x slabs (+ zero slab)] per part
  uint8_t* vring = base + C::XTS;          // 2 v tiles
  uint8_t* cring = vring + 2 * C::VTS;     // adjoint core slabs
  StageTail& st = *reinterpret_cast<StageTail*>(cring + (size_t)C::ARING * C::ASET);
  Bars& x = st.bars;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int h = blockIdx.x / p.ntiles, tile = blockIdx.x % p.ntiles;
  const int B = p.batch, b0 = tile * TS;
  const int t0 = p.t_begin[h], t1 = p.t_end[h];
  const int nsteps = t1 - t0;
  const int n = p.n;
  auto step_t = [&](int q) { return t1 - 1 - q; };
  auto site_of = [&](int q) { return p.half_site[h] + p.half_dir[h] * step_t(q); };

  if (tid == 0) {
    for (int i = 0; i < C::ARING; ++i) {
      ptx::mbar_init(ptx::smem_addr(&x.full[i]), 1);
      ptx::mbar_init(ptx::smem_addr(&x.empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(ptx::smem_addr(&x.vfull[i]), 1);
      ptx::mbar_init(ptx::smem_addr(&x.vempty[i]), 1);
    }
    ptx::mbar_init(ptx::smem_addr(&x.acc_full), 1);
    ptx::mbar_init(ptx::smem_addr(&x.final_bar), 1);
    x.abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_addr(&x.tmem_base), C::ACOLS);
    ptx::tmem_relinquish();
  }
  for (int i = tid; i < C::XTS / 16; i += NTHREADS) reinterpret_cast<uint4*>(xt)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();

  if (warp == NEPI / 32) {
    // ---------------- producer: per step the core slabs, then the v tile
    if ((tid & 31) == 0) {
      int g = 0, q = 0;
      bool stop = false;
      for (; q < nsteps && !stop; ++q) {
        const int t = step_t(q);
        for (int ks = 0; ks < C::XSL; ++ks, ++g) {
          const int slot = g % C::ARING;
          if ((g >= C::ARING &&
               !ptx::mbar_wait(ptx::smem_addr(&x.empty[slot]), (uint32_t)(((g / C::ARING) - 1) & 1), p.status)) ||
              *(volatile int32_t*)&x.abort) {
            x.abort = 1;
            stop = true;
            break;
          }
          const uint32_t bar = ptx::smem_addr(&x.full[slot]);
          ptx::mbar_arrive_expect_tx(bar, C::ASET);
          ptx::bulk_copy_g2s(ptx::smem_addr(cring + (size_t)slot * C::ASET),
                             p.images[h] + ((size_t)t * C::XSL + ks) * C::ASET, C::ASET, bar);
        }
        if (stop) break;
        const int vs = q & 1;
        if ((q >= 2 && !ptx::mbar_wait(ptx::smem_addr(&x.vempty[vs]), (uint32_t)(((q >> 1) - 1) & 1), p.status)) ||
            *(volatile int32_t*)&x.abort) {
          x.abort = 1;
          break;
        }
        const uint32_t bar = ptx::smem_addr(&x.vfull[vs]);
        ptx::mbar_arrive_expect_tx(bar, C::VTS);
        ptx::bulk_copy_g2s(ptx::smem_addr(vring + (size_t)vs * C::VTS),
                           p.vseg[h] + ((size_t)(t - t0) * p.ntiles + tile) * C::VTS, C::VTS, bar);
      }
      // let every copy issued land before the CTA can leave
      for (int gg = g - C::ARING < 0 ? 0 : g - C::ARING; gg < g; ++gg)
        ptx::mbar_wait(ptx::smem_addr(&x.full[gg % C::ARING]), (uint32_t)((gg / C::ARING) & 1), p.status);
      // v tiles issued: those of steps 0 .. q-1 (a break leaves q at the step not issued)
      for (int qq = q - 2 < 0 ? 0 : q - 2; qq < q; ++qq)
        ptx::mbar_wait(ptx::smem_addr(&x.vfull[qq & 1]), (uint32_t)((qq >> 1) & 1), p.status);
    }
    __syncwarp();
  } else {
    const int r = tid & (TS - 1), hc = tid >> 7;
    const int b = b0 + r;
    const bool live = b < B;
    const int c0 = hc * C::HC;
    float g[C::HC];
#pragma unroll
    for (int k = 0; k < C::HC; ++k) g[k] = live ? p.state[h][(int64_t)b * CHI + c0 + k] : 0.0f;
    // x of the step q: Phi_s(x at that step's site) g / sc into columns (s, c0 + k)
    auto write_xtile = [&](int q) {
      const float xp = st.px[q % PXS][r];
      const float f[2] = {cospif(0.5f * xp), sinpif(0.5f * xp)};
      const float scl = live ? p.sc[h][(int64_t)step_t(q) * B + b] : 1.0f;
      const float inv = __frcp_rn(scl);  // scales are powers of two: exact
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int g8 = 0; g8 < C::HC / 8; ++g8) {
          float w[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) w[e] = f[s] * g[g8 * 8 + e] * inv;
          const int col = s * CHI + c0 + g8 * 8;
          put8<C::PARTS>(xt, C::XPART, (uint32_t)((col >> 6) * SLAB_V) + sw128(r, (col >> 3) & 7), w);
        }
    };
    stage_pixels(st.px, p.pixels, n, B, b0, 0, nsteps, site_of);
    epi_barrier();
    if (nsteps > 0) write_xtile(0);
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    epi_barrier();
    ptx::tc_fence_after();
    const uint32_t tmem = x.tmem_base;
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t xaddr = ptx::smem_addr(xt), vaddr = ptx::smem_addr(vring), caddr = ptx::smem_addr(cring);
    constexpr uint32_t idesc1 = ptx::idesc_bf16_f32(128, CHI);
    constexpr uint32_t idesc2 = ptx::idesc_bf16_f32(128, C::KPAD, 1, 1);
    constexpr int LDN = C::HC >= 32 ? 32 : 16;
    constexpr int GLD = C::KPAD / 2 >= 32 ? 32 : 16;  // gradient columns per TMEM load
    const int mrow = r;  // gradient row (x column) of this lane in M half 0
    // this tile's share of step t's core gradient, from accumulator `buf`
    auto drain_grad = [&](int t, int buf) {
      float* gbase = p.grad[h] + (size_t)t * CHI * 2 * CHI;
#pragma unroll
      for (int mh = 0; mh < C::MH; ++mh) {
        const int m = mh * 128 + mrow;
        if (m < 2 * CHI) {
#pragma unroll
          for (int c = 0; c < C::KPAD / 2; c += GLD) {
            const int k0 = hc * (C::KPAD / 2) + c;
            if (k0 < CHI) {
              uint32_t u[GLD];
              tmem_ld<GLD>(lane_base + (uint32_t)(C::A2OFF + buf * C::MH * C::KPAD + mh * C::KPAD + k0), u);
              ptx::tmem_ld_wait();
#pragma unroll
              for (int e = 0; e < GLD; ++e)
                if (k0 + e < CHI) red_add(gbase + (size_t)(k0 + e) * 2 * CHI + m, __uint_as_float(u[e]));
            }
          }
        }
      }
    };

    bool ok = true;
    int gs = 0;
    // thread 0: both products of step qq (issued as soon as the x tile holds its operand)
    auto issue = [&](int qq) {
      bool w = true;
      // g'[b, k] = sum_m x[b, m] L[k, m]
      for (int ks = 0; ks < C::XSL && w; ++ks, ++gs) {
        const int slot = gs % C::ARING;
        w = ptx::mbar_wait(ptx::smem_addr(&x.full[slot]), (uint32_t)((gs / C::ARING) & 1), p.status);
        if (!w) break;
        ptx::tc_fence_after();
        const uint32_t bs = caddr + (uint32_t)(slot * C::ASET);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t ao = xaddr + (uint32_t)(ks * SLAB_V + kk * 32);
          const uint64_t ah = ptx::sw128_kmajor_desc(ao), bh = ptx::sw128_kmajor_desc(bs + kk * 32);
          ptx::mma_bf16(tmem, ah, bh, idesc1, (ks | kk) ? 1u : 0u);
          if (SPLIT) {
            ptx::mma_bf16(tmem, ptx::sw128_kmajor_desc(ao + C::XPART), bh, idesc1, 1u);
            ptx::mma_bf16(tmem, ah, ptx::sw128_kmajor_desc(bs + C::ASLAB + kk * 32), idesc1, 1u);
          }
        }
        ptx::mma_commit(ptx::smem_addr(&x.empty[slot]));
      }
      // dL[m, k] = sum_b x[b, m] v[b, k]: both operands MN-major (the
      // K-major x tile read transposed; the v tile as the forward wrote it)
      const int vs = qq & 1;
      if (w) w = ptx::mbar_wait(ptx::smem_addr(&x.vfull[vs]), (uint32_t)((qq >> 1) & 1), p.status);
      if (w) {
        ptx::tc_fence_after();
        const uint32_t vb = vaddr + (uint32_t)(vs * C::VTS);
#pragma unroll
        for (int mh = 0; mh < C::MH; ++mh) {
          const uint32_t d = tmem + (uint32_t)(C::A2OFF + ((qq & 1) % C::A2BUF) * C::MH * C::KPAD + mh * C::KPAD);
#pragma unroll
          for (int kk = 0; kk < TS / 16; ++kk) {
            const uint32_t ao = xaddr + (uint32_t)(mh * 2 * SLAB_V + kk * 2048);
            const uint32_t bo = vb + (uint32_t)(kk * 2048);
            const uint64_t ah = ptx::sw128_mnmajor_desc(ao, SLAB_V, 1024);
            const uint64_t bh = ptx::sw128_mnmajor_desc(bo, SLAB_V, 1024);
            ptx::mma_bf16(d, ah, bh, idesc2, kk ? 1u : 0u);
            if (SPLIT) {
              ptx::mma_bf16(d, ptx::sw128_mnmajor_desc(ao + C::XPART, SLAB_V, 1024), bh, idesc2, 1u);
              ptx::mma_bf16(d, ah, ptx::sw128_mnmajor_desc(bo + C::VT, SLAB_V, 1024), idesc2, 1u);
            }
          }
        }
        ptx::mma_commit(ptx::smem_addr(&x.vempty[vs]));
        ptx::mma_commit(ptx::smem_addr(&x.acc_full));
      } else {
        x.abort = 1;
        ptx::mbar_arrive(ptx::smem_addr(&x.acc_full));
      }
    };
    if (nsteps > 0 && tid == 0) issue(0);
    __syncwarp();
    for (int q = 0; q < nsteps && ok; ++q) {
      const int t = step_t(q);
      // pixels of steps q + 1 .. q + PXS (the x of the next step needs them)
      if ((q + 1) % PXS == 0 && q + 1 < nsteps) {
        stage_pixels(st.px, p.pixels, n, B, b0, q + 1, nsteps, site_of);
        epi_barrier();
      }
      const bool waited = ptx::mbar_wait(ptx::smem_addr(&x.acc_full), (uint32_t)(q & 1), p.status);
      if (!__all_sync(0xffffffffu, waited)) x.abort = 1;
      if (waited) {
        ptx::tc_fence_after();
#pragma unroll
        for (int c = 0; c < C::HC; c += LDN) {
          uint32_t u[LDN];
          tmem_ld<LDN>(lane_base + (uint32_t)(c0 + c), u);
          ptx::tmem_ld_wait();
#pragma unroll
          for (int e = 0; e < LDN; ++e) g[c + e] = __uint_as_float(u[e]);
        }
        if (C::A2BUF == 1) drain_grad(t, 0);
        if (q + 1 < nsteps) write_xtile(q + 1);
      }
      ptx::fence_proxy_async_smem();
      ptx::tc_fence_before();
      ok = ptx::named_barrier_or(1, NEPI, *(volatile int32_t*)&x.abort != 0) == false;
      ptx::tc_fence_after();
      if (tid == 0 && ok && q + 1 < nsteps) issue(q + 1);
      __syncwarp();
      // with two accumulators this step's gradient is drained while the next
      // step's products run (its buffer is rewritten two steps later, after
      // the next barrier)
      if (C::A2BUF == 2 && waited && ok) drain_grad(t, q & 1);
    }
    if (live) {
#pragma unroll
      for (int k = 0; k < C::HC; k += 4)
        *reinterpret_cast<float4*>(p.state[h] + (int64_t)b * CHI + c0 + k) = make_float4(g[k], g[k + 1], g[k + 2], g[k + 3]);
    }
    if (tid == 0) {
      ptx::mma_commit(ptx::smem_addr(&x.final_bar));
      ptx::mbar_wait(ptx::smem_addr(&x.final_bar), 0u, p.status);
    }
    __syncwarp();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(x.tmem_base, C::ACOLS);
  }
}

// dcore[site] from the step's accumulated gradient G[t][k][(s, j)]: the left
// half's core is L itself (A[k, s, j]), the right half's its transpose
// (A[j, s, k]).
__global__ void cls_scatter_kernel(const __grid_constant__ ClsScatterParams p) {
  int t = blockIdx.x, h = 0;
  if (t >= p.T[0]) {
    t -= p.T[0];
    h = 1;
  }
  const int site = h == 0 ? t : p.n - 1 - t;
  const int Da = p.bond[site], Dc = p.bond[site + 1], chi = p.chi;
  const float* __restrict__ G = p.grad[h] + (size_t)t * chi * 2 * chi;
  float* __restrict__ d = p.dcore[site];
  const int total = Da * 2 * Dc;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int c = i % Dc, s = (i / Dc) & 1, a = i / (2 * Dc);
    d[i] = h == 0 ? G[(size_t)a * 2 * chi + s * chi + c] : G[(size_t)c * 2 * chi + s * chi + a];
  }
}

template <int CHI, int SPLIT>
int launch_fwd(const ClsTcParams& p, cudaStream_t s) {
  const size_t smem = fwd_smem_bytes<CHI, SPLIT>();
  static std::atomic<uint64_t> attr{0};
  if (!smem_limit_once((const void*)cls_fwd_tc<CHI, SPLIT>, smem, &attr)) return TN_ERR_CUDA;
  cls_fwd_tc<CHI, SPLIT><<<2 * p.ntiles, NTHREADS, smem, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

template <int CHI, int SPLIT>
int launch_adj(const ClsTcParams& p, cudaStream_t s) {
  if constexpr (Cfg<CHI, SPLIT>::ARING < 2) {
    return TN_ERR_UNSUPPORTED;
  } else {
    const size_t smem = adj_smem_bytes<CHI, SPLIT>();
    static std::atomic<uint64_t> attr{0};
    if (!smem_limit_once((const void*)cls_adj_tc<CHI, SPLIT>, smem, &attr)) return TN_ERR_CUDA;
    cls_adj_tc<CHI, SPLIT><<<2 * p.ntiles, NTHREADS, smem, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
  }
}

}  // namespace

size_t cls_fwd_image_bytes(int chi, int split) {
  const int kpad = chi < 64 ? 64 : chi;
  return (size_t)(2 * chi) * kpad * 2 * (split ? 2 : 1);
}

size_t cls_adj_image_bytes(int chi, int split) { return (size_t)chi * (2 * chi) * 2 * (split ? 2 : 1); }

size_t cls_vtile_bytes(int chi, int split) {
  const int kpad = chi < 64 ? 64 : chi;
  return (size_t)TS * kpad * 2 * (split ? 2 : 1);
}

int cls_pack(const ClsPackParams& p, cudaStream_t s) {
  const int steps = p.T[0] > p.T[1] ? p.T[0] : p.T[1];
  if (steps <= 0) return TN_OK;
  cls_pack_kernel<<<dim3((unsigned)steps, 2), 256, 0, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int cls_fwd_tc_launch(int chi, int split, const ClsTcParams& p, cudaStream_t s) {
  if (p.t_end[0] <= p.t_begin[0] && p.t_end[1] <= p.t_begin[1]) return TN_OK;
  if (chi == 32) return split ? launch_fwd<32, 1>(p, s) : launch_fwd<32, 0>(p, s);
  if (chi == 64) return split ? launch_fwd<64, 1>(p, s) : launch_fwd<64, 0>(p, s);
  if (chi == 128) return split ? launch_fwd<128, 1>(p, s) : launch_fwd<128, 0>(p, s);
  return TN_ERR_UNSUPPORTED;
}

bool cls_adj_tc_supported(int chi, int split) {
  if (chi == 32) return split ? Cfg<32, 1>::ARING >= 2 : Cfg<32, 0>::ARING >= 2;
  if (chi == 64) return split ? Cfg<64, 1>::ARING >= 2 : Cfg<64, 0>::ARING >= 2;
  if (chi == 128) return split ? Cfg<128, 1>::ARING >= 2 : Cfg<128, 0>::ARING >= 2;
  return false;
}

int cls_adj_tc_launch(int chi, int split, const ClsTcParams& p, cudaStream_t s) {
  if (p.t_end[0] <= p.t_begin[0] && p.t_end[1] <= p.t_begin[1]) return TN_OK;
  if (chi == 32) return split ? launch_adj<32, 1>(p, s) : launch_adj<32, 0>(p, s);
  if (chi == 64) return split ? launch_adj<64, 1>(p, s) : launch_adj<64, 0>(p, s);
  if (chi == 128) return split ? launch_adj<128, 1>(p, s) : launch_adj<128, 0>(p, s);
  return TN_ERR_UNSUPPORTED;
}

int cls_scatter_grad(const ClsScatterParams& p, cudaStream_t s) {
  const int blocks = p.T[0] + p.T[1];
  if (blocks <= 0) return TN_OK;
  cls_scatter_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace tn
