// Persistent energy sweep: <psi|H|psi> and <psi|psi> of one MPS (Sec. II,
// Fig. 3a) in ONE cooperative launch for the whole chain. Every CTA stays
// resident from the first site to the last; the environment, its packed bf16
// image and the per-site intermediates stay in device memory that the 129 MB
// L2 holds at these bonds, and the sites' four phases are separated by
// device-wide barriers instead of kernel launches:
//   (A) pack L (with its largest magnitude, the site's exact rescale) and
//       the site's core in the two operand layouts of (i) and (iii);
//   (B) tcgen05 GEMM  T1[(w, a'), (s, b)] = sum_a L[(w, a'), a] A[a, (s, b)];
//   (C) step (ii) into (iii)'s packed operand (mpo_step.cuh);
//   (D) tcgen05 GEMM  L'[(w', b), b'] = sum_{(a', s')} T2 A[(a', s'), b'].
// A GEMM phase: CTA c takes output tiles c, c + grid, ... (128 x 128); one
// thread streams the packed blocks of each 64-wide shared slab into a ring of
// shared-memory stages (1-D bulk copies) and issues the MMAs, eight warps
// drain the TMEM accumulator (double-buffered across tiles) and store the
// float32 result. BF16X3 issues hi*hi, hi*lo, lo*hi per step and promotes the
// accumulator into registers every 512 shared indices, as the grouped GEMM.
// Every wait (mbarriers and the device-wide barrier) is bounded; on expiry
// the status word records TN_ERR_TIMEOUT and every CTA winds down.
#include <string.h>

#include <algorithm>

#include "mpo_step.cuh"
#include "packed.h"
#include "ptx.cuh"
#include "tn_internal.h"

namespace tn {
namespace {

constexpr int PS_THREADS = 384;  // 12 warps: warp 0 copies + MMAs, warp 1 TMEM, warps 4..11 drain TMEM
constexpr int PS_EPI0 = 4;       // first draining warp
constexpr int PS_EPI = 8;        // draining warps: two per TMEM lane quadrant, 64 columns each
constexpr int PS_KC = 8;         // BF16X3: slabs between promotions (512 shared indices)
constexpr int PS_BLOCK = 16384;  // one packed block: 128 rows x 64 shared indices of bf16
constexpr int PS_MAX_SITES = 512;
constexpr uint32_t PS_TMEM_COLS = 256;  // two 128-column accumulators

template <int SPLIT>
struct PsCfg {
  // BF16: P and Q hi (32 KB) per stage; BF16X3: hi and lo of both (64 KB)
  static constexpr int OPS = SPLIT ? 4 : 2;
  static constexpr int STAGES = SPLIT ? 3 : 6;
  static constexpr int STAGE_BYTES = OPS * PS_BLOCK;
};

struct PsSite {
  const float* A;  // core (Da, d, Db), row-major
  int32_t Da, Db, wa, wb;
  int32_t woff, pad;  // the site's extended MPO at Wx + woff
  // the core packed once per launch: for (i) at Cp + a1_off, for (iii) at
  // Cp + a3_off (bytes); its first pack chunk in the launch's numbering
  int64_t a1_off, a3_off, chunk0;
};

struct PsParams {
  int32_t n, d;
  const float* Wx;       // extended MPO of every site
  float* L[2];           // environments, (wa, Da, Da) / (wb, Db, Db) row-major
  float* T1;             // (wa, Da, d, Db)
  uint8_t* Lp;           // packed L: rows (w, a'), shared a (MN-major blocks)
  uint8_t* T2p;          // packed T2 for (iii): rows (w', b), shared a' d + s' (MN-major blocks)
  uint8_t* Cp;           // every site's packed cores (K-major blocks)
  int64_t Lp_lo, T2p_lo, Cp_lo;  // byte distance from a hi block to its lo block (BF16X3)
  int64_t chunks;        // pack chunks of all the cores
  unsigned* bits;        // per site: bits of the largest |L| entering it
  double* lg;            // float64 log-scale
  unsigned* bar;         // device-wide barrier counter (zero at launch)
  double* result;        // {energy, log-scale, norm, log-scale}
  int* status;
  PsSite site[PS_MAX_SITES];
};

struct __align__(8) PsAux {
  uint64_t full[8];       // stage s holds its blocks
  uint64_t empty[8];      // the MMAs that read stage s are complete
  uint64_t acc_full[2];   // accumulator b holds a finished chunk
  uint64_t acc_empty[2];  // the draining warps have read accumulator b
  uint64_t final_bar;     // every MMA of the launch is complete
  uint32_t tmem_base;
  volatile int32_t abort;
};

__device__ __forceinline__ uint32_t ld_acquire_gpu(const unsigned* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Device-wide barrier of the cooperative grid (all threads of every CTA):
// arrival `epoch` completes when the counter at `bar` reaches (epoch + 1) *
// gridDim.x. Writes before it are visible after it to every CTA's generic
// loads and to the bulk copies (async proxy) that read packed blocks.
// Bounded: after limit_ns of waiting the status word records TN_ERR_TIMEOUT,
// *abort is set and false is returned everywhere in this CTA (the CTAs that
// did arrive time out too and wind down).
__device__ bool grid_barrier(unsigned* bar, uint32_t& epoch, int* status, uint64_t limit_ns, volatile int32_t* abort) {
  fence_proxy_async_global();
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t target = (epoch + 1) * gridDim.x;
    atomicAdd(bar, 1u);
    if (ld_acquire_gpu(bar) < target) {
      const uint64_t t0 = ptx::globaltimer();
      for (uint32_t i = 1;; ++i) {
        if (ld_acquire_gpu(bar) >= target) break;
        if ((i & 63u) == 0u && ptx::globaltimer() - t0 > limit_ns) {
          ptx::set_status(status, TN_ERR_TIMEOUT);
          *abort = 1;
          break;
        }
      }
    }
    __threadfence();
  }
  ++epoch;
  __syncthreads();
  fence_proxy_async_global();
  return *abort == 0;
}

__device__ __forceinline__ bool grid_sync(const PsParams& p, uint32_t& epoch, PsAux& x) {
  return grid_barrier(p.bar, epoch, p.status, ptx::kWaitLimitNs, &x.abort);
}

// Failure-path check of the device-wide barrier: CTA 1 of a two-CTA
// cooperative launch leaves without arriving, so CTA 0's wait runs out.
__global__ void grid_barrier_timeout_kernel(unsigned* bar, int* status, uint64_t limit_ns) {
  __shared__ volatile int32_t abort;
  if (threadIdx.x == 0) abort = 0;
  __syncthreads();
  if (blockIdx.x != 0) return;
  uint32_t epoch = 0;
  grid_barrier(bar, epoch, status, limit_ns, &abort);
}

__device__ __forceinline__ uint32_t ps_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// One K-major packed operand written by the pack phase: element (r, k) of
// an R x K matrix at src[r_off(r) + k_off(k)], stored in whole 16 KB blocks
// of 128 rows x 64 shared indices (128-byte swizzle, as the grouped GEMM's
// packed blocks), zeros at every position past R or K.
struct PsPack {
  const float* src;
  uint8_t* hi;
  int64_t lo;       // byte distance to the lo plane, 0: none
  int32_t R, K, tiles, slabs;
  // row r = r1 * rd0 + r0 (r0 < rd0): offset r1 * rs1 + r0 * rs0; shared k likewise
  int32_t rd0, ks0_div;
  int64_t rs1, rs0, kq1, kq0;
};

__device__ __forceinline__ int32_t ceil_div(int32_t a, int32_t b) { return (a + b - 1) / b; }

// Chunks of one packed operand: (tile, 8-wide k group of the slab, row in the
// tile), rows fastest, so consecutive threads read consecutive rows at one
// shared index (the row digit r0 is the source's unit-stride one).
__device__ __forceinline__ int64_t pack_chunks(const PsPack& q) { return (int64_t)q.tiles * q.slabs * 8 * 128; }

__device__ __forceinline__ float pack_chunk(const PsPack& q, int64_t e, float amax) {
  const int32_t rr = (int32_t)(e & 127);
  int64_t rest = e >> 7;
  const int32_t g = (int32_t)(rest & 7);
  rest >>= 3;
  const int32_t sl = (int32_t)(rest % q.slabs), t = (int32_t)(rest / q.slabs);
  const int32_t r = t * 128 + rr, k0 = sl * 64 + g * 8;
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = 0.0f;
  if (r < q.R) {
    const int32_t r1 = r / q.rd0, r0 = r - r1 * q.rd0;
    const float* row = q.src + r1 * q.rs1 + r0 * q.rs0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int32_t k = k0 + j;
      if (k < q.K) {
        const int32_t k1 = k / q.ks0_div, kk = k - k1 * q.ks0_div;
        v[j] = __ldg(row + k1 * q.kq1 + kk * q.kq0);
      }
    }
  }
  uint4 h;
  h.x = ps_bf16x2(v[0], v[1]);
  h.y = ps_bf16x2(v[2], v[3]);
  h.z = ps_bf16x2(v[4], v[5]);
  h.w = ps_bf16x2(v[6], v[7]);
  const size_t off = ((size_t)t * q.slabs + sl) * PS_BLOCK +
                     (size_t)((rr >> 3) * 1024 + (rr & 7) * 128 + ((g ^ (rr & 7)) << 4));
  *reinterpret_cast<uint4*>(q.hi + off) = h;
  if (q.lo) {
    const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&h);
    uint4 l;
    l.x = ps_bf16x2(v[0] - __low2float(hb[0]), v[1] - __high2float(hb[0]));
    l.y = ps_bf16x2(v[2] - __low2float(hb[1]), v[3] - __high2float(hb[1]));
    l.z = ps_bf16x2(v[4] - __low2float(hb[2]), v[5] - __high2float(hb[2]));
    l.w = ps_bf16x2(v[6] - __low2float(hb[3]), v[7] - __high2float(hb[3]));
    *reinterpret_cast<uint4*>(q.hi + q.lo + off) = l;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) amax = fmaxf(amax, fabsf(v[j]));
  return amax;
}

// The pack jobs of a site's core: q1 for (i) (rows (s, b), shared a: A[a, s,
// b] at (a d + s) Db + b) and q3 for (iii) (rows b', shared a' d + s': at
// (a' d + s') Db + b'), at their places in the cores region.
__device__ __forceinline__ void core_packs(const PsParams& p, const PsSite& st, int32_t d, PsPack* q1, PsPack* q3) {
  if (q1) {
    q1->src = st.A;
    q1->hi = p.Cp + st.a1_off;
    q1->lo = p.Cp_lo;
    q1->R = d * st.Db;
    q1->K = st.Da;
    q1->rd0 = st.Db;
    q1->rs1 = st.Db;
    q1->rs0 = 1;
    q1->ks0_div = st.Da;
    q1->kq1 = 0;
    q1->kq0 = (int64_t)d * st.Db;
    q1->tiles = ceil_div(q1->R, 128);
    q1->slabs = ceil_div(q1->K, 64);
  }
  if (q3) {
    q3->src = st.A;
    q3->hi = p.Cp + st.a3_off;
    q3->lo = p.Cp_lo;
    q3->R = st.Db;
    q3->K = d * st.Da;
    q3->rd0 = st.Db;
    q3->rs1 = 0;
    q3->rs0 = 1;
    q3->ks0_div = q3->K;
    q3->kq1 = 0;
    q3->kq0 = st.Db;
    q3->tiles = ceil_div(q3->R, 128);
    q3->slabs = ceil_div(q3->K, 64);
  }
}

// One 16-byte chunk (8 rows at one shared index) of the first environment
// L[w, a, a'] as an MN-major operand (row w Da + a', shared a), zeros past R
// or K; chunks numbered (tile, slab, row group, k), k fastest.
__device__ __forceinline__ void pack_mn_chunk(const float* L, int32_t Da, int32_t R, int32_t K, int32_t slabs,
                                              uint8_t* hi, int64_t lo, int64_t e) {
  const int32_t kk = (int32_t)(e & 63);
  int64_t rest = e >> 6;
  const int32_t mg = (int32_t)(rest & 15);
  rest >>= 4;
  const int32_t sl = (int32_t)(rest % slabs), t = (int32_t)(rest / slabs);
  const int32_t k = sl * 64 + kk;
  float v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int32_t r = t * 128 + mg * 8 + j;
    v[j] = 0.0f;
    if (r < R && k < K) {
      const int32_t w = r / Da, a2 = r - w * Da;
      v[j] = L[((int64_t)w * Da + k) * Da + a2];
    }
  }
  uint4 h, l;
  uint32_t* hp = reinterpret_cast<uint32_t*>(&h);
  uint32_t* lp = reinterpret_cast<uint32_t*>(&l);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    hp[j] = ps_bf16x2(v[2 * j], v[2 * j + 1]);
    const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162*>(&hp[j]);
    lp[j] = ps_bf16x2(v[2 * j] - __low2float(hb), v[2 * j + 1] - __high2float(hb));
  }
  const size_t off = ((size_t)t * slabs + sl) * PS_BLOCK + mn_block_chunk(mg, kk);
  *reinterpret_cast<uint4*>(hi + off) = h;
  if (lo) *reinterpret_cast<uint4*>(hi + lo + off) = l;
}

// One GEMM phase: C[r, c] = sum_k P[r, k] Q[c, k] over whole packed blocks
// (P K-major, or MN-major when p_mn; Q K-major), output tiles of 128 x 128.
struct PsGemm {
  const uint8_t* P;
  const uint8_t* Q;
  int64_t P_lo, Q_lo;  // byte distance from a hi block to its lo block (BF16X3)
  float* C;
  int32_t ldc, R, N;   // C row stride; rows of P (result rows) and of Q (result columns)
  int32_t tp, tq, slabs, p_mn;
  // (iii): the result is also the next site's first operand of (i), written
  // here as whole MN-major blocks (row w' Db + b', shared index b), and its
  // largest magnitude goes to *maxbits; Pn null: none
  uint8_t* Pn;
  int64_t Pn_lo;
  int32_t Db, pn_slabs;
  unsigned* maxbits;
};

// Pipeline positions kept across the phases of the launch: slabs through the
// stage ring (producer), accumulator chunks (producer and draining warps).
struct PsPipe {
  uint32_t issued, consumed, gc;
};

// Producer and MMA issuer of a GEMM phase (one thread). Keeps STAGES - 1
// slabs of copies in flight ahead of the slab being multiplied; a slab's
// MMAs are queued before the thread waits to refill a stage.
template <int SPLIT>
__device__ bool gemm_issue(const PsGemm& g, uint32_t stage0, PsAux& x, uint32_t tmem, PsPipe& pp, int* status) {
  using C = PsCfg<SPLIT>;
  constexpr int S = C::STAGES;
  const uint32_t idesc = ptx::idesc_bf16_f32(128, 128, g.p_mn, 0);
  const int nks = g.slabs, chunk = SPLIT ? PS_KC : nks;
  for (int u = blockIdx.x; u < g.tp * g.tq; u += gridDim.x) {
    const int tpi = u / g.tq, tqi = u - tpi * g.tq;
    const uint8_t* pb = g.P + (size_t)tpi * g.slabs * PS_BLOCK;
    const uint8_t* qb = g.Q + (size_t)tqi * g.slabs * PS_BLOCK;
    const uint32_t first = pp.consumed;  // this unit's slab ks is global slab first + ks
    auto issue = [&](int ks) -> bool {
      const uint32_t gsl = first + (uint32_t)ks, st = gsl % S;
      // the stage's previous contents: read by MMAs that must be complete
      if (gsl >= (uint32_t)S && !ptx::mbar_wait(ptx::smem_addr(&x.empty[st]), ((gsl / S) - 1u) & 1u, status))
        return false;
      const uint32_t full = ptx::smem_addr(&x.full[st]), dst = stage0 + st * C::STAGE_BYTES;
      ptx::mbar_arrive_expect_tx(full, (uint32_t)C::STAGE_BYTES);
      ptx::bulk_copy_g2s(dst, pb + (size_t)ks * PS_BLOCK, PS_BLOCK, full);
      ptx::bulk_copy_g2s(dst + PS_BLOCK, qb + (size_t)ks * PS_BLOCK, PS_BLOCK, full);
      if (SPLIT) {
        ptx::bulk_copy_g2s(dst + 2 * PS_BLOCK, pb + g.P_lo + (size_t)ks * PS_BLOCK, PS_BLOCK, full);
        ptx::bulk_copy_g2s(dst + 3 * PS_BLOCK, qb + g.Q_lo + (size_t)ks * PS_BLOCK, PS_BLOCK, full);
      }
      ++pp.issued;
      return true;
    };
    for (int ks = 0; ks < S - 1 && ks < nks; ++ks)
      if (!issue(ks)) return false;
    uint32_t b = 0;
    for (int ks = 0; ks < nks; ++ks) {
      const bool start = ks % chunk == 0;
      if (start) {
        // the accumulator this chunk overwrites has been drained
        b = pp.gc & 1u;
        if (!ptx::mbar_wait(ptx::smem_addr(&x.acc_empty[b]), ((pp.gc >> 1) & 1u) ^ 1u, status)) return false;
      }
      const uint32_t gsl = first + (uint32_t)ks, st = gsl % S;
      if (!ptx::mbar_wait(ptx::smem_addr(&x.full[st]), (gsl / S) & 1u, status)) return false;
      ptx::tc_fence_after();
      const uint32_t sa = stage0 + st * C::STAGE_BYTES, dt = tmem + b * 128u;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t pd = g.p_mn ? ptx::sw128_mnmajor_desc(sa + kk * 2048, 8192, 1024)
                                   : ptx::sw128_kmajor_desc(sa + kk * 32);
        const uint64_t qd = ptx::sw128_kmajor_desc(sa + PS_BLOCK + kk * 32);
        ptx::mma_bf16(dt, pd, qd, idesc, (start && kk == 0) ? 0u : 1u);
        if (SPLIT) {
          const uint64_t pl = g.p_mn ? ptx::sw128_mnmajor_desc(sa + 2 * PS_BLOCK + kk * 2048, 8192, 1024)
                                     : ptx::sw128_kmajor_desc(sa + 2 * PS_BLOCK + kk * 32);
          const uint64_t ql = ptx::sw128_kmajor_desc(sa + 3 * PS_BLOCK + kk * 32);
          ptx::mma_bf16(dt, pd, ql, idesc, 1u);
          ptx::mma_bf16(dt, pl, qd, idesc, 1u);
        }
      }
      ptx::mma_commit(ptx::smem_addr(&x.empty[st]));
      ++pp.consumed;
      if (ks % chunk == chunk - 1 || ks == nks - 1) {
        ptx::mma_commit(ptx::smem_addr(&x.acc_full[b]));
        ++pp.gc;
      }
      // the next copies go to the stage of slab ks - 1, whose MMAs complete
      // while this slab's, queued behind them, keep the tensor pipe busy
      if (ks + S - 1 < nks && !issue(ks + S - 1)) return false;
    }
  }
  return true;
}

// Draining warps of a GEMM phase: warp (PS_EPI0 + 4 grp + quad) reads TMEM
// lanes quad * 32 .. + 31 (one result row per thread), columns grp * 64 ..
// + 63; BF16X3 adds each chunk's partial sums into float32 registers.
template <int SPLIT>
__device__ bool gemm_drain(const PsGemm& g, PsAux& x, uint32_t tmem, PsPipe& pp, int* status) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quad = warp & 3, grp = (warp - PS_EPI0) >> 2;
  const int nks = g.slabs, nchunks = SPLIT ? (nks + PS_KC - 1) / PS_KC : 1;
  const bool vec = (g.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(g.C) & 15) == 0;
  float mx = 0.0f;  // largest |value| written to the next site's operand
  for (int u = blockIdx.x; u < g.tp * g.tq; u += gridDim.x) {
    const int tpi = u / g.tq, tqi = u - tpi * g.tq;
    const int row = tpi * 128 + quad * 32 + lane, col0 = tqi * 128 + grp * 64;
    float* dst = g.C + (size_t)row * g.ldc + col0;
    const int ncol = g.N - col0;  // valid columns of this thread's 64
    auto store = [&](int h, const float* v) {
      if (row >= g.R || ncol <= 32 * h) return;
      if (vec && ncol >= 32 * h + 32) {
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *reinterpret_cast<float4*>(dst + 32 * h + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (32 * h + j < ncol) dst[32 * h + j] = v[j];
      }
    };
    // 32 result columns of this thread's row into the next site's packed
    // operand: row (w', b) of L' at shared index b, columns b' as rows
    auto pack_out = [&](int h, const float* v) {
      if (!g.Pn || row >= g.R) return;
      const int cb = col0 + 32 * h;
      if (cb >= g.N) return;
      const int wq = row / g.Db, b = row - wq * g.Db, kk = b & 63;
      const size_t slab_off = (size_t)(b >> 6) * PS_BLOCK;
      if ((g.Db & 63) == 0) {
        // rows r0 .. r0 + 31 of one tile: four 16-byte chunks
        const int r0 = wq * g.Db + cb;
        const size_t base = (size_t)(r0 >> 7) * g.pn_slabs * PS_BLOCK + slab_off;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const size_t off = base + mn_block_chunk(((r0 & 127) >> 3) + c, kk);
          uint4 hv, lv;
          uint32_t* hp = reinterpret_cast<uint32_t*>(&hv);
          uint32_t* lp = reinterpret_cast<uint32_t*>(&lv);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float a = v[8 * c + 2 * j], e2 = v[8 * c + 2 * j + 1];
            hp[j] = ps_bf16x2(a, e2);
            const __nv_bfloat162 hb = *reinterpret_cast<const __nv_bfloat162*>(&hp[j]);
            lp[j] = ps_bf16x2(a - __low2float(hb), e2 - __high2float(hb));
            mx = fmaxf(mx, fmaxf(fabsf(a), fabsf(e2)));
          }
          *reinterpret_cast<uint4*>(g.Pn + off) = hv;
          if (g.Pn_lo) *reinterpret_cast<uint4*>(g.Pn + g.Pn_lo + off) = lv;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (cb + j >= g.N) continue;
          const int r = wq * g.Db + cb + j;
          const size_t off = (size_t)(r >> 7) * g.pn_slabs * PS_BLOCK + slab_off +
                             mn_block_chunk((r & 127) >> 3, kk) + 2 * (r & 7);
          const __nv_bfloat16 hb = __float2bfloat16_rn(v[j]);
          *reinterpret_cast<__nv_bfloat16*>(g.Pn + off) = hb;
          if (g.Pn_lo)
            *reinterpret_cast<__nv_bfloat16*>(g.Pn + g.Pn_lo + off) = __float2bfloat16_rn(v[j] - __bfloat162float(hb));
          mx = fmaxf(mx, fabsf(v[j]));
        }
      }
    };
    float acc[SPLIT ? 64 : 1];
#pragma unroll
    for (int j = 0; j < (SPLIT ? 64 : 1); ++j) acc[j] = 0.0f;
    for (int c = 0; c < nchunks; ++c) {
      const uint32_t b = pp.gc & 1u;
      const bool w = ptx::mbar_wait(ptx::smem_addr(&x.acc_full[b]), (pp.gc >> 1) & 1u, status);
      if (!__all_sync(0xffffffffu, w)) return false;
      ptx::tc_fence_after();
      const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + b * 128u + (uint32_t)(grp * 64);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t r[32];
        ptx::tmem_ld_32x32b_x32(ta + 32u * h, r);
        ptx::tmem_ld_wait();
        if (SPLIT) {
#pragma unroll
          for (int j = 0; j < 32; ++j) acc[32 * h + j] += __uint_as_float(r[j]);
        } else {
          float v[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
          store(h, v);
          pack_out(h, v);
        }
      }
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ptx::smem_addr(&x.acc_empty[b]));
      ++pp.gc;
    }
    if (SPLIT) {
      store(0, acc);
      store(1, acc + 32);
      pack_out(0, acc);
      pack_out(1, acc + 32);
    }
  }
  if (g.maxbits) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > 0.0f) atomicMax(g.maxbits, __float_as_uint(mx));
  }
  return true;
}

template <int SPLIT>
__device__ bool gemm_phase(const PsGemm& g, uint32_t stage0, PsAux& x, uint32_t tmem, PsPipe& pp, int* status) {
  const int warp = threadIdx.x >> 5;
  bool ok = true;
  if (threadIdx.x == 0) ok = gemm_issue<SPLIT>(g, stage0, x, tmem, pp, status);
  else if (warp >= PS_EPI0) ok = gemm_drain<SPLIT>(g, x, tmem, pp, status);
  if (!ok) x.abort = 1;
  return ok;
}

// The whole sweep. Grid: one CTA per SM (cooperative launch).
template <int SPLIT>
__global__ void __launch_bounds__(PS_THREADS, 1) expect_persistent_kernel(const __grid_constant__ PsParams p) {
  using C = PsCfg<SPLIT>;
  extern __shared__ uint8_t ps_smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ps_smem_raw) + 1023) & ~uintptr_t(1023));
  PsAux& x = *reinterpret_cast<PsAux*>(smem + (size_t)C::STAGES * C::STAGE_BYTES);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int st = 0; st < C::STAGES; ++st) {
      ptx::mbar_init(ptx::smem_addr(&x.full[st]), 1);   // the producer's transaction arrival
      ptx::mbar_init(ptx::smem_addr(&x.empty[st]), 1);  // the MMA issuer's commit
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&x.acc_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&x.acc_empty[b]), PS_EPI);
    }
    ptx::mbar_init(ptx::smem_addr(&x.final_bar), 1);
    x.abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_addr(&x.tmem_base), PS_TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = x.tmem_base, stage0 = ptx::smem_addr(smem);
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, gstride = (int64_t)gridDim.x * blockDim.x;
  const int32_t d = p.d;
  PsPipe pp{0u, 0u, 0u};
  uint32_t epoch = 0;
  int cur = 0;
  // (0) every site's core in the two operand layouts, and the first
  // environment (1 in each channel) as the first site's MN-major operand
  for (int64_t e = gtid; e < p.chunks; e += gstride) {
    int lo = 0, hi = p.n - 1;  // the site whose chunks hold e
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.site[mid].chunk0 <= e) lo = mid;
      else hi = mid - 1;
    }
    const PsSite& st = p.site[lo];
    PsPack q;
    core_packs(p, st, d, &q, nullptr);
    const int64_t c1 = pack_chunks(q);
    int64_t k = e - st.chunk0;
    if (k >= c1) {
      core_packs(p, st, d, nullptr, &q);
      k -= c1;
    }
    pack_chunk(q, k, 0.0f);
  }
  {
    const PsSite& s0 = p.site[0];
    const int32_t R = s0.wa * s0.Da, K = s0.Da, tiles = ceil_div(R, 128), slabs = ceil_div(K, 64);
    for (int64_t e = gtid; e < (int64_t)tiles * slabs * 16 * 64; e += gstride)
      pack_mn_chunk(p.L[0], s0.Da, R, K, slabs, p.Lp, SPLIT ? p.Lp_lo : 0, e);
  }
  bool ok = grid_sync(p, epoch, x);
  for (int i = 0; i < p.n && ok; ++i) {
    const PsSite& st = p.site[i];
    const int32_t Da = st.Da, Db = st.Db, wa = st.wa, wb = st.wb;
    const int32_t slabs1 = ceil_div(Da, 64), slabs3 = ceil_div(d * Da, 64);
    // (B) T1[(w, a'), (s, b)] = sum_a L[(w, a'), a] A[a, (s, b)]
    PsGemm g;
    memset(&g, 0, sizeof(g));
    g.P = p.Lp;
    g.Q = p.Cp + st.a1_off;
    g.P_lo = p.Lp_lo;
    g.Q_lo = p.Cp_lo;
    g.C = p.T1;
    g.ldc = d * Db;
    g.R = wa * Da;
    g.N = d * Db;
    g.tp = ceil_div(g.R, 128);
    g.tq = ceil_div(g.N, 128);
    g.slabs = slabs1;
    g.p_mn = 1;
    gemm_phase<SPLIT>(g, stage0, x, tmem, pp, p.status);
    if (!(ok = grid_sync(p, epoch, x))) break;
    // (C) T2 = 2^-e W' T1, straight into (iii)'s packed first operand; zeros
    // at the shared indices past Db of the next site's operand of (i)
    StepIIPack q2;
    q2.T1 = p.T1;
    q2.W = p.Wx + st.woff;
    q2.maxbits = i > 0 ? p.bits + i : nullptr;
    q2.lg = p.lg;
    q2.hi = p.T2p;
    q2.lo = SPLIT ? p.T2p + p.T2p_lo : nullptr;
    q2.Da = Da;
    q2.Db = Db;
    q2.wa = wa;
    q2.wb = wb;
    q2.d = d;
    q2.tiles = ceil_div(wb * Db, 128);
    q2.slabs = slabs3;
    q2.ps = 1;
    q2.pa = d;
    q2.pad = 0;
    step_ii_pack(q2, gtid, gstride, blockIdx.x == 0 && threadIdx.x == 0);
    const int32_t nslabs = ceil_div(Db, 64), npad = nslabs * 64 - Db;
    if (i + 1 < p.n && npad > 0) {
      const int64_t nz = (int64_t)ceil_div(wb * Db, 128) * 16 * npad;
      for (int64_t e = gtid; e < nz; e += gstride) {
        const int32_t kk = Db + (int32_t)(e % npad);
        const int64_t rest = e / npad;
        const int32_t mg = (int32_t)(rest & 15), t = (int32_t)(rest >> 4);
        const size_t off = ((size_t)t * nslabs + (kk >> 6)) * PS_BLOCK + mn_block_chunk(mg, kk & 63);
        *reinterpret_cast<uint4*>(p.Lp + off) = make_uint4(0u, 0u, 0u, 0u);
        if (SPLIT) *reinterpret_cast<uint4*>(p.Lp + p.Lp_lo + off) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    if (!(ok = grid_sync(p, epoch, x))) break;
    // (D) L'[(w', b), b'] = sum_{(a', s')} T2[(w', b), (a', s')] A[(a', s'), b'];
    // L' also packed as the next site's operand of (i), with its largest magnitude
    g.P = p.T2p;
    g.Q = p.Cp + st.a3_off;
    g.P_lo = p.T2p_lo;
    g.Q_lo = p.Cp_lo;
    g.C = p.L[cur ^ 1];
    g.ldc = Db;
    g.R = wb * Db;
    g.N = Db;
    g.tp = q2.tiles;
    g.tq = ceil_div(Db, 128);
    g.slabs = slabs3;
    g.p_mn = 1;
    if (i + 1 < p.n) {
      g.Pn = p.Lp;
      g.Pn_lo = SPLIT ? p.Lp_lo : 0;
      g.Db = Db;
      g.pn_slabs = nslabs;
      g.maxbits = p.bits + i + 1;
    }
    gemm_phase<SPLIT>(g, stage0, x, tmem, pp, p.status);
    if (!(ok = grid_sync(p, epoch, x))) break;
    cur ^= 1;
  }
  if (ok && blockIdx.x == 0 && threadIdx.x == 0) {
    const float* L = p.L[cur];
    p.result[0] = (double)L[0];
    p.result[1] = *p.lg;
    p.result[2] = (double)L[1];
    p.result[3] = *p.lg;
  }
  // wind down: copies still in flight land, every MMA completes, then TMEM is freed
  if (threadIdx.x == 0) {
    for (uint32_t q = pp.consumed; q < pp.issued; ++q)
      ptx::mbar_wait(ptx::smem_addr(&x.full[q % C::STAGES]), (q / C::STAGES) & 1u, p.status);
    ptx::mma_commit(ptx::smem_addr(&x.final_bar));
    ptx::mbar_wait(ptx::smem_addr(&x.final_bar), 0u, p.status);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, PS_TMEM_COLS);
  }
}

}  // namespace

size_t ps_blocks(int64_t R, int64_t K) { return (size_t)((R + 127) / 128) * (size_t)((K + 63) / 64) * PS_BLOCK; }

// One plane (hi or lo) of every site's packed cores: the core as (i)'s
// second operand (d Db rows, Da shared) then as (iii)'s (Db rows, d Da shared).
size_t cores_plane_bytes(const tn_mps* psi) {
  size_t b = 0;
  for (int i = 0; i < psi->n; ++i)
    b += ps_blocks(psi->d * psi->bond[i + 1], psi->bond[i]) + ps_blocks(psi->bond[i + 1], psi->d * psi->bond[i]);
  return align256(b);
}

size_t expect_persistent_cores_bytes(const tn_mps* psi) { return 2 * cores_plane_bytes(psi); }

bool expect_persistent_ok(const tn_mps* psi, const tn_mpo* H, int prec) {
  if (prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return false;
  if (psi->n > PS_MAX_SITES) return false;
  for (int i = 0; i <= H->n; ++i)
    if ((H->bond[i] + 1) * psi->d > 8) return false;
  return true;
}

int expect_persistent(const tn_mps* psi, const tn_mpo* H, int prec, const ExpectBuffers& w, double* result,
                      cudaStream_t s) {
  if (!expect_persistent_ok(psi, H, prec)) return TN_ERR_UNSUPPORTED;
  const bool split = prec == TN_PREC_BF16X3;
  PsParams p;
  memset(&p, 0, sizeof(p));
  p.n = psi->n;
  p.d = (int32_t)psi->d;
  p.Wx = w.Wx;
  p.L[0] = w.L0;
  p.L[1] = w.L1;
  p.T1 = w.T1;
  // packed regions, laid out for the largest bond: L (hi, lo) in scratch,
  // T2 (hi, lo) in scratch3; every site's cores (hi plane, then lo) in cores
  int64_t Wm = 1, D = 1;
  for (int i = 0; i <= H->n; ++i) Wm = std::max(Wm, H->bond[i]);
  for (int i = 0; i <= psi->n; ++i) D = std::max(D, psi->bond[i]);
  const int64_t W1 = Wm + 1, d = psi->d;
  const size_t bl = align256(ps_blocks(W1 * D, D)), bt = align256(ps_blocks(W1 * D, d * D));
  const size_t bc = cores_plane_bytes(psi);
  if (w.scratch_bytes < 2 * bl || w.scratch3_bytes < 2 * bt || w.cores_bytes < 2 * bc) return TN_ERR_WORKSPACE;
  p.Lp = w.scratch;
  p.Lp_lo = split ? (int64_t)bl : 0;
  p.T2p = w.scratch3;
  p.T2p_lo = split ? (int64_t)bt : 0;
  p.Cp = w.cores;
  p.Cp_lo = split ? (int64_t)bc : 0;
  p.bits = w.bits;
  p.lg = w.lg;
  p.bar = w.bar;
  p.result = result;
  p.status = status_word();
  for (int i = 0; i < psi->n; ++i) {
    PsSite& st = p.site[i];
    st.A = psi->cores[i];
    st.Da = (int32_t)psi->bond[i];
    st.Db = (int32_t)psi->bond[i + 1];
    st.wa = (int32_t)(H->bond[i] + 1);
    st.wb = (int32_t)(H->bond[i + 1] + 1);
    st.woff = (int32_t)w.woff[(size_t)i];
  }
  // the cores' places and pack chunks, site by site
  size_t off = 0;
  int64_t chunks = 0;
  for (int i = 0; i < psi->n; ++i) {
    PsSite& st = p.site[i];
    const int64_t Da = st.Da, Db = st.Db;
    st.a1_off = (int64_t)off;
    off += ps_blocks(d * Db, Da);
    st.a3_off = (int64_t)off;
    off += ps_blocks(Db, d * Da);
    st.chunk0 = chunks;
    chunks += (int64_t)(ps_blocks(d * Db, Da) + ps_blocks(Db, d * Da)) / PS_BLOCK * 1024;
  }
  p.chunks = chunks;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return TN_ERR_CUDA;
  const size_t smem = 1024 + (size_t)(split ? PsCfg<1>::STAGES * PsCfg<1>::STAGE_BYTES
                                            : PsCfg<0>::STAGES * PsCfg<0>::STAGE_BYTES) +
                      sizeof(PsAux);
  const void* fn = split ? (const void*)expect_persistent_kernel<1> : (const void*)expect_persistent_kernel<0>;
  static std::atomic<uint64_t> attr[2];
  if (!smem_limit_once(fn, smem, &attr[split ? 1 : 0])) return TN_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, PS_THREADS, smem) != cudaSuccess || per_sm < 1)
    return TN_ERR_UNSUPPORTED;
  // the device-wide barrier counts arrivals from zero
  if (cudaMemsetAsync(w.bar, 0, sizeof(unsigned), s) != cudaSuccess) return TN_ERR_CUDA;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)sms);
  cfg.blockDim = dim3(PS_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = split ? cudaLaunchKernelEx(&cfg, expect_persistent_kernel<1>, p)
                              : cudaLaunchKernelEx(&cfg, expect_persistent_kernel<0>, p);
  return e == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace tn

extern "C" int tn_check_grid_barrier_timeout(uint64_t limit_ns, void* counter, void* stream) {
  if (!counter || (reinterpret_cast<uintptr_t>(counter) & 3)) return TN_ERR_ARG;
  const uint64_t lo = 10000000ull, hi = 2000000000ull;
  uint64_t lim = limit_ns < lo ? lo : (limit_ns > hi ? hi : limit_ns);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(counter, 0, sizeof(unsigned), s) != cudaSuccess) return TN_ERR_CUDA;
  unsigned* bar = static_cast<unsigned*>(counter);
  int* status = tn::status_word();
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tn::grid_barrier_timeout_kernel, bar, status, lim) == cudaSuccess ? TN_OK
                                                                                                   : TN_ERR_CUDA;
}
