// Matrix product state sweeps: <bra|ket> (transfer sweep) and <psi|H|psi>
// (MPO left-environment sweep), with per-site rescaling and a float64
// running log-scale (Sec. II, Fig. 3a; MPS as a sparse 2^N vector, Sec. IV.A).
//
// Chains with every bond <= 64 run the whole inner-product sweep in one CTA:
// the environment and the per-site intermediate stay in shared memory from
// site to site. Larger bonds run each per-site contraction through
// tn_contract's kernels (tcgen05 for BF16/BF16X3), with the environment in a
// caller workspace, followed by a two-kernel rescale.
//
// The energy sweep carries <psi|psi> along as one more MPO channel: the MPO
// is extended by a channel that maps to itself with the identity operator
// (W'[w, w'] = W[w, w'] on the original channels, W'[wa, wb] = identity), so
// the environment channel wa of L is the norm environment and one sweep of
// three contractions per site gives both results. Its rescaling is deferred
// and exact: after step (iii) the largest magnitude of the new environment
// is found (one pass); the next site's step (ii) multiplies its output by
// 2^-e, e the binary exponent of that maximum (the contractions are linear in
// L, so scaling T2 scales everything downstream), and adds e ln 2 to the
// float64 log-scale.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "mpo_step.cuh"
#include "packed.h"
#include "tn_internal.h"

namespace tn {
namespace {

constexpr int SMALL_D = 64;      // largest bond of the one-CTA sweep
constexpr int64_t PERSISTENT_MAX_BOND = 512;  // largest bond of the persistent energy sweep
constexpr int SMALL_PHYS = 4;    // largest physical dim of the one-CTA sweep
constexpr int SMALL_MAXN = 1024; // sites passed by value to the one-CTA sweep
constexpr int SMALL_THREADS = 256;

struct SmallChain {
  int32_t n, d;
  int32_t bb[SMALL_MAXN + 1];
  int32_t bk[SMALL_MAXN + 1];
  const float* bra[SMALL_MAXN];
  const float* ket[SMALL_MAXN];
};

__device__ __forceinline__ uint32_t ptx_smem(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float m = 0.0f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
  return m;
}

// One CTA: E (Da x Dak) -> T[a,s,bk] = sum_ak E[a,ak] ket[ak,s,bk]
//                       -> E'[b,bk] = sum_{a,s} bra[a,s,b] T[a,s,bk]
// -> divide by max|E'| and add its log to the float64 log-scale.
__global__ void __launch_bounds__(SMALL_THREADS)
mps_inner_small_kernel(const __grid_constant__ SmallChain c, double* result) {
  extern __shared__ float sm[];
  float* E = sm;
  float* E2 = E + SMALL_D * SMALL_D;
  float* T = E2 + SMALL_D * SMALL_D;
  __shared__ float red[SMALL_THREADS / 32];
  const int tid = threadIdx.x;
  if (tid == 0) E[0] = 1.0f;
  double lg = 0.0;
  __syncthreads();
  const int d = c.d;
  for (int i = 0; i < c.n; ++i) {
    const int Da = c.bb[i], Db = c.bb[i + 1], Dak = c.bk[i], Dbk = c.bk[i + 1];
    const float* __restrict__ K = c.ket[i];
    const float* __restrict__ Br = c.bra[i];
    const int nt = Da * d * Dbk;
    for (int idx = tid; idx < nt; idx += SMALL_THREADS) {
      const int bk = idx % Dbk, rest = idx / Dbk, s = rest % d, a = rest / d;
      float acc = 0.0f;
      for (int ak = 0; ak < Dak; ++ak) acc = fmaf(E[a * Dak + ak], __ldg(K + (ak * d + s) * Dbk + bk), acc);
      T[idx] = acc;
    }
    __syncthreads();
    const int ne = Db * Dbk;
    float mx = 0.0f;
    for (int idx = tid; idx < ne; idx += SMALL_THREADS) {
      const int bk = idx % Dbk, b = idx / Dbk;
      float acc = 0.0f;
      for (int as = 0; as < Da * d; ++as) acc = fmaf(__ldg(Br + as * Db + b), T[as * Dbk + bk], acc);
      E2[idx] = acc;
      mx = fmaxf(mx, fabsf(acc));
    }
    const float m = block_max(mx, red);
    const float sc = m > 0.0f ? m : 1.0f;
    for (int idx = tid; idx < ne; idx += SMALL_THREADS) E[idx] = E2[idx] / sc;
    lg += (double)logf(sc);
    __syncthreads();
  }
  if (tid == 0) {
    result[0] = (double)E[0];
    result[1] = lg;
  }
}

// The same sweep with both cores of every site staged in shared memory: the
// cores of site i+1 are copied in (cp.async, no registers) while site i is
// contracted, and each thread computes four consecutive outputs along the
// ket bond, so every shared-memory operand read feeds four FMAs.
// Dynamic shared memory: E, E2 (emax floats each), T (tmax), two ket and two
// bra core buffers (cmax each).
struct StagedSizes {
  int32_t emax, tmax, cmax;
};

__device__ __forceinline__ void cp_async_f32(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(ptx_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(ptx_smem(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copies n floats global -> shared by all threads of the block.
__device__ __forceinline__ void stage_core(float* dst, const float* __restrict__ src, int n) {
  const bool v16 = ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && ((n & 3) == 0);
  if (v16) {
    for (int i = threadIdx.x * 4; i < n; i += SMALL_THREADS * 4) cp_async_16(dst + i, src + i);
  } else {
    for (int i = threadIdx.x; i < n; i += SMALL_THREADS) cp_async_f32(dst + i, src + i);
  }
}

__global__ void __launch_bounds__(SMALL_THREADS)
mps_inner_staged_kernel(const __grid_constant__ SmallChain c, StagedSizes z, double* result) {
  extern __shared__ __align__(16) float smf[];
  float* E = smf;
  float* E2 = E + z.emax;
  float* T = E2 + z.emax;
  float* const kbuf = T + z.tmax;          // ket cores of sites i (i & 1) and i + 1
  float* const bbuf = kbuf + 2 * z.cmax;   // bra cores, likewise
  __shared__ float red[SMALL_THREADS / 32];
  const int tid = threadIdx.x;
  const int d = c.d;
  if (tid == 0) E[0] = 1.0f;
  double lg = 0.0;
  stage_core(kbuf, c.ket[0], c.bk[0] * d * c.bk[1]);
  stage_core(bbuf, c.bra[0], c.bb[0] * d * c.bb[1]);
  cp_async_commit();
  for (int i = 0; i < c.n; ++i) {
    const int Da = c.bb[i], Db = c.bb[i + 1], Dak = c.bk[i], Dbk = c.bk[i + 1];
    cp_async_wait_all();
    __syncthreads();  // site i's cores (and E) visible to all; buffers of site i-1 free
    if (i + 1 < c.n) {
      stage_core(kbuf + ((i + 1) & 1) * z.cmax, c.ket[i + 1], Dbk * d * c.bk[i + 2]);
      stage_core(bbuf + ((i + 1) & 1) * z.cmax, c.bra[i + 1], Db * d * c.bb[i + 2]);
    }
    cp_async_commit();
    const float* K = kbuf + (i & 1) * z.cmax;
    const float* Br = bbuf + (i & 1) * z.cmax;
    // T[a, s, bk] = sum_ak E[a, ak] K[ak, s, bk], four bk per thread when Dbk % 4 == 0
    const int w = (Dbk & 3) == 0 ? 4 : 1;
    const int qn = Dbk / w;
    const int nt = Da * d * qn;
    for (int idx = tid; idx < nt; idx += SMALL_THREADS) {
      const int q = idx % qn, rest = idx / qn, sidx = rest % d, a = rest / d;
      const int bk = q * w;
      if (w == 4) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int ak = 0; ak < Dak; ++ak) {
          const float e = E[a * Dak + ak];
          const float4 k4 = *reinterpret_cast<const float4*>(K + (ak * d + sidx) * Dbk + bk);
          acc.x = fmaf(e, k4.x, acc.x);
          acc.y = fmaf(e, k4.y, acc.y);
          acc.z = fmaf(e, k4.z, acc.z);
          acc.w = fmaf(e, k4.w, acc.w);
        }
        *reinterpret_cast<float4*>(T + (a * d + sidx) * Dbk + bk) = acc;
      } else {
        float acc = 0.0f;
        for (int ak = 0; ak < Dak; ++ak) acc = fmaf(E[a * Dak + ak], K[(ak * d + sidx) * Dbk + bk], acc);
        T[(a * d + sidx) * Dbk + bk] = acc;
      }
    }
    __syncthreads();
    // E2[b, bk] = sum_{a, s} Br[a, s, b] T[a, s, bk]
    const int ne = Db * qn;
    float mx = 0.0f;
    for (int idx = tid; idx < ne; idx += SMALL_THREADS) {
      const int q = idx % qn, b = idx / qn;
      const int bk = q * w;
      if (w == 4) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int as = 0; as < Da * d; ++as) {
          const float br = Br[as * Db + b];
          const float4 t4 = *reinterpret_cast<const float4*>(T + as * Dbk + bk);
          acc.x = fmaf(br, t4.x, acc.x);
          acc.y = fmaf(br, t4.y, acc.y);
          acc.z = fmaf(br, t4.z, acc.z);
          acc.w = fmaf(br, t4.w, acc.w);
        }
        *reinterpret_cast<float4*>(E2 + b * Dbk + bk) = acc;
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(acc.x), fabsf(acc.y)), fmaxf(fabsf(acc.z), fabsf(acc.w))));
      } else {
        float acc = 0.0f;
        for (int as = 0; as < Da * d; ++as) acc = fmaf(Br[as * Db + b], T[as * Dbk + bk], acc);
        E2[b * Dbk + bk] = acc;
        mx = fmaxf(mx, fabsf(acc));
      }
    }
    const float m = block_max(mx, red);
    const float sc = m > 0.0f ? m : 1.0f;
    for (int idx = tid; idx < Db * Dbk; idx += SMALL_THREADS) E[idx] = E2[idx] / sc;
    lg += (double)logf(sc);
  }
  cp_async_wait_all();
  __syncthreads();
  if (tid == 0) {
    result[0] = (double)E[0];
    result[1] = lg;
  }
}

// ------------------------------------------------------------ rescale pair
// Largest |x| of x[0..n) into *bits (float bits; nonnegative floats order as
// unsigned integers). *bits starts at 0.
__global__ void absmax_kernel(const float* __restrict__ x, int64_t n, unsigned* bits) {
  __shared__ float red[32];
  float m = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
  m = block_max(m, red);
  if (threadIdx.x == 0) atomicMax(bits, __float_as_uint(m));
}

// x /= max (if nonzero); one thread adds log(max) to *log_acc.
__global__ void scale_kernel(float* __restrict__ x, int64_t n, const unsigned* bits, double* log_acc) {
  const float m = __uint_as_float(*bits);
  const float sc = m > 0.0f ? m : 1.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = x[i] / sc;
  if (blockIdx.x == 0 && threadIdx.x == 0) *log_acc += log((double)sc);
}

// E[0] = 1 (a 1x1 or 1x1x1 environment), log-scales and max slots zeroed.
__global__ void init_sweep_kernel(float* E, double* log_acc, int nlog, unsigned* bits, int nbits) {
  for (int i = threadIdx.x; i < nbits; i += blockDim.x) bits[i] = 0u;
  if (threadIdx.x < nlog) log_acc[threadIdx.x] = 0.0;
  if (threadIdx.x == 0) E[0] = 1.0f;
}

// result[2j] = (double)env_j[0], result[2j+1] = log_acc[j].
__global__ void finish_kernel(const float* e0, const double* l0, const float* e1, const double* l1,
                              double* result) {
  if (threadIdx.x == 0) {
    result[0] = (double)e0[0];
    result[1] = l0[0];
    if (e1) {
      result[2] = (double)e1[0];
      result[3] = l1[0];
    }
  }
}

int rescale(float* x, int64_t n, unsigned* bits, double* log_acc, cudaStream_t s) {
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((n + threads - 1) / threads, 1024);
  absmax_kernel<<<blocks, threads, 0, s>>>(x, n, bits);
  scale_kernel<<<blocks, threads, 0, s>>>(x, n, bits, log_acc);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int check_chain(const tn_mps* m) {
  if (!m || m->n < 1 || m->d < 1 || !m->bond || !m->cores) return TN_ERR_ARG;
  if (m->bond[0] != 1 || m->bond[m->n] != 1) return TN_ERR_ARG;
  for (int i = 0; i < m->n; ++i) {
    if (m->bond[i + 1] < 1 || !m->cores[i]) return TN_ERR_ARG;
  }
  return TN_OK;
}

int64_t max_bond(const tn_mps* m) {
  int64_t x = 1;
  for (int i = 0; i <= m->n; ++i) x = std::max(x, m->bond[i]);
  return x;
}

tn_tensor tensor3(float* p, int64_t a, int64_t b, int64_t c) {
  tn_tensor t;
  const int64_t sh[3] = {a, b, c};
  tn_tensor_init(&t, p, 3, sh);
  return t;
}
tn_tensor tensor2(float* p, int64_t a, int64_t b) {
  tn_tensor t;
  const int64_t sh[2] = {a, b};
  tn_tensor_init(&t, p, 2, sh);
  return t;
}
tn_tensor tensor4(float* p, int64_t a, int64_t b, int64_t c, int64_t d) {
  tn_tensor t;
  const int64_t sh[4] = {a, b, c, d};
  tn_tensor_init(&t, p, 4, sh);
  return t;
}

// ---------------------------------------------------- energy sweep kernels
constexpr int MPO_MAXN = 1024;   // sites of one extended-MPO build
constexpr int MPO_MAXWD = 32;    // (extended MPO bond) x d of the step (ii) kernel

// The extended MPO of every site: W'[w, w', s, s'] = W[w, w', s, s'] for
// w < wa, w' < wb; W'[wa, wb, s, s'] = (s == s'); 0 elsewhere.
struct MpoExtParams {
  int32_t n, d;
  int32_t wb[MPO_MAXN + 1];
  const float* W[MPO_MAXN];
  int64_t off[MPO_MAXN];
  float* out;
};

__global__ void mpo_extend_kernel(const __grid_constant__ MpoExtParams p) {
  const int i = blockIdx.x;
  const int wa = p.wb[i], wb = p.wb[i + 1], d = p.d;
  const int wa2 = wa + 1, wb2 = wb + 1;
  float* o = p.out + p.off[i];
  const int total = wa2 * wb2 * d * d;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int s2 = e % d, s = (e / d) % d, w2 = (e / (d * d)) % wb2, w = e / (d * d * wb2);
    float v = 0.0f;
    if (w < wa && w2 < wb) v = p.W[i][((w * wb + w2) * d + s) * d + s2];
    else if (w == wa && w2 == wb) v = s == s2 ? 1.0f : 0.0f;
    o[e] = v;
  }
}


// Offsets are 32-bit: the host checks that T1 and T2 hold fewer than 2^31
// elements. Thread c takes column (a', b) = (c / Db, c % Db); WD bounds both
// (extended MPO bond) x d, so the sums unroll fully at the MPO's own size.
template <int WD>
__device__ __forceinline__ void step_ii(const StepII& q, int64_t first, int64_t stride, bool log_thread) {
  __shared__ float Ws[WD][WD];     // [(w, s)][(w', s')], zero past the MPO
  __shared__ int32_t koff[WD];     // T1 offset of (w, s): (w Da d + s) Db
  const int wad = q.wa * q.d, wbd = q.wb * q.d, d = q.d;
  const int32_t Da = (int32_t)q.Da, Db = (int32_t)q.Db;
  for (int e = threadIdx.x; e < WD * WD; e += blockDim.x) {
    const int k = e / WD, m = e - k * WD;
    float v = 0.0f;
    if (k < wad && m < wbd) {
      const int w = k / d, s = k - w * d, w2 = m / d, s2 = m - w2 * d;
      v = q.W[((w * q.wb + w2) * d + s) * d + s2];
    }
    Ws[k][m] = v;
  }
  for (int k = threadIdx.x; k < WD; k += blockDim.x) {
    const int w = k / d, s = k - w * d;
    koff[k] = k < wad ? (w * Da * d + s) * Db : 0;
  }
  __syncthreads();
  int e = 0;
  if (q.maxbits) e = pow2_exponent(__uint_as_float(*q.maxbits));
  const float inv = __int_as_float((127 - e) << 23);
  if (log_thread && q.maxbits) *q.lg += (double)e * 0.69314718055994530942;
  const int32_t cols = Da * Db, mstride = Da * Db;
  const float* __restrict__ T1 = q.T1;
  float* __restrict__ T2 = q.T2;
  // at the smallest width the whole MPO lives in registers
  constexpr int WR = WD == 8 ? 8 : 1;
  float wr[WR][WR];
#pragma unroll
  for (int k = 0; k < WR; ++k)
#pragma unroll
    for (int m = 0; m < WR; ++m) wr[k][m] = Ws[k][m];
  int32_t ko[WD];
#pragma unroll
  for (int k = 0; k < WD; ++k) ko[k] = koff[k];
  for (int32_t c = (int32_t)first; c < cols; c += (int32_t)stride) {
    const int32_t a = c / Db, b = c - a * Db;
    const int32_t base1 = a * d * Db + b;
    float t[WD];
#pragma unroll
    for (int k = 0; k < WD; ++k) t[k] = k < wad ? __ldg(T1 + base1 + ko[k]) : 0.0f;
#pragma unroll
    for (int m = 0; m < WD; ++m) {
      if (m < wbd) {
        float acc = 0.0f;
#pragma unroll
        for (int k = 0; k < WD; ++k) acc = fmaf(WD == 8 ? wr[k % WR][m % WR] : Ws[k][m], t[k], acc);
        T2[m * mstride + c] = acc * inv;
      }
    }
  }
}

template <int WD>
__global__ void __launch_bounds__(256) mpo_step_ii_kernel(const __grid_constant__ StepII q) {
  step_ii<WD>(q, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
              blockIdx.x == 0 && threadIdx.x == 0);
}

__global__ void __launch_bounds__(256) step_ii_pack_kernel(const __grid_constant__ StepIIPack q) {
  step_ii_pack(q, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
               blockIdx.x == 0 && threadIdx.x == 0);
}

// Grouped form: blockIdx.y picks the chain's descriptor.
__global__ void __launch_bounds__(256) step_ii_pack_grouped(const StepIIPack* __restrict__ descs) {
  const StepIIPack q = descs[blockIdx.y];
  step_ii_pack(q, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
               blockIdx.x == 0 && threadIdx.x == 0);
}

// Work items of one chain's step_ii_pack (8-column groups, or columns).
int64_t step_ii_pack_items(int64_t Da, int64_t Db) { return Db % 8 == 0 ? Da * (Db / 8) : Da * Db; }

// Grouped form: blockIdx.y picks the chain's descriptor.
template <int WD>
__global__ void __launch_bounds__(256) mpo_step_ii_grouped(const StepII* __restrict__ descs) {
  const StepII q = descs[blockIdx.y];
  step_ii<WD>(q, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
              blockIdx.x == 0 && threadIdx.x == 0);
}

// The unroll width of step (ii): the smallest of 8, 16, 32 covering both
// (extended MPO bond) x d.
int step_ii_width(int64_t wad, int64_t wbd) {
  const int64_t m = std::max(wad, wbd);
  return m <= 8 ? 8 : (m <= 16 ? 16 : 32);
}

int launch_step_ii(const StepII& q, cudaStream_t s) {
  const int64_t cols = q.Da * q.Db;
  // a few columns per thread: the block's setup (the MPO into registers) is
  // then spread over more work
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cols + 1023) / 1024, 1216));
  switch (step_ii_width((int64_t)q.wa * q.d, (int64_t)q.wb * q.d)) {
    case 8: mpo_step_ii_kernel<8><<<grid, 256, 0, s>>>(q); break;
    case 16: mpo_step_ii_kernel<16><<<grid, 256, 0, s>>>(q); break;
    default: mpo_step_ii_kernel<32><<<grid, 256, 0, s>>>(q); break;
  }
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

// Energy sweep workspace: L0, L1 ((W+1) D^2), T1, T2 ((W+1) D d D), n max
// slots, the log-scale, the extended MPO, and scratch for the packed bf16
// operands of the largest contraction (sized for BF16X3).
struct ExpectWs2 {
  float *L0, *L1, *T1, *T2, *Wx;
  unsigned* bits;
  unsigned* bar;  // the persistent sweep's device-wide barrier counter
  double* lg;
  uint8_t* scratch;
  size_t scratch_bytes;
  uint8_t* scratch3;  // BF16 / BF16X3 with step (ii) fused: (iii)'s packed operands
  size_t scratch3_bytes;
  uint8_t* cores;     // the persistent sweep: every site's packed cores
  size_t cores_bytes;
  size_t bytes;
  std::vector<int64_t> woff;
};

ExpectWs2 expect2_layout(uint8_t* base, const tn_mps* psi, const tn_mpo* H) {
  ExpectWs2 w;
  int64_t Wm = 1;
  for (int i = 0; i <= H->n; ++i) Wm = std::max(Wm, H->bond[i]);
  const int64_t W1 = Wm + 1, D = max_bond(psi), d = psi->d;
  size_t off = 0;
  auto take = [&](size_t b) { uint8_t* p = base ? base + off : nullptr; off += align256(b); return p; };
  w.L0 = reinterpret_cast<float*>(take(sizeof(float) * W1 * D * D));
  w.L1 = reinterpret_cast<float*>(take(sizeof(float) * W1 * D * D));
  w.T1 = reinterpret_cast<float*>(take(sizeof(float) * W1 * D * d * D));
  w.T2 = reinterpret_cast<float*>(take(sizeof(float) * W1 * D * d * D));
  w.bits = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * (size_t)psi->n));
  w.lg = reinterpret_cast<double*>(take(sizeof(double) * 2));
  w.bar = reinterpret_cast<unsigned*>(take(sizeof(unsigned)));
  int64_t tot = 0;
  for (int i = 0; i < H->n; ++i) {
    w.woff.push_back(tot);
    tot += (H->bond[i] + 1) * (H->bond[i + 1] + 1) * d * d;
  }
  w.Wx = reinterpret_cast<float*>(take(sizeof(float) * (size_t)tot));
  // (i) (W+1) D x D by D x dD and (iii) (W+1) D x dD by dD x D, packed
  w.scratch_bytes = std::max(packed_scratch_bound(W1 * D, d * D, D, TN_PREC_BF16X3),
                             packed_scratch_bound(W1 * D, D, d * D, TN_PREC_BF16X3));
  w.scratch = take(w.scratch_bytes);
  // step (iii) of the fused sweep: T2 in whole MN-major blocks and the core,
  // packed while the previous contraction's operands are still in use
  w.scratch3_bytes = packed_scratch_bound(W1 * D, D, d * D, TN_PREC_BF16X3);
  w.scratch3 = take(w.scratch3_bytes);
  w.cores_bytes = D <= PERSISTENT_MAX_BOND ? expect_persistent_cores_bytes(psi) : 0;
  w.cores = take(w.cores_bytes);
  w.bytes = off;
  return w;
}

// L[w, 0, 0] = 1 for the first site's channels (the MPO's left boundary and
// the norm channel), log-scale and max slots zeroed.
__global__ void expect_init_kernel(float* L, int channels, double* lg, unsigned* bits, int nbits) {
  for (int i = threadIdx.x; i < nbits; i += blockDim.x) bits[i] = 0u;
  if (threadIdx.x < 2) lg[threadIdx.x] = 0.0;
  if (threadIdx.x < channels) L[threadIdx.x] = 1.0f;
}

// result = {L[0] (energy channel), lg, L[1] (norm channel), lg} of the final
// (wN + 1) x 1 x 1 environment (wN = 1).
__global__ void expect_finish_kernel(const float* L, const double* lg, double* result) {
  if (threadIdx.x == 0) {
    result[0] = (double)L[0];
    result[1] = lg[0];
    result[2] = (double)L[1];
    result[3] = lg[0];
  }
}

bool small_ok(const tn_mps* bra, const tn_mps* ket) {
  return bra->n <= SMALL_MAXN && bra->d <= SMALL_PHYS && max_bond(bra) <= SMALL_D && max_bond(ket) <= SMALL_D;
}

// Workspace of the contraction-kernel inner sweep: E0, E1 (Dmax^2 each),
// T (Dmax d Dmax), n max slots, one log-scale, and scratch for the packed
// bf16 operands of the largest contraction (sized for BF16X3, the larger).
struct InnerWs {
  float *E0, *E1, *T;
  unsigned* bits;
  double* lg;
  uint8_t* scratch;
  size_t scratch_bytes;
  size_t bytes;
};

InnerWs inner_layout(uint8_t* base, int64_t D, int64_t d, int n) {
  InnerWs w;
  size_t off = 0;
  auto take = [&](size_t b) { uint8_t* p = base ? base + off : nullptr; off += align256(b); return p; };
  w.E0 = reinterpret_cast<float*>(take(sizeof(float) * D * D));
  w.E1 = reinterpret_cast<float*>(take(sizeof(float) * D * D));
  w.T = reinterpret_cast<float*>(take(sizeof(float) * D * d * D));
  w.bits = reinterpret_cast<unsigned*>(take(sizeof(unsigned) * (size_t)n));
  w.lg = reinterpret_cast<double*>(take(sizeof(double) * 2));
  // T = E psi (D x D by D x dD) and E' = psi T (D x dD by dD x D)
  w.scratch_bytes = std::max(packed_scratch_bound(D, d * D, D, TN_PREC_BF16X3),
                             packed_scratch_bound(D, D, d * D, TN_PREC_BF16X3));
  w.scratch = take(w.scratch_bytes);
  w.bytes = off;
  return w;
}

// Inner-product sweep through the contraction kernels. Leaves the final 1x1
// environment in *final_env and the log-scale in w.lg[0].
int inner_sweep(const tn_mps* bra, const tn_mps* ket, int prec, const InnerWs& w, float** final_env,
                cudaStream_t s) {
  init_sweep_kernel<<<1, 256, 0, s>>>(w.E0, w.lg, 1, w.bits, bra->n);
  if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
  float* E = w.E0;
  float* E2 = w.E1;
  const int64_t d = bra->d;
  for (int i = 0; i < bra->n; ++i) {
    const int64_t Da = bra->bond[i], Db = bra->bond[i + 1], Dak = ket->bond[i], Dbk = ket->bond[i + 1];
    tn_tensor tE = tensor2(E, Da, Dak);
    tn_tensor tK = tensor3(ket->cores[i], Dak, d, Dbk);
    tn_tensor tT = tensor3(w.T, Da, d, Dbk);
    const int l1a[1] = {1}, l1b[1] = {0};
    int rc = contract_internal(&tE, l1a, &tK, l1b, 1, &tT, prec, s, w.scratch, w.scratch_bytes);
    if (rc != TN_OK) return rc;
    tn_tensor tB = tensor3(bra->cores[i], Da, d, Db);
    tn_tensor tE2 = tensor2(E2, Db, Dbk);
    const int l2a[2] = {0, 1}, l2b[2] = {0, 1};
    rc = contract_internal(&tB, l2a, &tT, l2b, 2, &tE2, prec, s, w.scratch, w.scratch_bytes);
    if (rc != TN_OK) return rc;
    rc = rescale(E2, Db * Dbk, w.bits + i, w.lg, s);
    if (rc != TN_OK) return rc;
    std::swap(E, E2);
  }
  *final_env = E;
  return TN_OK;
}

// The fused energy sweep's support: BF16 / BF16X3, and (extended MPO bond)
// x d <= 8 on both sides of every site (step (ii) keeps all its channels of 8
// columns in registers).
bool fused_expect_ok(const tn_mps* psi, const tn_mpo* H, int prec) {
  if (prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return false;
  for (int i = 0; i <= H->n; ++i)
    if ((H->bond[i] + 1) * psi->d > 8) return false;
  return true;
}

// The energy sweep runs as one persistent launch (mps_persistent.cu) when
// it supports the chain and the bond is at most 512: there its phases are
// short and a launch boundary per phase costs more than a device-wide
// barrier (measured, N = 100: chi = 512 BF16X3 4.7 -> 4.1 ms, BF16 3.35 ->
// 3.2 ms; chi = 256 even). At chi = 1024 the per-site launches, with their
// warp-specialised GEMM and 256-wide BF16 tiles, are faster (BF16X3 10.8
// against 13.6 ms).
bool use_persistent(const tn_mps* psi, const tn_mpo* H, int prec) {
  return max_bond(psi) <= PERSISTENT_MAX_BOND && expect_persistent_ok(psi, H, prec);
}

// Output tile width of a sweep contraction on the BF16 GEMM: 256 columns
// (each P block feeds twice the columns) when that still makes a work unit
// for every SM, else 128 (measured: chi = 1024 BF16 sweep 7.4 -> 6.1 ms with
// 256-wide tiles, chi = 256 2.2 -> 2.5 ms with too few units).
int wide_tile(const ContractDesc& d) {
  const int64_t rp = p_is_b(d) ? d.N : d.M, rq = p_is_b(d) ? d.M : d.N;
  const int64_t units = (rp + 127) / 128 * ((rq + 255) / 256) * d.splits;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    sms = 152;
  return rq >= 256 && units >= sms ? 256 : 128;
}

// Energy sweep with step (ii) fused into the packing of step (iii)'s first
// operand. Per site, four launches: one pack launch (L, with its largest
// magnitude for this site's rescale, the core for (i) and the core for
// (iii)), the GEMM of (i), step (ii) writing T2 as packed bf16 blocks, the
// GEMM of (iii). Leaves the final environment in *final_env.
int expect_sweep_fused(const tn_mps* psi, const tn_mpo* H, int prec, const ExpectWs2& w, float** final_env,
                       cudaStream_t s) {
  const int n = psi->n;
  const int64_t d = psi->d;
  float* L = w.L0;
  float* L2 = w.L1;
  int rc;
  for (int i = 0; i < n; ++i) {
    const int64_t Da = psi->bond[i], Db = psi->bond[i + 1], wa = H->bond[i] + 1, wb = H->bond[i + 1] + 1;
    // (i) T1[w, a', s, b] = sum_a L[w, a, a'] A[a, s, b]
    tn_tensor tL = tensor3(L, wa, Da, Da);
    tn_tensor tA = tensor3(psi->cores[i], Da, d, Db);
    tn_tensor tT1 = tensor4(w.T1, wa, Da, d, Db);
    const int la1[1] = {1}, lb1[1] = {0};
    ContractDesc d1;
    if ((rc = plan_contract(&tL, la1, &tA, lb1, 1, &tT1, &d1)) != TN_OK) return rc;
    plan_units(&d1, min_units_single());
    SinglePacked s1;
    if ((rc = plan_single_packed(d1, prec, false, wide_tile(d1), w.scratch, w.scratch_bytes, &s1)) != TN_OK)
      return rc;
    // (iii) L'[w', b, b'] = sum_{a', s'} T2[w', s', a', b] A[a', s', b'] (T2's
    // float32 layout stands in for the planner; its blocks come from (ii))
    tn_tensor tT2 = tensor4(w.T2, wb, d, Da, Db);
    tn_tensor tL2 = tensor3(L2, wb, Db, Db);
    const int la3[2] = {1, 2}, lb3[2] = {1, 0};
    ContractDesc d3;
    if ((rc = plan_contract(&tT2, la3, &tA, lb3, 2, &tL2, &d3)) != TN_OK) return rc;
    // BF16X3: whole k ranges per tile (measured at chi = 1024: 11.5 -> 10.8 ms;
    // the split in two left its float32 atomics and the zeroing on the path);
    // BF16 keeps the split, which its 256-wide tiles need to fill the SMs
    plan_units(&d3, prec == TN_PREC_BF16X3 ? 1 : min_units_single());
    SinglePacked s3;
    if ((rc = plan_single_packed(d3, prec, true, wide_tile(d3), w.scratch3, w.scratch3_bytes, &s3)) != TN_OK)
      return rc;
    // the shared index of (iii): legs (s', a') in the planner's order; rows (w', b)
    if (d3.nk != 2 || d3.nm != 2 || d3.M != wb * Db || d3.K != d * Da) return TN_ERR_UNSUPPORTED;
    StepIIPack q;
    memset(&q, 0, sizeof(q));
    q.T1 = w.T1;
    q.W = w.Wx + w.woff[(size_t)i];
    q.maxbits = i > 0 ? w.bits + i : nullptr;
    q.lg = w.lg;
    q.hi = s3.ja.hi;
    q.lo = s3.ja.lo;
    q.Da = (int32_t)Da;
    q.Db = (int32_t)Db;
    q.wa = (int32_t)wa;
    q.wb = (int32_t)wb;
    q.d = (int32_t)d;
    q.tiles = s3.ja.tiles;
    q.slabs = s3.ja.slabs;
    step_iii_places(Da, Db, d, d3.kstrA, &q.ps, &q.pa);
    // L (and its largest magnitude: this site's rescale), then both cores
    if ((rc = launch_pack_jobs(&s1.ja, i > 0 ? w.bits + i : nullptr, &s1.jb, &s3.jb, s)) != TN_OK) return rc;
    if ((rc = launch_gemm_single(s1.g, prec, s)) != TN_OK) return rc;
    const int64_t items = step_ii_pack_items(Da, Db);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 1216));
    step_ii_pack_kernel<<<grid, 256, 0, s>>>(q);
    if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
    if ((rc = launch_gemm_single(s3.g, prec, s)) != TN_OK) return rc;
    std::swap(L, L2);
  }
  *final_env = L;
  return TN_OK;
}

}  // namespace

int launch_mpo_step_ii_grouped(const StepII* descs, int count, int64_t max_cols, int64_t wad, int64_t wbd,
                               cudaStream_t s) {
  if (count <= 0) return TN_OK;
  // a few columns per thread and at most 64 blocks per chain: the small
  // chains' blocks would otherwise mostly start, load the MPO and leave
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_cols + 1023) / 1024, 64)), (unsigned)count);
  switch (step_ii_width(wad, wbd)) {
    case 8: mpo_step_ii_grouped<8><<<grid, 256, 0, s>>>(descs); break;
    case 16: mpo_step_ii_grouped<16><<<grid, 256, 0, s>>>(descs); break;
    default: mpo_step_ii_grouped<32><<<grid, 256, 0, s>>>(descs); break;
  }
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

void step_iii_places(int64_t Da, int64_t Db, int64_t d, const int64_t* kstrA, int32_t* ps, int32_t* pa) {
  // the innermost shared leg is s' (stride Da Db in T2) or a' (stride Db);
  // with Da = 1 only s' varies and either order gives k = s'
  const bool s_inner = Da > 1 && kstrA[1] == Da * Db;
  *ps = s_inner ? 1 : (int32_t)Da;
  *pa = s_inner ? (int32_t)d : 1;
}

int launch_step_ii_pack_grouped(const StepIIPack* descs, int count, int64_t max_items, cudaStream_t s) {
  if (count <= 0) return TN_OK;
  // at most 64 blocks per chain (the small chains' blocks would mostly start and leave)
  const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((max_items + 255) / 256, 64)), (unsigned)count);
  step_ii_pack_grouped<<<grid, 256, 0, s>>>(descs);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int launch_mpo_extend(const tn_mpo* H, float* out, const int64_t* off, cudaStream_t s) {
  if (H->n > MPO_MAXN) return TN_ERR_UNSUPPORTED;
  MpoExtParams mp;
  memset(&mp, 0, sizeof(mp));
  mp.n = H->n;
  mp.d = H->d;
  for (int i = 0; i <= H->n; ++i) mp.wb[i] = (int32_t)H->bond[i];
  for (int i = 0; i < H->n; ++i) {
    mp.W[i] = H->cores[i];
    mp.off[i] = off[i];
  }
  mp.out = out;
  mpo_extend_kernel<<<H->n, 128, 0, s>>>(mp);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

bool mpo_extend_supported(const tn_mpo* H) {
  if (H->n > MPO_MAXN) return false;
  for (int i = 0; i <= H->n; ++i)
    if ((H->bond[i] + 1) * H->d > MPO_MAXWD) return false;
  return true;
}

}  // namespace tn

using namespace tn;

extern "C" {

size_t tn_mps_inner_workspace_bytes(const tn_mps* bra, const tn_mps* ket) {
  if (check_chain(bra) != TN_OK || check_chain(ket) != TN_OK) return 0;
  if (small_ok(bra, ket)) return 0;
  const int64_t D = std::max(max_bond(bra), max_bond(ket));
  return inner_layout(nullptr, D, bra->d, bra->n).bytes;
}

int tn_mps_inner(const tn_mps* bra, const tn_mps* ket, int prec, void* workspace, size_t ws_bytes,
                 double* result, void* stream) {
  int rc;
  if ((rc = check_chain(bra)) != TN_OK || (rc = check_chain(ket)) != TN_OK) return rc;
  if (bra->n != ket->n || bra->d != ket->d || !result) return TN_ERR_ARG;
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (small_ok(bra, ket)) {
    SmallChain c;
    c.n = bra->n;
    c.d = bra->d;
    for (int i = 0; i <= bra->n; ++i) {
      c.bb[i] = (int32_t)bra->bond[i];
      c.bk[i] = (int32_t)ket->bond[i];
    }
    for (int i = 0; i < bra->n; ++i) {
      c.bra[i] = bra->cores[i];
      c.ket[i] = ket->cores[i];
    }
    // staged variant when its buffers fit: E, E2, T and four core buffers
    StagedSizes z{1, 1, 1};
    for (int i = 0; i < bra->n; ++i) {
      z.emax = std::max(z.emax, c.bb[i + 1] * c.bk[i + 1]);
      z.emax = std::max(z.emax, c.bb[i] * c.bk[i]);
      z.tmax = std::max(z.tmax, c.bb[i] * c.d * c.bk[i + 1]);
      z.cmax = std::max(z.cmax, std::max(c.bb[i] * c.d * c.bb[i + 1], c.bk[i] * c.d * c.bk[i + 1]));
    }
    // every buffer starts on a 16-byte boundary
    z.emax = (z.emax + 3) & ~3;
    z.tmax = (z.tmax + 3) & ~3;
    z.cmax = (z.cmax + 3) & ~3;
    const size_t staged = sizeof(float) * (2 * (size_t)z.emax + z.tmax + 4 * (size_t)z.cmax);
    constexpr size_t STAGED_MAX = 200 * 1024;
    if (staged <= STAGED_MAX) {
      static std::atomic<uint64_t> attr2{0};
      if (!smem_limit_once((const void*)mps_inner_staged_kernel, STAGED_MAX, &attr2)) return TN_ERR_CUDA;
      mps_inner_staged_kernel<<<1, SMALL_THREADS, staged, s>>>(c, z, result);
      return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
    }
    const size_t smem = sizeof(float) * (2 * SMALL_D * SMALL_D + SMALL_D * SMALL_PHYS * SMALL_D);
    static std::atomic<uint64_t> attr{0};
    if (!smem_limit_once((const void*)mps_inner_small_kernel, smem, &attr)) return TN_ERR_CUDA;
    mps_inner_small_kernel<<<1, SMALL_THREADS, smem, s>>>(c, result);
    return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
  }
  const int64_t D = std::max(max_bond(bra), max_bond(ket));
  InnerWs w = inner_layout(static_cast<uint8_t*>(workspace), D, bra->d, bra->n);
  if (!workspace || ws_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;
  float* env = nullptr;
  rc = inner_sweep(bra, ket, prec, w, &env, s);
  if (rc != TN_OK) return rc;
  finish_kernel<<<1, 32, 0, s>>>(env, w.lg, nullptr, nullptr, result);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

size_t tn_mps_expect_workspace_bytes(const tn_mps* psi, const tn_mpo* H) {
  if (check_chain(psi) != TN_OK || !H || !H->bond || H->n != psi->n) return 0;
  return expect2_layout(nullptr, psi, H).bytes;
}

int tn_mps_expect(const tn_mps* psi, const tn_mpo* H, int prec, void* workspace, size_t ws_bytes,
                  double* result, void* stream) {
  int rc;
  if ((rc = check_chain(psi)) != TN_OK) return rc;
  if (!H || !H->bond || !H->cores || H->n != psi->n || H->d != psi->d || !result) return TN_ERR_ARG;
  if (H->bond[0] != 1 || H->bond[H->n] != 1) return TN_ERR_ARG;
  for (int i = 0; i < H->n; ++i)
    if (H->bond[i + 1] < 1 || !H->cores[i]) return TN_ERR_ARG;
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  const int n = psi->n;
  const int64_t d = psi->d;
  if (!mpo_extend_supported(H)) return TN_ERR_UNSUPPORTED;
  {
    int64_t Wm = 1;
    for (int i = 0; i <= n; ++i) Wm = std::max(Wm, H->bond[i]);
    const int64_t D = max_bond(psi);
    if ((Wm + 1) * D * d * D >= (int64_t(1) << 31)) return TN_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ExpectWs2 w = expect2_layout(static_cast<uint8_t*>(workspace), psi, H);
  if (!workspace || ws_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;

  // the extended MPO (one more channel: the norm)
  if ((rc = launch_mpo_extend(H, w.Wx, w.woff.data(), s)) != TN_OK) return rc;
  expect_init_kernel<<<1, 256, 0, s>>>(w.L0, (int)(H->bond[0] + 1), w.lg, w.bits, n);
  if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
  float* L = w.L0;
  float* L2 = w.L1;
  if (use_persistent(psi, H, prec)) {
    ExpectBuffers b;
    b.L0 = w.L0;
    b.L1 = w.L1;
    b.T1 = w.T1;
    b.Wx = w.Wx;
    b.woff = w.woff.data();
    b.bits = w.bits;
    b.lg = w.lg;
    b.bar = w.bar;
    b.scratch = w.scratch;
    b.scratch_bytes = w.scratch_bytes;
    b.scratch3 = w.scratch3;
    b.scratch3_bytes = w.scratch3_bytes;
    b.cores = w.cores;
    b.cores_bytes = w.cores_bytes;
    return expect_persistent(psi, H, prec, b, result, s);
  }
  if (fused_expect_ok(psi, H, prec)) {
    if ((rc = expect_sweep_fused(psi, H, prec, w, &L, s)) != TN_OK) return rc;
    expect_finish_kernel<<<1, 32, 0, s>>>(L, w.lg, result);
    return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
  }
  for (int i = 0; i < n; ++i) {
    const int64_t Da = psi->bond[i], Db = psi->bond[i + 1], wa = H->bond[i] + 1, wb = H->bond[i + 1] + 1;
    // (i) T1[w, a', s, b] = sum_a L[w, a, a'] A[a, s, b]
    tn_tensor tL = tensor3(L, wa, Da, Da);
    tn_tensor tA = tensor3(psi->cores[i], Da, d, Db);
    tn_tensor tT1 = tensor4(w.T1, wa, Da, d, Db);
    const int la1[1] = {1}, lb1[1] = {0};
    if ((rc = contract_internal(&tL, la1, &tA, lb1, 1, &tT1, prec, s, w.scratch, w.scratch_bytes)) != TN_OK)
      return rc;
    // (ii) T2[w', s', a', b] = 2^-e sum_{w,s} W'[w, w', s, s'] T1[w, a', s, b]
    StepII q;
    memset(&q, 0, sizeof(q));
    q.T1 = w.T1;
    q.T2 = w.T2;
    q.W = w.Wx + w.woff[(size_t)i];
    q.Da = Da;
    q.Db = Db;
    q.wa = (int32_t)wa;
    q.wb = (int32_t)wb;
    q.d = (int32_t)d;
    q.maxbits = i > 0 ? w.bits + (i - 1) : nullptr;
    q.lg = w.lg;
    if ((rc = launch_step_ii(q, s)) != TN_OK) return rc;
    // (iii) L'[w', b, b'] = sum_{a', s'} T2[w', s', a', b] A[a', s', b']
    tn_tensor tT2 = tensor4(w.T2, wb, d, Da, Db);
    tn_tensor tL2 = tensor3(L2, wb, Db, Db);
    const int la3[2] = {1, 2}, lb3[2] = {1, 0};
    if ((rc = contract_internal(&tT2, la3, &tA, lb3, 2, &tL2, prec, s, w.scratch, w.scratch_bytes)) != TN_OK)
      return rc;
    // the largest |L'|: applied, exactly, in the next site's step (ii)
    if (i + 1 < n) {
      const int64_t nl = wb * Db * Db;
      absmax_kernel<<<(unsigned)std::min<int64_t>((nl + 255) / 256, 1024), 256, 0, s>>>(L2, nl, w.bits + i);
      if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
    }
    std::swap(L, L2);
  }
  expect_finish_kernel<<<1, 32, 0, s>>>(L, w.lg, result);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // extern "C"
