// FP32 tensordot with a small first operand: C[m, n] = sum_k A(m, k) B(k, n)
// (Sec. III.B.4) for M <= 16 and K <= 16 and any N -- the shape of the MPO
// step of an environment sweep (the MPO core against the environment: a few
// results per environment element, a few shared indices). A tiled kernel
// would spend almost all of a 128-row tile on padding; here A is gathered
// once per CTA into shared memory and each thread takes one column n: it
// reads B's K values of that column through the leg strides and writes the
// M results, consecutive threads on consecutive n (coalesced along the
// row-major result when B's last free leg has unit stride). Exact float32
// FMA, K terms in ascending shared-index order.
#include "gather.cuh"
#include "tn_internal.h"

namespace tn {
namespace {

constexpr int SK_THREADS = 256;

__global__ void __launch_bounds__(SK_THREADS) skinny_contract_kernel(const __grid_constant__ ContractDesc d) {
  __shared__ float As[SKINNY_MAX][SKINNY_MAX];
  __shared__ int32_t kB[SKINNY_MAX];
  const int t = threadIdx.x;
  const int M = (int)d.M, K = (int)d.K;
  if (t < M * K) {
    const int m = t / K, k = t - m * K;
    As[m][k] = d.A[leg_offset((uint32_t)m, d.nm, d.mdim, d.mstr) + leg_offset((uint32_t)k, d.nk, d.kdim, d.kstrA)];
  }
  if (t < K) kB[t] = (int32_t)leg_offset((uint32_t)t, d.nk, d.kdim, d.kstrB);
  __syncthreads();
  const float* __restrict__ B = d.B;
  float* __restrict__ C = d.C;
  for (int64_t n = (int64_t)blockIdx.x * SK_THREADS + t; n < d.N; n += (int64_t)gridDim.x * SK_THREADS) {
    const int64_t bo = leg_offset((uint32_t)n, d.nn, d.ndim, d.nstr);
    float b[SKINNY_MAX];
#pragma unroll
    for (int k = 0; k < SKINNY_MAX; ++k) b[k] = k < K ? __ldg(B + bo + kB[k]) : 0.0f;
#pragma unroll
    for (int m = 0; m < SKINNY_MAX; ++m) {
      if (m >= M) break;
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < SKINNY_MAX; ++k)
        if (k < K) acc = fmaf(As[m][k], b[k], acc);
      C[(int64_t)m * d.N + n] = acc;
    }
  }
}

// Grouped form: blockIdx.y picks the contraction of the uploaded list (all
// with M, K <= SKINNY_MAX), blockIdx.x strides over its columns.
__global__ void __launch_bounds__(SK_THREADS) skinny_contract_grouped(const ContractDesc* __restrict__ descs) {
  __shared__ float As[SKINNY_MAX][SKINNY_MAX];
  __shared__ int32_t kB[SKINNY_MAX];
  __shared__ ContractDesc sd;
  const int t = threadIdx.x;
  {
    const int nwords = (int)(sizeof(ContractDesc) / sizeof(int32_t));
    const int32_t* src = reinterpret_cast<const int32_t*>(descs + blockIdx.y);
    int32_t* dst = reinterpret_cast<int32_t*>(&sd);
    for (int i = t; i < nwords; i += SK_THREADS) dst[i] = src[i];
  }
  __syncthreads();
  const ContractDesc& d = sd;
  const int M = (int)d.M, K = (int)d.K;
  if ((int64_t)blockIdx.x * SK_THREADS >= d.N) return;  // uniform: this contraction has fewer columns
  if (t < M * K) {
    const int m = t / K, k = t - m * K;
    As[m][k] = d.A[leg_offset((uint32_t)m, d.nm, d.mdim, d.mstr) + leg_offset((uint32_t)k, d.nk, d.kdim, d.kstrA)];
  }
  if (t < K) kB[t] = (int32_t)leg_offset((uint32_t)t, d.nk, d.kdim, d.kstrB);
  __syncthreads();
  const float* __restrict__ B = d.B;
  float* __restrict__ C = d.C;
  for (int64_t n = (int64_t)blockIdx.x * SK_THREADS + t; n < d.N; n += (int64_t)gridDim.x * SK_THREADS) {
    const int64_t bo = leg_offset((uint32_t)n, d.nn, d.ndim, d.nstr);
    float b[SKINNY_MAX];
#pragma unroll
    for (int k = 0; k < SKINNY_MAX; ++k) b[k] = k < K ? __ldg(B + bo + kB[k]) : 0.0f;
#pragma unroll
    for (int m = 0; m < SKINNY_MAX; ++m) {
      if (m >= M) break;
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < SKINNY_MAX; ++k)
        if (k < K) acc = fmaf(As[m][k], b[k], acc);
      C[(int64_t)m * d.N + n] = acc;
    }
  }
}

}  // namespace

int launch_contract_skinny_grouped(const ContractDesc* descs, int count, int64_t max_n, cudaStream_t stream) {
  if (count <= 0 || max_n <= 0) return TN_OK;
  if (count > 65535) return TN_ERR_UNSUPPORTED;
  const int64_t blocks = (max_n + SK_THREADS - 1) / SK_THREADS;
  // about eight CTAs per SM over the whole group
  const int64_t want = (152 * 8 + count - 1) / count;
  const unsigned gx = (unsigned)(blocks < want ? blocks : (want < 1 ? 1 : want));
  skinny_contract_grouped<<<dim3(gx, (unsigned)count), SK_THREADS, 0, stream>>>(descs);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int launch_contract_skinny(const ContractDesc& d, cudaStream_t stream) {
  if (d.M > SKINNY_MAX || d.K > SKINNY_MAX || d.M <= 0 || d.K <= 0) return TN_ERR_ARG;
  const int64_t blocks = (d.N + SK_THREADS - 1) / SK_THREADS;
  const unsigned grid = (unsigned)(blocks < 152 * 8 ? blocks : 152 * 8);
  skinny_contract_kernel<<<grid, SK_THREADS, 0, stream>>>(d);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace tn
