// FP32 pairwise tensordot on the CUDA cores (exact float32 FMA path).
//
// C[m, n] = sum_k A(m, k) B(k, n) over the flattened shared legs
// (Sec. III.B.2 / III.B.4). Operands are gathered in place through their leg
// strides (no transposed copy): per 128x128 output tile, row offsets of A's
// free legs and column offsets of B's free legs are decoded once, and the
// offsets of each 16-wide slab of shared indices are decoded into a small
// shared-memory table one slab ahead. Register-tiled 8x8 outer products,
// double-buffered shared memory.
#include "gather.cuh"
#include "ptx.cuh"

namespace tn {
namespace {

constexpr int BM = SIMT_BM, BN = SIMT_BN, BK = 16, NT = 256;

struct SimtSmem {
  float As[2][BK][BM + 4];
  float Bs[2][BK][BN + 4];
  int32_t rowA[BM];
  int32_t colB[BN];
  int32_t kA[2][BK];
  int32_t kB[2][BK];
  ContractDesc d;
  UnitCoord uc;
  int idx;
};

__device__ __forceinline__ void fill_k(SimtSmem& s, int buf, int64_t k0) {
  const int t = threadIdx.x;
  if (t < 2 * BK) {
    const int j = t & (BK - 1);
    const int64_t k = s.uc.k_begin + k0 + j;
    int32_t off = -1;
    if (k < s.uc.k_end) {
      off = (int32_t)((t < BK) ? leg_offset((uint32_t)k, s.d.nk, s.d.kdim, s.d.kstrA)
                               : leg_offset((uint32_t)k, s.d.nk, s.d.kdim, s.d.kstrB));
    }
    if (t < BK) s.kA[buf][j] = off;
    else s.kB[buf][j] = off;
  }
}

__device__ __forceinline__ void load_regs(const SimtSmem& s, int buf, float (&ra)[8], float (&rb)[8]) {
  const int t = threadIdx.x;
  const float* __restrict__ A = s.d.A;
  const float* __restrict__ B = s.d.B;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int r, k;
    if (s.d.a_kfast) { k = t & (BK - 1); r = (t >> 4) + 16 * i; }
    else { r = t & (BM - 1); k = (t >> 7) + 2 * i; }
    const int32_t ko = s.kA[buf][k], ro = s.rowA[r];
    ra[i] = (ko >= 0 && ro >= 0) ? __ldg(A + (ro + ko)) : 0.0f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int c, k;
    if (s.d.b_kfast) { k = t & (BK - 1); c = (t >> 4) + 16 * i; }
    else { c = t & (BN - 1); k = (t >> 7) + 2 * i; }
    const int32_t ko = s.kB[buf][k], co = s.colB[c];
    rb[i] = (ko >= 0 && co >= 0) ? __ldg(B + (co + ko)) : 0.0f;
  }
}

__device__ __forceinline__ void store_regs(SimtSmem& s, int buf, const float (&ra)[8], const float (&rb)[8]) {
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int r, k;
    if (s.d.a_kfast) { k = t & (BK - 1); r = (t >> 4) + 16 * i; }
    else { r = t & (BM - 1); k = (t >> 7) + 2 * i; }
    s.As[buf][k][r] = ra[i];
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int c, k;
    if (s.d.b_kfast) { k = t & (BK - 1); c = (t >> 4) + 16 * i; }
    else { c = t & (BN - 1); k = (t >> 7) + 2 * i; }
    s.Bs[buf][k][c] = rb[i];
  }
}

__global__ void __launch_bounds__(NT, 2)
simt_contract_kernel(const __grid_constant__ ContractDesc single, const ContractDesc* group,
                     const int32_t* unit_desc) {
  __shared__ __align__(16) SimtSmem s;
  const int64_t tile = fetch_desc(single, group, unit_desc, (int64_t)blockIdx.x, &s.d, &s.idx);
  const int t = threadIdx.x;
  if (t == 0) s.uc = decode_unit(s.d, tile, BM, BN);
  __syncthreads();
  const int64_t m0 = s.uc.m0, n0 = s.uc.n0;

  if (t < BM) {
    const int64_t m = m0 + t;
    s.rowA[t] = (m < s.d.M) ? (int32_t)leg_offset((uint32_t)m, s.d.nm, s.d.mdim, s.d.mstr) : -1;
  } else {
    const int64_t n = n0 + (t - BM);
    s.colB[t - BM] = (n < s.d.N) ? (int32_t)leg_offset((uint32_t)n, s.d.nn, s.d.ndim, s.d.nstr) : -1;
  }
  const int64_t nkt = (s.uc.k_end - s.uc.k_begin + BK - 1) / BK;
  fill_k(s, 0, 0);
  __syncthreads();

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

  float ra[8], rb[8];
  if (nkt > 0) {
    load_regs(s, 0, ra, rb);
    store_regs(s, 0, ra, rb);
    if (nkt > 1) fill_k(s, 1, BK);
  }
  __syncthreads();

  const int ty = t >> 4, tx = t & 15;
  for (int64_t kt = 0; kt < nkt; ++kt) {
    const int cur = (int)(kt & 1);
    if (kt + 1 < nkt) load_regs(s, cur ^ 1, ra, rb);
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&s.As[cur][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&s.As[cur][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&s.Bs[cur][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&s.Bs[cur][k][64 + tx * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nkt) store_regs(s, cur ^ 1, ra, rb);
    if (kt + 2 < nkt) fill_k(s, cur, (kt + 2) * BK);
    __syncthreads();
  }

  float* __restrict__ C = s.d.C;
  const int64_t N = s.d.N;
  const bool vec = ((N & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
  const bool accumulate = s.d.splits > 1;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= s.d.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = n0 + h * 64 + tx * 4;
      if (n < N)
        emit4(C + m * N + n, vec, N - n, accumulate, acc[i][h * 4 + 0], acc[i][h * 4 + 1],
              acc[i][h * 4 + 2], acc[i][h * 4 + 3]);
    }
  }
}

__global__ void zero_kernel(const ZeroRange* ranges) {
  const ZeroRange r = ranges[blockIdx.x];
  float* p = r.ptr;
  int64_t n = r.count;
  int64_t head = 0;
  while (head < n && (reinterpret_cast<uintptr_t>(p + head) & 15) != 0) ++head;
  for (int64_t i = threadIdx.x; i < head; i += blockDim.x) p[i] = 0.0f;
  const int64_t nv = (n - head) / 4;
  float4* q = reinterpret_cast<float4*>(p + head);
  for (int64_t i = threadIdx.x; i < nv; i += blockDim.x) q[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t i = head + nv * 4 + threadIdx.x; i < n; i += blockDim.x) p[i] = 0.0f;
}

}  // namespace

int launch_zero(const ZeroRange* ranges, int n, cudaStream_t stream) {
  if (n <= 0) return TN_OK;
  zero_kernel<<<(unsigned)n, 512, 0, stream>>>(ranges);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int launch_contract_simt(const ContractDesc& single, const ContractDesc* group, const int32_t* unit_desc,
                         int64_t total_tiles, cudaStream_t stream) {
  if (total_tiles <= 0) return TN_OK;
  if (total_tiles > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (group && !unit_desc) return TN_ERR_ARG;
  simt_contract_kernel<<<(unsigned)total_tiles, NT, 0, stream>>>(single, group, unit_desc);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace tn
