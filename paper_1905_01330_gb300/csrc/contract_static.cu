// Grouped contraction for callers that cannot allocate device memory.
//
// tn_contract_grouped_static runs the same kernels as tn_group_plan_run, but
// the work list those kernels read (one descriptor per contraction, plus the
// results to zero for split-K) lives in a fixed array inside this library
// instead of a caller workspace. It is for code that must not call
// cudaMalloc: code whose device memory all belongs to another framework's
// pool (a stray cudaMalloc there can exceed the pool's budget, and it
// synchronises the device, stalling every stream the caller is overlapping),
// and code on a latency-bound path that can only launch kernels.
//
// The array costs every GPU that loads the library STATIC_SCRATCH_BYTES of
// device memory until the process exits. All calls share it, so two calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on it; calls on one stream are ordered and safe.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "tn_internal.h"

namespace tn {
namespace {

constexpr size_t STATIC_SCRATCH_BYTES = 4u << 20;  // 4 MiB
constexpr int STATIC_MAX_SPECS = 4096;
constexpr int64_t STATIC_MAX_UNITS = 1 << 20;  // bound of the host staging map; the array bounds it further

static __device__ __align__(256) unsigned char g_static_scratch[STATIC_SCRATCH_BYTES];

// Host staging for the work list (no heap allocation per call).
static ContractDesc h_descs[STATIC_MAX_SPECS];
static ZeroRange h_zero[STATIC_MAX_SPECS];
static int32_t h_units[STATIC_MAX_UNITS];
static std::mutex h_lock;

// Device address of g_static_scratch on each device, looked up once per
// device (with that device current) on the first call there.
static unsigned char* scratch_ptr[64] = {nullptr};

int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TN_ERR_CUDA;
  if (!scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return TN_ERR_CUDA;
    scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = scratch_ptr[dev];
  return TN_OK;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" int tn_contract_grouped_static(const tn_contract_spec* specs, int nspecs, int prec, void* stream) {
  if (nspecs < 0 || (nspecs > 0 && !specs)) return TN_ERR_ARG;
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  if (nspecs > STATIC_MAX_SPECS) return TN_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The work list is copied from host staging arrays that the next call
  // overwrites: a captured copy would replay whatever list was staged last.
  // So a capturing stream is refused before anything is enqueued.
  if (stream_capturing(s)) return TN_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> guard(h_lock);
  unsigned char* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != TN_OK) return rc;

  int nd = 0, nz = 0;
  for (int i = 0; i < nspecs; ++i) {
    const tn_contract_spec& sp = specs[i];
    if (sp.nshared < 0 || sp.nshared > TN_MAX_RANK) return TN_ERR_ARG;
    int la[TN_MAX_RANK], lb[TN_MAX_RANK];
    for (int j = 0; j < sp.nshared; ++j) {
      la[j] = sp.legsA[j];
      lb[j] = sp.legsB[j];
    }
    ContractDesc d;
    rc = plan_contract(&sp.A, la, &sp.B, lb, sp.nshared, &sp.C, &d);
    if (rc != TN_OK) return rc;
    if (d.M == 0 || d.N == 0) continue;
    if (d.K == 0) {  // empty shared index: the result is zero
      h_zero[nz++] = ZeroRange{d.C, d.M * d.N};
      continue;
    }
    plan_units(&d, 1);
    h_descs[nd++] = d;
  }
  // largest work units first, as the allocating entry point does
  auto unit_work = [](const ContractDesc& d) {
    return (double)std::min<int64_t>(d.M, TC_BM) * (double)std::min<int64_t>(d.N, TC_BN) *
           (double)std::min<int64_t>(d.K, d.k_per_split);
  };
  std::stable_sort(h_descs, h_descs + nd,
                   [&](const ContractDesc& a, const ContractDesc& b) { return unit_work(a) > unit_work(b); });
  int64_t tiles = 0;
  for (int i = 0; i < nd; ++i) {
    h_descs[i].tile_begin = tiles;
    tiles += (int64_t)h_descs[i].tiles_m * h_descs[i].tiles_n * h_descs[i].splits;
    if (h_descs[i].splits > 1) h_zero[nz++] = ZeroRange{h_descs[i].C, h_descs[i].M * h_descs[i].N};
  }
  if (tiles > STATIC_MAX_UNITS) return TN_ERR_UNSUPPORTED;
  const size_t desc_bytes = align256(sizeof(ContractDesc) * (size_t)nd);
  const size_t zero_bytes = align256(sizeof(ZeroRange) * (size_t)nz);
  if (desc_bytes + zero_bytes + sizeof(int32_t) * (size_t)tiles > STATIC_SCRATCH_BYTES) return TN_ERR_UNSUPPORTED;
  for (int i = 0; i < nd; ++i) {
    const int64_t n = (int64_t)h_descs[i].tiles_m * h_descs[i].tiles_n * h_descs[i].splits;
    for (int64_t k = 0; k < n; ++k) h_units[h_descs[i].tile_begin + k] = i;
  }

  // Every call rewrites the whole work list it reads; nothing in the array
  // needs to start at zero. Pageable sources: each copy returns once staged.
  if (nd > 0 && cudaMemcpyAsync(scratch, h_descs, sizeof(ContractDesc) * (size_t)nd, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess)
    return TN_ERR_CUDA;
  ZeroRange* zdev = reinterpret_cast<ZeroRange*>(scratch + desc_bytes);
  if (nz > 0 && cudaMemcpyAsync(zdev, h_zero, sizeof(ZeroRange) * (size_t)nz, cudaMemcpyHostToDevice, s) !=
                    cudaSuccess)
    return TN_ERR_CUDA;
  int32_t* map = reinterpret_cast<int32_t*>(scratch + desc_bytes + zero_bytes);
  if (tiles > 0 && cudaMemcpyAsync(map, h_units, sizeof(int32_t) * (size_t)tiles, cudaMemcpyHostToDevice, s) !=
                       cudaSuccess)
    return TN_ERR_CUDA;
  if (nz > 0 && (rc = launch_zero(zdev, nz, s)) != TN_OK) return rc;
  if (tiles == 0) return TN_OK;
  const ContractDesc* g = reinterpret_cast<const ContractDesc*>(scratch);
  if (prec == TN_PREC_FP32) return launch_contract_simt(h_descs[0], g, map, tiles, s);
  return launch_contract_tc(h_descs[0], g, map, tiles, prec, s);
}
