// extern "C" entry points of libtn.so for pairwise and grouped contractions.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "packed.h"
#include "ptx.cuh"
#include "tn_internal.h"

namespace tn {

__device__ int g_status;

int* status_word() {
  static int* ptrs[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!ptrs[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<int*>(p);
  }
  return ptrs[dev];
}

// One contraction alone should still fill the GPU when its K allows: ask for
// at least two work units per SM.
static int64_t min_units_single() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 148;
  }
  return 2 * (int64_t)sms;
}

static int launch_one(const ContractDesc& d, int prec, cudaStream_t stream) {
  const int64_t tiles = (int64_t)d.tiles_m * d.tiles_n * d.splits;
  if (prec == TN_PREC_FP32) return launch_contract_simt(d, nullptr, nullptr, tiles, stream);
  return launch_contract_tc(d, nullptr, nullptr, tiles, prec, stream);
}

}  // namespace tn

using namespace tn;

// A grouped contraction. FP32 plans launch the single-pass float32 kernel
// over `descs`; BF16 / BF16X3 plans launch pack + GEMM over `pp` (the
// operands packed once into bf16 blocks inside the workspace).
struct tn_group_plan {
  std::vector<ContractDesc> descs;  // launched specs, largest first, tile_begin set
  std::vector<ContractDesc> zeros;  // specs with an empty shared index (K = 0): C = 0
  std::vector<ZeroRange> zero_ranges;  // results zeroed on the device before the launch
  std::vector<int32_t> unit_desc;      // descriptor (or GEMM) index of every work unit
  tn::PackedPlan pp;                   // packed path (BF16 / BF16X3)
  bool packed = false;
  int prec = TN_PREC_FP32;
  int64_t total_tiles = 0;
  double flops = 0.0, bytes = 0.0;
};

extern "C" {

int tn_tensor_init(tn_tensor* t, void* data, int rank, const int64_t* shape) {
  if (!t || rank < 0 || rank > TN_MAX_RANK || (rank > 0 && !shape)) return TN_ERR_ARG;
  memset(t, 0, sizeof(*t));
  t->data = data;
  t->rank = rank;
  t->dtype = TN_F32;
  for (int i = 0; i < rank; ++i) t->shape[i] = shape[i];
  return TN_OK;
}

const char* tn_status_string(int status) {
  switch (status) {
    case TN_OK: return "ok";
    case TN_ERR_ARG: return "invalid argument";
    case TN_ERR_SHAPE: return "shape mismatch";
    case TN_ERR_UNSUPPORTED: return "unsupported";
    case TN_ERR_CUDA: return "CUDA error";
    case TN_ERR_TIMEOUT: return "device wait timed out";
    case TN_ERR_WORKSPACE: return "workspace missing or too small";
    default: return "unknown status";
  }
}

}  // extern "C"

namespace tn {
namespace {
// Waits on a freshly initialised mbarrier whose phase nobody completes.
__global__ void wait_timeout_kernel(uint64_t limit_ns, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    ptx::mbar_init(ptx::smem_addr(&bar), 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  ptx::mbar_wait_for(ptx::smem_addr(&bar), 0u, status, limit_ns);
}
}  // namespace
}  // namespace tn

extern "C" {

int tn_check_wait_timeout(uint64_t limit_ns, void* stream) {
  const uint64_t lo = 10000000ull, hi = 2000000000ull;
  const uint64_t lim = limit_ns < lo ? lo : (limit_ns > hi ? hi : limit_ns);
  tn::wait_timeout_kernel<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(lim, status_word());
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int tn_sync_status(void* stream) {
  if (cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) return TN_ERR_CUDA;
  int* w = status_word();
  if (!w) return TN_ERR_CUDA;
  int h = 0;
  if (cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TN_ERR_CUDA;
  if (h != 0) {
    const int zero = 0;
    if (cudaMemcpy(w, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return TN_ERR_CUDA;
  }
  return h;
}

int tn_contract(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                int nshared, const tn_tensor* C, int prec, void* stream) {
  return tn::contract_internal(A, legsA, B, legsB, nshared, C, prec, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

int tn::contract_internal(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                          int nshared, const tn_tensor* C, int prec, cudaStream_t s) {
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  ContractDesc d;
  int rc = plan_contract(A, legsA, B, legsB, nshared, C, &d);
  if (rc != TN_OK) return rc;
  if (d.M == 0 || d.N == 0) return TN_OK;
  if (d.K == 0)
    return cudaMemsetAsync(d.C, 0, sizeof(float) * (size_t)(d.M * d.N), s) == cudaSuccess ? TN_OK
                                                                                          : TN_ERR_CUDA;
  plan_units(&d, min_units_single());
  if (d.splits > 1 &&
      cudaMemsetAsync(d.C, 0, sizeof(float) * (size_t)(d.M * d.N), s) != cudaSuccess)
    return TN_ERR_CUDA;
  return launch_one(d, prec, s);
}

extern "C" {

int tn_group_plan_create(const tn_contract_spec* specs, int nspecs, int prec, tn_group_plan** plan) {
  return tn::group_plan_create_ex(specs, nspecs, prec, true, plan);
}

}  // extern "C"

int tn::group_plan_create_ex(const tn_contract_spec* specs, int nspecs, int prec, bool allow_packed,
                             tn_group_plan** plan) {
  if (!plan) return TN_ERR_ARG;
  *plan = nullptr;
  if (nspecs < 0 || (nspecs > 0 && !specs)) return TN_ERR_ARG;
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  tn_group_plan* p = new (std::nothrow) tn_group_plan();
  if (!p) return TN_ERR_ARG;
  p->prec = prec;
  p->descs.reserve((size_t)nspecs);
  for (int i = 0; i < nspecs; ++i) {
    const tn_contract_spec& sp = specs[i];
    if (sp.nshared < 0 || sp.nshared > TN_MAX_RANK) { delete p; return TN_ERR_ARG; }
    int la[TN_MAX_RANK], lb[TN_MAX_RANK];
    for (int j = 0; j < sp.nshared; ++j) { la[j] = sp.legsA[j]; lb[j] = sp.legsB[j]; }
    ContractDesc d;
    int rc = plan_contract(&sp.A, la, &sp.B, lb, sp.nshared, &sp.C, &d);
    if (rc != TN_OK) { delete p; return rc; }
    if (d.M == 0 || d.N == 0) continue;
    p->bytes += 4.0 * ((double)d.M * d.K + (double)d.K * d.N + (double)d.M * d.N);
    if (d.K == 0) { p->zeros.push_back(d); continue; }
    p->flops += 2.0 * (double)d.M * (double)d.N * (double)d.K;
    plan_units(&d, 1);
    p->descs.push_back(d);
  }
  // largest work units first, so the tail of the launch is made of small ones
  if (prec != TN_PREC_FP32 && allow_packed) {
    p->packed = true;
    for (const auto& d : p->descs) {
      const int rc = plan_packed(d, prec, &p->pp);
      if (rc != TN_OK) { delete p; return rc; }
    }
    // largest units first: tensor time plus memory time of one unit
    auto cost = [](const GemmDesc& g) {
      const double pr = (double)std::min<int64_t>(g.RP, 128), qr = (double)std::min<int64_t>(g.RQ, 128);
      const double k = 64.0 * std::min<int64_t>(g.slabs, g.slabs_per_split);
      return 2.0 * pr * qr * k / 1500.0 + (2.0 * (pr + qr) * k + 4.0 * pr * qr) / 5.0;
    };
    std::stable_sort(p->pp.gemms.begin(), p->pp.gemms.end(),
                     [&](const GemmDesc& a, const GemmDesc& b) { return cost(a) > cost(b); });
    int64_t t = 0;
    for (auto& g : p->pp.gemms) {
      g.tile_begin = t;
      t += (int64_t)g.tiles_p * g.tiles_q * g.splits;
      if (g.splits > 1) p->zero_ranges.push_back(ZeroRange{g.C, g.RP * g.RQ});
    }
    p->total_tiles = t;
    if (t > 0x7FFFFFFF) { delete p; return TN_ERR_UNSUPPORTED; }
    p->unit_desc.resize((size_t)t);
    for (size_t i = 0; i < p->pp.gemms.size(); ++i) {
      const GemmDesc& g = p->pp.gemms[i];
      const int64_t n = (int64_t)g.tiles_p * g.tiles_q * g.splits;
      std::fill(p->unit_desc.begin() + g.tile_begin, p->unit_desc.begin() + g.tile_begin + n, (int32_t)i);
    }
    *plan = p;
    return TN_OK;
  }
  auto unit_work = [](const ContractDesc& d) {
    return (double)std::min<int64_t>(d.M, TC_BM) * (double)std::min<int64_t>(d.N, TC_BN) *
           (double)std::min<int64_t>(d.K, d.k_per_split);
  };
  std::stable_sort(p->descs.begin(), p->descs.end(), [&](const ContractDesc& a, const ContractDesc& b) {
    return unit_work(a) > unit_work(b);
  });
  int64_t t = 0;
  for (auto& d : p->descs) {
    d.tile_begin = t;
    t += (int64_t)d.tiles_m * d.tiles_n * d.splits;
    if (d.splits > 1) p->zero_ranges.push_back(ZeroRange{d.C, d.M * d.N});
  }
  p->total_tiles = t;
  if (t > 0x7FFFFFFF) { delete p; return TN_ERR_UNSUPPORTED; }
  p->unit_desc.resize((size_t)t);
  for (size_t i = 0; i < p->descs.size(); ++i) {
    const ContractDesc& d = p->descs[i];
    const int64_t n = (int64_t)d.tiles_m * d.tiles_n * d.splits;
    std::fill(p->unit_desc.begin() + d.tile_begin, p->unit_desc.begin() + d.tile_begin + n, (int32_t)i);
  }
  *plan = p;
  return TN_OK;
}

extern "C" {

// Workspace layout (each part 256-byte aligned): descriptors (ContractDesc,
// or GemmDesc when packed) | zero ranges | unit -> descriptor map |
// (packed:) pack jobs | pack units | packed blocks.
static size_t zero_offset(const tn_group_plan* plan) {
  return plan->packed ? align256(sizeof(GemmDesc) * plan->pp.gemms.size())
                      : align256(sizeof(ContractDesc) * plan->descs.size());
}
static size_t map_offset(const tn_group_plan* plan) {
  return zero_offset(plan) + align256(sizeof(ZeroRange) * plan->zero_ranges.size());
}
static size_t jobs_offset(const tn_group_plan* plan) {
  return map_offset(plan) + align256(sizeof(int32_t) * plan->unit_desc.size());
}
static size_t punits_offset(const tn_group_plan* plan) {
  return jobs_offset(plan) + align256(sizeof(PackJob) * plan->pp.jobs.size());
}
static size_t packed_offset(const tn_group_plan* plan) {
  return punits_offset(plan) + align256(sizeof(PackUnit) * plan->pp.units.size());
}

size_t tn_group_plan_workspace_bytes(const tn_group_plan* plan) {
  if (!plan) return 0;
  if (plan->packed) return packed_offset(plan) + plan->pp.packed_bytes;
  return map_offset(plan) + sizeof(int32_t) * plan->unit_desc.size();
}

double tn_group_plan_flops(const tn_group_plan* plan) { return plan ? plan->flops : 0.0; }
int tn_group_plan_launches(const tn_group_plan* plan) {
  if (!plan) return 0;
  const int main = plan->total_tiles > 0 ? (plan->packed ? 2 : 1) : 0;
  return main + (plan->zero_ranges.empty() ? 0 : 1);
}
double tn_group_plan_bytes(const tn_group_plan* plan) { return plan ? plan->bytes : 0.0; }

static int check_ws(const tn_group_plan* plan, void* ws, size_t bytes) {
  const size_t need = tn_group_plan_workspace_bytes(plan);
  if (need == 0) return TN_OK;
  if (!ws || bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TN_ERR_WORKSPACE;
  return TN_OK;
}

int tn_group_plan_upload(const tn_group_plan* plan, void* workspace, size_t bytes, void* stream) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws(plan, workspace, bytes);
  if (rc != TN_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // pageable sources: each call returns once the bytes are staged, so the
  // plan may be destroyed right after it
  uint8_t* base = static_cast<uint8_t*>(workspace);
  if (plan->packed) {
    // device addresses of the packed blocks, patched into copies of the lists
    uint8_t* packed = base + packed_offset(plan);
    std::vector<GemmDesc> g = plan->pp.gemms;
    for (auto& e : g) {
      e.P = packed + e.P_off;
      e.Q = packed + e.Q_off;
    }
    std::vector<PackJob> j = plan->pp.jobs;
    for (size_t i = 0; i < j.size(); ++i) {
      j[i].hi = packed + plan->pp.job_hi_off[i];
      j[i].lo = plan->pp.job_lo_off[i] == SIZE_MAX ? nullptr : packed + plan->pp.job_lo_off[i];
    }
    if ((!g.empty() && cudaMemcpyAsync(base, g.data(), sizeof(GemmDesc) * g.size(), cudaMemcpyHostToDevice, s) !=
                           cudaSuccess) ||
        (!j.empty() && cudaMemcpyAsync(base + jobs_offset(plan), j.data(), sizeof(PackJob) * j.size(),
                                       cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        (!plan->pp.units.empty() &&
         cudaMemcpyAsync(base + punits_offset(plan), plan->pp.units.data(), sizeof(PackUnit) * plan->pp.units.size(),
                         cudaMemcpyHostToDevice, s) != cudaSuccess))
      return TN_ERR_CUDA;
  } else if (!plan->descs.empty() &&
             cudaMemcpyAsync(workspace, plan->descs.data(), sizeof(ContractDesc) * plan->descs.size(),
                             cudaMemcpyHostToDevice, s) != cudaSuccess) {
    return TN_ERR_CUDA;
  }
  if (!plan->zero_ranges.empty() &&
      cudaMemcpyAsync(static_cast<uint8_t*>(workspace) + zero_offset(plan), plan->zero_ranges.data(),
                      sizeof(ZeroRange) * plan->zero_ranges.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TN_ERR_CUDA;
  if (!plan->unit_desc.empty() &&
      cudaMemcpyAsync(static_cast<uint8_t*>(workspace) + map_offset(plan), plan->unit_desc.data(),
                      sizeof(int32_t) * plan->unit_desc.size(), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TN_ERR_CUDA;
  return TN_OK;
}

int tn_group_plan_run(const tn_group_plan* plan, void* workspace, size_t bytes, void* stream) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws(plan, workspace, bytes);
  if (rc != TN_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (const auto& z : plan->zeros)
    if (cudaMemsetAsync(z.C, 0, sizeof(float) * (size_t)(z.M * z.N), s) != cudaSuccess) return TN_ERR_CUDA;
  if (plan->total_tiles == 0) return TN_OK;
  if (!plan->zero_ranges.empty()) {
    rc = launch_zero(reinterpret_cast<const ZeroRange*>(static_cast<uint8_t*>(workspace) + zero_offset(plan)),
                     (int)plan->zero_ranges.size(), s);
    if (rc != TN_OK) return rc;
  }
  const int32_t* map = reinterpret_cast<const int32_t*>(static_cast<uint8_t*>(workspace) + map_offset(plan));
  if (plan->packed) {
    uint8_t* base = static_cast<uint8_t*>(workspace);
    rc = launch_pack(reinterpret_cast<const PackJob*>(base + jobs_offset(plan)),
                     reinterpret_cast<const PackUnit*>(base + punits_offset(plan)), (int64_t)plan->pp.units.size(), s);
    if (rc != TN_OK) return rc;
    return launch_packed_gemm(reinterpret_cast<const GemmDesc*>(base), map, plan->total_tiles, plan->prec, s);
  }
  const ContractDesc* g = static_cast<const ContractDesc*>(workspace);
  if (plan->prec == TN_PREC_FP32) return launch_contract_simt(plan->descs[0], g, map, plan->total_tiles, s);
  return launch_contract_tc(plan->descs[0], g, map, plan->total_tiles, plan->prec, s);
}

void tn_group_plan_destroy(tn_group_plan* plan) { delete plan; }

}  // extern "C"
