// extern "C" entry points of libtn.so for pairwise and grouped contractions.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
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
int64_t min_units_single() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 152;
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
  std::vector<uint8_t> ext_p;          // per descriptor: its A written by the caller (MN-major blocks)
  tn::PackedSchedule sched[3];         // packed schedules: thin (min(M, N) < 128), short k (<= 512), long k
  // list sizes and packed bytes of the largest layout (workspace offsets):
  // the schedule with the longest lists, nothing fused
  size_t reserve_zero = 0, reserve_units = 0, reserve_punits = 0, reserve_packed = 0;
  uint64_t signature = 0;              // shapes of the specs (tuning cache key)
  bool packed = false;
  int prec = TN_PREC_FP32;
  int64_t total_tiles = 0;
  int64_t packed_tiles = 0;            // units of the GEMM on packed P; the fused GEMM's follow them
  bool skinny = false;                 // FP32, every contraction with M, K <= SKINNY_MAX
  int64_t max_n = 0;
  // offset tables of the P operand of every contraction that may take the
  // fused GEMM (BF16, narrower side at most 128 rows): element offsets of
  // its row and shared-index runs in `ctab`, -1 for the others
  std::vector<int32_t> ctab;
  std::vector<int64_t> ctab_r, ctab_k;
  // the fused TMA GEMM's tiling of every contraction whose P allows one
  // (BF16, narrower side at most 64 rows, P in device memory): its box and
  // the index of P's tensor map in `tmaps`, -1 for the others
  std::vector<tn::TmaBox> boxes;
  std::vector<int64_t> box_map;
  std::vector<tn::TmaMap> tmaps;
  int64_t tma_tiles = 0;               // first unit of the fused TMA GEMM (after the other fused ones)
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

size_t tn_contract_workspace_bytes(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                                   int nshared, const tn_tensor* C, int prec) {
  if (prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return 0;
  ContractDesc d;
  if (plan_contract(A, legsA, B, legsB, nshared, C, &d) != TN_OK) return 0;
  if (d.M == 0 || d.N == 0 || d.K == 0) return 0;
  plan_units(&d, min_units_single());
  return packed_single_bytes(d, prec);
}

int tn_contract_ws(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB, int nshared,
                   const tn_tensor* C, int prec, void* workspace, size_t bytes, void* stream) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!workspace) return tn::contract_internal(A, legsA, B, legsB, nshared, C, prec, s);
  if (reinterpret_cast<uintptr_t>(workspace) & 255) return TN_ERR_WORKSPACE;
  if (prec == TN_PREC_BF16 || prec == TN_PREC_BF16X3) {
    const size_t need = tn_contract_workspace_bytes(A, legsA, B, legsB, nshared, C, prec);
    if (bytes < need) return TN_ERR_WORKSPACE;
  }
  return tn::contract_internal(A, legsA, B, legsB, nshared, C, prec, s, workspace, bytes);
}

}  // extern "C"

int tn::contract_internal(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                          int nshared, const tn_tensor* C, int prec, cudaStream_t s, void* scratch,
                          size_t scratch_bytes) {
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  ContractDesc d;
  int rc = plan_contract(A, legsA, B, legsB, nshared, C, &d);
  if (rc != TN_OK) return rc;
  if (d.M == 0 || d.N == 0) return TN_OK;
  if (d.K == 0)
    return cudaMemsetAsync(d.C, 0, sizeof(float) * (size_t)(d.M * d.N), s) == cudaSuccess ? TN_OK
                                                                                          : TN_ERR_CUDA;
  // FP32 with a small first operand and a long second one (an MPO core
  // against an environment): one thread per result column
  if (prec == TN_PREC_FP32 && d.M <= SKINNY_MAX && d.K <= SKINNY_MAX && d.N >= 4096)
    return launch_contract_skinny(d, s);
  plan_units(&d, min_units_single());
  if (prec != TN_PREC_FP32 && scratch && packed_single_bytes(d, prec) <= scratch_bytes)
    return contract_packed_single(d, prec, scratch, scratch_bytes, s);
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

namespace {

// Schedule class of a contraction: 0 thin (fewer than 128 rows on one side),
// 1 short shared index (K <= 512: bound by writing C), 2 the rest.
int spec_class(const ContractDesc& d) {
  if (std::min(d.M, d.N) < 128) return 0;
  return d.K <= 512 ? 1 : 2;
}

tn::PackedSchedule default_schedule(int cls) {
  tn::PackedSchedule sc;
  sc.store16 = cls == 2 ? 1 : 0;  // measured: whole-sector stores help long-k specs only
  return sc;
}

// (Re)builds a packed plan's GEMM list, zero ranges and unit map from its
// contractions under its schedules. The GEMMs on packed P come first, the
// fused ones (P rounded inside the GEMM) after them; each launch numbers its
// units from 0.
int build_packed(tn_group_plan* p, bool allow_fuse = true) {
  p->pp = tn::PackedPlan();
  p->zero_ranges.clear();
  for (size_t i = 0; i < p->descs.size(); ++i) {
    ContractDesc d = p->descs[i];
    const tn::PackedSchedule& sc = p->sched[spec_class(d)];
    plan_units_packed(&d, sc.long_k != 0);
    const int64_t rt = p->ctab_r.empty() ? -1 : p->ctab_r[i], kt = p->ctab_k.empty() ? -1 : p->ctab_k[i];
    const int64_t bm = p->box_map.empty() ? -1 : p->box_map[i];
    const bool ext = !p->ext_p.empty() && p->ext_p[i] != 0;
    const int rc = plan_packed(d, p->prec, sc, allow_fuse && !ext, rt, kt, bm >= 0 ? &p->boxes[i] : nullptr, bm,
                               &p->pp, ext);
    if (rc != TN_OK) return rc;
  }
  // largest units first: tensor time plus memory time of one unit
  auto cost = [](const GemmDesc& g) {
    const double pr = (double)std::min<int64_t>(g.RP, 128), qr = (double)std::min<int64_t>(g.RQ, g.q_tile);
    const double k = 64.0 * std::min<int64_t>(g.slabs, g.slabs_per_split);
    return 2.0 * pr * qr * k / 1500.0 + (2.0 * (pr + qr) * k + 4.0 * pr * qr) / 5.0;
  };
  // launch of a GEMM: 0 on packed P, 1 fused (converters' copies), 2 fused TMA
  auto kind = [](const GemmDesc& g) { return g.pjob < 0 ? 0 : (g.tmap_idx < 0 ? 1 : 2); };
  std::stable_sort(p->pp.gemms.begin(), p->pp.gemms.end(), [&](const GemmDesc& a, const GemmDesc& b) {
    if (kind(a) != kind(b)) return kind(a) < kind(b);
    return cost(a) > cost(b);
  });
  // each launch numbers its units from 0
  int64_t t = 0, start[3] = {-1, -1, -1};
  for (auto& g : p->pp.gemms) {
    const int k = kind(g);
    if (start[k] < 0) start[k] = t;
    g.tile_begin = t - start[k];
    t += (int64_t)g.tiles_p * g.tiles_q * g.splits;
    if (g.splits > 1) p->zero_ranges.push_back(ZeroRange{g.C, g.RP * g.RQ});
  }
  p->tma_tiles = start[2] < 0 ? t : start[2];
  p->packed_tiles = start[1] < 0 ? p->tma_tiles : start[1];
  p->total_tiles = t;
  if (t > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  p->unit_desc.assign((size_t)t, 0);
  for (size_t i = 0; i < p->pp.gemms.size(); ++i) {
    const GemmDesc& g = p->pp.gemms[i];
    const int64_t n = (int64_t)g.tiles_p * g.tiles_q * g.splits;
    const int64_t b = g.tile_begin + start[kind(g)];
    std::fill(p->unit_desc.begin() + b, p->unit_desc.begin() + b + n, (int32_t)i);
  }
  return TN_OK;
}

// Host-side tuning cache: schedules picked by tn_group_plan_autotune, keyed
// by precision and the specs' shapes; a later plan of the same shapes starts
// from them.
std::mutex g_tune_lock;
struct TunedSchedules {
  tn::PackedSchedule sc[3];
};
std::map<uint64_t, TunedSchedules> g_tune_cache;

uint64_t plan_signature(const tn_group_plan* p) {
  uint64_t h = 1469598103934665603ull ^ (uint64_t)p->prec;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  for (const auto& d : p->descs) {
    mix((uint64_t)d.M);
    mix((uint64_t)d.N);
    mix((uint64_t)d.K);
  }
  return h;
}

}  // namespace

int tn::group_plan_create_ex(const tn_contract_spec* specs, int nspecs, int prec, bool allow_packed,
                             tn_group_plan** plan, const uint8_t* ext_p) {
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
    if (d.K == 0) {
      if (ext_p && ext_p[i]) { delete p; return TN_ERR_ARG; }
      p->zeros.push_back(d);
      continue;
    }
    p->flops += 2.0 * (double)d.M * (double)d.N * (double)d.K;
    plan_units(&d, 1);
    p->descs.push_back(d);
    p->ext_p.push_back(ext_p && ext_p[i] ? 1 : 0);
  }
  const bool any_ext = std::find(p->ext_p.begin(), p->ext_p.end(), (uint8_t)1) != p->ext_p.end();
  if (any_ext && (prec == TN_PREC_FP32 || !allow_packed)) { delete p; return TN_ERR_ARG; }
  // largest work units first, so the tail of the launch is made of small ones
  if (prec != TN_PREC_FP32 && allow_packed) {
    p->packed = true;
    p->signature = plan_signature(p);
    if (prec == TN_PREC_BF16) {
      p->ctab_r.assign(p->descs.size(), -1);
      p->ctab_k.assign(p->descs.size(), -1);
      p->boxes.assign(p->descs.size(), tn::TmaBox());
      p->box_map.assign(p->descs.size(), -1);
      for (size_t i = 0; i < p->descs.size(); ++i) {
        const ContractDesc& d = p->descs[i];
        if (p->ext_p[i]) continue;  // never fused
        tn::TmaMap m;
        if (std::min(d.M, d.N) <= 64 && tn::plan_tma_box(d, &p->boxes[i], &m)) {
          p->box_map[i] = (int64_t)p->tmaps.size();
          p->tmaps.push_back(m);
        } else if (std::min(d.M, d.N) <= 128) {
          tn::fused_tables(d, &p->ctab, &p->ctab_r[i], &p->ctab_k[i]);
        }
      }
    }
    // the workspace is laid out for the schedule with the longest lists
    // (64-wide tiles, 32-slab k ranges), nothing fused (the most packed
    // bytes) or everything that can be (the fused TMA GEMM's tiles may be
    // shorter than 128 rows), so any schedule fits it
    for (auto& sc : p->sched) sc = tn::PackedSchedule{64, 0, 0};
    for (int f = 0; f < 2; ++f) {
      int rc = build_packed(p, f == 1);
      if (rc != TN_OK) { delete p; return rc; }
      p->reserve_zero = std::max(p->reserve_zero, p->zero_ranges.size());
      p->reserve_units = std::max(p->reserve_units, p->unit_desc.size());
      p->reserve_punits = std::max(p->reserve_punits, p->pp.units.size());
      p->reserve_packed = std::max(p->reserve_packed, p->pp.packed_bytes);
    }
    for (int c = 0; c < 3; ++c) p->sched[c] = default_schedule(c);
    {
      std::lock_guard<std::mutex> lk(g_tune_lock);
      auto it = g_tune_cache.find(p->signature);
      if (it != g_tune_cache.end())
        for (int c = 0; c < 3; ++c) p->sched[c] = it->second.sc[c];
    }
    const int rc = build_packed(p);
    if (rc != TN_OK) { delete p; return rc; }
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
  // FP32 plans whose contractions all have a small first operand (the MPO
  // step of a batch of environment sweeps) run one thread per result column
  if (prec == TN_PREC_FP32 && !p->descs.empty()) {
    p->skinny = true;
    for (const auto& d : p->descs) {
      if (d.M > SKINNY_MAX || d.K > SKINNY_MAX) p->skinny = false;
      p->max_n = std::max(p->max_n, d.N);
    }
  }
  *plan = p;
  return TN_OK;
}

extern "C" {

// Workspace layout (each part 256-byte aligned): descriptors (ContractDesc,
// or GemmDesc when packed) | zero ranges | unit -> descriptor map |
// (packed:) pack jobs | pack units | offset tables | tensor maps | the
// GEMMs' unit counters | packed blocks.
static size_t zero_offset(const tn_group_plan* plan) {
  return plan->packed ? align256(sizeof(GemmDesc) * plan->pp.gemms.size())
                      : align256(sizeof(ContractDesc) * plan->descs.size());
}
static size_t map_offset(const tn_group_plan* plan) {
  const size_t nz = plan->packed ? plan->reserve_zero : plan->zero_ranges.size();
  return zero_offset(plan) + align256(sizeof(ZeroRange) * nz);
}
static size_t jobs_offset(const tn_group_plan* plan) {
  const size_t nu = plan->packed ? plan->reserve_units : plan->unit_desc.size();
  return map_offset(plan) + align256(sizeof(int32_t) * nu);
}
static size_t punits_offset(const tn_group_plan* plan) {
  return jobs_offset(plan) + align256(sizeof(PackJob) * plan->pp.jobs.size());
}
static size_t tables_offset(const tn_group_plan* plan) {
  return punits_offset(plan) + align256(sizeof(PackUnit) * plan->reserve_punits);
}
static size_t tmaps_offset(const tn_group_plan* plan) {
  return tables_offset(plan) + align256(sizeof(int32_t) * plan->ctab.size());
}
static size_t ctr_offset(const tn_group_plan* plan) {
  return tmaps_offset(plan) + align256(sizeof(tn::TmaMap) * plan->tmaps.size());
}
static size_t packed_offset(const tn_group_plan* plan) {
  return ctr_offset(plan) + (plan->packed ? 256 : 0);
}

size_t tn_group_plan_workspace_bytes(const tn_group_plan* plan) {
  if (!plan) return 0;
  if (plan->packed) return packed_offset(plan) + plan->reserve_packed;
  return map_offset(plan) + sizeof(int32_t) * plan->unit_desc.size();
}

double tn_group_plan_flops(const tn_group_plan* plan) { return plan ? plan->flops : 0.0; }
static int launch_count(const tn_group_plan* plan);
int tn_group_plan_launches(const tn_group_plan* plan) { return plan ? launch_count(plan) : 0; }
double tn_group_plan_bytes(const tn_group_plan* plan) { return plan ? plan->bytes : 0.0; }

// Bytes of the work lists alone (without the packed blocks).
static size_t list_bytes(const tn_group_plan* plan) {
  return plan->packed ? packed_offset(plan) : tn_group_plan_workspace_bytes(plan);
}

static int check_ws_need(size_t need, void* ws, size_t bytes) {
  if (need == 0) return TN_OK;
  if (!ws || bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TN_ERR_WORKSPACE;
  return TN_OK;
}

static int check_ws(const tn_group_plan* plan, void* ws, size_t bytes) {
  const size_t need = tn_group_plan_workspace_bytes(plan);
  if (need == 0) return TN_OK;
  if (!ws || bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255) != 0) return TN_ERR_WORKSPACE;
  return TN_OK;
}

}  // extern "C"

// Upload with the packed blocks at `packed` (inside the workspace, or a
// separate region shared by plans that run one after another).
// The schedule-independent lists: the fused GEMM's offset tables and the
// fused TMA GEMM's tensor maps.
static int upload_tables(const tn_group_plan* plan, uint8_t* base, cudaStream_t s) {
  if (!plan->ctab.empty() &&
      cudaMemcpyAsync(base + tables_offset(plan), plan->ctab.data(), sizeof(int32_t) * plan->ctab.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TN_ERR_CUDA;
  if (!plan->tmaps.empty() &&
      cudaMemcpyAsync(base + tmaps_offset(plan), plan->tmaps.data(), sizeof(tn::TmaMap) * plan->tmaps.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TN_ERR_CUDA;
  return TN_OK;
}

static int upload_impl(const tn_group_plan* plan, void* workspace, uint8_t* packed, cudaStream_t s,
                       bool with_tables = true) {
  // pageable sources: each call returns once the bytes are staged, so the
  // plan may be destroyed right after it -- and a capturing stream is refused
  if (stream_capturing(s)) return TN_ERR_UNSUPPORTED;
  uint8_t* base = static_cast<uint8_t*>(workspace);
  if (plan->packed) {
    // device addresses of the packed blocks, patched into copies of the lists
    std::vector<GemmDesc> g = plan->pp.gemms;
    for (auto& e : g) {
      e.P = packed + e.P_off;
      e.Q = packed + e.Q_off;
      e.tmap = e.tmap_idx >= 0 ? base + tmaps_offset(plan) + sizeof(tn::TmaMap) * (size_t)e.tmap_idx : nullptr;
    }
    std::vector<PackJob> j = plan->pp.jobs;
    const int32_t* tabs = reinterpret_cast<const int32_t*>(base + tables_offset(plan));
    for (size_t i = 0; i < j.size(); ++i) {
      j[i].hi = plan->pp.job_hi_off[i] == SIZE_MAX ? nullptr : packed + plan->pp.job_hi_off[i];
      j[i].lo = plan->pp.job_lo_off[i] == SIZE_MAX ? nullptr : packed + plan->pp.job_lo_off[i];
      j[i].rtab = j[i].rtab_off >= 0 ? tabs + j[i].rtab_off : nullptr;
      j[i].ktab = j[i].ktab_off >= 0 ? tabs + j[i].ktab_off : nullptr;
    }
    if (with_tables && upload_tables(plan, base, s) != TN_OK) return TN_ERR_CUDA;
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

size_t tn::group_plan_list_bytes(const tn_group_plan* plan) { return plan ? list_bytes(plan) : 0; }
size_t tn::group_plan_packed_bytes(const tn_group_plan* plan) {
  return plan && plan->packed ? plan->reserve_packed : 0;
}

int tn::group_plan_ext_layout(const tn_group_plan* plan, int i, ExtPLayout* out) {
  if (!plan || !out || !plan->packed || i < 0 || (size_t)i >= plan->descs.size() || !plan->ext_p[(size_t)i])
    return TN_ERR_ARG;
  const size_t j = 2 * (size_t)i;  // A's job: two jobs per contraction, in order
  const tn::PackJob& job = plan->pp.jobs[j];
  const ContractDesc& d = plan->descs[(size_t)i];
  memset(out, 0, sizeof(*out));
  out->hi_off = (int64_t)plan->pp.job_hi_off[j];
  out->lo_off = plan->pp.job_lo_off[j] == SIZE_MAX ? -1 : (int64_t)plan->pp.job_lo_off[j];
  out->tiles = job.tiles;
  out->slabs = job.slabs;
  out->nk = d.nk;
  for (int q = 0; q < d.nk; ++q) {
    out->kdim[q] = d.kdim[q];
    out->kstrA[q] = d.kstrA[q];
  }
  return TN_OK;
}

int tn::group_plan_upload_shared(const tn_group_plan* plan, void* lists, size_t bytes, void* packed,
                                 cudaStream_t s) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws_need(list_bytes(plan), lists, bytes);
  if (rc != TN_OK) return rc;
  if (plan->packed && plan->pp.packed_bytes > 0 && (!packed || (reinterpret_cast<uintptr_t>(packed) & 255)))
    return TN_ERR_WORKSPACE;
  return upload_impl(plan, lists, static_cast<uint8_t*>(packed), s);
}

extern "C" {

int tn_group_plan_upload(const tn_group_plan* plan, void* workspace, size_t bytes, void* stream) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws(plan, workspace, bytes);
  if (rc != TN_OK) return rc;
  return upload_impl(plan, workspace, static_cast<uint8_t*>(workspace) + packed_offset(plan),
                     static_cast<cudaStream_t>(stream));
}

}  // extern "C"

static int run_impl(const tn_group_plan* plan, void* workspace, cudaStream_t s);

int tn::group_plan_run_shared(const tn_group_plan* plan, void* lists, size_t bytes, cudaStream_t s) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws_need(list_bytes(plan), lists, bytes);
  if (rc != TN_OK) return rc;
  return run_impl(plan, lists, s);
}

extern "C" {

int tn_group_plan_run(const tn_group_plan* plan, void* workspace, size_t bytes, void* stream) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws(plan, workspace, bytes);
  if (rc != TN_OK) return rc;
  return run_impl(plan, workspace, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// The launch sequence of a run: [zeroing of split results] [pack] then the
// contraction kernel (single-pass), or the GEMM on packed P and / or the
// fused GEMM.
enum LaunchKind { L_ZERO, L_PACK, L_CONTRACT, L_FUSED, L_TMA };
constexpr int MAX_LAUNCHES = 5;

static int launch_list(const tn_group_plan* plan, LaunchKind* kinds) {
  int n = 0;
  if (plan->total_tiles == 0) return 0;
  if (!plan->zero_ranges.empty()) kinds[n++] = L_ZERO;
  if (plan->packed) {
    if (!plan->pp.units.empty()) kinds[n++] = L_PACK;
    if (plan->packed_tiles > 0) kinds[n++] = L_CONTRACT;
    if (plan->tma_tiles > plan->packed_tiles) kinds[n++] = L_FUSED;
    if (plan->total_tiles > plan->tma_tiles) kinds[n++] = L_TMA;
    return n;
  }
  kinds[n++] = L_CONTRACT;
  return n;
}

static int launch_count(const tn_group_plan* plan) {
  LaunchKind kinds[MAX_LAUNCHES];
  return launch_list(plan, kinds);
}

static int run_one(const tn_group_plan* plan, void* workspace, LaunchKind k, cudaStream_t s) {
  uint8_t* base = static_cast<uint8_t*>(workspace);
  const int32_t* map = reinterpret_cast<const int32_t*>(base + map_offset(plan));
  switch (k) {
    case L_ZERO:
      return launch_zero(reinterpret_cast<const ZeroRange*>(base + zero_offset(plan)), (int)plan->zero_ranges.size(),
                         s);
    case L_PACK:
      return launch_pack(reinterpret_cast<const PackJob*>(base + jobs_offset(plan)),
                         reinterpret_cast<const PackUnit*>(base + punits_offset(plan)),
                         (int64_t)plan->pp.units.size(), s);
    case L_FUSED:
      return launch_fused_gemm(reinterpret_cast<const GemmDesc*>(base), map + plan->packed_tiles,
                               reinterpret_cast<const PackJob*>(base + jobs_offset(plan)),
                               plan->tma_tiles - plan->packed_tiles, s);
    case L_TMA:
      return launch_tma_gemm(reinterpret_cast<const GemmDesc*>(base), map + plan->tma_tiles,
                             plan->total_tiles - plan->tma_tiles,
                             reinterpret_cast<uint32_t*>(base + ctr_offset(plan)) + 1, s);
    default:
      break;
  }
  if (plan->packed)
    return launch_packed_gemm(reinterpret_cast<const GemmDesc*>(base), map, plan->packed_tiles, plan->prec,
                              reinterpret_cast<uint32_t*>(base + ctr_offset(plan)), s);
  const ContractDesc* g = reinterpret_cast<const ContractDesc*>(base);
  if (plan->prec == TN_PREC_FP32 && plan->skinny)
    return launch_contract_skinny_grouped(g, (int)plan->descs.size(), plan->max_n, s);
  if (plan->prec == TN_PREC_FP32) return launch_contract_simt(plan->descs[0], g, map, plan->total_tiles, s);
  return launch_contract_tc(plan->descs[0], g, map, plan->total_tiles, plan->prec, s);
}

static int run_impl(const tn_group_plan* plan, void* workspace, cudaStream_t s) {
  for (const auto& z : plan->zeros)
    if (cudaMemsetAsync(z.C, 0, sizeof(float) * (size_t)(z.M * z.N), s) != cudaSuccess) return TN_ERR_CUDA;
  LaunchKind kinds[MAX_LAUNCHES];
  const int n = launch_list(plan, kinds);
  for (int i = 0; i < n; ++i) {
    const int rc = run_one(plan, workspace, kinds[i], s);
    if (rc != TN_OK) return rc;
  }
  return TN_OK;
}

extern "C" {

int tn_group_plan_run_launch(const tn_group_plan* plan, void* workspace, size_t bytes, int index, void* stream) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws(plan, workspace, bytes);
  if (rc != TN_OK) return rc;
  LaunchKind kinds[MAX_LAUNCHES];
  const int n = launch_list(plan, kinds);
  if (index < 0 || index >= n) return TN_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (index == 0)
    for (const auto& z : plan->zeros)
      if (cudaMemsetAsync(z.C, 0, sizeof(float) * (size_t)(z.M * z.N), s) != cudaSuccess) return TN_ERR_CUDA;
  return run_one(plan, workspace, kinds[index], s);
}

const char* tn_group_plan_launch_name(const tn_group_plan* plan, int index) {
  if (!plan) return nullptr;
  LaunchKind kinds[MAX_LAUNCHES];
  const int n = launch_list(plan, kinds);
  if (index < 0 || index >= n) return nullptr;
  switch (kinds[index]) {
    case L_ZERO: return "zero";
    case L_PACK: return "pack";
    case L_FUSED: return "gemm_fused";
    case L_TMA: return "gemm_tma";
    default: return plan->packed ? "gemm" : "contract";
  }
}

double tn_group_plan_launch_bytes(const tn_group_plan* plan, int index) {
  if (!plan) return -1.0;
  LaunchKind kinds[MAX_LAUNCHES];
  const int n = launch_list(plan, kinds);
  if (index < 0 || index >= n) return -1.0;
  double b = 0.0;
  switch (kinds[index]) {
    case L_ZERO:
      for (const auto& z : plan->zero_ranges) b += 4.0 * (double)z.count;
      return b;
    case L_PACK: {
      const double out = plan->prec == TN_PREC_BF16X3 ? 4.0 : 2.0;  // hi (+ lo) per element
      for (size_t i = 0; i < plan->pp.jobs.size(); ++i)
        if (plan->pp.job_hi_off[i] != SIZE_MAX && !plan->pp.job_ext[i])
          b += (4.0 + out) * (double)plan->pp.jobs[i].R * (double)plan->pp.jobs[i].K;
      return b;
    }
    case L_FUSED:
    case L_TMA:
    case L_CONTRACT:
      break;
  }
  if (!plan->packed) {
    for (const auto& d : plan->descs)
      b += 4.0 * ((double)d.M * d.K + (double)d.K * d.N + (double)d.M * d.N);
    return b;
  }
  const int want = kinds[index] == L_CONTRACT ? 0 : (kinds[index] == L_FUSED ? 1 : 2);
  const bool fused = want > 0;
  const double pe = plan->prec == TN_PREC_BF16X3 ? 4.0 : 2.0;  // packed bytes per element
  for (const auto& g : plan->pp.gemms) {
    if ((g.pjob < 0 ? 0 : (g.tmap_idx < 0 ? 1 : 2)) != want) continue;
    const double K = (double)g.K;
    b += (fused ? 4.0 : pe) * (double)g.RP * K + pe * (double)g.RQ * K + 4.0 * (double)g.RP * (double)g.RQ;
  }
  return b;
}

}  // extern "C"

extern "C" {

int tn_group_plan_autotune(tn_group_plan* plan, void* workspace, size_t bytes, void* stream) {
  if (!plan) return TN_ERR_ARG;
  int rc = check_ws(plan, workspace, bytes);
  if (rc != TN_OK) return rc;
  if (!plan->packed || plan->total_tiles == 0) return TN_OK;  // nothing to choose
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* base = static_cast<uint8_t*>(workspace);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return TN_ERR_CUDA;
  }
  // one candidate: rebuild, upload, one warm run, the mean of two timed runs
  // the offset tables and tensor maps do not depend on the schedule: uploaded once
  if (upload_tables(plan, base, s) != TN_OK) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return TN_ERR_CUDA;
  }
  auto trial = [&](float* ms) -> int {
    int r = build_packed(plan);
    if (r == TN_OK) r = upload_impl(plan, workspace, base + packed_offset(plan), s, false);
    if (r == TN_OK) r = run_impl(plan, workspace, s);
    if (r == TN_OK && cudaEventRecord(e0, s) != cudaSuccess) r = TN_ERR_CUDA;
    for (int k = 0; k < 2 && r == TN_OK; ++k) r = run_impl(plan, workspace, s);
    if (r == TN_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                       cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
      r = TN_ERR_CUDA;
    return r;
  };
  bool has[3] = {false, false, false};
  for (const auto& d : plan->descs) has[spec_class(d)] = true;
  // candidates: tile width 128 / 64, epilogue shape, and (long-k class only)
  // whole or cut k ranges; coordinate descent over the three classes
  std::vector<tn::PackedSchedule> cand;
  for (int cls = 0; cls < 3 && rc == TN_OK; ++cls) {
    if (!has[cls]) continue;
    cand.clear();
    // 256-wide tiles (BF16): P is loaded once per 256 result columns
    for (int w : {128, 64, 256})
      for (int s16 : {0, 1})
        for (int lk : {1, 0})
          // (BF16 stores through the epilogue's shared-memory transpose in
          // both read shapes: one candidate each)
          if ((cls == 2 || lk == 1) && (w != 256 || (plan->prec == TN_PREC_BF16 && cls != 0)) &&
              !(s16 && plan->prec == TN_PREC_BF16 && cls != 0))
            cand.push_back(tn::PackedSchedule{w, lk, s16});
    float best = 0.0f;
    tn::PackedSchedule pick = plan->sched[cls];
    for (size_t c = 0; c < cand.size() && rc == TN_OK; ++c) {
      plan->sched[cls] = cand[c];
      float ms = 0.0f;
      rc = trial(&ms);
      if (rc == TN_OK && (c == 0 || ms < best)) {
        best = ms;
        pick = cand[c];
      }
    }
    plan->sched[cls] = pick;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != TN_OK) return rc;
  rc = build_packed(plan);
  if (rc == TN_OK) rc = upload_impl(plan, workspace, base + packed_offset(plan), s, false);
  if (rc != TN_OK) return rc;
  std::lock_guard<std::mutex> lk(g_tune_lock);
  TunedSchedules& t = g_tune_cache[plan->signature];
  for (int c = 0; c < 3; ++c) t.sc[c] = plan->sched[c];
  return TN_OK;
}

int tn_group_plan_set_schedule(tn_group_plan* plan, int cls, int tile_width, int long_k, int store16) {
  if (!plan || cls < 0 || cls > 2 || (tile_width != 64 && tile_width != 128 && tile_width != 256)) return TN_ERR_ARG;
  if (tile_width == 256 && plan->prec != TN_PREC_BF16) return TN_ERR_UNSUPPORTED;
  if (!plan->packed) return TN_OK;
  plan->sched[cls] = tn::PackedSchedule{tile_width, long_k ? 1 : 0, store16 ? 1 : 0};
  return build_packed(plan);
}

int tn_group_plan_schedule(const tn_group_plan* plan, int cls, int* tile_width, int* long_k, int* store16) {
  if (!plan || cls < 0 || cls > 2 || !tile_width || !long_k || !store16) return TN_ERR_ARG;
  const tn::PackedSchedule& sc = plan->sched[cls];
  *tile_width = plan->packed ? sc.q_tile : TC_BN;
  *long_k = plan->packed ? sc.long_k : 0;
  *store16 = plan->packed ? sc.store16 : 0;
  return TN_OK;
}

void tn_group_plan_destroy(tn_group_plan* plan) { delete plan; }

}  // extern "C"
