// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/tn.h"

namespace tn {

// GEMM view of one pairwise contraction (edge flattening, Sec. III.B.2):
//   C[m, n] = sum_k A(m, k) B(k, n)
// m runs over A's free legs (A's order, last fastest), n over B's free legs,
// k over the shared legs in `kdim` order (last fastest). Element addresses are
// sums of per-leg index * stride, so any leg permutation or stride pattern of
// the inputs is read in place.
struct ContractDesc {
  const float* A;
  const float* B;
  float* C;
  int64_t M, N, K;
  int32_t nm, nn, nk;
  int32_t a_kfast;   // 1: A's unit-stride direction is k (else m)
  int32_t b_kfast;   // 1: B's unit-stride direction is k (else n)
  int32_t tiles_m, tiles_n;
  int32_t splits;      // k ranges the shared index is cut into (split-K); results are summed
                       // into C with float32 atomic adds when > 1, so C is zeroed first
  int32_t pad0;
  int64_t k_per_split; // shared indices per k range (a multiple of 64)
  int64_t tile_begin;  // first global work unit of this spec in a grouped launch
  int64_t pad1;        // size a multiple of 16 bytes (bulk async copies)
  int32_t mdim[TN_MAX_RANK];
  int32_t ndim[TN_MAX_RANK];
  int32_t kdim[TN_MAX_RANK];
  int64_t mstr[TN_MAX_RANK];
  int64_t nstr[TN_MAX_RANK];
  int64_t kstrA[TN_MAX_RANK];
  int64_t kstrB[TN_MAX_RANK];
};

// Validates one contraction and fills its descriptor (tile counts for the
// given tile shape). Returns a TN_* status.
int plan_contract(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                  int nshared, const tn_tensor* C, ContractDesc* d);

// Launchers. `group` (device array of descriptors sorted by decreasing unit
// work, tile_begin filled) with `unit_desc` (device array: descriptor index of
// every global work unit) is used when non-null; otherwise `single` is.
// Work unit u of a spec: tn = u % tiles_n, tm = (u / tiles_n) % tiles_m,
// split = u / (tiles_n * tiles_m).
int launch_contract_simt(const ContractDesc& single, const ContractDesc* group, const int32_t* unit_desc,
                         int64_t total_tiles, cudaStream_t stream);
int launch_contract_tc(const ContractDesc& single, const ContractDesc* group, const int32_t* unit_desc,
                       int64_t total_tiles, int prec, cudaStream_t stream);
// FP32 contraction with a small first operand (M, K <= SKINNY_MAX; any N):
// one thread per result column, the first operand in shared memory.
constexpr int SKINNY_MAX = 16;
int launch_contract_skinny(const ContractDesc& d, cudaStream_t stream);
// The same over an uploaded list of `count` such contractions (max_n: the
// largest N among them).
int launch_contract_skinny_grouped(const ContractDesc* descs, int count, int64_t max_n, cudaStream_t stream);

// Tile shapes of the kernels (used by the planner to count tiles).
constexpr int SIMT_BM = 128, SIMT_BN = 128;
constexpr int TC_BM = 128, TC_BN = 128;
// Longest k range of one work unit, in 64-wide slabs: a spec whose shared
// index is longer is split so no single CTA serialises a huge K.
constexpr int MAX_SLABS_PER_UNIT = 32;

// Sets tiles_m/n, splits and k_per_split; `min_units` asks for at least that
// many work units when K is long enough to split (keeping >= 4 slabs per unit).
void plan_units(ContractDesc* d, int64_t min_units);
// Work units a lone contraction asks plan_units for (two per SM).
int64_t min_units_single();
// The same for the packed GEMM (longer k ranges when a spec has many tiles).
void plan_units_packed(ContractDesc* d, bool long_k);

// Zeroes the results of split specs: list of (pointer, element count).
struct ZeroRange {
  float* ptr;
  int64_t count;
};
int launch_zero(const ZeroRange* ranges, int n, cudaStream_t stream);

// tn_contract without the C-ABI wrapper (used by the chain sweeps). With a
// scratch buffer large enough for the packed operands (BF16 / BF16X3), the
// contraction runs as pack + GEMM; otherwise on the single-pass kernels.
int contract_internal(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                      int nshared, const tn_tensor* C, int prec, cudaStream_t stream, void* scratch = nullptr,
                      size_t scratch_bytes = 0);

// tn_group_plan_create; allow_packed = false keeps BF16 / BF16X3 plans on
// the single-launch kernel, whose workspace holds only the work list.
// ext_p (or null): per spec, nonzero when its first operand A is written by
// the caller straight into the plan's packed region as whole MN-major
// blocks (BF16 / BF16X3 packed plans; A must be the GEMM's wider side): the
// plan packs no A for it and never fuses it.
int group_plan_create_ex(const tn_contract_spec* specs, int nspecs, int prec, bool allow_packed,
                         tn_group_plan** plan, const uint8_t* ext_p = nullptr);
// Where a caller-written A goes: spec `i` (numbered among the specs with a
// nonempty result), its blocks at packed + hi_off (+ lo_off for BF16X3; -1
// none), `tiles` x `slabs` blocks of 16 KB (block (t, s) at t * slabs + s),
// and the plan's order of its shared legs (kdim, kstrA as planned).
struct ExtPLayout {
  int64_t hi_off, lo_off;
  int32_t tiles, slabs, nk, pad;
  int32_t kdim[TN_MAX_RANK];
  int64_t kstrA[TN_MAX_RANK];
};
int group_plan_ext_layout(const tn_group_plan* plan, int i, ExtPLayout* out);

// Plans that run one after another on a stream can share one region for
// their packed bf16 blocks: the lists go to `lists` (group_plan_list_bytes),
// the blocks to `packed` (group_plan_packed_bytes, 256-byte aligned).
size_t group_plan_list_bytes(const tn_group_plan* plan);
size_t group_plan_packed_bytes(const tn_group_plan* plan);
int group_plan_upload_shared(const tn_group_plan* plan, void* lists, size_t bytes, void* packed, cudaStream_t s);
int group_plan_run_shared(const tn_group_plan* plan, void* lists, size_t bytes, cudaStream_t s);

// Step (ii) of an energy sweep with a deferred, exact rescale (mps.cu):
//   T2[w', s', a', b] = 2^-e sum_{w,s} W'[w, w', s, s'] T1[w, a', s, b],
// W' the MPO extended by the norm channel, e the binary exponent of *maxbits
// (the largest |L| entering the site; null at the first site), e ln 2 added
// to *lg by one thread.
struct StepII {
  const float* T1;
  float* T2;
  const float* W;
  int64_t Da, Db;
  int32_t wa, wb, d, pad;
  const unsigned* maxbits;
  double* lg;
};
// Step (ii) written straight into step (iii)'s packed operand (mps.cu):
// T2 is the first operand P of (iii) with row r = w' Db + b and shared index
// k = s' ps + a' pa, rounded to bf16 (and its remainder to bf16 for BF16X3)
// and stored as whole MN-major 128-row x 64-k blocks, block (tile, slab) at
// hi + (tile slabs + slab) 16 KB; positions past the last shared index are
// written as zeros. (Extended MPO bond) x d <= 8 on both sides.
struct StepIIPack {
  const float* T1;          // [wa][Da][d][Db], row-major
  const float* W;           // the site's extended MPO [wa][wb][d][d]
  const unsigned* maxbits;  // bits of the largest |L| (null: no rescale)
  double* lg;               // float64 log-scale: e ln 2 added
  uint8_t* hi;
  uint8_t* lo;              // BF16X3, else null
  int32_t Da, Db, wa, wb, d;
  int32_t tiles, slabs;     // of P: rows wb Db, shared indices d Da
  int32_t ps, pa;           // place values of s' and a' in the shared index
  int32_t pad;
};
// One launch for `count` chains (blockIdx.y: the chain); max_items: the
// largest work of one chain (Da Db / 8 columns groups, or Da Db).
int launch_step_ii_pack_grouped(const StepIIPack* descs, int count, int64_t max_items, cudaStream_t s);
// The place values (ps, pa) of s' and a' in the shared index of step (iii),
// from the planner's order of its two shared legs (kstrA of T2[w', s', a', b]).
void step_iii_places(int64_t Da, int64_t Db, int64_t d, const int64_t* kstrA, int32_t* ps, int32_t* pa);

// The energy sweep as one persistent cooperative launch (mps_persistent.cu):
// BF16 / BF16X3, at most 512 sites, (extended MPO bond) x d <= 8. Buffers
// from the energy sweep's workspace: environments L0 / L1 (with the first
// site's L0 = 1 in its channels), T1, the extended MPO Wx (site i at
// woff[i]), per-site max slots `bits` and the log-scale `lg` (zeroed), the
// barrier counter `bar` (4 bytes), the packed regions `scratch` / `scratch3`
// and `cores` (every site's core packed once per call).
struct ExpectBuffers {
  float *L0, *L1, *T1;
  const float* Wx;
  const int64_t* woff;
  unsigned* bits;
  double* lg;
  unsigned* bar;
  uint8_t* scratch;
  size_t scratch_bytes;
  uint8_t* scratch3;
  size_t scratch3_bytes;
  uint8_t* cores;  // every site's packed cores (expect_persistent_cores_bytes)
  size_t cores_bytes;
};
bool expect_persistent_ok(const tn_mps* psi, const tn_mpo* H, int prec);
size_t expect_persistent_cores_bytes(const tn_mps* psi);
int expect_persistent(const tn_mps* psi, const tn_mpo* H, int prec, const ExpectBuffers& w, double* result,
                      cudaStream_t s);

// wad, wbd: (extended MPO bond) x d on either side of the site.
int launch_mpo_step_ii_grouped(const StepII* descs, int count, int64_t max_cols, int64_t wad, int64_t wbd,
                               cudaStream_t s);
// The extended MPO W' of every site of H into out + off[i] (floats):
// W'[w, w', s, s'] = W[w, w', s, s'] on the original channels, the identity
// on the added channel (bond + 1 of every bond).
int launch_mpo_extend(const tn_mpo* H, float* out, const int64_t* off, cudaStream_t s);
bool mpo_extend_supported(const tn_mpo* H);

// Device status word (first error wins); defined in api.cu.
int* status_word();

// Bytes rounded up to the 256-byte alignment every workspace region keeps.
inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// True when `s` is being captured into a CUDA graph (or the query fails, as
// it does on the legacy stream while another stream captures). Calls that
// copy host lists which do not outlive them (plan uploads) refuse such a
// stream: a captured copy would replay from freed host memory.
// Raises kernel fn's dynamic shared-memory limit to `bytes` the first time it
// is launched on the current device: the attribute belongs to the function as
// loaded on each device, so `done` (one per kernel, static at the call site)
// keeps one bit per device. False when the device or the call fails.
inline bool smem_limit_once(const void* fn, size_t bytes, std::atomic<uint64_t>* done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  const uint64_t bit = uint64_t(1) << dev;
  if (done->load(std::memory_order_acquire) & bit) return true;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return false;
  done->fetch_or(bit, std::memory_order_acq_rel);
  return true;
}

inline bool stream_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return st != cudaStreamCaptureStatusNone;
}

}  // namespace tn
