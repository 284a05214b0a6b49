// Two-launch grouped contraction (pack + tcgen05 GEMM on packed bf16 blocks):
// device work-list records and the host plan that lays them out.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "tn_internal.h"

namespace tn {

// One operand of one contraction, packed K-major: block (tile, slab) holds
// rows tile*128 .. +127 and shared indices slab*64 .. +63 as bf16 in the
// 128-byte-swizzled layout (8-row atoms of 1 KB), at hi + (tile * slabs +
// slab) * block_bytes. Rows past the operand's end are not stored (a block
// of a 1..127-row operand is ceil8(rows) * 128 bytes); shared indices past K
// are stored as zeros.
struct PackJob {
  const float* src;
  uint8_t* hi;            // device: bf16(x) blocks
  uint8_t* lo;            // device: bf16(x - bf16(x)) blocks (BF16X3), else null
  int64_t R, K;           // rows (free-leg extent) and shared extent
  int64_t block_bytes;
  int32_t tiles, slabs;
  int32_t nr, nk;         // free legs and shared legs
  int32_t rfast, kfast;   // the source's unit stride is the last free / shared leg
  int32_t rdim[TN_MAX_RANK];
  int32_t kdim[TN_MAX_RANK];
  int64_t rstr[TN_MAX_RANK];
  int64_t kstr[TN_MAX_RANK];
};

// Blocks first .. first+count-1 of one job, packed by one CTA.
struct PackUnit {
  int32_t job, first, count, pad;
};

// One contraction as D[i, j] = sum_k P[i, k] Q[j, k] on packed operands, P
// feeding the MMA's 128 rows and Q its columns; C[i * ci + j * cj] = D[i, j].
struct GemmDesc {
  const uint8_t* P;       // device: P hi blocks
  const uint8_t* Q;       // device: Q hi blocks
  float* C;
  int64_t P_lo, Q_lo;     // byte distance from a hi block to its lo block
  int64_t ci, cj;         // element strides of C along i and j
  int64_t RP, RQ;         // rows of P and of Q
  int64_t P_block, Q_block;
  int64_t tile_begin;     // first global work unit
  uint64_t P_off, Q_off;  // host: offsets of the hi blocks in the packed region
  int32_t tiles_p, tiles_q, slabs, splits, slabs_per_split;
  int32_t q_tile;         // rows of Q per unit (the output tile's width): 128 or 64
  int32_t store16;        // C row-major along j: drain TMEM as 16-lane x 256-bit blocks
                          // (whole-sector stores) instead of one row per thread
  int32_t pad;
};

// Schedule of the packed GEMM for one class of contractions: the output
// tile width (rows of Q per unit), whether a spec with many tiles keeps each
// tile's whole k range in one unit, and the epilogue's TMEM read shape.
// Picked by tn_group_plan_autotune.
struct PackedSchedule {
  int32_t q_tile = 128;
  int32_t long_k = 1;
  int32_t store16 = 0;
};

struct PackedPlan {
  std::vector<PackJob> jobs;       // two per contraction (A, B)
  std::vector<size_t> job_hi_off;  // offsets in the packed region
  std::vector<size_t> job_lo_off;  // SIZE_MAX when absent
  std::vector<PackUnit> units;
  std::vector<GemmDesc> gemms;     // one per contraction, in contraction order
  size_t packed_bytes = 0;
};

// Appends contraction d (units already planned by plan_units) to the plan
// under schedule sc (tile width and epilogue shape).
int plan_packed(const ContractDesc& d, int prec, const PackedSchedule& sc, PackedPlan* pp);

int launch_pack(const PackJob* jobs, const PackUnit* units, int64_t nunits, cudaStream_t s);

// One contraction through pack + GEMM with its lists passed by value
// (launch-only, capturable): packed blocks go to `scratch` (256-byte
// aligned, at least packed_single_bytes(d, prec)); d's units are planned.
size_t packed_single_bytes(const ContractDesc& d, int prec);
// Upper bound of packed_single_bytes for an M x K by K x N contraction.
size_t packed_scratch_bound(int64_t M, int64_t N, int64_t K, int prec);
int contract_packed_single(const ContractDesc& d, int prec, void* scratch, size_t bytes, cudaStream_t s);
int launch_packed_gemm(const GemmDesc* descs, const int32_t* map, int64_t units, int prec, cudaStream_t s);

}  // namespace tn
