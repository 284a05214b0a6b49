// Two-launch grouped contraction (pack + tcgen05 GEMM on packed bf16 blocks):
// device work-list records and the host plan that lays them out.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "tn_internal.h"

namespace tn {

// One operand of one contraction, packed K-major: block (tile, slab) holds
// rows tile*128 .. +127 and shared indices slab*kw .. +kw-1 (kw = 64 unless
// the other operand is read by the fused TMA GEMM) as bf16 in the
// 128-byte-swizzled layout (8-row atoms of 1 KB, 64 positions per row), at
// hi + (tile * slabs + slab) * block_bytes. Rows past the operand's end are
// not stored (a block of a 1..127-row operand is ceil8(rows) * 128 bytes);
// positions past kw or past K are stored as zeros.
struct PackJob {
  const float* src;
  uint8_t* hi;            // device: bf16(x) blocks
  uint8_t* lo;            // device: bf16(x - bf16(x)) blocks (BF16X3), else null
  int64_t R, K;           // rows (free-leg extent) and shared extent
  int64_t block_bytes;
  int32_t tiles, slabs;
  int32_t nr, nk;         // free legs and shared legs
  int32_t rfast, kfast;   // the source's unit stride is the last free / shared leg
  int32_t vec4;           // 16-byte copies: 1 along k, 2 along rows (every 4 consecutive
                          // elements from a 4-aligned index are contiguous and 16-byte
                          // aligned), 0 none
  int32_t rg, nbv;        // pack: rows per block, and blocks packed at once (nbv * rg <= 128)
  int32_t kw;             // shared indices per slab: 64, or the width of the TMA box of the
                          // fused TMA GEMM's P (positions kw .. 63 of a slab are zeros)
  int32_t pad_kw;
  const int32_t* rtab;    // device (fused P only): source offset of every row, R entries
  const int32_t* ktab;    // and of every shared index, K entries (32-byte aligned, zero-padded
                          // to whole 64-wide slabs)
  int64_t rtab_off, ktab_off;  // host: their element offsets in the plan's table region, -1 none
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
  int64_t tile_begin;     // first work unit (numbered per launch)
  int64_t K;              // shared extent (host: algorithmic bytes)
  uint64_t P_off, Q_off;  // host: offsets of the hi blocks in the packed region
  int32_t tiles_p, tiles_q, slabs, splits, slabs_per_split;
  int32_t q_tile;         // rows of Q per unit (the output tile's width): 64, 128, or 256 (BF16)
  int32_t store16;        // C row-major along j: drain TMEM as 16-lane x 256-bit blocks
                          // (whole-sector stores) instead of one row per thread
  int32_t pjob;           // fused: index of P's job in the job list (P is read as float32
                          // and rounded inside the GEMM, never packed); -1: P is packed
  int32_t p_mn;           // the P tile is MN-major (rows fastest), else K-major: fused with
                          // P contiguous along its rows, or packed P written by the caller
                          // as whole MN-major blocks (plan_single_packed)
  int32_t ph;             // rows of P per tile: 128, or the TMA box's height (fused TMA GEMM)
  int32_t kw;             // shared indices per slab: 64, or the TMA box's width
  int32_t bkmask;         // fused TMA GEMM: bit i set when dimension i of P's tensor map
                          // walks a shared leg (else a free leg, or a unit padding dimension)
  uint32_t bdim[5];       // extent of each tensor-map dimension, and the place value of its
  uint32_t bplace[5];     // leg in the flattened row or shared index (coordinate i of the box
                          // at row r0, shared index k0 = (r0 or k0) / bplace[i] % bdim[i])
  int32_t bk0, bk1, bkstep;  // the next box: bkstep more along map dimension bk0, carries
                             // into the dimensions up to bk1 (the shared legs)
  int32_t nsb;            // fused TMA GEMM: slabs per box (P with few rows: the staged
                          // tile holds nsb k-blocks of ceil8(ph) rows), else 1
  const void* tmap;       // device: P's tensor map (fused TMA GEMM), else null
  int64_t tmap_idx;       // host: its index in the plan's tensor-map list, -1 none
};

// The fused TMA GEMM's tiling of a contraction's P: tiles of ph rows x kw
// shared indices, each one box of P's tensor map (the leg permutation is done
// by the TMA unit: the box's dimensions are P's legs, ordered so that the
// staged tile is row-major along k, or along the rows when P is contiguous
// along them).
struct TmaBox {
  int32_t ph, kw, p_mn, kmask;
  uint32_t dim[5], place[5];
  int32_t k0, k1, kstep, nsb;
};
// One encoded tensor map (the driver's 128-byte CUtensorMap, 64-byte aligned).
struct alignas(64) TmaMap {
  uint8_t bytes[128];
};
// Box tiling and tensor map of d's P for the fused TMA GEMM. False when P's
// layout does not allow one (more than five legs of extent > 1, no unit
// stride on its last free or last shared leg, strides or the innermost box
// extent not multiples of 16 bytes, a box narrower than 32 shared indices on
// a longer k, or no driver entry point to encode the map).
bool plan_tma_box(const ContractDesc& d, TmaBox* box, TmaMap* map);

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
  std::vector<uint8_t> job_ext;    // written by the caller (MN-major blocks), not packed
  std::vector<PackUnit> units;
  std::vector<GemmDesc> gemms;     // one per contraction, in contraction order
  size_t packed_bytes = 0;
};

// Appends contraction d (units already planned by plan_units) to the plan
// under schedule sc (tile width and epilogue shape). fuse (allowed): a BF16
// contraction whose narrower operand has at most 64 rows takes the fused
// GEMM -- every element of its wider operand P is read by exactly one work
// unit, so rounding P inside the GEMM repeats no conversion, where packing it
// would cost 4 more bytes per element than reading it once; P is then not
// packed, and its job (with the offset tables at rtab_off / ktab_off) is kept
// for the fused GEMM's converters (pjob).
// box (or null): the contraction's TMA tiling, taken when it is fused; its
// tensor map is entry `map` of the plan's list.
// ext_p: A is written by the caller as whole MN-major blocks (not packed,
// never fused); TN_ERR_UNSUPPORTED if A would be the GEMM's narrower side.
int plan_packed(const ContractDesc& d, int prec, const PackedSchedule& sc, bool fuse, int64_t rtab_off,
                int64_t ktab_off, const TmaBox* box, int64_t map, PackedPlan* pp, bool ext_p = false);

// The operand on the MMA's 128-row side of contraction d: B when it has more
// rows and A fewer than 128, else A.
inline bool p_is_b(const ContractDesc& d) { return d.N > d.M && d.M < 128; }

// Appends to `tab` the source offsets of every row (R entries) and every
// shared index (K entries) of d's P operand, for the fused GEMM's converters
// (they then read offsets instead of dividing composite indices by leg
// lengths); returns the element offsets of the two runs.
void fused_tables(const ContractDesc& d, std::vector<int32_t>* tab, int64_t* rtab_off, int64_t* ktab_off);

int launch_pack(const PackJob* jobs, const PackUnit* units, int64_t nunits, cudaStream_t s);

// One contraction through pack + GEMM with its lists passed by value
// (launch-only, capturable): packed blocks go to `scratch` (256-byte
// aligned, at least packed_single_bytes(d, prec)); d's units are planned.
size_t packed_single_bytes(const ContractDesc& d, int prec);
// Upper bound of packed_single_bytes for an M x K by K x N contraction.
size_t packed_scratch_bound(int64_t M, int64_t N, int64_t K, int prec);
int contract_packed_single(const ContractDesc& d, int prec, void* scratch, size_t bytes, cudaStream_t s);

// The pieces of contract_packed_single, for callers that fuse work around
// them (the energy sweep): d's pack jobs (A, B) and GEMM descriptor with the
// packed blocks at `base` (256-byte aligned, `bytes` long), nothing launched.
// p_mn: the first operand A is the GEMM's P (never its narrower side) and is
// written by the caller as whole MN-major blocks of MN_BLOCK_BYTES (rows
// fastest, see mn_block_chunk) at ja.hi (+ ja.lo for BF16X3) instead of being
// packed; TN_ERR_UNSUPPORTED if A would be the narrower side.
struct SinglePacked {
  PackJob ja, jb;
  GemmDesc g;
  bool swap;
};
// q_tile: the output tile's width (128, or 256 for BF16).
int plan_single_packed(const ContractDesc& d, int prec, bool p_mn, int q_tile, uint8_t* base, size_t bytes,
                       SinglePacked* sp);
size_t single_packed_bytes(const ContractDesc& d, int prec, bool p_mn);
// Packs up to three jobs in one launch (b, c: null for none); maxbits (or
// null): raised with atomicMax to the bits of the largest |value| of job a.
int launch_pack_jobs(const PackJob* a, unsigned* maxbits, const PackJob* b, const PackJob* c, cudaStream_t s);
// The GEMM of a planned single contraction (its result zeroed first when its
// shared index is split).
int launch_gemm_single(const GemmDesc& g, int prec, cudaStream_t s);

// MN-major packed block: 128 rows x 64 shared indices of bf16, 16 KB, in the
// 128-byte-swizzled MN-major layout the MMA reads through an MN-major
// descriptor (atoms of 8 k-rows x 64 rows, 128 bytes per k-row; the two
// 64-row halves 8 KB apart, 8-row k groups 1 KB apart). The 16-byte chunk of
// rows 8 mg .. 8 mg + 7 at shared index k starts at mn_block_chunk(mg, k);
// row r within it at 2 (r % 8) bytes.
constexpr int MN_BLOCK_BYTES = 16384;
__host__ __device__ inline uint32_t mn_block_chunk(int mg, int k) {
  return (uint32_t)((mg >> 3) * 8192 + (k >> 3) * 1024 + (k & 7) * 128 + (((mg & 7) ^ (k & 7)) << 4));
}
// unit_ctr (or null: units assigned statically): the device counter the
// launch's CTAs claim units from (zeroed here, before the launch, on the same
// stream).
int launch_packed_gemm(const GemmDesc* descs, const int32_t* map, int64_t units, int prec, uint32_t* unit_ctr,
                       cudaStream_t s);
// The fused GEMM (BF16): units whose P is read as float32 through jobs[pjob]
// and rounded to bf16 in shared memory, Q packed.
int launch_fused_gemm(const GemmDesc* descs, const int32_t* map, const PackJob* jobs, int64_t units,
                      cudaStream_t s);
// The fused TMA GEMM (BF16): units whose P tiles are boxes of its tensor map
// (GemmDesc::tmap), loaded as float32 and rounded to bf16 in shared memory;
// its CTAs claim units from the device counter unit_ctr (zeroed here, before
// the launch, on the same stream).
int launch_tma_gemm(const GemmDesc* descs, const int32_t* map, int64_t units, uint32_t* unit_ctr, cudaStream_t s);

}  // namespace tn
