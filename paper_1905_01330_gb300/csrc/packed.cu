// Grouped pairwise tensordot in two launches (bf16 operands, tcgen05):
//
//   1. pack: every operand of every contraction is gathered once through its
//      leg strides (the leg permutation and edge flattening of Sec. III.B.2
//      are folded into this gather), rounded to bf16 (and, for BF16X3, split
//      into hi + lo), and written as 128-row x 64-k blocks already in the
//      128-byte-swizzled K-major layout the MMA reads. HBM-bound: 4 bytes
//      read and 2 (hi) or 4 (hi + lo) written per element.
//   2. gemm: a persistent, warp-specialised tcgen05 kernel. Warp 0 moves
//      blocks into a ring of shared-memory stages with 1-D bulk async copies
//      (one copy per block: the layout needs no gather), warp 1 issues the
//      MMAs into a double-buffered TMEM accumulator, warps 2-9 drain TMEM and
//      write C while the next tile is multiplied.
//
// The per-tile float32 -> bf16 conversion of the single-launch kernel
// (contract_tc.cu) repeats for every output tile that reads an operand tile;
// here it happens once per element, and the MMA loop only moves bytes.
//
// The operand with more rows feeds the MMA's M side (128 TMEM lanes); the
// other one its N side, whose width per tile is cut to the rows present
// (multiple of 16), so a contraction with one thin side streams its wide
// operand at memory speed instead of filling a 128x128 tile with padding.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "gather.cuh"
#include "packed.h"
#include "ptx.cuh"

namespace tn {
namespace {

constexpr int PR = 128;                // rows per block
constexpr int PK = 64;                 // shared indices per block
constexpr int PBLOCK = PR * PK * 2;    // bytes of a full bf16 block (16 KB)
constexpr int PACK_THREADS = 256;

__device__ __forceinline__ uint32_t sw128_chunk(int r, int g) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t bf16x2_rn(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// ------------------------------------------------------------------- pack
// Each output chunk (one row, 8 consecutive shared indices: 16 bytes of
// bf16) is made by one thread from 8 float32 values it loads itself, so the
// blocks need no shared-memory staging and no barrier besides the one that
// publishes a block's offset tables. A thread takes PACK_CPT chunks per
// block and issues all their loads before converting any.
//  - Source with unit stride along k: a thread's 8 values are consecutive in
//    memory (two 16-byte loads when aligned); eight consecutive threads cover
//    a row's 64 shared indices, so a warp reads 4 x 256 contiguous bytes and
//    writes 4 whole 128-byte rows.
//  - Otherwise: consecutive threads take consecutive rows at the same 8
//    shared indices, so each of the 8 loads of a warp reads 32 consecutive
//    rows (128 contiguous bytes when the unit stride is along the rows).
constexpr int PACK_CPT = 4;  // chunks per thread and block (1024 chunks / 256 threads)

// A CTA packs "virtual blocks": J.nbv consecutive blocks of one tile at a
// time, J.rg rows each (nbv * rg <= 128). Operands with 128 rows or more (or
// more than 64) take one block at a time (rg = 128 or their row count); a
// narrow operand (at most 64 rows, e.g. the thin side of a contraction)
// takes 128 / rg of its slabs at once, so all threads have rows to pack.
struct PackSmem {
  int32_t roff[2][PR];           // source offset of each row of the tile (valid rows only)
  int32_t koff[2][PR * PK / 8];  // source offset of each shared index of the nbv slabs
  PackJob job;                   // the CTA's job, copied in once (its fields are read
                                 // throughout; from global memory each read would be a
                                 // long-latency load)
};
constexpr size_t PACK_SMEM = sizeof(PackSmem);

__device__ __forceinline__ void store_chunk(uint8_t* hi, uint8_t* lo, uint32_t off, const float (&v)[8]) {
  uint4 h;
  h.x = bf16x2_rn(v[0], v[1]);
  h.y = bf16x2_rn(v[2], v[3]);
  h.z = bf16x2_rn(v[4], v[5]);
  h.w = bf16x2_rn(v[6], v[7]);
  *reinterpret_cast<uint4*>(hi + off) = h;
  if (lo) {
    const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&h);
    uint4 l;
    l.x = bf16x2_rn(v[0] - __low2float(hb[0]), v[1] - __high2float(hb[0]));
    l.y = bf16x2_rn(v[2] - __low2float(hb[1]), v[3] - __high2float(hb[1]));
    l.z = bf16x2_rn(v[4] - __low2float(hb[2]), v[5] - __high2float(hb[2]));
    l.w = bf16x2_rn(v[6] - __low2float(hb[3]), v[7] - __high2float(hb[3]));
    *reinterpret_cast<uint4*>(lo + off) = l;
  }
}

// Virtual block: blocks b0 .. b0+nb-1 (nb <= J.nbv, one tile).
struct VBlock {
  int b0, nb, slab0, rv;  // first block, blocks, first slab, valid rows of the tile
};

__device__ __forceinline__ VBlock vblock(const PackJob& J, int b0, int nb) {
  VBlock v;
  const int tile = b0 / J.slabs;
  v.b0 = b0;
  v.nb = nb;
  v.slab0 = b0 - tile * J.slabs;
  const int64_t r0 = (int64_t)tile * PR;
  v.rv = (int)(J.R - r0 < PR ? J.R - r0 : PR);
  return v;
}

// Offset tables of virtual block v into slot `sl` (all threads).
__device__ __forceinline__ void block_tables(const PackJob& J, const VBlock& v, int sl, PackSmem& sm) {
  const int t = threadIdx.x;
  const int64_t r0 = (int64_t)(v.b0 / J.slabs) * PR;
  if (t < PR) sm.roff[sl][t] = t < v.rv ? (int32_t)leg_offset((uint32_t)(r0 + t), J.nr, J.rdim, J.rstr) : 0;
  // shared indices from thread 128 on, so one block's rows and shared
  // indices are decoded by different threads at once
  for (int e = t ^ PR; e < v.nb * PK; e += PACK_THREADS) {
    const int p = e & (PK - 1);
    const int64_t k = (int64_t)(v.slab0 + (e >> 6)) * J.kw + p;
    sm.koff[sl][e] = (p < J.kw && k < J.K) ? (int32_t)leg_offset((uint32_t)k, J.nk, J.kdim, J.kstr) : 0;
  }
}

// The chunks a thread makes for one virtual block: values and output
// coordinates (block -1: none).
struct ChunkRegs {
  float v[PACK_CPT][8];
  int rr[PACK_CPT], gg[PACK_CPT], bb[PACK_CPT];
};

// Loads this thread's chunks of virtual block v (tables in slot sl); zeros
// outside the valid rows and shared indices.
__device__ __forceinline__ void block_load(const PackJob& J, const VBlock& v, int sl, const PackSmem& sm,
                                           ChunkRegs& cr) {
  const int t = threadIdx.x;
  const float* __restrict__ src = J.src;
  const int32_t* roff = sm.roff[sl];
#pragma unroll
  for (int c = 0; c < PACK_CPT; ++c) {
    const int e = t + c * PACK_THREADS;
    int vr, grp;
    if (J.kfast) {
      vr = e >> 3;
      grp = e & 7;
    } else {
      vr = e & (PR - 1);
      grp = e >> 7;
    }
    const int bl = J.nbv == 1 ? 0 : vr / J.rg;
    const int r = vr - bl * J.rg;
    cr.rr[c] = r;
    cr.gg[c] = grp;
    cr.bb[c] = bl < v.nb ? bl : -1;
#pragma unroll
    for (int j = 0; j < 8; ++j) cr.v[c][j] = 0.0f;
    if (bl >= v.nb || r >= v.rv) continue;
    const int64_t kb = (int64_t)(v.slab0 + bl) * J.kw;
    const int kv = (int)(J.K - kb < J.kw ? J.K - kb : J.kw);
    const int32_t* koff = sm.koff[sl] + bl * PK;
    const int k0 = grp * 8;
    const float* rowp = src + roff[r];
    if (J.kfast && k0 + 7 < kv) {
      const int32_t ka = koff[k0];
      if (koff[k0 + 7] == ka + 7 && (reinterpret_cast<uintptr_t>(rowp + ka) & 15) == 0) {
        const float4 a = __ldg(reinterpret_cast<const float4*>(rowp + ka));
        const float4 d = __ldg(reinterpret_cast<const float4*>(rowp + ka) + 1);
        cr.v[c][0] = a.x; cr.v[c][1] = a.y; cr.v[c][2] = a.z; cr.v[c][3] = a.w;
        cr.v[c][4] = d.x; cr.v[c][5] = d.y; cr.v[c][6] = d.z; cr.v[c][7] = d.w;
        continue;
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (k0 + j < kv) cr.v[c][j] = __ldg(rowp + koff[k0 + j]);
  }
}

// Largest magnitude among this thread's loaded values (zeros stand in for
// positions outside the operand, so they never raise it).
__device__ __forceinline__ float chunk_absmax(const ChunkRegs& cr, float m) {
#pragma unroll
  for (int c = 0; c < PACK_CPT; ++c)
#pragma unroll
    for (int j = 0; j < 8; ++j) m = fmaxf(m, fabsf(cr.v[c][j]));
  return m;
}

// Converts and writes this thread's chunks of virtual block v (rows < ceil8(rv)).
__device__ __forceinline__ void block_write(const PackJob& J, const VBlock& v, const ChunkRegs& cr) {
  const int rs = (v.rv + 7) & ~7;
#pragma unroll
  for (int c = 0; c < PACK_CPT; ++c) {
    if (cr.bb[c] < 0 || cr.rr[c] >= rs) continue;
    const size_t b = (size_t)(v.b0 + cr.bb[c]);
    uint8_t* hi = J.hi + b * (size_t)J.block_bytes;
    uint8_t* lo = J.lo ? J.lo + b * (size_t)J.block_bytes : nullptr;
    store_chunk(hi, lo, sw128_chunk(cr.rr[c], cr.gg[c]), cr.v[c]);
  }
}

// Packs blocks first .. first+count-1 of job J (all threads of the CTA), one
// virtual block at a time. The offset tables of the next virtual block are
// decoded into the other slot while the loads of this one are in flight; one
// barrier per virtual block publishes them (and orders the reuse of a slot
// two virtual blocks later).
// MAX: also folds the largest |value| packed into *amax (this thread's).
template <bool MAX = false>
__device__ __forceinline__ void pack_blocks(const PackJob& J, int first, int count, PackSmem& sm,
                                            float* amax = nullptr) {
  if (count <= 0) return;
  const int nbv = J.nbv;
  VBlock v = vblock(J, first, min(nbv, count));
  block_tables(J, v, 0, sm);
  __syncthreads();
  ChunkRegs cr;
  for (int j = 0, sl = 0; j < count; j += nbv, sl ^= 1) {
    block_load(J, v, sl, sm, cr);
    if (MAX) *amax = chunk_absmax(cr, *amax);
    VBlock vn = v;
    if (j + nbv < count) {
      vn = vblock(J, first + j + nbv, min(nbv, count - j - nbv));
      block_tables(J, vn, sl ^ 1, sm);
    }
    block_write(J, v, cr);
    __syncthreads();
    v = vn;
  }
}

// Grouped form: one CTA per pack unit of the uploaded lists.
// Copies job J into shared memory (all threads, then a barrier).
__device__ __forceinline__ void stage_job(const PackJob& J, PackSmem& sm) {
  static_assert(sizeof(PackJob) % 4 == 0, "PackJob is copied as 32-bit words");
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&J);
  uint32_t* dst = reinterpret_cast<uint32_t*>(&sm.job);
  for (int i = threadIdx.x; i < (int)(sizeof(PackJob) / 4); i += PACK_THREADS) dst[i] = src[i];
  __syncthreads();
}

__global__ void __launch_bounds__(PACK_THREADS)
pack_kernel(const PackJob* __restrict__ jobs, const PackUnit* __restrict__ units) {
  extern __shared__ __align__(16) uint8_t pack_smem_raw[];
  PackSmem& sm = *reinterpret_cast<PackSmem*>(pack_smem_raw);
  const PackUnit un = units[blockIdx.x];
  stage_job(jobs[un.job], sm);
  pack_blocks(sm.job, un.first, un.count, sm);
}

// Single-contraction form: the jobs passed by value (nothing to upload, so
// the launch can be captured in a CUDA graph). CTAs 0 .. units_a-1 pack A,
// `per_a` blocks each; the next units_b pack B, `per_b` each; the rest pack
// the optional third job C (an operand of a later contraction packed in the
// same launch), `per_c` each. maxbits (or null): the bits of the largest
// |value| of A are raised to with atomicMax (non-negative floats order as
// their bit patterns do).
struct PackPair {
  PackJob a, b, c;
  int32_t units_a, units_b, per_a, per_b, per_c, pad;
  unsigned* maxbits;
};

__global__ void __launch_bounds__(PACK_THREADS)
pack_pair_kernel(const __grid_constant__ PackPair pp) {
  extern __shared__ __align__(16) uint8_t pack_smem_raw[];
  PackSmem& sm = *reinterpret_cast<PackSmem*>(pack_smem_raw);
  const int blk = (int)blockIdx.x;
  const int which = blk < pp.units_a ? 0 : (blk < pp.units_a + pp.units_b ? 1 : 2);
  stage_job(which == 0 ? pp.a : (which == 1 ? pp.b : pp.c), sm);
  const PackJob& J = sm.job;
  const int per = which == 0 ? pp.per_a : (which == 1 ? pp.per_b : pp.per_c);
  const int first = (blk - (which >= 1 ? pp.units_a : 0) - (which == 2 ? pp.units_b : 0)) * per;
  const int nb = J.tiles * J.slabs;
  if (which == 0 && pp.maxbits) {
    float m = 0.0f;
    pack_blocks<true>(J, first, min(per, nb - first), sm, &m);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(pp.maxbits, __float_as_uint(m));
    return;
  }
  pack_blocks(J, first, min(per, nb - first), sm);
}

// ------------------------------------------------------------------- gemm
// warp 0 copies, warp 1 issues the MMAs, then (fused GEMM only) eight
// converter warps, then the epilogue warps that drain TMEM: eight (two per
// lane quadrant, 64 of the tile's 128 columns each), or four in the fused
// GEMM (one per quadrant, all 128 columns: its tiles are narrow, and 14 warps
// leave each sub-partition's register file 128 registers per thread)
// BF16X3 promotes the TMEM accumulator into float32 registers every KC slabs
// (512 shared indices): the tensor core's float32 accumulation truncates, and
// over long k that error would exceed the split's own rounding error.
constexpr int KC = 8;

// Fused GEMM: eight converter warps copy each 128-row x 64-k float32 slab of
// P through its leg strides into a ring of XSLOTS staging slots (cp.async,
// XSLOTS - 1 slabs ahead of the one they round), then round it to bf16 into
// the stage the MMA reads. Each warp owns a fixed part of every slab -- its
// own rows, or its own 8 shared indices -- and runs ahead or behind the other
// warps at will: no barrier wider than a warp. Source offsets come from the
// job's precomputed row and shared-index tables, loaded into registers one
// slab before they are used, so no composite index is divided on the device.
// Each warp stages its part in its own fixed 4 KB of every slot, whatever the
// slab's layout or rows per warp, so a warp copying a later slab into a slot
// never overwrites what another warp has yet to round from it. Staging
// layouts of that 4 KB: "K" = up to 16 rows of 64 floats (256 B), the warp's
// rows, for sources contiguous along k (16-byte copies of 4 k, a warp's lanes
// on two 256-byte row runs) and for the 4-byte fallback (lanes on 32
// consecutive k); "R" = 8 k-rows of 128 floats (512 B), the warp's 8 shared
// indices, for sources contiguous along the rows (16-byte copies of 4 rows,
// lanes on one 512-byte run). Rounding reads and writes shared memory without
// bank conflicts in both.
constexpr int CONV_WARPS = 8;
// MN-major bf16 P tile (P contiguous along its rows): atoms of 8 k-rows x 64
// rows (128 B per k-row, 128-byte swizzle), the two 64-row halves MN_HALF
// bytes apart, 8-row k groups MN_KGROUP bytes apart
constexpr uint32_t MN_HALF = 8192;
constexpr uint32_t MN_KGROUP = 1024;
constexpr int XSLOTS = 4;
constexpr int XDIST = XSLOTS - 1;          // slabs copied ahead of the rounding
constexpr int XSLOT_BYTES = PR * PK * 4;   // 32 KB
constexpr int XPART = XSLOT_BYTES / CONV_WARPS;  // one converter warp's part of a slot (4 KB)
// Fused TMA GEMM: the same staging memory as a ring of bytes, each box at the
// next 128-byte boundary (wrapping to the ring's start rather than past its
// end), at most XBOXES boxes in it at once: more small boxes in flight than
// fixed slots would hold.
constexpr uint32_t XRING = XSLOTS * XSLOT_BYTES;  // 128 KB
constexpr int XBOXES = 8;
static_assert((XRING & (XRING - 1)) == 0, "ring size: a power of two");

// Ring position of the next box of `bytes` (rounded up to 128): advances the
// running position `v` (which counts the skipped tails too) and returns the
// box's start on it.
__device__ __forceinline__ uint64_t ring_take(uint64_t& v, uint32_t bytes) {
  const uint32_t b = (bytes + 127u) & ~127u;
  const uint32_t off = (uint32_t)(v & (XRING - 1));
  if (off + b > XRING) v += XRING - off;
  const uint64_t start = v;
  v += b;
  return start;
}

// FUSE: 0 -- P and Q packed; 1 -- P gathered by the converters' own copies
// (cp.async through offset tables); 2 -- P tiles loaded as boxes of its
// tensor map by one TMA warp, the converters only round.
template <int SPLIT, int FUSE>
struct GCfg {
  static constexpr int OPS = SPLIT ? 4 : 2;            // P hi, Q hi (, P lo, Q lo)
  // BF16 on packed operands: tiles up to 256 wide (Q up to two 128-row blocks)
  static constexpr bool WIDE = !SPLIT && !FUSE;
  static constexpr int STAGES = FUSE ? 3 : (SPLIT ? 3 : 4);
  // fused: P 16 KB + Q at most 64 rows (8 KB); fused TMA: P only (Q has a
  // ring of its own); wide: P 16 KB + Q 32 KB
  static constexpr int STAGE_BYTES =
      FUSE == 2 ? PBLOCK : (FUSE ? PBLOCK + PBLOCK / 2 : (WIDE ? 3 * PBLOCK : OPS * PBLOCK));
  // fused TMA GEMM: Q's blocks (at most 64 rows, 8 KB) in QSLOTS slots of
  // their own, copied as far ahead as the slots allow -- not gated by the
  // rounding of P, so their latency stays off the stages' turnaround
  static constexpr int QSLOTS = FUSE == 2 ? 4 : 0;
  static constexpr int QDIV = QSLOTS > 0 ? QSLOTS : 1;
  static constexpr int QSLOT_BYTES = PBLOCK / 2;
  static constexpr int ACC_COLS = WIDE ? 256 : 128;   // columns of one accumulator
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS; // two accumulators
  static constexpr int CONV = FUSE ? CONV_WARPS : 0;
  static constexpr int TMAW = FUSE == 2 ? 1 : 0;       // the warp issuing P's box loads
  // fused TMA GEMM: the converter warps form RGROUPS groups, each rounding
  // every RGROUPS-th box (two groups of four measured slower than one of
  // eight: the rounding is bound by throughput, not latency)
  static constexpr int RGROUPS = 1;
  static constexpr int RW = CONV / RGROUPS;            // warps rounding one box
  static constexpr int EPI0 = 2 + TMAW + CONV;         // first epilogue warp
  static constexpr int EPI = FUSE ? 4 : 8;             // epilogue warps
  static constexpr int ECOLS = ACC_COLS * 4 / EPI;     // at most this many accumulator columns per warp
  static constexpr int THREADS = 32 * (2 + TMAW + CONV + EPI);
  // BF16 on packed operands: each epilogue warp transposes its 32 x 32 blocks
  // through shared memory (16-byte chunks of a row XOR-permuted by row % 8:
  // 16-byte accesses conflict-free both ways), so a store instruction writes
  // four whole 128-byte row segments of C instead of 16 bytes in each of 32
  // rows
  // (and the fused TMA GEMM: its thin tiles' rows are short, so per-row
  // stores would touch 32 lines per instruction)
  static constexpr bool TR = !SPLIT && FUSE != 1;
  static constexpr int TR_BYTES = TR ? EPI * 32 * 32 * 4 : 0;
  static_assert(!(SPLIT && FUSE), "the fused GEMM is BF16 only");
};

template <int S>
struct GemmAux {
  uint64_t full[S];          // stage s holds its blocks
  uint64_t empty[S];         // the MMAs reading stage s are complete
  uint64_t xfull[XBOXES];    // fused TMA GEMM: box j (mod XBOXES) has landed in the ring
  uint64_t xempty[XBOXES];   // ... and the converters have rounded it
  uint64_t qfull[8];         // fused TMA GEMM: Q slot j holds its block
  uint64_t qempty[8];        // ... and the MMAs reading it are complete
  uint64_t uqfull[16];       // fused TMA GEMM: unit slot j (mod 16) is posted
  uint64_t uqempty[16];      // ... and every role has read it
  volatile int32_t uq[16];   // the posted units (-1: no more)
  uint64_t acc_full[2];      // accumulator b holds a finished chunk
  uint64_t acc_empty[2];     // the epilogue has drained accumulator b
  uint64_t final_bar;
  uint32_t tmem_base;
  volatile int32_t abort;
};

// This CTA's sequence of work units. Static: units blockIdx.x + n *
// gridDim.x. Dynamic (grouped launches of the GEMM on packed P and of the
// fused TMA GEMM): the first role to need a unit (the leader: the copy warp,
// or the box-load warp) claims units from a global counter, UQ_AHEAD ahead
// of the one it works on, and posts them in a ring of 16 slots; every other
// role (followers: one thread, or a whole warp of which lane 0 answers) reads
// them in order -- so a CTA that finishes early takes more units, and the
// launch ends when the work does rather than when the CTA with the most
// static units does. A follower reads unit n + 1 when it starts unit
// n (to load its descriptor early): claims stay at most UQ_AHEAD + 1 units
// ahead of the slowest role, within the ring. -1: none left.
constexpr int UQ = 16, UQ_AHEAD = 2;

template <int S>
struct UnitSeq {
  GemmAux<S>* x;
  uint32_t* ctr;
  int* status;
  int64_t total;
  uint32_t n, claimed;
  int mode;  // 0 static, 1 leader, 2 follower thread, 3 follower warp
  bool ended;

  __device__ __forceinline__ void claim() {
    if (ended) return;
    const uint32_t k = claimed, sl = k % UQ;
    if (!ptx::mbar_wait(ptx::smem_addr(&x->uqempty[sl]), ((k / UQ) & 1u) ^ 1u, status)) {
      x->abort = 1;
      ended = true;
      return;
    }
    const uint32_t u = atomicAdd(ctr, 1u);
    const int32_t v = (int64_t)u < total ? (int32_t)u : -1;
    x->uq[sl] = v;
    ptx::mbar_arrive(ptx::smem_addr(&x->uqfull[sl]));
    ++claimed;
    if (v < 0) ended = true;
  }
  __device__ __forceinline__ int64_t read(uint32_t k) {
    const uint32_t sl = k % UQ;
    if (mode == 1) return k < claimed ? (int64_t)x->uq[sl] : -1;
    bool ok = ptx::mbar_wait(ptx::smem_addr(&x->uqfull[sl]), (k / UQ) & 1u, status);
    if (mode == 3) ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
      x->abort = 1;
      return -1;
    }
    const int32_t v = x->uq[sl];
    if (mode == 3) __syncwarp();
    if (mode == 2 || (threadIdx.x & 31) == 0) ptx::mbar_arrive(ptx::smem_addr(&x->uqempty[sl]));
    return v;
  }
  __device__ __forceinline__ int64_t at_static(uint32_t k) const {
    const int64_t u = (int64_t)blockIdx.x + (int64_t)k * gridDim.x;
    return u < total ? u : -1;
  }
  __device__ __forceinline__ int64_t first() {
    n = 0;
    if (mode == 0) return at_static(0);
    if (mode == 1)
      for (int k = 0; k <= UQ_AHEAD; ++k) claim();
    return read(0);
  }
  __device__ __forceinline__ int64_t next() {
    ++n;
    if (mode == 0) return at_static(n);
    if (mode == 1) claim();
    return read(n);
  }
};

template <int S>
__device__ __forceinline__ UnitSeq<S> unit_seq(GemmAux<S>& x, uint32_t* ctr, int* status, int64_t total, int mode) {
  UnitSeq<S> q;
  q.x = &x;
  q.ctr = ctr;
  q.status = status;
  q.total = total;
  q.n = q.claimed = 0;
  q.mode = mode;
  q.ended = false;
  return q;
}

// Offsets of the 4-byte fallback copies (each converter warp its own).
struct ConvTables {
  int32_t roff[CONV_WARPS][16];  // the warp's 16 rows of the unit
  int32_t koff[CONV_WARPS][PK];  // the slab's 64 shared indices
};

template <int SPLIT, int FUSE>
constexpr size_t gemm_smem_bytes() {
  using C = GCfg<SPLIT, FUSE>;
  return 1024 + (size_t)C::STAGES * C::STAGE_BYTES + (size_t)C::QSLOTS * C::QSLOT_BYTES +
         (FUSE ? (size_t)XSLOTS * XSLOT_BYTES : 0) + (FUSE == 1 ? sizeof(ConvTables) : 0) + (size_t)C::TR_BYTES +
         sizeof(GemmAux<C::STAGES>);
}
static_assert(GCfg<0, 2>::QSLOTS <= 8, "Q slots: barrier pairs");
static_assert(gemm_smem_bytes<0, 2>() <= 227 * 1024, "fused TMA GEMM: shared memory");

struct GUnit {
  int64_t p0, q0;        // first row of P and of Q
  int32_t ks0, nks;      // first slab and slab count
};

// Unit u of descriptor d (u < 2^31: the host rejects larger launches); 32-bit
// division, far cheaper on the device than 64-bit. D: GemmDesc or one of the
// per-role views below.
template <class D>
__device__ __forceinline__ GUnit gunit(const D& d, int64_t u) {
  GUnit g;
  const uint32_t uu = (uint32_t)u, nq = (uint32_t)d.tiles_q, np = (uint32_t)d.tiles_p;
  const uint32_t rest = uu / nq, tq = uu - rest * nq;
  const uint32_t split = rest / np, tp = rest - split * np;
  g.p0 = (int64_t)tp * d.ph;
  g.q0 = (int64_t)tq * d.q_tile;
  g.ks0 = (int32_t)(split * (uint32_t)d.slabs_per_split);
  g.nks = (int32_t)(d.slabs - g.ks0 < d.slabs_per_split ? d.slabs - g.ks0 : d.slabs_per_split);
  return g;
}

__device__ __forceinline__ uint32_t rows_bytes(int64_t rows_left) {
  const int64_t r = rows_left < PR ? rows_left : PR;
  return (uint32_t)(((r + 7) & ~int64_t(7)) * 128);
}

// The descriptor of global unit u: from the uploaded list, or the by-value
// single descriptor when there is no list.
__device__ __forceinline__ GemmDesc load_desc(const GemmDesc& single, const GemmDesc* descs, const int32_t* map,
                                              int64_t u) {
  return descs ? descs[__ldg(map + u)] : single;
}

// The fields of a unit's descriptor the epilogue uses, loaded one by one (a
// copy of the whole descriptor, current and next, would hold ~80 registers).
struct EpiDesc {
  float* C;
  int64_t ci, cj, RP, RQ, tile_begin;
  int32_t tiles_q, tiles_p, slabs, slabs_per_split, q_tile, splits, store16, ph;
};

__device__ __forceinline__ EpiDesc load_epi(const GemmDesc& single, const GemmDesc* descs, const int32_t* map,
                                           int64_t u) {
  const GemmDesc* d = descs ? descs + __ldg(map + u) : &single;
  EpiDesc e;
  e.C = d->C;
  e.ci = d->ci;
  e.cj = d->cj;
  e.RP = d->RP;
  e.RQ = d->RQ;
  e.tile_begin = d->tile_begin;
  e.tiles_q = d->tiles_q;
  e.tiles_p = d->tiles_p;
  e.slabs = d->slabs;
  e.slabs_per_split = d->slabs_per_split;
  e.q_tile = d->q_tile;
  e.splits = d->splits;
  e.store16 = d->store16;
  e.ph = d->ph;
  return e;
}

// What the fused TMA GEMM's box-load warp reads of a unit's descriptor.
struct TmaDesc {
  const void* tmap;
  int64_t tile_begin;
  int32_t tiles_q, tiles_p, slabs, slabs_per_split, q_tile, ph, kw, bkmask, bk0, bk1, bkstep, nsb;
  uint32_t bdim[5], bplace[5];
};

__device__ __forceinline__ TmaDesc load_tma(const GemmDesc* descs, const int32_t* map, int64_t u) {
  const GemmDesc* d = descs + __ldg(map + u);
  TmaDesc e;
  e.tmap = d->tmap;
  e.tile_begin = d->tile_begin;
  e.tiles_q = d->tiles_q;
  e.tiles_p = d->tiles_p;
  e.slabs = d->slabs;
  e.slabs_per_split = d->slabs_per_split;
  e.q_tile = d->q_tile;
  e.ph = d->ph;
  e.kw = d->kw;
  e.bkmask = d->bkmask;
  e.bk0 = d->bk0;
  e.bk1 = d->bk1;
  e.bkstep = d->bkstep;
  e.nsb = d->nsb;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    e.bdim[i] = d->bdim[i];
    e.bplace[i] = d->bplace[i];
  }
  return e;
}

// What its rounding warps read.
struct RoundDesc {
  int64_t tile_begin;
  int32_t tiles_q, tiles_p, slabs, slabs_per_split, q_tile, ph, kw, p_mn, nsb;
};

__device__ __forceinline__ RoundDesc load_round(const GemmDesc* descs, const int32_t* map, int64_t u) {
  const GemmDesc* d = descs + __ldg(map + u);
  RoundDesc e;
  e.tile_begin = d->tile_begin;
  e.tiles_q = d->tiles_q;
  e.tiles_p = d->tiles_p;
  e.slabs = d->slabs;
  e.slabs_per_split = d->slabs_per_split;
  e.q_tile = d->q_tile;
  e.ph = d->ph;
  e.kw = d->kw;
  e.p_mn = d->p_mn;
  e.nsb = d->nsb;
  return e;
}

// Walks this CTA's (unit, slab) pairs in the order the copy warp and the MMA
// issuer consume them: the slab's first row and shared index, its valid rows
// and shared indices, the source job, its copy mode (PackJob::vec4), and
// whether it is the first slab of its unit.
struct ConvIter {
  int64_t u, total, p0, R, K;
  const float* src;
  const int32_t* rtab;
  const int32_t* ktab;
  int32_t ks, nks, ks0, mode;

  __device__ __forceinline__ void load(const GemmDesc* descs, const int32_t* map, const PackJob* jobs) {
    if (u >= total) return;
    const GemmDesc& d = descs[__ldg(map + u)];
    const GUnit g = gunit(d, u - d.tile_begin);
    p0 = g.p0;
    ks0 = g.ks0;
    nks = g.nks;
    ks = 0;
    const PackJob& J = jobs[d.pjob];
    src = J.src;
    rtab = J.rtab;
    ktab = J.ktab;
    R = J.R;
    K = J.K;
    mode = J.vec4;
  }
  __device__ __forceinline__ void next(const GemmDesc* descs, const int32_t* map, const PackJob* jobs) {
    if (++ks == nks) {
      u += gridDim.x;
      load(descs, map, jobs);
    }
  }
  __device__ __forceinline__ bool valid() const { return u < total; }
  __device__ __forceinline__ int64_t k0() const { return (int64_t)(ks0 + ks) * PK; }
  __device__ __forceinline__ int rv() const { return (int)(R - p0 < PR ? R - p0 : PR); }
  // shared indices left from this slab on: K - k0 < 2^31 (operands span
  // fewer than 2^31 elements), so 32-bit arithmetic suffices
  __device__ __forceinline__ int kv() const {
    const int left = (int)K - (ks0 + ks) * PK;
    return left < PK ? left : PK;
  }
  // what rounding needs, in one word: valid (bit 0), copy mode (bits 1-2),
  // valid rows (bits 3-10), valid shared indices (11-17)
  __device__ __forceinline__ uint32_t info() const {
    return valid() ? 1u | ((uint32_t)mode << 1) | ((uint32_t)rv() << 3) | ((uint32_t)kv() << 11) : 0u;
  }
};

// The table entries converter warp cw (lane l) needs for the slab `it`
// points at: mode 1 -- row (l / 16) + 2i of its rows (i < rpw / 2, on the
// unit's first slab) and shared index 4(l % 16); mode 2 -- row group l (4
// rows, on the first slab) and shared indices 8cw + i. Mode 0 keeps its
// tables in shared memory (ConvTables).
struct ConvRegs {
  int32_t r[8], k[8];
};

// Rows per converter warp in layout K: a tile's valid rows spread evenly over
// the eight warps (an even count, at most 16), so a tile with few rows takes
// proportionally less time.
__device__ __forceinline__ int conv_rpw(int rv) { return rv >= PR ? 16 : ((((rv + 7) >> 3) + 1) & ~1); }

// Row entries past the operand's end are read at its last row (always in
// bounds), shared-index entries past K in the run's zero padding; neither is
// used, so no select waits on the loads, which land while the current slab is
// rounded.
__device__ __forceinline__ void conv_fetch(const ConvIter& it, int cw, int l, ConvRegs& cr) {
  if (!it.valid() || it.mode == 0) return;
  const int64_t k0 = it.k0(), rl = it.R - 1;
  if (it.mode == 1) {
    if (it.ks == 0) {
      const int rpw = conv_rpw(it.rv());
#pragma unroll
      for (int i = 0; i < 8; ++i) cr.r[i] = __ldg(it.rtab + min(it.p0 + rpw * cw + (l >> 4) + 2 * i, rl));
    }
    cr.k[0] = __ldg(it.ktab + k0 + 4 * (l & 15));  // inside the padded run
  } else {
    if (it.ks == 0) cr.r[0] = __ldg(it.rtab + min(it.p0 + 4 * l, rl));
    // the run is 32-byte aligned and padded to whole slabs (fused_tables)
    const int4* kp = reinterpret_cast<const int4*>(it.ktab + k0 + 8 * cw);
    const int4 k03 = __ldg(kp), k47 = __ldg(kp + 1);
    cr.k[0] = k03.x;
    cr.k[1] = k03.y;
    cr.k[2] = k03.z;
    cr.k[3] = k03.w;
    cr.k[4] = k47.x;
    cr.k[5] = k47.y;
    cr.k[6] = k47.z;
    cr.k[7] = k47.w;
  }
}

// Converter warp cw issues its copies of slab `it` into staging slot `xs`
// (shared address), with the table entries in cr (modes 1 and 2).
__device__ __forceinline__ void conv_copy(const ConvIter& it, const ConvRegs& cr, int cw, int l, ConvTables& tb,
                                          uint32_t xs) {
  const int rv = it.rv(), kv = it.kv();
  const float* __restrict__ src = it.src;
  const int rpw = conv_rpw(rv);
  if (it.mode == 1) {
    // rpw rows x 16 chunks of 4 k; an instruction covers two 256-byte rows.
    // Chunk q lands at position q ^ ((q >> 3) & 1) of its row (see conv_round).
    const int q = l & 15;
    const uint32_t dst = xs + (uint32_t)(cw * XPART + (l >> 4) * 256 + ((q ^ ((q >> 3) & 1)) << 4));
    const float* base = src + cr.k[0];
    if (rv == PR && kv == PK) {
#pragma unroll
      for (int i = 0; i < 8; ++i) ptx::cp_async16(dst + i * 512, base + cr.r[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = rpw * cw + (l >> 4) + 2 * i;
        if (2 * i < rpw && r < rv && 4 * q < kv) ptx::cp_async16(dst + i * 512, base + cr.r[i]);
      }
    }
  } else if (it.mode == 2) {
    // 8 k-rows x 32 chunks of 4 rows; an instruction covers one 512-byte k-row
    const uint32_t dst = xs + (uint32_t)(cw * XPART + l * 16);
    const float* base = src + cr.r[0];
    if (rv == PR && kv == PK) {
#pragma unroll
      for (int i = 0; i < 8; ++i) ptx::cp_async16(dst + i * 512, base + cr.k[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i)
        if (8 * cw + i < kv && 4 * l < rv) ptx::cp_async16(dst + i * 512, base + cr.k[i]);
    }
  } else {
    // rpw rows x 64 k, one float each; an instruction covers 32 consecutive k
    int32_t* roff = tb.roff[cw];
    int32_t* koff = tb.koff[cw];
    const int64_t k0 = it.k0();
    __syncwarp();  // the previous slab's copies have read the tables
    if (it.ks == 0 && l < rpw) roff[l] = rpw * cw + l < rv ? __ldg(it.rtab + it.p0 + rpw * cw + l) : 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) koff[l + 32 * h] = l + 32 * h < kv ? __ldg(it.ktab + k0 + l + 32 * h) : 0;
    __syncwarp();
    for (int i = 0; i < 2 * rpw; ++i) {
      const int e = l + 32 * i, rl = e >> 6, k = e & 63, r = rpw * cw + rl;
      const int qk = k >> 2, pos = qk ^ ((qk >> 3) & 1);  // chunk position, as in mode 1
      if (r < rv && k < kv)
        ptx::cp_async4(xs + (uint32_t)(cw * XPART + rl * 256 + pos * 16 + 4 * (k & 3)), src + roff[rl] + koff[k]);
    }
  }
}

// Converter warp cw rounds its part of a staged slab (info word w, slot
// `xs`) into the bf16 P tile `pt`; zeros outside the valid rows and shared
// indices (rows past the end could hold anything -- their products are never
// stored -- but shared indices past the end must be zero). All shared-memory
// loads are issued before the first store.
__device__ __forceinline__ void conv_round(uint32_t w, int cw, int l, const uint8_t* xs, uint8_t* pt) {
  const int mode = (int)((w >> 1) & 3), rv = (int)((w >> 3) & 255), kv = (int)((w >> 11) & 127);
  const bool full = rv == PR && kv == PK;
  float v[4][8];
  if (mode != 2) {
    // chunk (r, g) = row r, k 8g .. 8g+7 of the warp's rpw rows; an
    // instruction takes 4 rows x 8 chunks. The copies stored the two 16-byte
    // halves of chunk g swapped when g >= 4 (hf = 1), so reading the half at
    // position 2g + hf first takes k 8g .. 8g+3 and spreads the
    // instruction's loads over all eight bank groups
    const int g = l & 7, hf = (g >> 2) & 1, rpw = conv_rpw(rv);
    if (rpw < 16) {
      // few rows: chunks (l / 8) + 4i of the warp's rows, i < rpw / 4 (the
      // same bank-group order of the two 16-byte halves as below)
      for (int i = 0; 4 * i < rpw; ++i) {
        const int rl = (l >> 3) + 4 * i, r = rpw * cw + rl;
        if (rl >= rpw) continue;
        const uint8_t* row = xs + cw * XPART + rl * 256 + g * 32;
        const float4 lo = *reinterpret_cast<const float4*>(row + 16 * hf);
        const float4 hi = *reinterpret_cast<const float4*>(row + 16 * (1 - hf));
        float u[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (!(r < rv && 8 * g + j < kv)) u[j] = 0.0f;
        store_chunk(pt, nullptr, sw128_chunk(r, g), u);
      }
      return;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint8_t* row = xs + cw * XPART + ((l >> 3) + 4 * i) * 256 + g * 32;
      const float4 lo = *reinterpret_cast<const float4*>(row + 16 * hf);
      const float4 hi = *reinterpret_cast<const float4*>(row + 16 * (1 - hf));
      v[i][0] = lo.x; v[i][1] = lo.y; v[i][2] = lo.z; v[i][3] = lo.w;
      v[i][4] = hi.x; v[i][5] = hi.y; v[i][6] = hi.z; v[i][7] = hi.w;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = 16 * cw + (l >> 3) + 4 * i;
      if (!full) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (!(r < rv && 8 * g + j < kv)) v[i][j] = 0.0f;
      }
      store_chunk(pt, nullptr, sw128_chunk(r, g), v[i]);
    }
  } else {
    // MN-major tile: the warp's k group g = cw (8 k-rows), rows 4l .. 4l+3
    // of each: one 16-byte load of 4 rows per k-row, rounded to 4 bf16 and
    // stored as 8 bytes at row group l / 2 (k-row chunks XOR-swizzled by k %
    // 8, as the MN-major descriptor reads them). Shared indices past kv are
    // zeros; rows past rv are never stored, so they may hold anything.
    const int g = cw, mg = l >> 1;
    const uint32_t base = (uint32_t)((mg >> 3) * MN_HALF + g * MN_KGROUP + (l & 1) * 8);
    float4 f[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = *reinterpret_cast<const float4*>(xs + cw * XPART + j * 512 + l * 16);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool ok = full || 8 * g + j < kv;
      uint2 h;
      h.x = ok ? bf16x2_rn(f[j].x, f[j].y) : 0u;
      h.y = ok ? bf16x2_rn(f[j].z, f[j].w) : 0u;
      *reinterpret_cast<uint2*>(pt + base + j * 128 + (((mg & 7) ^ j) << 4)) = h;
    }
  }
}

// Fused TMA GEMM: warp wi of the NW warps rounding one staged box (shared
// address xs) writes its part of the bf16 P tile (shared address pt).
// p_mn = 0: the box is ph rows x nsb * kw shared indices, row-major along k,
// covering nsb slabs; slab j of row r goes to row j * ceil8(ph) + r of the
// tile (the MMA reads slab j's k-block from that row on). Lane l takes
// shared indices 4q .. 4q+3 (q = l % 16) of each slab of rows r0 + 2 NW i
// (r0 = 2 wi + l / 16) and writes them K-major (zeros at q >= kw / 4): rows
// 2 NW apart are 2 NW / 8 swizzle atoms (of 1 KB) apart at the same position
// in their atom, as are k-blocks (ceil8(ph) rows apart), so both addresses
// advance by steps. At most 8 (slab, row) pairs per lane: nsb * ceil(ph / 16)
// <= 8 (the planner's bound). p_mn = 1 (one slab): the box is kw k-rows x ph
// rows, row-major along the rows; lane l takes rows 4l .. 4l+3 of the k-rows
// of 8-row groups wi + NW j and writes them MN-major (zeros at k >= kw). Rows
// past ph are left as they are: their products are never stored. Both read
// each 16-byte run of the box with consecutive lanes on consecutive runs, and
// write whole 128-byte rows of the tile per 16 lanes: no bank conflicts.
// Loads go out 8 at a time before their conversions.
template <int NW>
__device__ __forceinline__ void round_box(int p_mn, int ph, int kw, int nsb, int wi, int l, uint32_t xs,
                                          uint32_t pt) {
  float4 v[8];
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!p_mn) {
    static_assert((2 * NW) % 8 == 0, "rows of one step: whole swizzle atoms");
    const int q = l & 15, r0 = 2 * wi + (l >> 4);
    const bool kin = q < (kw >> 2);
    const int wrow = nsb * kw;                          // floats per staged row
    const uint32_t ld0 = xs + (uint32_t)((r0 * wrow + 4 * q) * 4);
    const uint32_t ldrow = (uint32_t)(2 * NW * wrow * 4), ldslab = (uint32_t)(kw * 4);
    const uint32_t st0 = pt + sw128_chunk(r0, q >> 1) + 8 * (q & 1);
    constexpr uint32_t strow = 2 * NW / 8 * 1024;
    const uint32_t stslab = (uint32_t)(((ph + 7) & ~7) * 128);
    const int nrows = ph - r0;  // this lane's rows: r0 + 2 NW i < ph
    const int ni = (ph - 2 * wi + 2 * NW - 1) / (2 * NW);  // row steps of this warp (uniform)
    if (ni <= 0) return;
    if (nsb == 1) {
#pragma unroll
      for (int h = 0; h < 64 / NW; h += 8) {
        if (h >= ni) break;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int ii = h + i;
          v[i] = (2 * NW * ii < nrows && kin) ? ptx::ld_shared_v4(ld0 + (uint32_t)ii * ldrow) : zero;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int ii = h + i;
          if (2 * NW * ii < nrows)
            ptx::st_shared_v2(st0 + (uint32_t)ii * strow, bf16x2_rn(v[i].x, v[i].y), bf16x2_rn(v[i].z, v[i].w));
        }
      }
    } else {
      // (slab j, row step i) pairs t = j * ni + i, t < nsb * ni <= 8
      const int nt = nsb * ni;
      int j = 0, i = 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v[t] = (t < nt && 2 * NW * i < nrows && kin)
                   ? ptx::ld_shared_v4(ld0 + (uint32_t)i * ldrow + (uint32_t)j * ldslab)
                   : zero;
        if (++i == ni) { i = 0; ++j; }
      }
      j = 0;
      i = 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (t < nt && 2 * NW * i < nrows)
          ptx::st_shared_v2(st0 + (uint32_t)i * strow + (uint32_t)j * stslab, bf16x2_rn(v[t].x, v[t].y),
                            bf16x2_rn(v[t].z, v[t].w));
        if (++i == ni) { i = 0; ++j; }
      }
    }
  } else {
    const int m = 4 * l;
    if (m >= ph) return;
    const uint32_t ldstep = (uint32_t)(ph * 4);
    const int mg = (m & 63) >> 3;
#pragma unroll
    for (int gi = 0; gi < 8 / NW; ++gi) {
      const int g = wi + NW * gi;  // 8-row k group
      const uint32_t ld0 = xs + (uint32_t)((8 * g * ph + m) * 4);
      const int kin = kw - 8 * g;  // k-rows of the group inside the box
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) v[jj] = jj < kin ? ptx::ld_shared_v4(ld0 + (uint32_t)jj * ldstep) : zero;
      const uint32_t st0 = pt + (uint32_t)((m >> 6) * MN_HALF + g * MN_KGROUP + (m & 7) * 2);
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        ptx::st_shared_v2(st0 + jj * 128 + ((mg ^ jj) << 4), bf16x2_rn(v[jj].x, v[jj].y),
                          bf16x2_rn(v[jj].z, v[jj].w));
    }
  }
}

template <int SPLIT, int FUSE>
__global__ void __launch_bounds__(GCfg<SPLIT, FUSE>::THREADS, 1)
packed_gemm_kernel(const __grid_constant__ GemmDesc single, const GemmDesc* __restrict__ descs,
                   const int32_t* __restrict__ map, const PackJob* __restrict__ jobs, int64_t total_units,
                   uint32_t* unit_ctr, int* status) {
  using Cf = GCfg<SPLIT, FUSE>;
  constexpr int S = Cf::STAGES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // after the stages: fused TMA -- Q's slots; fused -- the staging slots
  // (or ring), then (converters' copies) their tables; BF16 on packed
  // operands -- the epilogue's transpose buffers; then the barriers
  uint8_t* qring = smem + (size_t)S * Cf::STAGE_BYTES;
  uint8_t* xstage = qring + (size_t)Cf::QSLOTS * Cf::QSLOT_BYTES;
  ConvTables& tb = *reinterpret_cast<ConvTables*>(xstage + (FUSE ? (size_t)XSLOTS * XSLOT_BYTES : 0));
  uint8_t* trb = xstage + (FUSE ? (size_t)XSLOTS * XSLOT_BYTES : 0) + (FUSE == 1 ? sizeof(ConvTables) : 0);
  float* trbuf = reinterpret_cast<float*>(trb);
  GemmAux<S>& x = *reinterpret_cast<GemmAux<S>*>(trb + Cf::TR_BYTES);
  const uint32_t stage0 = ptx::smem_addr(smem), qring0 = ptx::smem_addr(qring);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;

  if (t == 0) {
    for (int s = 0; s < S; ++s) {
      // the copy warp's transaction arrival (unless Q has its own slots) and
      // one per converter warp rounding the stage's P
      ptx::mbar_init(ptx::smem_addr(&x.full[s]), (FUSE == 2 ? 0 : 1) + Cf::RW);
      ptx::mbar_init(ptx::smem_addr(&x.empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&x.acc_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&x.acc_empty[b]), Cf::EPI);
    }
    if (unit_ctr)
      for (int q = 0; q < UQ; ++q) {
        ptx::mbar_init(ptx::smem_addr(&x.uqfull[q]), 1);  // the leader's post
        // every other role's read: MMA issuer, epilogue warps (and, fused
        // TMA, the copy thread and the rounding warps)
        ptx::mbar_init(ptx::smem_addr(&x.uqempty[q]), FUSE == 2 ? 2 + Cf::CONV + Cf::EPI : 1 + Cf::EPI);
      }
    for (int q = 0; q < Cf::QSLOTS; ++q) {
      ptx::mbar_init(ptx::smem_addr(&x.qfull[q]), 1);   // the copy's transaction arrival
      ptx::mbar_init(ptx::smem_addr(&x.qempty[q]), 1);  // the MMA issuer's commit
    }
    if (FUSE == 2)
      for (int q = 0; q < XBOXES; ++q) {
        ptx::mbar_init(ptx::smem_addr(&x.xfull[q]), 1);           // the TMA warp's transaction arrival
        ptx::mbar_init(ptx::smem_addr(&x.xempty[q]), Cf::RW);     // one per warp rounding the box
      }
    ptx::mbar_init(ptx::smem_addr(&x.final_bar), 1);
    x.abort = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 1) {
    ptx::tmem_alloc(ptx::smem_addr(&x.tmem_base), Cf::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = x.tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t gs = 0;
      // each role loads the descriptor of its next unit while the current
      // one runs, so unit boundaries do not wait on global-memory latency
      UnitSeq<S> us = unit_seq(x, unit_ctr, status, total_units, !unit_ctr ? 0 : (FUSE == 2 ? 2 : 1));
      int64_t u = us.first(), un = 0;
      GemmDesc dn = load_desc(single, descs, map, u >= 0 ? u : 0);
      for (; u >= 0 && !x.abort; u = un) {
        const GemmDesc d = dn;
        un = us.next();
        if (un >= 0) dn = load_desc(single, descs, map, un);
        const GUnit g = gunit(d, u - d.tile_begin);
        const int64_t qleft = d.RQ - g.q0 < d.q_tile ? d.RQ - g.q0 : d.q_tile;
        // a 256-wide tile takes its Q rows from two consecutive 128-row blocks
        // an MN-major packed P block is stored whole (its two 64-row halves 8 KB apart)
        const uint32_t pb = FUSE ? 0u : (d.p_mn ? (uint32_t)PBLOCK : rows_bytes(d.RP - g.p0)), qb = rows_bytes(qleft);
        const uint32_t qb2 = qleft > PR ? rows_bytes(qleft - PR) : 0u;
        const uint32_t tx = (pb + qb + qb2) * (SPLIT ? 2u : 1u);
        const uint8_t* pbase = d.P + ((g.p0 / PR) * d.slabs + g.ks0) * d.P_block;
        // a 64-row tile starts 64 rows (8 atoms, 8 KB) into its 128-row block
        const uint8_t* qbase = d.Q + ((g.q0 / PR) * d.slabs + g.ks0) * d.Q_block + (g.q0 % PR) * 128;
        bool ok = true;
        const int step = FUSE == 2 ? d.nsb : 1;  // slabs per stage
        for (int ks = 0; ks < g.nks; ks += step, ++gs) {
          if (FUSE == 2) {
            // Q alone (the box's slabs: consecutive blocks), into its own slot
            const int qs = (int)(gs % Cf::QDIV);
            if (!ptx::mbar_wait(ptx::smem_addr(&x.qempty[qs]), ((gs / Cf::QDIV) & 1u) ^ 1u, status)) {
              ok = false;
              break;
            }
            const uint32_t qf = ptx::smem_addr(&x.qfull[qs]);
            const uint32_t qbytes = (uint32_t)(step - 1) * (uint32_t)d.Q_block + qb;
            ptx::mbar_arrive_expect_tx(qf, qbytes);
            ptx::bulk_copy_g2s(qring0 + (uint32_t)qs * Cf::QSLOT_BYTES, qbase + ks * d.Q_block, qbytes, qf);
            continue;
          }
          const int s = (int)(gs % S);
          if (!ptx::mbar_wait(ptx::smem_addr(&x.empty[s]), ((gs / S) & 1u) ^ 1u, status)) { ok = false; break; }
          const uint32_t full = ptx::smem_addr(&x.full[s]);
          const uint32_t st = stage0 + (uint32_t)s * Cf::STAGE_BYTES;
          ptx::mbar_arrive_expect_tx(full, tx);
          if (!FUSE) ptx::bulk_copy_g2s(st, pbase + ks * d.P_block, pb, full);
          ptx::bulk_copy_g2s(st + PBLOCK, qbase + ks * d.Q_block, qb, full);
          if (qb2) ptx::bulk_copy_g2s(st + 2 * PBLOCK, qbase + (d.slabs + ks) * d.Q_block, qb2, full);
          if (SPLIT) {
            ptx::bulk_copy_g2s(st + 2 * PBLOCK, pbase + d.P_lo + ks * d.P_block, pb, full);
            ptx::bulk_copy_g2s(st + 3 * PBLOCK, qbase + d.Q_lo + ks * d.Q_block, qb, full);
          }
        }
        if (!ok) { x.abort = 1; break; }
      }
      // copies still in flight land before the CTA can exit
      if (FUSE == 2) {
        const uint32_t first = gs > (uint32_t)Cf::QDIV ? gs - (uint32_t)Cf::QDIV : 0u;
        for (uint32_t q = first; q < gs; ++q)
          ptx::mbar_wait(ptx::smem_addr(&x.qfull[q % Cf::QDIV]), (q / Cf::QDIV) & 1u, status);
      } else {
        const uint32_t first = gs > (uint32_t)S ? gs - (uint32_t)S : 0u;
        for (uint32_t q = first; q < gs; ++q)
          ptx::mbar_wait(ptx::smem_addr(&x.full[q % S]), (q / S) & 1u, status);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t gs = 0, gc = 0;
      UnitSeq<S> us = unit_seq(x, unit_ctr, status, total_units, unit_ctr ? 2 : 0);
      int64_t u = us.first(), un = 0;
      GemmDesc dn = load_desc(single, descs, map, u >= 0 ? u : 0);
      for (; u >= 0 && !x.abort; u = un) {
        const GemmDesc d = dn;
        un = us.next();
        if (un >= 0) dn = load_desc(single, descs, map, un);
        const GUnit g = gunit(d, u - d.tile_begin);
        const int64_t qrows = d.RQ - g.q0 < d.q_tile ? d.RQ - g.q0 : d.q_tile;
        const int nmma = (int)((qrows + 15) & ~int64_t(15));
        const uint32_t idesc = ptx::idesc_bf16_f32(PR, nmma, d.p_mn, 0);
        const int chunk = SPLIT ? KC : g.nks;
        const int step = FUSE == 2 ? d.nsb : 1;  // slabs per stage
        // fused TMA: slab j of a stage at row j * ceil8(ph) of the P tile,
        // and Q's block j after the first j blocks of its slot
        const uint32_t pslab = (uint32_t)(((d.ph + 7) & ~7) * 128), qslab = (uint32_t)d.Q_block;
        bool ok = true;
        for (int c0 = 0; c0 < g.nks && ok; c0 += chunk, ++gc) {
          const int b = (int)(gc & 1);
          if (!ptx::mbar_wait(ptx::smem_addr(&x.acc_empty[b]), ((gc >> 1) & 1u) ^ 1u, status)) { ok = false; break; }
          ptx::tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * Cf::ACC_COLS);
          const int c1 = min(g.nks, c0 + chunk);
          for (int ks = c0; ks < c1; ks += step, ++gs) {
            const int s = (int)(gs % S), qs = (int)(gs % Cf::QDIV);
            if (!ptx::mbar_wait(ptx::smem_addr(&x.full[s]), (gs / S) & 1u, status)) { ok = false; break; }
            if (FUSE == 2 && !ptx::mbar_wait(ptx::smem_addr(&x.qfull[qs]), (gs / Cf::QDIV) & 1u, status)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t st = stage0 + (uint32_t)s * Cf::STAGE_BYTES;
            const uint32_t qst = FUSE == 2 ? qring0 + (uint32_t)qs * Cf::QSLOT_BYTES : st + PBLOCK;
            for (int j = 0; j < step; ++j) {
              const uint32_t pj = st + (uint32_t)j * pslab, qj = qst + (uint32_t)j * qslab;
#pragma unroll
              for (int kk = 0; kk < PK / 16; ++kk) {
                if (16 * kk >= d.kw) break;  // positions past kw are zeros on both sides
                const uint64_t pd = d.p_mn ? ptx::sw128_mnmajor_desc(pj + kk * 2 * MN_KGROUP, MN_HALF, MN_KGROUP)
                                           : ptx::sw128_kmajor_desc(pj + kk * 32);
                const uint64_t qd = ptx::sw128_kmajor_desc(qj + kk * 32);
                ptx::mma_bf16(dt, pd, qd, idesc, (ks == c0 && j == 0 && kk == 0) ? 0u : 1u);
                if (SPLIT) {
                  const uint64_t pl =
                      d.p_mn ? ptx::sw128_mnmajor_desc(st + 2 * PBLOCK + kk * 2 * MN_KGROUP, MN_HALF, MN_KGROUP)
                             : ptx::sw128_kmajor_desc(st + 2 * PBLOCK + kk * 32);
                  const uint64_t ql = ptx::sw128_kmajor_desc(st + 3 * PBLOCK + kk * 32);
                  ptx::mma_bf16(dt, pd, ql, idesc, 1u);
                  ptx::mma_bf16(dt, pl, qd, idesc, 1u);
                }
              }
            }
            ptx::mma_commit(ptx::smem_addr(&x.empty[s]));
            if (FUSE == 2) ptx::mma_commit(ptx::smem_addr(&x.qempty[qs]));
          }
          if (!ok) break;
          ptx::mma_commit(ptx::smem_addr(&x.acc_full[b]));
        }
        if (!ok) { x.abort = 1; break; }
      }
      // every MMA of this thread completes before TMEM is released
      ptx::mma_commit(ptx::smem_addr(&x.final_bar));
      ptx::mbar_wait(ptx::smem_addr(&x.final_bar), 0u, status);
    }
  } else if (FUSE == 2 && warp == 2) {
    // ------------------------------------------------------------ P box loads
    // one box per slab into the staging ring, as far ahead of the rounding
    // as the ring's bytes and its XBOXES barrier pairs allow; the box's
    // coordinates are the mixed-radix digits of its first row and first
    // shared index over P's legs
    if (lane == 0) {
      const uint32_t xs0 = ptx::smem_addr(xstage);
      uint32_t gx = 0, old = 0;  // next box; oldest box not known to be rounded
      uint64_t v = 0, vs[XBOXES];
      for (int q = 0; q < XBOXES; ++q) vs[q] = 0;
      UnitSeq<S> us = unit_seq(x, unit_ctr, status, total_units, 1);
      int64_t u = us.first(), un = 0;
      TmaDesc dn = load_tma(descs, map, u >= 0 ? u : 0);
      for (; u >= 0 && !x.abort; u = un) {
        const TmaDesc d = dn;
        un = us.next();
        if (un >= 0) dn = load_tma(descs, map, un);
        const GUnit g = gunit(d, u - d.tile_begin);
        // the unit's first box by division, the next ones by stepping the
        // shared legs' coordinates like an odometer (no division per slab)
        int32_t c[5];
        const uint32_t r0 = (uint32_t)g.p0, k0 = (uint32_t)g.ks0 * (uint32_t)d.kw;
#pragma unroll
        for (int i = 0; i < 5; ++i) c[i] = (int32_t)((((d.bkmask >> i) & 1) ? k0 : r0) / d.bplace[i] % d.bdim[i]);
        const uint32_t bytes = (uint32_t)(d.ph * d.kw * d.nsb * 4);
        bool ok = true;
        for (int ks = 0; ks < g.nks; ks += d.nsb, ++gx) {
          if (ks > 0) {
            int32_t add = d.bkstep;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              if (i < d.bk0 || i > d.bk1 || add == 0) continue;
              c[i] += add;
              add = 0;
              if (c[i] >= (int32_t)d.bdim[i]) {
                c[i] -= (int32_t)d.bdim[i];
                add = 1;
              }
            }
          }
          // room for the box: the boxes it would overwrite, and the one whose
          // barriers it takes, have been rounded
          const uint64_t start = ring_take(v, bytes);
          while (old < gx && (gx - old >= (uint32_t)XBOXES || start + bytes - vs[old % XBOXES] > XRING)) {
            if (!ptx::mbar_wait(ptx::smem_addr(&x.xempty[old % XBOXES]), (old / XBOXES) & 1u, status)) {
              ok = false;
              break;
            }
            ++old;
          }
          if (!ok) break;
          const int sl = (int)(gx % XBOXES);
          vs[sl] = start;
          const uint32_t xf = ptx::smem_addr(&x.xfull[sl]);
          ptx::mbar_arrive_expect_tx(xf, bytes);
          ptx::tma_load_5d(xs0 + (uint32_t)(start & (XRING - 1)), d.tmap, c[0], c[1], c[2], c[3], c[4], xf);
        }
        if (!ok) {
          x.abort = 1;
          break;
        }
      }
      // boxes still in flight land before the CTA can exit
      for (uint32_t q = old; q < gx; ++q) ptx::mbar_wait(ptx::smem_addr(&x.xfull[q % XBOXES]), (q / XBOXES) & 1u, status);
    }
  } else if (FUSE == 2 && warp < Cf::EPI0) {
    // ------------------------------------------------------------ rounding
    const int cw = warp - 2 - Cf::TMAW;
    const uint32_t xs0 = ptx::smem_addr(xstage);
    const uint32_t grp = (uint32_t)(cw / Cf::RW);  // this warp rounds boxes grp, grp + RGROUPS, ..
    const int wi = cw % Cf::RW;
    uint32_t gx = 0;
    uint64_t v = 0;  // the ring positions, taken in the TMA warp's order
    bool ok = true;
    UnitSeq<S> us = unit_seq(x, unit_ctr, status, total_units, 3);
    int64_t u = us.first(), un = 0;
    RoundDesc dn = load_round(descs, map, u >= 0 ? u : 0);
    for (; u >= 0 && ok && !x.abort; u = un) {
      const RoundDesc d = dn;
      un = us.next();
      if (un >= 0) dn = load_round(descs, map, un);
      const GUnit g = gunit(d, u - d.tile_begin);
      const uint32_t bytes = (uint32_t)(d.ph * d.kw * d.nsb * 4);
      for (int ks = 0; ks < g.nks; ks += d.nsb, ++gx) {
        const uint64_t start = ring_take(v, bytes);
        if (gx % Cf::RGROUPS != grp) continue;
        const int sl = (int)(gx % XBOXES), s = (int)(gx % S);
        const bool w = ptx::mbar_wait(ptx::smem_addr(&x.xfull[sl]), (gx / XBOXES) & 1u, status) &&
                       ptx::mbar_wait(ptx::smem_addr(&x.empty[s]), ((gx / S) & 1u) ^ 1u, status);
        if (!__all_sync(0xffffffffu, w)) {
          ok = false;
          break;
        }
        round_box<Cf::RW>(d.p_mn, d.ph, d.kw, d.nsb, wi, lane, xs0 + (uint32_t)(start & (XRING - 1)),
                          stage0 + (uint32_t)s * Cf::STAGE_BYTES);
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          ptx::mbar_arrive(ptx::smem_addr(&x.full[s]));
          ptx::mbar_arrive(ptx::smem_addr(&x.xempty[sl]));
        }
      }
    }
    if (!ok) x.abort = 1;
  } else if (FUSE == 1 && warp < Cf::EPI0) {
    // ------------------------------------------------------------ converters
    const int cw = warp - 2;
    const uint32_t xs0 = ptx::smem_addr(xstage);
    ConvIter itr;  // the next slab to copy
    itr.u = blockIdx.x;
    itr.total = total_units;
    itr.ks = itr.nks = itr.ks0 = itr.mode = 0;
    itr.p0 = itr.R = itr.K = 0;
    itr.src = nullptr;
    itr.rtab = itr.ktab = nullptr;
    itr.load(descs, map, jobs);
    ConvRegs cr;
#pragma unroll
    for (int i = 0; i < 8; ++i) cr.r[i] = cr.k[i] = 0;
    conv_fetch(itr, cw, lane, cr);
    // copies of the slab XDIST ahead (one commit group per slab, empty
    // groups included), then the table entries of the slab after it
    auto issue = [&](int sl) -> uint32_t {
      const uint32_t info = itr.info();
      if (itr.valid()) {
        conv_copy(itr, cr, cw, lane, tb, xs0 + (uint32_t)(sl * XSLOT_BYTES));
        itr.next(descs, map, jobs);
        conv_fetch(itr, cw, lane, cr);
      }
      ptx::cp_async_commit();
      return info;
    };
    uint32_t w[XDIST + 1];
#pragma unroll
    for (int d = 0; d < XDIST; ++d) w[d] = issue(d);
    uint32_t gs = 0;
    int sl = 0;  // slot of slab gs; slab gs + XDIST goes to the slot before it
    while ((w[0] & 1u) && !x.abort) {
      w[XDIST] = issue(sl == 0 ? XSLOTS - 1 : sl - 1);
      ptx::cp_async_wait<XDIST>();  // this thread's copies of slab gs have landed
      __syncwarp();                 // ... and those of the whole warp
      const int s = (int)(gs % S);
      const bool ok = __all_sync(0xffffffffu, ptx::mbar_wait(ptx::smem_addr(&x.empty[s]), ((gs / S) & 1u) ^ 1u,
                                                             status));
      if (!ok) {
        x.abort = 1;
        break;
      }
      conv_round(w[0], cw, lane, xstage + (size_t)sl * XSLOT_BYTES, smem + (size_t)s * Cf::STAGE_BYTES);
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(ptx::smem_addr(&x.full[s]));
      ++gs;
#pragma unroll
      for (int d = 0; d < XDIST; ++d) w[d] = w[d + 1];
      sl = sl == XSLOTS - 1 ? 0 : sl + 1;
    }
    ptx::cp_async_wait<0>();
  } else {
    // ------------------------------------------------------------ epilogue
    const int quad = warp & 3;            // TMEM lanes quad*32 .. quad*32+31
    constexpr int ECOLS = Cf::ECOLS;
    const int grp = (warp - Cf::EPI0) >> 2;  // column group of this warp (eight warps: two groups)
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    uint32_t gc = 0;
    UnitSeq<S> us = unit_seq(x, unit_ctr, status, total_units, unit_ctr ? 3 : 0);
    int64_t u = us.first(), un = 0;
    EpiDesc dn = load_epi(single, descs, map, u >= 0 ? u : 0);
    for (; u >= 0 && !x.abort; u = un) {
      const EpiDesc d = dn;
      un = us.next();
      if (un >= 0) dn = load_epi(single, descs, map, un);
      const GUnit g = gunit(d, u - d.tile_begin);
      const int64_t i = g.p0 + quad * 32 + lane;            // row of P this thread owns
      // rows of this tile: ph of them (fewer at P's end)
      const int64_t rend = d.RP - g.p0 < d.ph ? d.RP : g.p0 + d.ph;
      const int64_t qcols = d.RQ - g.q0 < d.q_tile ? d.RQ - g.q0 : d.q_tile;
      // columns of the tile this warp drains: eight warps split the tile
      // width in two (the 64-column reads of the 16x256b shape: in 64s)
      // (BF16 on packed operands stores through the shared-memory
      // transpose instead: whole 128-byte row segments)
      const bool rows16 = !Cf::TR && d.cj == 1 && d.store16 != 0;
      const int span = Cf::EPI == 8 ? d.q_tile / 2 : d.q_tile;
      const int gspan = rows16 && span < 64 ? 64 : span;
      const int col0 = grp * gspan;
      const int chunk = SPLIT ? KC : g.nks;
      const int nchunks = (g.nks + chunk - 1) / chunk;
      const bool accumulate = d.splits > 1;
      float* __restrict__ C = d.C;
      // 16-byte stores along a row of C: C row-major along j, rows 16-byte aligned
      const bool vec = d.cj == 1 && ((d.ci & 3) == 0) && (((reinterpret_cast<uintptr_t>(C) >> 2) + g.q0) & 3) == 0;
      float acc[SPLIT ? ECOLS : 1];
#pragma unroll
      for (int j = 0; j < (SPLIT ? ECOLS : 1); ++j) acc[j] = 0.0f;
      // Writes columns col .. col+31 of row i (this thread's values r):
      // 16-byte stores along a row of C, or, with the roles swapped, one
      // store per column with the warp's lanes on consecutive addresses.
      auto emit = [&](int col, const float* r) {
        if (i >= rend) return;
        const int64_t nrem = qcols - col;
        if (d.cj == 1) {
          float* dst = C + i * d.ci + g.q0 + col;
          if (vec && !accumulate && nrem >= 32) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(dst + j) = make_float4(r[j], r[j + 1], r[j + 2], r[j + 3]);
            return;
          }
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (j < nrem) emit4(dst + j, vec, nrem - j, accumulate, r[j], r[j + 1], r[j + 2], r[j + 3]);
        } else {
          float* dst = C + i * d.ci + (g.q0 + col) * d.cj;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < nrem) {
              if (accumulate) atomicAdd(dst + j * d.cj, r[j]);
              else dst[j * d.cj] = r[j];
            }
          }
        }
      };
      // C row-major along j, transposed through shared memory: this warp's 32
      // rows x 32 columns written row per lane (chunk c of row r at slot
      // c ^ (r % 8)), read back 4 rows x 8 lanes x 16 bytes per store
      // instruction
      float* tr = trbuf + (warp - Cf::EPI0) * (32 * 32);
      auto emit_tr = [&](int col, const float* r) {
        __syncwarp();  // the previous block has been read back
#pragma unroll
        for (int c = 0; c < 8; ++c)
          *reinterpret_cast<float4*>(tr + lane * 32 + ((c ^ (lane & 7)) << 2)) =
              make_float4(r[4 * c], r[4 * c + 1], r[4 * c + 2], r[4 * c + 3]);
        __syncwarp();
        const int64_t nrem = qcols - col;
        const int q = lane & 7;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const int rr = it * 4 + (lane >> 3);
          const int64_t row = g.p0 + quad * 32 + rr;
          if (row >= rend || 4 * q >= nrem) continue;
          const float4 v4 = *reinterpret_cast<const float4*>(tr + rr * 32 + ((q ^ (rr & 7)) << 2));
          emit4(C + row * d.ci + g.q0 + col + 4 * q, vec, nrem - 4 * q, accumulate, v4.x, v4.y, v4.z, v4.w);
        }
      };
      // C row-major along j: the accumulator is read as 16-lane x 256-bit
      // blocks, so each thread holds two consecutive columns of two rows and
      // a warp's store covers 8 rows x 32 contiguous bytes (whole sectors).
      const bool vec2 = rows16 && ((d.ci & 1) == 0) && (((reinterpret_cast<uintptr_t>(C) >> 2) + g.q0) & 1) == 0 &&
                        ((reinterpret_cast<uintptr_t>(C) & 7) == 0);
      // values r[4j..4j+3] of lane half h (rows +0 and +8), columns
      // cbase + 8j + 2(lane % 4) + {0, 1} (a block of 64 columns)
      auto emit16 = [&](int h, const float* r, int cbase) {
        const int64_t row = g.p0 + quad * 32 + h * 16 + (lane >> 2);
        const int cq = cbase + 2 * (lane & 3);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = cq + 8 * j;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int64_t rr = row + 8 * e;
            if (rr >= rend || c >= qcols) continue;
            float* dst = C + rr * d.ci + g.q0 + c;
            const float a = r[4 * j + 2 * e], bq = r[4 * j + 2 * e + 1];
            if (accumulate) {
              atomicAdd(dst, a);
              if (c + 1 < qcols) atomicAdd(dst + 1, bq);
            } else if (vec2 && c + 1 < qcols) {
              *reinterpret_cast<float2*>(dst) = make_float2(a, bq);
            } else {
              dst[0] = a;
              if (c + 1 < qcols) dst[1] = bq;
            }
          }
        }
      };
      bool ok = true;
      for (int c = 0; c < nchunks; ++c, ++gc) {
        const int b = (int)(gc & 1);
        const bool w = ptx::mbar_wait(ptx::smem_addr(&x.acc_full[b]), (gc >> 1) & 1u, status);
        if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
        ptx::tc_fence_after();
        if (rows16) {
#pragma unroll
          for (int blk = 0; blk < ECOLS / 64; ++blk) {
            const int cbase = col0 + 64 * blk;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (64 * blk < gspan && cbase < qcols) {  // uniform across the warp
                uint32_t r[32];
                ptx::tmem_ld_16x256b_x8(tmem + ((uint32_t)(quad * 32 + h * 16) << 16) + (uint32_t)(b * Cf::ACC_COLS + cbase),
                                        r);
                ptx::tmem_ld_wait();
                if (SPLIT) {
#pragma unroll
                  for (int j = 0; j < 32; ++j) acc[blk * 64 + h * 32 + j] += __uint_as_float(r[j]);
                } else {
                  float v[32];
#pragma unroll
                  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                  emit16(h, v, cbase);
                }
              }
            }
          }
        } else {
          const uint32_t ta = tmem + lane_base + (uint32_t)(b * Cf::ACC_COLS + col0);
          if constexpr (SPLIT) {
#pragma unroll
            for (int cb = 0; cb < ECOLS / 32; ++cb) {
              if (32 * cb < gspan && col0 + cb * 32 < qcols) {  // uniform across the warp
                uint32_t r[32];
                ptx::tmem_ld_32x32b_x32(ta + (uint32_t)(cb * 32), r);
                ptx::tmem_ld_wait();
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[cb * 32 + j] += __uint_as_float(r[j]);
              }
            }
          } else {
            // one 32-column block at a time (a loop, not unrolled: one
            // block's registers live at once)
#pragma unroll 1
            for (int cb = 0; cb < ECOLS / 32; ++cb) {
              if (32 * cb < gspan && col0 + cb * 32 < qcols) {  // uniform across the warp
                uint32_t r[32];
                ptx::tmem_ld_32x32b_x32(ta + (uint32_t)(cb * 32), r);
                ptx::tmem_ld_wait();
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
                if (Cf::TR && d.cj == 1) emit_tr(col0 + cb * 32, v);
                else emit(col0 + cb * 32, v);
              }
            }
          }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(ptx::smem_addr(&x.acc_empty[b]));
      }
      if (!ok) { x.abort = 1; break; }
      if (SPLIT) {
        if (rows16) {
#pragma unroll
          for (int blk = 0; blk < ECOLS / 64; ++blk)
#pragma unroll
            for (int h = 0; h < 2; ++h)
              if (64 * blk < gspan && col0 + 64 * blk < qcols) emit16(h, &acc[blk * 64 + h * 32], col0 + 64 * blk);
        } else {
#pragma unroll
          for (int cb = 0; cb < ECOLS / 32; ++cb)
            if (32 * cb < gspan && col0 + cb * 32 < qcols) emit(col0 + cb * 32, &acc[cb * 32]);
        }
      }
    }
  }

  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, Cf::TMEM_COLS);
  }
}

// Both pack kernels take PACK_SMEM of dynamic shared memory (above the 48 KB
// default); set once per device.
bool pack_attr() {
  static std::atomic<uint64_t> done_pack{0}, done_pair{0};
  if (!smem_limit_once((const void*)pack_kernel, PACK_SMEM, &done_pack) ||
      !smem_limit_once((const void*)pack_pair_kernel, PACK_SMEM, &done_pair))
    return false;
  return true;
}

int sm_count() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 152;
  }
  return sms;
}

template <int SPLIT, int FUSE>
int launch_gemm(const GemmDesc& single, const GemmDesc* descs, const int32_t* map, const PackJob* jobs,
                int64_t units, cudaStream_t s, uint32_t* unit_ctr = nullptr) {
  const size_t smem = gemm_smem_bytes<SPLIT, FUSE>();
  static std::atomic<uint64_t> attr{0};
  if (!smem_limit_once((const void*)packed_gemm_kernel<SPLIT, FUSE>, smem, &attr)) return TN_ERR_CUDA;
  const int64_t sms = sm_count();
  const unsigned grid = (unsigned)(units < sms ? units : sms);
  packed_gemm_kernel<SPLIT, FUSE>
      <<<grid, GCfg<SPLIT, FUSE>::THREADS, smem, s>>>(single, descs, map, jobs, units, unit_ctr, status_word());
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace

int launch_pack(const PackJob* jobs, const PackUnit* units, int64_t nunits, cudaStream_t s) {
  if (nunits <= 0) return TN_OK;
  if (nunits > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (!pack_attr()) return TN_ERR_CUDA;
  pack_kernel<<<(unsigned)nunits, PACK_THREADS, PACK_SMEM, s>>>(jobs, units);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int launch_packed_gemm(const GemmDesc* descs, const int32_t* map, int64_t units, int prec, uint32_t* unit_ctr,
                       cudaStream_t s) {
  if (units <= 0) return TN_OK;
  if (units > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  // the launch's CTAs claim units from this counter
  if (unit_ctr && cudaMemsetAsync(unit_ctr, 0, sizeof(uint32_t), s) != cudaSuccess) return TN_ERR_CUDA;
  GemmDesc none;
  memset(&none, 0, sizeof(none));
  if (prec == TN_PREC_BF16) return launch_gemm<0, 0>(none, descs, map, nullptr, units, s, unit_ctr);
  return launch_gemm<1, 0>(none, descs, map, nullptr, units, s, unit_ctr);
}

int launch_fused_gemm(const GemmDesc* descs, const int32_t* map, const PackJob* jobs, int64_t units,
                      cudaStream_t s) {
  if (units <= 0) return TN_OK;
  if (units > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (!descs || !map || !jobs) return TN_ERR_ARG;
  GemmDesc none;
  memset(&none, 0, sizeof(none));
  return launch_gemm<0, 1>(none, descs, map, jobs, units, s);
}

int launch_tma_gemm(const GemmDesc* descs, const int32_t* map, int64_t units, uint32_t* unit_ctr, cudaStream_t s) {
  if (units <= 0) return TN_OK;
  if (units > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (!descs || !map || !unit_ctr) return TN_ERR_ARG;
  // the launch's CTAs claim units from this counter
  if (cudaMemsetAsync(unit_ctr, 0, sizeof(uint32_t), s) != cudaSuccess) return TN_ERR_CUDA;
  GemmDesc none;
  memset(&none, 0, sizeof(none));
  return launch_gemm<0, 2>(none, descs, map, nullptr, units, s, unit_ctr);
}

namespace {

// Pack job of one operand of d (rows: its free legs; k: the shared legs).
PackJob make_job(const ContractDesc& d, const float* src, int64_t R, int nr, const int32_t* rdim,
                 const int64_t* rstr, const int64_t* kstr) {
  PackJob j;
  memset(&j, 0, sizeof(j));
  j.src = src;
  j.R = R;
  j.K = d.K;
  j.tiles = (int32_t)((R + PR - 1) / PR);
  j.kw = PK;
  j.slabs = (int32_t)((d.K + PK - 1) / PK);
  j.block_bytes = R >= PR ? PBLOCK : ((R + 7) & ~int64_t(7)) * 128;
  j.rg = R >= PR ? PR : (int32_t)((R + 7) & ~int64_t(7));
  j.nbv = (R >= PR || j.rg > PR / 2) ? 1 : PR / j.rg;
  j.nr = nr;
  j.nk = d.nk;
  for (int q = 0; q < nr; ++q) {
    j.rdim[q] = rdim[q];
    j.rstr[q] = rstr[q];
  }
  for (int q = 0; q < d.nk; ++q) {
    j.kdim[q] = d.kdim[q];
    j.kstr[q] = kstr[q];
  }
  j.kfast = (d.nk > 0 && kstr[d.nk - 1] == 1) ? 1 : 0;
  j.rfast = (nr > 0 && rstr[nr - 1] == 1) ? 1 : 0;
  // 16-byte copies along the unit-stride leg: it is the last shared (or
  // free) leg with a length divisible by 4, every other stride is a multiple
  // of 4 elements, and the base is 16-byte aligned
  int mode = 0;
  if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
    if (j.kfast && d.kdim[d.nk - 1] % 4 == 0) mode = 1;
    else if (j.rfast && rdim[nr - 1] % 4 == 0) mode = 2;
    for (int q = 0; q < nr && mode; ++q)
      if (!(mode == 2 && q == nr - 1) && rdim[q] > 1 && rstr[q] % 4 != 0) mode = 0;
    for (int q = 0; q < d.nk && mode; ++q)
      if (!(mode == 1 && q == d.nk - 1) && d.kdim[q] > 1 && kstr[q] % 4 != 0) mode = 0;
  }
  j.vec4 = mode;
  j.rtab_off = j.ktab_off = -1;
  return j;
}

// Pack blocks per CTA: about 256 KB of float32 reads (a block reads twice
// its bf16 bytes); measured best among 64, 128, 256 and 512 KB. At most 16
// virtual blocks.
int32_t blocks_per_unit(const PackJob& j) {
  return (int32_t)std::max<int64_t>(1, std::min<int64_t>(16 * j.nbv, 262144 / (2 * j.block_bytes)));
}

size_t job_bytes(const PackJob& j) { return (size_t)j.tiles * j.slabs * j.block_bytes; }

// GEMM descriptor of contraction d over packed A (ja) and B (jb): the side
// with more rows is P (the MMA's 128 rows). Offsets are left to the caller.
GemmDesc make_gemm(const ContractDesc& d, const PackJob& ja, const PackJob& jb, int q_tile, bool* swapped) {
  const bool swap = p_is_b(d);
  GemmDesc g;
  memset(&g, 0, sizeof(g));
  g.C = d.C;
  g.RP = swap ? d.N : d.M;
  g.RQ = swap ? d.M : d.N;
  g.ci = swap ? 1 : d.N;
  g.cj = swap ? d.N : 1;
  const PackJob& jp = swap ? jb : ja;
  const PackJob& jq = swap ? ja : jb;
  g.P_block = jp.block_bytes;
  g.Q_block = jq.block_bytes;
  g.q_tile = q_tile == 64 ? 64 : (q_tile == 256 ? 256 : PR);
  g.tiles_p = jp.tiles;
  g.tiles_q = (int32_t)((g.RQ + g.q_tile - 1) / g.q_tile);
  g.slabs = ja.slabs;
  g.splits = d.splits;
  g.slabs_per_split = (int32_t)(d.k_per_split / PK);
  g.pjob = -1;
  g.p_mn = 0;
  g.ph = PR;
  g.kw = PK;
  g.bkmask = 0;
  g.nsb = 1;
  g.tmap = nullptr;
  g.tmap_idx = -1;
  g.K = d.K;
  *swapped = swap;
  return g;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when the driver does not provide it.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

}  // namespace

bool plan_tma_box(const ContractDesc& d, TmaBox* box, TmaMap* map) {
  static_assert(sizeof(TmaMap) == sizeof(CUtensorMap), "tensor map size");
  const bool swap = p_is_b(d);
  const float* src = swap ? d.B : d.A;
  if (!src || (reinterpret_cast<uintptr_t>(src) & 15) || d.K <= 0) return false;
  // device memory only (host-resident operands keep the converters' copies)
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, src) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (pa.type != cudaMemoryTypeDevice) return false;
  // P's legs of extent > 1: free legs in the order they flatten into the row
  // index, shared legs in the order they flatten into k (last fastest)
  struct Leg {
    int64_t dim, str, place;
    bool k;
  };
  Leg rl[TN_MAX_RANK], kl[TN_MAX_RANK];
  int nr = 0, nk = 0;
  const int nfree = swap ? d.nn : d.nm;
  const int32_t* fdim = swap ? d.ndim : d.mdim;
  const int64_t* fstr = swap ? d.nstr : d.mstr;
  const int64_t* kstr = swap ? d.kstrB : d.kstrA;
  int64_t place = 1;
  for (int q = nfree - 1; q >= 0; --q) {
    if (fdim[q] > 1) rl[nr++] = Leg{fdim[q], fstr[q], place, false};
    place *= fdim[q];
  }
  place = 1;
  for (int q = d.nk - 1; q >= 0; --q) {
    if (d.kdim[q] > 1) kl[nk++] = Leg{d.kdim[q], kstr[q], place, true};
    place *= d.kdim[q];
  }
  // rl / kl now run fastest first
  if (nr + nk == 0 || nr + nk > 5) return false;
  // box extents, fastest leg first: whole legs while they fit, then the
  // largest divisor of the next leg that fits, then 1 -- so the boxes tile
  // the flattened index exactly, each one a run of consecutive rows (or k)
  auto extents = [](const Leg* l, int n, int64_t cap, int64_t* b) -> int64_t {
    int64_t e = 1;
    int q = 0;
    for (; q < n && e * l[q].dim <= cap; ++q) {
      b[q] = l[q].dim;
      e *= l[q].dim;
    }
    if (q < n) {
      int64_t m = cap / e;
      while (l[q].dim % m) --m;
      b[q] = m;
      e *= m;
      for (++q; q < n; ++q) b[q] = 1;
    }
    return e;
  };
  int64_t rb[TN_MAX_RANK], kb[TN_MAX_RANK];
  const int64_t H = extents(rl, nr, PR, rb), W = extents(kl, nk, PK, kb);
  const int64_t RQ = swap ? d.M : d.N;
  // narrow boxes on a long k would multiply Q's packed slabs, short ones on
  // many rows the work units
  const int64_t RP = swap ? d.N : d.M;
  if ((W < 32 && W < d.K) || (H < 32 && H < RP)) return false;
  // the unit-stride leg leads: the last shared leg (tile row-major along k)
  // or else the last free leg (tile row-major along the rows)
  int mode = 0;
  if (nk && kl[0].str == 1) mode = 1;
  else if (nr && rl[0].str == 1) mode = 2;
  if (!mode) return false;
  // P with few rows, staged row-major along k: one box covers nsb
  // consecutive slabs (k extent nsb * W, a box of its own), its k-blocks
  // stacked as nsb x ceil8(H) rows of the bf16 tile; bounded by the tile's
  // 128 rows, the rounding's 8 loads per lane, Q's 8 KB slot and the TMA's
  // 256 elements per dimension
  int64_t nsb = 1;
  if (mode == 1) {
    const int64_t H8 = (H + 7) & ~int64_t(7), ni = (H + 15) / 16, qblk = ((RQ + 7) & ~int64_t(7)) * 128;
    int64_t cap = std::min<int64_t>(std::min<int64_t>(PR / H8, 8 / ni), std::min<int64_t>(8192 / qblk, d.K / W));
    for (int64_t c = cap; c > 1; --c) {
      int64_t kb2[TN_MAX_RANK];
      if (extents(kl, nk, c * W, kb2) != c * W) continue;
      bool fits = true;
      for (int q = 0; q < nk; ++q) fits = fits && kb2[q] <= 256;
      if (!fits) continue;
      nsb = c;
      for (int q = 0; q < nk; ++q) kb[q] = kb2[q];
      break;
    }
  }
  // tensor-map dimensions, fastest first
  Leg dl[5];
  int64_t db[5];
  int n = 0;
  const Leg* first = mode == 1 ? kl : rl;
  const Leg* second = mode == 1 ? rl : kl;
  const int64_t* fb = mode == 1 ? kb : rb;
  const int64_t* sb = mode == 1 ? rb : kb;
  const int n1 = mode == 1 ? nk : nr, n2 = mode == 1 ? nr : nk;
  for (int q = 0; q < n1; ++q, ++n) {
    dl[n] = first[q];
    db[n] = fb[q];
  }
  for (int q = 0; q < n2; ++q, ++n) {
    dl[n] = second[q];
    db[n] = sb[q];
  }
  // TMA: the innermost box extent a multiple of 16 bytes (so is every
  // coordinate along it: multiples of that extent), other strides too
  if (db[0] % 4) return false;
  int64_t span = 1;
  for (int q = 0; q < n; ++q) {
    if (q > 0 && (dl[q].str % 4 || dl[q].str <= 0)) return false;
    span += (dl[q].dim - 1) * dl[q].str;
  }
  cuuint64_t gdim[5], gstr[4];
  cuuint32_t bdim[5], estr[5] = {1, 1, 1, 1, 1};
  const int64_t pad_str = (span + 3) / 4 * 4;  // unit padding dimensions: any multiple of 16 bytes
  box->kmask = 0;
  for (int q = 0; q < 5; ++q) {
    const bool real = q < n;
    gdim[q] = real ? (cuuint64_t)dl[q].dim : 1;
    bdim[q] = real ? (cuuint32_t)db[q] : 1;
    if (q > 0) gstr[q - 1] = (cuuint64_t)(4 * (real ? dl[q].str : pad_str));
    box->dim[q] = real ? (uint32_t)dl[q].dim : 1;
    box->place[q] = real ? (uint32_t)dl[q].place : 1;
    if (real && dl[q].k) box->kmask |= 1 << q;
  }
  box->ph = (int32_t)H;
  box->kw = (int32_t)W;
  box->nsb = (int32_t)nsb;
  box->p_mn = mode == 2 ? 1 : 0;
  // the shared legs' map dimensions, fastest first, and the first one whose
  // box is not the whole leg: the next slab advances it by its box extent
  box->k0 = box->k1 = -1;
  box->kstep = 0;
  for (int q = 0; q < n; ++q) {
    if (!dl[q].k) continue;
    box->k1 = q;
    if (box->k0 < 0 && db[q] < dl[q].dim) {
      box->k0 = q;
      box->kstep = (int32_t)db[q];
    }
  }
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  CUtensorMap m;
  if (enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float*>(src), gdim, gstr, bdim, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  memcpy(map->bytes, &m, sizeof(m));
  return true;
}

// Host side: pack jobs (two per contraction), their block units, and the GEMM
// descriptors, with block storage as offsets in the plan's packed region.
void fused_tables(const ContractDesc& d, std::vector<int32_t>* tab, int64_t* rtab_off, int64_t* ktab_off) {
  const bool b = p_is_b(d);
  const int nr = b ? d.nn : d.nm;
  const int32_t* rdim = b ? d.ndim : d.mdim;
  const int64_t* rstr = b ? d.nstr : d.mstr;
  const int64_t* kstr = b ? d.kstrB : d.kstrA;
  const int64_t R = b ? d.N : d.M;
  // odometer over the legs, last leg fastest (offsets fit 32 bits: the
  // planner rejects operands spanning 2^31 elements or more)
  auto run = [&](int64_t n, int nl, const int32_t* dims, const int64_t* str) {
    int32_t idx[TN_MAX_RANK] = {0};
    int64_t off = 0;
    for (int64_t i = 0; i < n; ++i) {
      tab->push_back((int32_t)off);
      for (int q = nl - 1; q >= 0; --q) {
        off += str[q];
        if (++idx[q] < dims[q]) break;
        off -= (int64_t)dims[q] * str[q];
        idx[q] = 0;
      }
    }
  };
  *rtab_off = (int64_t)tab->size();
  run(R, nr, rdim, rstr);
  // the shared-index run starts on a 32-byte boundary and is padded with
  // zeros to whole 64-wide slabs, so a converter reads the 8 entries of its
  // k-rows as two aligned 16-byte loads, never past the run
  while (tab->size() % 8) tab->push_back(0);
  *ktab_off = (int64_t)tab->size();
  run(d.K, d.nk, d.kdim, kstr);
  while ((tab->size() - (size_t)*ktab_off) % PK) tab->push_back(0);
}

int plan_packed(const ContractDesc& d, int prec, const PackedSchedule& sc, bool fuse, int64_t rtab_off,
                int64_t ktab_off, const TmaBox* box, int64_t map, PackedPlan* pp, bool ext_p) {
  PackJob ja = make_job(d, d.A, d.M, d.nm, d.mdim, d.mstr, d.kstrA);
  PackJob jb = make_job(d, d.B, d.N, d.nn, d.ndim, d.nstr, d.kstrB);
  if ((int64_t)ja.tiles * ja.slabs > 0x7FFFFFFF || (int64_t)jb.tiles * jb.slabs > 0x7FFFFFFF)
    return TN_ERR_UNSUPPORTED;
  bool swap = false;
  GemmDesc g = make_gemm(d, ja, jb, sc.q_tile, &swap);
  if (ext_p) {
    if (swap) return TN_ERR_UNSUPPORTED;
    ja.block_bytes = PBLOCK;
    g.P_block = PBLOCK;
    fuse = false;
  }
  fuse = fuse && prec == TN_PREC_BF16 && g.RQ <= PR / 2 &&
         ((rtab_off >= 0 && ktab_off >= 0) || (box && map >= 0));
  const bool tma = fuse && box && map >= 0;
  if (tma) {
    // P in boxes of box->ph rows x box->kw shared indices; Q packed in
    // slabs of the same width, so slab ks of both covers k = ks * kw ..
    PackJob& jq = swap ? ja : jb;
    jq.kw = box->kw;
    jq.slabs = (int32_t)(d.K / box->kw);
    if ((int64_t)jq.tiles * jq.slabs > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
    g.ph = box->ph;
    g.kw = box->kw;
    g.tiles_p = (int32_t)(g.RP / box->ph);
    g.slabs = jq.slabs;
    // the unit's k range: about as many shared indices as the schedule's,
    // in whole boxes
    int64_t per = std::max<int64_t>(1, d.k_per_split / box->kw);
    per = (per + box->nsb - 1) / box->nsb * box->nsb;
    g.slabs_per_split = (int32_t)std::min<int64_t>(per, g.slabs);
    g.nsb = box->nsb;
    g.splits = (int32_t)((g.slabs + g.slabs_per_split - 1) / g.slabs_per_split);
    g.p_mn = box->p_mn;
    g.bkmask = box->kmask;
    for (int i = 0; i < 5; ++i) {
      g.bdim[i] = box->dim[i];
      g.bplace[i] = box->place[i];
    }
    g.bk0 = box->k0;
    g.bk1 = box->k1;
    g.bkstep = box->kstep;
    g.tmap_idx = map;
  }
  // a fused contraction packs Q only: P (A, or B when swapped) is read by
  // the fused GEMM's converters
  const bool pack_a = !(fuse && !swap) && !ext_p, pack_b = !(fuse && swap);
  const size_t bytes_a = (pack_a || ext_p) ? (size_t)ja.tiles * ja.slabs * ja.block_bytes : 0;
  const size_t bytes_b = pack_b ? (size_t)jb.tiles * jb.slabs * jb.block_bytes : 0;
  const bool split = prec == TN_PREC_BF16X3;
  // storage offsets (relative to the packed region): A hi, B hi, A lo, B lo
  const size_t off_a = pp->packed_bytes;
  size_t off = off_a + align256(bytes_a);
  const size_t off_b = off;
  off += align256(bytes_b);
  size_t off_alo = 0, off_blo = 0;
  if (split) {
    off_alo = off;
    off += align256(bytes_a);
    off_blo = off;
    off += align256(bytes_b);
  }
  pp->packed_bytes = off;

  const int ja_idx = (int)pp->jobs.size();
  pp->jobs.push_back(ja);
  pp->jobs.push_back(jb);
  if (fuse) {
    PackJob& jp = pp->jobs[(size_t)ja_idx + (swap ? 1 : 0)];
    jp.rtab_off = rtab_off;
    jp.ktab_off = ktab_off;
  }
  pp->job_hi_off.push_back((pack_a || ext_p) ? off_a : SIZE_MAX);
  pp->job_hi_off.push_back(pack_b ? off_b : SIZE_MAX);
  pp->job_lo_off.push_back(split ? off_alo : SIZE_MAX);
  pp->job_lo_off.push_back(split ? off_blo : SIZE_MAX);
  pp->job_ext.push_back(ext_p ? 1 : 0);
  pp->job_ext.push_back(0);
  for (int w = 0; w < 2; ++w) {
    if (!(w == 0 ? pack_a : pack_b)) continue;
    const PackJob& j = pp->jobs[(size_t)ja_idx + w];
    const int32_t nb = j.tiles * j.slabs;
    const int32_t per = blocks_per_unit(j);
    for (int32_t f = 0; f < nb; f += per) pp->units.push_back(PackUnit{ja_idx + w, f, std::min(per, nb - f), 0});
  }

  g.store16 = sc.store16;
  g.P_off = swap ? off_b : off_a;
  g.Q_off = swap ? off_a : off_b;
  g.P_lo = split ? (int64_t)(swap ? off_blo : off_alo) - (int64_t)g.P_off : 0;
  g.Q_lo = split ? (int64_t)(swap ? off_alo : off_blo) - (int64_t)g.Q_off : 0;
  g.pjob = fuse ? ja_idx + (swap ? 1 : 0) : -1;
  if (!tma) g.p_mn = (fuse && pp->jobs[(size_t)ja_idx + (swap ? 1 : 0)].vec4 == 2) || ext_p ? 1 : 0;
  pp->gemms.push_back(g);
  return TN_OK;
}

size_t packed_single_bytes(const ContractDesc& d, int prec) {
  const PackJob ja = make_job(d, d.A, d.M, d.nm, d.mdim, d.mstr, d.kstrA);
  const PackJob jb = make_job(d, d.B, d.N, d.nn, d.ndim, d.nstr, d.kstrB);
  const size_t planes = prec == TN_PREC_BF16X3 ? 2 : 1;
  return planes * (align256(job_bytes(ja)) + align256(job_bytes(jb)));
}

size_t packed_scratch_bound(int64_t M, int64_t N, int64_t K, int prec) {
  const size_t planes = prec == TN_PREC_BF16X3 ? 2 : 1;
  const size_t slabs = (size_t)((K + PK - 1) / PK);
  const size_t ra = (size_t)((M + PR - 1) / PR) * PR, rb = (size_t)((N + PR - 1) / PR) * PR;
  return planes * (align256(ra * slabs * PK * 2) + align256(rb * slabs * PK * 2));
}

int plan_single_packed(const ContractDesc& d, int prec, bool p_mn, int q_tile, uint8_t* base, size_t bytes,
                       SinglePacked* sp) {
  if (prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  PackJob ja = make_job(d, d.A, d.M, d.nm, d.mdim, d.mstr, d.kstrA);
  PackJob jb = make_job(d, d.B, d.N, d.nn, d.ndim, d.nstr, d.kstrB);
  if ((int64_t)ja.tiles * ja.slabs > 0x7FFFFFFF || (int64_t)jb.tiles * jb.slabs > 0x7FFFFFFF)
    return TN_ERR_UNSUPPORTED;
  bool swap = false;
  // 256-wide tiles: BF16 only (the BF16X3 accumulator is promoted into
  // registers, which hold 128 columns)
  GemmDesc g = make_gemm(d, ja, jb, prec == TN_PREC_BF16 ? q_tile : PR, &swap);
  if (p_mn) {
    // P (the first operand: never the MMA's narrower side here) written by
    // the caller as whole MN-major blocks
    if (swap) return TN_ERR_UNSUPPORTED;
    ja.block_bytes = PBLOCK;
    g.P_block = PBLOCK;
    g.p_mn = 1;
  }
  const bool split = prec == TN_PREC_BF16X3;
  const size_t ba = align256(job_bytes(ja)), bb = align256(job_bytes(jb));
  if (!base || (reinterpret_cast<uintptr_t>(base) & 255) || bytes < (split ? 2 : 1) * (ba + bb))
    return TN_ERR_WORKSPACE;
  ja.hi = base;
  jb.hi = base + ba;
  ja.lo = split ? base + ba + bb : nullptr;
  jb.lo = split ? base + 2 * ba + bb : nullptr;
  g.P = swap ? jb.hi : ja.hi;
  g.Q = swap ? ja.hi : jb.hi;
  g.P_lo = split ? (swap ? jb.lo - jb.hi : ja.lo - ja.hi) : 0;
  g.Q_lo = split ? (swap ? ja.lo - ja.hi : jb.lo - jb.hi) : 0;
  g.tile_begin = 0;
  if ((int64_t)g.tiles_p * g.tiles_q * g.splits > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  sp->ja = ja;
  sp->jb = jb;
  sp->g = g;
  sp->swap = swap;
  return TN_OK;
}

size_t single_packed_bytes(const ContractDesc& d, int prec, bool p_mn) {
  PackJob ja = make_job(d, d.A, d.M, d.nm, d.mdim, d.mstr, d.kstrA);
  const PackJob jb = make_job(d, d.B, d.N, d.nn, d.ndim, d.nstr, d.kstrB);
  if (p_mn) ja.block_bytes = PBLOCK;
  const size_t planes = prec == TN_PREC_BF16X3 ? 2 : 1;
  return planes * (align256(job_bytes(ja)) + align256(job_bytes(jb)));
}

int launch_pack_jobs(const PackJob* a, unsigned* maxbits, const PackJob* b, const PackJob* c, cudaStream_t s) {
  PackPair pp;
  memset(&pp, 0, sizeof(pp));
  const PackJob* jobs[3] = {a, b, c};
  int64_t blocks = 0;
  for (const PackJob* j : jobs)
    if (j) blocks += (int64_t)j->tiles * j->slabs;
  // jobs alone on the GPU: units of fewer blocks when that is what it takes
  // to give every SM a few (a large operand in units of 8 blocks left two
  // thirds of the SMs idle and the rest latency-bound)
  const int32_t cap = (int32_t)std::max<int64_t>(1, blocks / (4 * (int64_t)sm_count()));
  int64_t units[3] = {0, 0, 0};
  int32_t per[3] = {1, 1, 1};
  for (int q = 0; q < 3; ++q) {
    if (!jobs[q]) continue;
    per[q] = std::min(blocks_per_unit(*jobs[q]), cap);
    units[q] = ((int64_t)jobs[q]->tiles * jobs[q]->slabs + per[q] - 1) / per[q];
  }
  const int64_t total = units[0] + units[1] + units[2];
  if (total == 0) return TN_OK;
  if (total > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (a) pp.a = *a;
  if (b) pp.b = *b;
  if (c) pp.c = *c;
  pp.units_a = (int32_t)units[0];
  pp.units_b = (int32_t)units[1];
  pp.per_a = per[0];
  pp.per_b = per[1];
  pp.per_c = per[2];
  pp.maxbits = a ? maxbits : nullptr;
  if (!pack_attr()) return TN_ERR_CUDA;
  pack_pair_kernel<<<(unsigned)total, PACK_THREADS, PACK_SMEM, s>>>(pp);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int launch_gemm_single(const GemmDesc& g, int prec, cudaStream_t s) {
  if (g.splits > 1 && cudaMemsetAsync(g.C, 0, sizeof(float) * (size_t)(g.RP * g.RQ), s) != cudaSuccess)
    return TN_ERR_CUDA;
  const int64_t units = (int64_t)g.tiles_p * g.tiles_q * g.splits;
  if (units <= 0) return TN_OK;
  if (prec == TN_PREC_BF16) return launch_gemm<0, 0>(g, nullptr, nullptr, nullptr, units, s);
  if (prec == TN_PREC_BF16X3) return launch_gemm<1, 0>(g, nullptr, nullptr, nullptr, units, s);
  return TN_ERR_ARG;
}

int contract_packed_single(const ContractDesc& d, int prec, void* scratch, size_t bytes, cudaStream_t s) {
  SinglePacked sp;
  int rc = plan_single_packed(d, prec, false, PR, static_cast<uint8_t*>(scratch), bytes, &sp);
  if (rc != TN_OK) return rc;
  if ((rc = launch_pack_jobs(&sp.ja, nullptr, &sp.jb, nullptr, s)) != TN_OK) return rc;
  return launch_gemm_single(sp.g, prec, s);
}

}  // namespace tn
