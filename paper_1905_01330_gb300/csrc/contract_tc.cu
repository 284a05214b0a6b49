// Pairwise tensordot on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// C[m, n] = sum_k A(m, k) B(k, n) over the flattened shared legs
// (Sec. III.B.2 / III.B.4), float32 in and out, bf16 operands with float32
// accumulation in tensor memory (TMEM):
//   BF16   : one MMA per 16-wide k step on bf16(A), bf16(B);
//   BF16X3 : x = hi + lo (hi = bf16(x), lo = bf16(x - hi)); three MMAs per
//            k step, Ahi*Bhi + Ahi*Blo + Alo*Bhi, into the same accumulator.
//
// Persistent kernel: one 1024-thread CTA per SM walks the work units
// blockIdx.x, blockIdx.x + gridDim.x, ... (a unit is one 128x128 output tile
// and one k range; the host sorts units largest first). Barriers and TMEM are
// set up once per CTA; the next unit's descriptor is fetched by a 1-D bulk
// async copy while the current unit runs.
//
// Every thread is a converter: the CTA gathers 128x64 float32 slabs of A and B
// in place through the operands' leg strides (the permutation is folded into
// the gather: no transposed copy exists anywhere), rounds them to bf16 (and
// splits them), and stores them into the 128-byte-swizzled K-major shared-
// memory layout the MMA descriptors describe, in a ring of stages. The offset
// tables of the next slabs are decoded ahead, and for BF16 the loads of slab
// k+1 can stay in flight while slab k is converted (PIPE). A named barrier closes each
// slab; right after it one thread issues the slab's tcgen05.mma instructions
// (the barrier orders every converter's fenced stores before them) and
// commits them to the stage's `empty` barrier, which the converters wait on
// before they reuse the stage. After a unit's k loop the 16 warps drain TMEM
// and write C. 32 warps (64 registers each; the register file is split
// between the SM's four sub-partitions) with one unit per thread and operand:
// the many resident warps hide the gather's latency.
// Every mbarrier wait is bounded (2 s of wall time); on expiry the kernel
// records TN_ERR_TIMEOUT, stops all units, frees its TMEM and returns.
#include <cuda_bf16.h>

#include "gather.cuh"
#include "ptx.cuh"

namespace tn {
namespace {

constexpr int BM = TC_BM, BN = TC_BN, BK = 64;
constexpr int UNITS = BM * (BK / 8);     // (row, 8-wide k group) units of one operand slab
constexpr int TILE_BYTES = BM * BK * 2;  // one 128x64 bf16 operand tile (16 KB)
constexpr int KMAX = MAX_SLABS_PER_UNIT * BK;  // longest k range of a work unit (2048)
// BF16X3 promotes the tensor-core accumulator into float32 registers every
// KC k-slabs (KC * 64 = 256 shared indices): the tensor core's float32
// accumulation truncates, and over long K that error (linear in the number
// of accumulation steps) would exceed the split's own rounding error.
constexpr int KC = 4;

// Threads per CTA: BF16 runs 32 warps (64 registers each, one unit per
// thread and operand; the resident warps hide the gather latency); BF16X3
// runs 16 warps (128 registers: its promoted partial sums need them) with two
// units per thread. (PIPE = true would keep the loads of slab k+1 in flight
// while slab k is converted; at these register budgets it spills, so both
// paths rely on resident warps instead.)
template <int NT>
struct Shape {
  static constexpr int UPT = UNITS / NT;          // units per thread and operand
  static constexpr int WCOLS = BN / (NT / 128);   // accumulator columns each warp drains
};

template <int SPLIT>
struct Cfg {
  static constexpr int NT = SPLIT ? 512 : 1024;
  static constexpr bool PIPE = false;
  static constexpr int STAGES = SPLIT ? 3 : 4;
  static constexpr int OPS = SPLIT ? 4 : 2;                  // tiles per stage: Ahi, Bhi (, Alo, Blo)
  static constexpr int STAGE_BYTES = OPS * TILE_BYTES;
  static constexpr uint32_t TMEM_COLS = SPLIT ? 2 * BN : BN; // f32 accumulators, 128 lanes each
};

template <int S>
struct TcAux {
  ContractDesc dslot[2];    // descriptors of this and the next unit (16-byte aligned)
  int32_t rowA[BM];
  int32_t rowB[BN];
  int32_t kA[KMAX];          // shared-index offsets of the unit's k range, A
  int32_t kB[KMAX];          // and B (-1 past the range's end)
  int8_t kcA[KMAX / 8];      // 1: the 8-wide k group is unit-stride in A
  int8_t kcB[KMAX / 8];
  uint64_t empty[S];        // the MMAs reading stage s are complete
  uint64_t accum;           // a unit's accumulator is final
  uint64_t chunk_full[2];   // BF16X3: accumulator buffer b holds a finished chunk
  uint64_t desc_bar[2];     // descriptor slot b has landed
  uint64_t final_bar;       // all MMAs of the issuing thread are complete
  uint32_t tmem_base;
  int32_t abort;            // a bounded wait expired somewhere in the CTA
};

template <int SPLIT>
constexpr size_t tc_smem_bytes() {
  using C = Cfg<SPLIT>;
  return 1024 /* alignment slack */ + (size_t)C::STAGES * C::STAGE_BYTES + sizeof(TcAux<C::STAGES>);
}

// Byte offset of the 16-byte chunk (row r, k group g) in a 128B-swizzled
// K-major tile: 8-row atoms of 1024 B, rows of 128 B, chunk index XOR row%8.
__device__ __forceinline__ uint32_t sw128_chunk(int r, int g) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((g ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// k-group contiguity: the 8 indices k0..k0+7 are all < k_end and consecutive
// in memory (innermost shared leg has unit stride and the group does not wrap).
__device__ __forceinline__ int group_contiguous(const ContractDesc& d, int64_t k0, int64_t k_end,
                                                const int64_t* kstr) {
  if (d.nk == 0 || k0 + 8 > k_end) return 0;
  const int last = d.nk - 1;
  if (kstr[last] != 1) return 0;
  const uint32_t dl = (uint32_t)d.kdim[last];
  return (((uint32_t)k0 % dl) + 8 <= dl) ? 1 : 0;
}

// Shared-index offsets of the unit's whole k range (at most KMAX), decoded
// once per unit by all threads, and the unit-stride flag of every 8-group.
template <int NT, class Aux>
__device__ __forceinline__ void fill_tables(const ContractDesc& d, const UnitCoord& uc, Aux& x) {
  const int64_t len = uc.k_end - uc.k_begin;
  const int64_t padded = ((len + BK - 1) / BK) * BK;
  for (int e = threadIdx.x; e < 2 * padded; e += NT) {
    const bool isA = e < padded;
    const int jj = isA ? e : e - (int)padded;
    const int64_t k = uc.k_begin + jj;
    const int64_t* kstr = isA ? d.kstrA : d.kstrB;
    const int32_t off = (jj < len) ? (int32_t)leg_offset((uint32_t)k, d.nk, d.kdim, kstr) : -1;
    if (isA) x.kA[jj] = off;
    else x.kB[jj] = off;
    if ((jj & 7) == 0) {
      const int8_t c = (int8_t)group_contiguous(d, k, uc.k_end, kstr);
      if (isA) x.kcA[jj >> 3] = c;
      else x.kcB[jj >> 3] = c;
    }
  }
}

// Staged layouts. An operand whose unit-stride axis is a shared leg (kfast)
// is staged K-major: a unit is 8 consecutive k of one row, stored as one
// 16-byte chunk of a 128-byte-swizzled K-major tile. An operand whose
// unit-stride axis is a free leg is staged MN-major: a unit is 8 consecutive
// rows at one k, one 16-byte chunk of a 128-byte-swizzled MN-major tile
// (atoms of 8 k-rows x 64 MN elements; the two 64-row halves 8 KB apart,
// 8-row k groups 1 KB apart). Either way the gather reads 32 contiguous bytes
// per unit when the memory layout allows, and consecutive threads walk the
// unit-stride direction.
constexpr uint32_t MN_HALF_BYTES = 8192;  // MN-major: stride between the 64-row halves
constexpr uint32_t MN_KGROUP_BYTES = 1024;  // MN-major: stride between 8-row k groups

__device__ __forceinline__ uint32_t sw128_mn_chunk(int mg, int k) {
  return (uint32_t)((mg >> 3) * MN_HALF_BYTES + (k >> 3) * MN_KGROUP_BYTES + (k & 7) * 128 +
                    (((mg & 7) ^ (k & 7)) << 4));
}

// Rows r0 .. r0+7 of a free-leg index are all present and consecutive in memory.
__device__ __forceinline__ bool row_group_regular(int64_t r0, int64_t R, int n, const int32_t* dims,
                                                  const int64_t* strides) {
  if (n == 0 || r0 + 8 > R || strides[n - 1] != 1) return false;
  const uint32_t dl = (uint32_t)dims[n - 1];
  return ((uint32_t)r0 % dl) + 8 <= dl;
}

// What a thread keeps for a whole work unit, per operand and unit: the base
// pointer of its row (K-major) or 8-row group (MN-major; null when the group
// is not regular), its k group (K-major) or k (MN-major), its row group
// (MN-major), and the swizzled shared-memory offset its values go to.
template <int NT>
struct ThreadUnits {
  static constexpr int UPT = Shape<NT>::UPT;
  const float* pa[UPT];
  const float* pb[UPT];
  uint16_t ga[UPT], gb[UPT];
  uint8_t ma[UPT], mb[UPT];
  uint32_t oa[UPT], ob[UPT];
};

template <int NT>
__device__ __forceinline__ void unit_of(int kfast, const float* base, const int32_t* rows, int64_t row0, int64_t R,
                                        int nr, const int32_t* rdims, const int64_t* rstr, int t, int i,
                                        const float*& p, uint16_t& g, uint8_t& mg, uint32_t& off) {
  const int uu = t + NT * i;
  if (kfast) {
    const int r = uu >> 3;
    g = uu & 7;
    mg = 0;
    p = rows[r] >= 0 ? base + rows[r] : nullptr;
    off = sw128_chunk(r, g);
  } else {
    mg = uu & 15;
    g = uu >> 4;  // the unit's k within the slab
    p = row_group_regular(row0 + 8 * mg, R, nr, rdims, rstr) ? base + rows[8 * mg] : nullptr;
    off = sw128_mn_chunk(mg, g);
  }
}

template <int NT, class Aux>
__device__ __forceinline__ ThreadUnits<NT> thread_units(const ContractDesc& d, const Aux& x, int64_t m0, int64_t n0,
                                                        int t) {
  ThreadUnits<NT> u;
#pragma unroll
  for (int i = 0; i < Shape<NT>::UPT; ++i) {
    unit_of<NT>(d.a_kfast, d.A, x.rowA, m0, d.M, d.nm, d.mdim, d.mstr, t, i, u.pa[i], u.ga[i], u.ma[i], u.oa[i]);
    unit_of<NT>(d.b_kfast, d.B, x.rowB, n0, d.N, d.nn, d.ndim, d.nstr, t, i, u.pb[i], u.gb[i], u.mb[i], u.ob[i]);
  }
  return u;
}

__device__ __forceinline__ void load8(const float* p, float (&v)[8]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// K-major unit: 8 consecutive k of one row.
__device__ __forceinline__ void load_kmajor(const float* row, const int32_t* koff, int contiguous, float (&v)[8]) {
  if (!row) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.0f;
    return;
  }
  const float* p = row + koff[0];
  if (contiguous && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    load8(p, v);
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int32_t ko = koff[j];
    v[j] = (ko >= 0) ? __ldg(row + ko) : 0.0f;
  }
}

// MN-major unit: 8 consecutive rows (group mg) at one shared offset ko.
__device__ __forceinline__ void load_mnmajor(const float* base, const float* grp, const int32_t* rows, int mg,
                                             int32_t ko, float (&v)[8]) {
  if (ko < 0) {
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.0f;
    return;
  }
  if (grp && (reinterpret_cast<uintptr_t>(grp + ko) & 15) == 0) {
    load8(grp + ko, v);
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int32_t ro = rows[8 * mg + j];
    v[j] = (ro >= 0) ? __ldg(base + (ro + ko)) : 0.0f;
  }
}

// Slab kt of the unit: entries kt*64 .. kt*64+63 of the unit's tables.
template <int NT, class Aux>
__device__ __forceinline__ void load_slab(const ContractDesc& d, const Aux& x, int kt, const ThreadUnits<NT>& tu,
                                          float (&va)[Shape<NT>::UPT][8], float (&vb)[Shape<NT>::UPT][8]) {
  constexpr int UPT = Shape<NT>::UPT;
  const int k0 = kt * BK;
#pragma unroll
  for (int i = 0; i < UPT; ++i) {
    if (d.a_kfast) load_kmajor(tu.pa[i], &x.kA[k0 + tu.ga[i] * 8], x.kcA[(k0 >> 3) + tu.ga[i]], va[i]);
    else load_mnmajor(d.A, tu.pa[i], x.rowA, tu.ma[i], x.kA[k0 + tu.ga[i]], va[i]);
  }
#pragma unroll
  for (int i = 0; i < UPT; ++i) {
    if (d.b_kfast) load_kmajor(tu.pb[i], &x.kB[k0 + tu.gb[i] * 8], x.kcB[(k0 >> 3) + tu.gb[i]], vb[i]);
    else load_mnmajor(d.B, tu.pb[i], x.rowB, tu.mb[i], x.kB[k0 + tu.gb[i]], vb[i]);
  }
}

// Descriptor of the 16-wide k step kk of an operand tile at `tile`.
__device__ __forceinline__ uint64_t operand_desc(int kfast, uint32_t tile, int kk) {
  return kfast ? ptx::sw128_kmajor_desc(tile + kk * 32)
               : ptx::sw128_mnmajor_desc(tile + kk * 2 * MN_KGROUP_BYTES, MN_HALF_BYTES, MN_KGROUP_BYTES);
}

template <int SPLIT>
__device__ __forceinline__ void store_group(uint8_t* hi_tile, uint8_t* lo_tile, uint32_t off, const float (&v)[8]) {
  uint4 h;
  h.x = pack_bf16x2(v[0], v[1]);
  h.y = pack_bf16x2(v[2], v[3]);
  h.z = pack_bf16x2(v[4], v[5]);
  h.w = pack_bf16x2(v[6], v[7]);
  *reinterpret_cast<uint4*>(hi_tile + off) = h;
  if (SPLIT) {
    const __nv_bfloat162* hb = reinterpret_cast<const __nv_bfloat162*>(&h);
    uint4 l;
    l.x = pack_bf16x2(v[0] - __low2float(hb[0]), v[1] - __high2float(hb[0]));
    l.y = pack_bf16x2(v[2] - __low2float(hb[1]), v[3] - __high2float(hb[1]));
    l.z = pack_bf16x2(v[4] - __low2float(hb[2]), v[5] - __high2float(hb[2]));
    l.w = pack_bf16x2(v[6] - __low2float(hb[3]), v[7] - __high2float(hb[3]));
    *reinterpret_cast<uint4*>(lo_tile + off) = l;
  }
}

template <int SPLIT, int NT>
__device__ __forceinline__ void store_slab(uint8_t* st, const ThreadUnits<NT>& tu, const float (&va)[Shape<NT>::UPT][8],
                                           const float (&vb)[Shape<NT>::UPT][8]) {
  constexpr int UPT = Shape<NT>::UPT;
#pragma unroll
  for (int i = 0; i < UPT; ++i) store_group<SPLIT>(st, st + 2 * TILE_BYTES, tu.oa[i], va[i]);
#pragma unroll
  for (int i = 0; i < UPT; ++i) store_group<SPLIT>(st + TILE_BYTES, st + 3 * TILE_BYTES, tu.ob[i], vb[i]);
}

// Writes (splits == 1) or accumulates (split-K) WCOLS consecutive results of
// row m starting at column n0 + col.
// WCOLS consecutive accumulator columns of this warp's 32 lanes.
template <int WCOLS>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[WCOLS]) {
  if constexpr (WCOLS == 32) ptx::tmem_ld_32x32b_x32(taddr, r);
  else ptx::tmem_ld_32x32b_x16(taddr, r);
}

template <int WCOLS>
__device__ __forceinline__ void write_row(const ContractDesc& d, int64_t m, int64_t n0, int col,
                                          const uint32_t (&r)[WCOLS]) {
  if (m >= d.M) return;
  float* __restrict__ C = d.C;
  const int64_t N = d.N;
  const bool vec = ((N & 3) == 0) && ((reinterpret_cast<uintptr_t>(C) & 15) == 0);
  const bool accumulate = d.splits > 1;
  float* dst = C + m * N + n0 + col;
  const int64_t nrem = N - (n0 + col);
#pragma unroll
  for (int i = 0; i < WCOLS; i += 4)
    if (i < nrem)
      emit4(dst + i, vec, nrem - i, accumulate, __uint_as_float(r[i]), __uint_as_float(r[i + 1]),
            __uint_as_float(r[i + 2]), __uint_as_float(r[i + 3]));
}

template <int SPLIT>
__global__ void __launch_bounds__(Cfg<SPLIT>::NT, 1)
tc_contract_kernel(const __grid_constant__ ContractDesc single, const ContractDesc* group,
                   const int32_t* unit_desc, int64_t total_units, int* status) {
  using C = Cfg<SPLIT>;
  constexpr int S = C::STAGES;
  constexpr int NT = C::NT;
  constexpr int UPT = Shape<NT>::UPT;
  constexpr int WCOLS = Shape<NT>::WCOLS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  TcAux<S>& x = *reinterpret_cast<TcAux<S>*>(smem + (size_t)S * C::STAGE_BYTES);

  const int t = threadIdx.x;
  const int warp = t >> 5, lane = t & 31;
  const bool grouped = group != nullptr;
  constexpr uint32_t DESC_BYTES = (uint32_t)sizeof(ContractDesc);
  static_assert(sizeof(ContractDesc) % 16 == 0, "bulk copies move multiples of 16 bytes");
  const bool issuer = (t == 0);    // issues the MMAs
  const bool fetcher = (t == 32);  // prefetches descriptors

  if (issuer) {
    for (int s = 0; s < S; ++s) ptx::mbar_init(ptx::smem_addr(&x.empty[s]), 1);
    ptx::mbar_init(ptx::smem_addr(&x.accum), 1);
    for (int b = 0; b < 2; ++b) {
      ptx::mbar_init(ptx::smem_addr(&x.chunk_full[b]), 1);
      ptx::mbar_init(ptx::smem_addr(&x.desc_bar[b]), 1);
    }
    ptx::mbar_init(ptx::smem_addr(&x.final_bar), 1);
    x.abort = 0;
    ptx::fence_mbar_init();
    if (grouped) {
      ptx::mbar_arrive_expect_tx(ptx::smem_addr(&x.desc_bar[0]), DESC_BYTES);
      ptx::bulk_copy_g2s(ptx::smem_addr(&x.dslot[0]), group + unit_desc[blockIdx.x], DESC_BYTES,
                         ptx::smem_addr(&x.desc_bar[0]));
    } else {
      x.dslot[0] = single;
      x.dslot[1] = single;
    }
  }
  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_addr(&x.tmem_base), C::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  // the fetcher keeps the descriptor index of the unit after next in a
  // register, so its global load overlaps a whole unit
  int next_idx = 0;
  if (fetcher && grouped && blockIdx.x + gridDim.x < total_units) next_idx = unit_desc[blockIdx.x + gridDim.x];
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = x.tmem_base;
  const uint32_t stage0 = ptx::smem_addr(smem);
  const int q = warp & 3, cb = warp >> 2;  // TMEM lane quadrant and WCOLS-column block of this warp

  uint32_t g_slab = 0;   // slabs processed by this CTA (stage ring position)
  uint32_t g_chunk = 0;  // BF16X3 accumulator chunks processed by this CTA
  uint32_t j = 0;        // units processed by this CTA
  for (int64_t u = blockIdx.x; u < total_units; u += gridDim.x, ++j) {
    if (x.abort) break;  // uniform: read after the barrier that ends each unit
    const int slot = grouped ? (int)(j & 1) : 0;
    // prefetch the next unit's descriptor into the other slot (free: every
    // thread finished the previous unit before the barrier that ended it)
    if (fetcher && grouped && u + gridDim.x < total_units) {
      ptx::mbar_arrive_expect_tx(ptx::smem_addr(&x.desc_bar[slot ^ 1]), DESC_BYTES);
      ptx::bulk_copy_g2s(ptx::smem_addr(&x.dslot[slot ^ 1]), group + next_idx, DESC_BYTES,
                         ptx::smem_addr(&x.desc_bar[slot ^ 1]));
      const int64_t u2 = u + 2 * (int64_t)gridDim.x;
      if (u2 < total_units) next_idx = unit_desc[u2];
    }
    bool ok = true;
    if (grouped) ok = ptx::mbar_wait(ptx::smem_addr(&x.desc_bar[slot]), (j >> 1) & 1u, status);
    ok = __syncthreads_and(ok) != 0;  // CTA-uniform: every thread runs the same slab count
    const ContractDesc& d = x.dslot[slot];
    const UnitCoord uc = decode_unit(d, ok ? u - d.tile_begin : 0, BM, BN);
    const int64_t m0 = uc.m0, n0 = uc.n0;
    const int64_t nkt = ok ? (uc.k_end - uc.k_begin + BK - 1) / BK : 0;
    const int64_t nchunks = (nkt + KC - 1) / KC;

    if (t < BM) {
      const int64_t m = m0 + t;
      x.rowA[t] = (m < d.M) ? (int32_t)leg_offset((uint32_t)m, d.nm, d.mdim, d.mstr) : -1;
    } else if (t < BM + BN) {
      const int64_t n = n0 + (t - BM);
      x.rowB[t - BM] = (n < d.N) ? (int32_t)leg_offset((uint32_t)n, d.nn, d.ndim, d.nstr) : -1;
    }
    float acc[SPLIT ? WCOLS : 1];
#pragma unroll
    for (int i = 0; i < (SPLIT ? WCOLS : 1); ++i) acc[i] = 0.0f;
    // BF16X3: adds finished chunk c of this unit (accumulator buffer c & 1)
    // into acc; the MMAs that reuse the buffer are issued after a later
    // barrier, so program order protects it
    auto drain = [&](int64_t c) -> bool {
      const uint32_t cg = g_chunk + (uint32_t)c;
      const int b = (int)(cg & 1);
      const bool w = ptx::mbar_wait(ptx::smem_addr(&x.chunk_full[b]), (cg >> 1) & 1u, status);
      if (!__all_sync(0xffffffffu, w)) return false;
      ptx::tc_fence_after();
      uint32_t r[WCOLS];
      tmem_ld_cols<WCOLS>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + cb * WCOLS), r);
      ptx::tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < WCOLS; ++i) acc[i] += __uint_as_float(r[i]);
      ptx::tc_fence_before();
      return true;
    };
    int64_t next_drain = 0;

    ThreadUnits<NT> tu;  // filled once the row tables are published (prologue barrier)
    // two register sets used in turn (the loop below is unrolled by two), so
    // the loads of slab k+1 are consumed only in the next slab's step
    float ra0[UPT][8], rb0[UPT][8], ra1[UPT][8], rb1[UPT][8];
    // One slab: decode tables ahead, gather (pipelined: the next slab into
    // the other set), wait for the stage, convert and store the current set,
    // close the slab with the barrier, issue its MMAs. Returns false when a
    // bounded wait expired anywhere in the CTA.
    auto slab = [&](int64_t kt, float (&cur_a)[UPT][8], float (&cur_b)[UPT][8], float (&nxt_a)[UPT][8],
                    float (&nxt_b)[UPT][8]) -> bool {
      const uint32_t gs = g_slab + (uint32_t)kt;
      const int s = (int)(gs % S);
      const uint32_t round = gs / S;
      if (C::PIPE) {
        if (kt + 1 < nkt) load_slab<NT>(d, x, (int)kt + 1, tu, nxt_a, nxt_b);
      } else {
        load_slab<NT>(d, x, (int)kt, tu, cur_a, cur_b);
      }
      bool drained_ok = true;
      if (SPLIT && (kt % KC) == 0 && kt / KC >= 2) drained_ok = drain(next_drain++);
      // the stage's previous MMAs must be complete before it is rewritten
      const bool waited = ptx::mbar_wait(ptx::smem_addr(&x.empty[s]), (round & 1u) ^ 1u, status) && drained_ok;
      if (waited) {
        store_slab<SPLIT, NT>(smem + (size_t)s * C::STAGE_BYTES, tu, cur_a, cur_b);
        ptx::fence_proxy_async_smem();
      }
      // every thread reaches this barrier once per slab; a wait that expired
      // anywhere stops all of them together
      ptx::tc_fence_before();
      if (ptx::named_barrier_or(1, NT, !waited)) return false;
      if (issuer) {
        ptx::tc_fence_after();
        const int64_t c = kt / KC;
        const uint32_t cg = g_chunk + (uint32_t)c;
        const uint32_t d_tmem = SPLIT ? tmem + (uint32_t)((cg & 1) * BN) : tmem;
        const bool fresh = SPLIT ? (kt % KC) == 0 : (kt == 0);
        const uint32_t idesc = ptx::idesc_bf16_f32(BM, BN, d.a_kfast ? 0 : 1, d.b_kfast ? 0 : 1);
        const uint32_t a_hi = stage0 + (uint32_t)(s * C::STAGE_BYTES);
        const uint32_t b_hi = a_hi + TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t ad = operand_desc(d.a_kfast, a_hi, kk);
          const uint64_t bd = operand_desc(d.b_kfast, b_hi, kk);
          ptx::mma_bf16(d_tmem, ad, bd, idesc, (fresh && kk == 0) ? 0u : 1u);
          if (SPLIT) {
            const uint64_t al = operand_desc(d.a_kfast, a_hi + 2 * TILE_BYTES, kk);
            const uint64_t bl = operand_desc(d.b_kfast, b_hi + 2 * TILE_BYTES, kk);
            ptx::mma_bf16(d_tmem, ad, bl, idesc, 1u);
            ptx::mma_bf16(d_tmem, al, bd, idesc, 1u);
          }
        }
        ptx::mma_commit(ptx::smem_addr(&x.empty[s]));
        if (SPLIT && ((kt % KC) == KC - 1 || kt == nkt - 1)) ptx::mma_commit(ptx::smem_addr(&x.chunk_full[cg & 1]));
      }
      __syncwarp();
      return true;
    };
    // prologue: the unit's offset tables (and, pipelined, the registers of
    // slab 0)
    if (nkt > 0) fill_tables<NT>(d, uc, x);
    ptx::named_barrier(1, NT);
    tu = thread_units<NT>(d, x, m0, n0, t);
    if (C::PIPE && nkt > 0) load_slab<NT>(d, x, 0, tu, ra0, rb0);
    for (int64_t kt = 0; kt < nkt; kt += 2) {
      if (!slab(kt, ra0, rb0, ra1, rb1)) { ok = false; break; }
      if (kt + 1 < nkt && !slab(kt + 1, ra1, rb1, ra0, rb0)) { ok = false; break; }
    }
    // one arrival per unit on accum: a commit tracking this unit's MMAs, or a
    // plain arrive when none were issued
    if (issuer) {
      if (ok && nkt > 0) ptx::mma_commit(ptx::smem_addr(&x.accum));
      else ptx::mbar_arrive(ptx::smem_addr(&x.accum));
    }
    __syncwarp();

    // -------------------------------------------------------------- epilogue
    if (SPLIT) {
      for (; ok && next_drain < nchunks; ++next_drain) ok = drain(next_drain);
    }
    const bool acc_ready = ptx::mbar_wait(ptx::smem_addr(&x.accum), j & 1u, status) && ok;
    if (__all_sync(0xffffffffu, acc_ready) && nkt > 0) {  // tcgen05.ld is warp-collective
      ptx::tc_fence_after();
      const int64_t m = m0 + q * 32 + lane;
      uint32_t r[WCOLS];
      if (SPLIT) {
#pragma unroll
        for (int i = 0; i < WCOLS; ++i) r[i] = __float_as_uint(acc[i]);
      } else {
        tmem_ld_cols<WCOLS>(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(cb * WCOLS), r);
        ptx::tmem_ld_wait();
      }
      write_row<WCOLS>(d, m, n0, cb * WCOLS, r);
    }
    if (!ok || !acc_ready) x.abort = 1;
    g_slab += (uint32_t)nkt;
    g_chunk += (uint32_t)nchunks;
    // end of unit: TMEM drained, descriptor slot and offset tables free
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
  }

  // every MMA of the issuing thread has completed before TMEM is released
  if (warp == 0) {
    if (issuer) {
      ptx::mma_commit(ptx::smem_addr(&x.final_bar));
      ptx::mbar_wait(ptx::smem_addr(&x.final_bar), 0u, status);
    }
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
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

template <int SPLIT>
int launch_tc(const ContractDesc& single, const ContractDesc* group, const int32_t* unit_desc, int64_t units,
              cudaStream_t stream) {
  const size_t smem = tc_smem_bytes<SPLIT>();
  static std::atomic<uint64_t> attr{0};
  if (!smem_limit_once((const void*)tc_contract_kernel<SPLIT>, smem, &attr)) return TN_ERR_CUDA;
  const int64_t resident = (int64_t)sm_count();
  const unsigned grid = (unsigned)(units < resident ? units : resident);
  tc_contract_kernel<SPLIT><<<grid, Cfg<SPLIT>::NT, smem, stream>>>(single, group, unit_desc, units, status_word());
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace

int launch_contract_tc(const ContractDesc& single, const ContractDesc* group, const int32_t* unit_desc,
                       int64_t total_tiles, int prec, cudaStream_t stream) {
  if (total_tiles <= 0) return TN_OK;
  if (total_tiles > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (group && !unit_desc) return TN_ERR_ARG;
  if (prec == TN_PREC_BF16) return launch_tc<0>(single, group, unit_desc, total_tiles, stream);
  if (prec == TN_PREC_BF16X3) return launch_tc<1>(single, group, unit_desc, total_tiles, stream);
  return TN_ERR_ARG;
}

}  // namespace tn
