// <psi_k|H|psi_k> and <psi_k|psi_k> for a batch of MPS with uneven bond
// dimensions and one shared MPO (the environment sweep of Sec. II / Fig. 3a
// applied to many chains at once). The norm rides along as one more MPO
// channel (the MPO extended by an identity channel, as in tn_mps_expect).
// Every site step of every chain goes into grouped launches, so the launch
// count per site does not grow with the batch: (i) one grouped contraction,
// (ii) one grouped float32 kernel that also applies the previous site's
// deferred power-of-two rescale, (iii) one grouped contraction, then one
// grouped max-abs pass over the count new environments. BF16 / BF16X3 with
// an extended MPO of (bond) x d <= 8: step (ii) writes each chain's T2
// straight into the (iii) plan's packed region as its first operand (whole
// MN-major blocks), so that plan packs only the cores.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "tn_internal.h"

namespace tn {
namespace {

// One environment whose largest magnitude is wanted after a site: *bits
// holds the running max (float bits) and starts at 0.
struct Segment {
  float* x;
  int64_t n;
  unsigned* bits;
  double* lg;
};

__device__ float seg_block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float m = 0.0f;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmaxf(m, red[i]);
  return m;
}

// grid (blocks per segment, segments)
__global__ void seg_absmax_kernel(const Segment* __restrict__ segs) {
  __shared__ float red[32];
  const Segment s = segs[blockIdx.y];
  float m = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(s.x[i]));
  m = seg_block_max(m, red);
  if (threadIdx.x == 0) atomicMax(s.bits, __float_as_uint(m));
}

// Per chain: the starting environment, 1 in each of its channels (the MPO's
// left boundary and the norm channel).
struct ChainInit {
  float* L;
  int32_t channels, pad;
};

__global__ void grouped_init_kernel(const ChainInit* __restrict__ c, int count, double* lg, int nlg,
                                    unsigned* bits, int64_t nbits) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = t; i < nbits; i += stride) bits[i] = 0u;
  for (int64_t i = t; i < nlg; i += stride) lg[i] = 0.0;
  for (int64_t i = t; i < count; i += stride)
    for (int w = 0; w < c[i].channels; ++w) c[i].L[w] = 1.0f;
}

// Per chain: where the final environment ended (channel 0: the energy,
// channel 1: the norm).
struct ChainFinal {
  const float* L;
};

__global__ void grouped_finish_kernel(const ChainFinal* __restrict__ f, int count, const double* __restrict__ lg,
                                      double* result) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
    result[4 * k + 0] = (double)f[k].L[0];
    result[4 * k + 1] = lg[k];
    result[4 * k + 2] = (double)f[k].L[1];
    result[4 * k + 3] = lg[k];
  }
}

tn_tensor make_tensor(float* p, int rank, const int64_t* sh) {
  tn_tensor t;
  tn_tensor_init(&t, p, rank, sh);
  return t;
}

tn_contract_spec make_spec(const tn_tensor& A, std::initializer_list<int> la, const tn_tensor& B,
                           std::initializer_list<int> lb, const tn_tensor& C) {
  tn_contract_spec s;
  memset(&s, 0, sizeof(s));
  s.A = A;
  s.B = B;
  s.C = C;
  s.nshared = (int32_t)la.size();
  int j = 0;
  for (int v : la) s.legsA[j++] = v;
  j = 0;
  for (int v : lb) s.legsB[j++] = v;
  return s;
}

int64_t chain_max_bond(const tn_mps& m) {
  int64_t x = 1;
  for (int i = 0; i <= m.n; ++i) x = std::max(x, m.bond[i]);
  return x;
}

int check_one(const tn_mps& m) {
  if (m.n < 1 || m.d < 1 || !m.bond || !m.cores) return TN_ERR_ARG;
  if (m.bond[0] != 1 || m.bond[m.n] != 1) return TN_ERR_ARG;
  for (int i = 0; i < m.n; ++i)
    if (m.bond[i + 1] < 1 || !m.cores[i]) return TN_ERR_ARG;
  return TN_OK;
}

struct PlanDeleter {
  void operator()(tn_group_plan* p) const { tn_group_plan_destroy(p); }
};
using PlanPtr = std::unique_ptr<tn_group_plan, PlanDeleter>;

// Host-side layout of one grouped sweep: buffers of every chain, the site
// plans (two per site, their work lists only), one packed-operand region
// they share, the extended MPO, the step (ii) descriptors and the per-site
// max-abs tables.
struct GroupedSweep {
  struct ChainBufs {
    float *L[2], *T1, *T2;
  };
  int count = 0, n = 0;
  int64_t d = 0;
  std::vector<ChainBufs> bufs;
  std::vector<PlanPtr> plans;         // site-major: (i), (iii)
  std::vector<size_t> plan_off;       // workspace offset of each plan's work list
  std::vector<size_t> plan_bytes;
  std::vector<Segment> segs;          // n * count
  std::vector<StepII> steps;          // n * count
  // fused mode (BF16 / BF16X3, extended MPO bond x d <= 8): step (ii) writes
  // T2 straight into the (iii) plan's packed region
  bool fused = false;
  std::vector<StepIIPack> psteps;     // n * count (hi / lo: offsets in the packed region until laid out)
  std::vector<int64_t> max_items;     // per site: the largest step (ii) work of a chain
  std::vector<int64_t> max_cols;      // per site: the largest Da Db of the batch
  std::vector<ChainInit> inits;
  std::vector<ChainFinal> finals;
  std::vector<int64_t> woff;          // extended MPO of every site
  size_t off_lg = 0, off_bits = 0, off_segs = 0, off_steps = 0, off_psteps = 0, off_init = 0, off_final = 0,
         off_packed = 0;
  size_t off_w = 0, total = 0;
  size_t packed_bytes = 0;  // largest packed-operand region of one plan
  int64_t nbits = 0;
};

// Builds the layout of a workspace at `base` (the plans' work lists decide
// its size, so they are built even when only the size is wanted; nothing is
// dereferenced on the host).
int build_sweep(const tn_mps* psis, int count, const tn_mpo* H, int prec, uint8_t* base, GroupedSweep* g) {
  if (!psis || count < 1 || count > 16384 || !H || !H->bond || !H->cores) return TN_ERR_ARG;
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  const int n = psis[0].n;
  const int64_t d = psis[0].d;
  for (int k = 0; k < count; ++k) {
    int rc = check_one(psis[k]);
    if (rc != TN_OK) return rc;
    if (psis[k].n != n || psis[k].d != d) return TN_ERR_ARG;
  }
  if (H->n != n || H->d != d || H->bond[0] != 1 || H->bond[n] != 1) return TN_ERR_ARG;
  int64_t Wm = 1;
  for (int i = 0; i < n; ++i) {
    if (H->bond[i + 1] < 1 || !H->cores[i]) return TN_ERR_ARG;
    Wm = std::max(Wm, H->bond[i + 1]);
  }
  if (!mpo_extend_supported(H)) return TN_ERR_UNSUPPORTED;
  const int64_t W1 = Wm + 1;
  for (int k = 0; k < count; ++k) {
    const int64_t D = chain_max_bond(psis[k]);
    if (W1 * D * d * D >= (int64_t(1) << 31)) return TN_ERR_UNSUPPORTED;  // 32-bit step (ii) offsets
  }
  g->count = count;
  g->n = n;
  g->d = d;
  g->fused = prec != TN_PREC_FP32;
  for (int i = 0; i <= n; ++i)
    if ((H->bond[i] + 1) * d > 8) g->fused = false;
  size_t off = 0;
  auto take = [&](size_t b) {
    uint8_t* p = base + off;
    off += align256(b);
    return reinterpret_cast<float*>(p);
  };
  g->bufs.resize((size_t)count);
  for (int k = 0; k < count; ++k) {
    const int64_t D = chain_max_bond(psis[k]);
    auto& b = g->bufs[(size_t)k];
    b.L[0] = take(sizeof(float) * W1 * D * D);
    b.L[1] = take(sizeof(float) * W1 * D * D);
    b.T1 = take(sizeof(float) * W1 * D * d * D);
    b.T2 = take(sizeof(float) * W1 * D * d * D);
  }
  int64_t wtot = 0;
  for (int i = 0; i < n; ++i) {
    g->woff.push_back(wtot);
    wtot += (H->bond[i] + 1) * (H->bond[i + 1] + 1) * d * d;
  }
  g->off_w = off;
  off += align256(sizeof(float) * (size_t)wtot);
  const float* Wx = reinterpret_cast<const float*>(base + g->off_w);
  g->off_lg = off;
  off += align256(sizeof(double) * (size_t)count);
  g->off_bits = off;
  g->nbits = (int64_t)n * count;
  off += align256(sizeof(unsigned) * (size_t)g->nbits);
  double* lg = reinterpret_cast<double*>(base + g->off_lg);
  unsigned* bits = reinterpret_cast<unsigned*>(base + g->off_bits);

  // site plans
  std::vector<tn_contract_spec> s1, s3;
  for (int i = 0; i < n; ++i) {
    s1.clear();
    s3.clear();
    const int64_t wa = H->bond[i] + 1, wb = H->bond[i + 1] + 1;
    int64_t mc = 1;
    for (int k = 0; k < count; ++k) {
      const tn_mps& m = psis[k];
      auto& b = g->bufs[(size_t)k];
      const int64_t Da = m.bond[i], Db = m.bond[i + 1];
      float* core = m.cores[i];
      const int64_t shA[3] = {Da, d, Db};
      const tn_tensor tA = make_tensor(core, 3, shA);
      const int64_t shL[3] = {wa, Da, Da}, shT1[4] = {wa, Da, d, Db};
      const int64_t shT2[4] = {wb, d, Da, Db}, shL2[3] = {wb, Db, Db};
      const tn_tensor tL = make_tensor(b.L[i & 1], 3, shL), tT1 = make_tensor(b.T1, 4, shT1);
      const tn_tensor tT2 = make_tensor(b.T2, 4, shT2);
      const tn_tensor tL2 = make_tensor(b.L[(i + 1) & 1], 3, shL2);
      // (i)   T1[w, a', s, b] = sum_a L[w, a, a'] psi[a, s, b]
      s1.push_back(make_spec(tL, {1}, tA, {0}, tT1));
      // (ii)  T2[w', s', a', b] = 2^-e sum_{w, s} W'[w, w', s, s'] T1[w, a', s, b]
      StepII q;
      memset(&q, 0, sizeof(q));
      q.T1 = b.T1;
      q.T2 = b.T2;
      q.W = Wx + g->woff[(size_t)i];
      q.Da = Da;
      q.Db = Db;
      q.wa = (int32_t)wa;
      q.wb = (int32_t)wb;
      q.d = (int32_t)d;
      q.maxbits = i > 0 ? bits + (size_t)count * (i - 1) + k : nullptr;
      q.lg = lg + k;
      g->steps.push_back(q);
      mc = std::max(mc, Da * Db);
      // (iii) L'[w', b, b'] = sum_{a', s'} T2[w', s', a', b] psi[a', s', b']
      s3.push_back(make_spec(tT2, {1, 2}, tA, {1, 0}, tL2));
      g->segs.push_back(Segment{b.L[(i + 1) & 1], wb * Db * Db, bits + (size_t)count * i + k, lg + k});
    }
    g->max_cols.push_back(mc);
    const std::vector<tn_contract_spec>* stages[2] = {&s1, &s3};
    const std::vector<uint8_t> ext((size_t)count, 1);
    for (int j = 0; j < 2; ++j) {
      tn_group_plan* p = nullptr;
      int rc = group_plan_create_ex(stages[j]->data(), (int)stages[j]->size(), prec, true, &p,
                                    j == 1 && g->fused ? ext.data() : nullptr);
      if (rc != TN_OK) return rc;
      g->plans.emplace_back(p);
      if (j == 1 && g->fused) {
        // step (ii) of every chain writes its T2 where the (iii) plan reads P
        int64_t mi = 1;
        for (int k = 0; k < count; ++k) {
          ExtPLayout lay;
          if ((rc = group_plan_ext_layout(p, k, &lay)) != TN_OK) return rc;
          const StepII& q0 = g->steps[(size_t)count * i + k];
          StepIIPack q;
          memset(&q, 0, sizeof(q));
          q.T1 = q0.T1;
          q.W = q0.W;
          q.maxbits = q0.maxbits;
          q.lg = q0.lg;
          // offsets for now; device addresses once the packed region is placed
          q.hi = reinterpret_cast<uint8_t*>((uintptr_t)lay.hi_off);
          q.lo = lay.lo_off < 0 ? nullptr : reinterpret_cast<uint8_t*>((uintptr_t)lay.lo_off);
          q.Da = (int32_t)q0.Da;
          q.Db = (int32_t)q0.Db;
          q.wa = q0.wa;
          q.wb = q0.wb;
          q.d = q0.d;
          q.tiles = lay.tiles;
          q.slabs = lay.slabs;
          if (lay.nk != 2) return TN_ERR_UNSUPPORTED;
          step_iii_places(q0.Da, q0.Db, d, lay.kstrA, &q.ps, &q.pa);
          g->psteps.push_back(q);
          mi = std::max(mi, q0.Db % 8 == 0 ? q0.Da * (q0.Db / 8) : q0.Da * q0.Db);
        }
        g->max_items.push_back(mi);
      }
      const size_t bytes = group_plan_list_bytes(p);
      g->plan_off.push_back(off);
      g->plan_bytes.push_back(bytes);
      off += align256(bytes);
      g->packed_bytes = std::max(g->packed_bytes, group_plan_packed_bytes(p));
    }
  }
  // one region for the packed operands of whichever plan is running (the
  // plans run one after another on the stream)
  g->off_packed = off;
  off += align256(g->packed_bytes);
  for (auto& q : g->psteps) {
    q.hi = base + g->off_packed + (uintptr_t)q.hi;
    if (q.lo) q.lo = base + g->off_packed + (uintptr_t)q.lo;
  }
  g->off_segs = off;
  off += align256(sizeof(Segment) * g->segs.size());
  g->off_steps = off;
  off += align256(sizeof(StepII) * g->steps.size());
  g->off_psteps = off;
  off += align256(sizeof(StepIIPack) * g->psteps.size());
  g->inits.resize((size_t)count);
  g->finals.resize((size_t)count);
  for (int k = 0; k < count; ++k) {
    g->inits[(size_t)k] = ChainInit{g->bufs[(size_t)k].L[0], (int32_t)(H->bond[0] + 1), 0};
    g->finals[(size_t)k] = ChainFinal{g->bufs[(size_t)k].L[n & 1]};
  }
  g->off_init = off;
  off += align256(sizeof(ChainInit) * (size_t)count);
  g->off_final = off;
  off += align256(sizeof(ChainFinal) * (size_t)count);
  g->total = off;
  return TN_OK;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

size_t tn_mps_expect_grouped_workspace_bytes(const tn_mps* psis, int count, const tn_mpo* H, int prec) {
  // sizes only: any 256-byte aligned base gives the same layout
  GroupedSweep g;
  if (build_sweep(psis, count, H, prec, reinterpret_cast<uint8_t*>(uintptr_t(1) << 20), &g) != TN_OK) return 0;
  return g.total;
}

}  // extern "C"

// A planned grouped sweep: the host layout (site plans, tables) built and its
// tables uploaded once; every run only launches. The MPO's core pointers are
// kept (its extension is rebuilt at every run, so values changed in place
// are picked up, as are the states' core values).
struct tn_expect_plan {
  tn::GroupedSweep g;
  uint8_t* base;
  size_t bytes;
  std::vector<int64_t> hbond;
  std::vector<float*> hcores;
  tn_mpo H;
};

namespace tn {
namespace {

int run_sweep(const tn_expect_plan* pl, double* result, cudaStream_t s) {
  const GroupedSweep& g = pl->g;
  uint8_t* base = pl->base;
  const int count = g.count;
  int rc;
  if ((rc = launch_mpo_extend(&pl->H, reinterpret_cast<float*>(base + g.off_w), g.woff.data(), s)) != TN_OK) return rc;
  double* lg = reinterpret_cast<double*>(base + g.off_lg);
  unsigned* bits = reinterpret_cast<unsigned*>(base + g.off_bits);
  grouped_init_kernel<<<64, 256, 0, s>>>(reinterpret_cast<const ChainInit*>(base + g.off_init), count, lg, count,
                                         bits, g.nbits);
  if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
  const Segment* segs = reinterpret_cast<const Segment*>(base + g.off_segs);
  const StepII* steps = reinterpret_cast<const StepII*>(base + g.off_steps);
  for (int i = 0; i < g.n; ++i) {
    const size_t p0 = (size_t)i * 2;
    if ((rc = group_plan_run_shared(g.plans[p0].get(), base + g.plan_off[p0], g.plan_bytes[p0], s)) != TN_OK)
      return rc;
    const StepII& q0 = g.steps[(size_t)count * i];
    if (g.fused) {
      const StepIIPack* psteps = reinterpret_cast<const StepIIPack*>(base + g.off_psteps);
      if ((rc = launch_step_ii_pack_grouped(psteps + (size_t)count * i, count, g.max_items[(size_t)i], s)) != TN_OK)
        return rc;
    } else if ((rc = launch_mpo_step_ii_grouped(steps + (size_t)count * i, count, g.max_cols[(size_t)i],
                                                (int64_t)q0.wa * q0.d, (int64_t)q0.wb * q0.d, s)) != TN_OK) {
      return rc;
    }
    if ((rc = group_plan_run_shared(g.plans[p0 + 1].get(), base + g.plan_off[p0 + 1], g.plan_bytes[p0 + 1], s)) !=
        TN_OK)
      return rc;
    if (i + 1 < g.n) {
      int64_t longest = 1;
      for (int k = 0; k < count; ++k) longest = std::max(longest, g.segs[(size_t)count * i + k].n);
      const dim3 grid((unsigned)std::min<int64_t>((longest + 2047) / 2048, 64), (unsigned)count);
      seg_absmax_kernel<<<grid, 256, 0, s>>>(segs + (size_t)count * i);
      if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
    }
  }
  grouped_finish_kernel<<<(count + 127) / 128, 128, 0, s>>>(reinterpret_cast<const ChainFinal*>(base + g.off_final),
                                                           count, lg, result);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

}  // namespace
}  // namespace tn

extern "C" {

int tn_mps_expect_grouped_plan(const tn_mps* psis, int count, const tn_mpo* H, int prec, void* workspace,
                               size_t ws_bytes, tn_expect_plan** plan, void* stream) {
  if (!plan) return TN_ERR_ARG;
  *plan = nullptr;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;
  // its tables are copied from host lists that live in the plan: not from a capture
  if (stream_capturing(static_cast<cudaStream_t>(stream))) return TN_ERR_UNSUPPORTED;
  std::unique_ptr<tn_expect_plan> pl(new tn_expect_plan());
  uint8_t* base = static_cast<uint8_t*>(workspace);
  GroupedSweep& g = pl->g;
  int rc = build_sweep(psis, count, H, prec, base, &g);
  if (rc != TN_OK) return rc;
  if (ws_bytes < g.total) return TN_ERR_WORKSPACE;
  pl->base = base;
  pl->bytes = ws_bytes;
  pl->hbond.assign(H->bond, H->bond + H->n + 1);
  pl->hcores.assign(H->cores, H->cores + H->n);
  pl->H = *H;
  pl->H.bond = pl->hbond.data();
  pl->H.cores = pl->hcores.data();
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // uploads: plan work lists, max-abs segments, step (ii) descriptors, init
  // and final tables
  for (size_t j = 0; j < g.plans.size(); ++j) {
    if (g.plan_bytes[j] == 0) continue;
    rc = group_plan_upload_shared(g.plans[j].get(), base + g.plan_off[j], g.plan_bytes[j], base + g.off_packed, s);
    if (rc != TN_OK) return rc;
  }
  if (cudaMemcpyAsync(base + g.off_segs, g.segs.data(), sizeof(Segment) * g.segs.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      cudaMemcpyAsync(base + g.off_steps, g.steps.data(), sizeof(StepII) * g.steps.size(), cudaMemcpyHostToDevice,
                      s) != cudaSuccess ||
      (!g.psteps.empty() && cudaMemcpyAsync(base + g.off_psteps, g.psteps.data(),
                                            sizeof(StepIIPack) * g.psteps.size(), cudaMemcpyHostToDevice,
                                            s) != cudaSuccess) ||
      cudaMemcpyAsync(base + g.off_init, g.inits.data(), sizeof(ChainInit) * g.inits.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + g.off_final, g.finals.data(), sizeof(ChainFinal) * g.finals.size(),
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TN_ERR_CUDA;
  *plan = pl.release();
  return TN_OK;
}

int tn_mps_expect_grouped_run(const tn_expect_plan* plan, double* result, void* stream) {
  if (!plan || !result) return TN_ERR_ARG;
  return run_sweep(plan, result, static_cast<cudaStream_t>(stream));
}

void tn_mps_expect_grouped_destroy(tn_expect_plan* plan) { delete plan; }

int tn_mps_expect_grouped(const tn_mps* psis, int count, const tn_mpo* H, int prec, void* workspace,
                          size_t ws_bytes, double* result, void* stream) {
  if (!result) return TN_ERR_ARG;
  tn_expect_plan* plan = nullptr;
  int rc = tn_mps_expect_grouped_plan(psis, count, H, prec, workspace, ws_bytes, &plan, stream);
  if (rc != TN_OK) return rc;
  rc = tn_mps_expect_grouped_run(plan, result, stream);
  tn_mps_expect_grouped_destroy(plan);
  return rc;
}

}  // extern "C"
