// MPS image classifier (Sec. IV.A): forward scores and the adjoint backward.
//
// Forward: the local feature map Phi(p) = (cos(pi p/2), sin(pi p/2)) of each
// pixel is contracted into the chain from both ends towards the label core.
// One step of a half-chain, for a tile of samples b and the site's core seen
// as L[k, s, j] (k the incoming bond, j the outgoing one):
//     v'_b[j] = sum_s Phi_s(x_b) sum_k v_b[k] L[k, s, j],
// then v'_b is divided by its largest magnitude and log(scale_b) is added to
// the sample's float64 log-scale. The two half-chain vectors meet at the
// label core: ftilde_b[l] = sum_{a,s,c} vL_b[a] C[a, s, l, c] Phi_s vR_b[c].
//
// Backward (adjoint): the same step with the transposed core and the recorded
// scale, g_b[k] = sum_s Phi_s sum_j L[k, s, j] g'_b[j] / scale_b, walks from
// the label core outwards; the core gradients are sums over the batch,
// dL[k, s, j] = sum_b v_b[k] Phi_s(x_b) g'_b[j] / scale_b, evaluated per
// checkpoint segment as one grouped tensordot (K = batch) on the engine of
// tn_contract. Sweep vectors are kept every `ckpt_every` steps and the steps
// in between are recomputed segment by segment (checkpointing).
#include <math.h>

#include <algorithm>
#include <vector>

#include "classifier_tc.h"
#include "tn_internal.h"

namespace tn {
namespace {

constexpr int CLS_MAXN = 1024;  // sites passed by value to the sweep kernel
constexpr int CLS_MAXCHI = 128;
constexpr int BT = 32;          // samples per CTA of the float32 sweep

struct SweepParams {
  int32_t n, batch, half, mode;  // half: 0 left (sites 0..ls-1), 1 right (n-1..ls+1); mode 0 fwd, 1 adjoint
  int32_t t_begin, t_end;        // steps [t_begin, t_end) in sweep order (adjoint runs them backwards)
  int32_t store_every;           // forward: keep the vector entering step t if (t - store_base) % store_every == 0
  int32_t store_base;
  int32_t bond[CLS_MAXN + 1];
  const float* core[CLS_MAXN];
  const float* pixels;  // [batch, n]
  float* state;         // [batch, chi]: vector in, vector out
  double* lam;          // [batch] forward log-scale, in/out
  float* store;         // forward: [slot][batch][chi]
  float* sc;            // [t][batch] per-step scale (forward writes, adjoint reads)
  float* xout;          // adjoint: [t - t_begin][batch][2 chi] operands of the core gradients
};

// One CTA sweeps BT samples of one half-chain over [t_begin, t_end).
template <int CHI>
__global__ void __launch_bounds__(2 * CHI)
cls_sweep_simt(const __grid_constant__ SweepParams p) {
  constexpr int NT = 2 * CHI;
  constexpr int GQ = CHI / 4;  // threads sharing one group of 4 samples
  extern __shared__ float smem[];
  float* Ls = smem;                       // [CHI][2][CHI]
  float* S = Ls + 2 * CHI * CHI;          // [BT][CHI + 1]
  float* phi = S + BT * (CHI + 1);        // [2][BT]
  float* scl = phi + 2 * BT;              // [BT]
  double* lam = reinterpret_cast<double*>(scl + BT + (BT & 1));  // [BT]
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * BT;
  const int B = p.batch;
  const int bq = tid / GQ, jq = tid % GQ;
  constexpr int SR = CHI + 1;

  for (int i = tid; i < BT * CHI; i += NT) {
    const int b = i / CHI, k = i % CHI;
    S[b * SR + k] = (b0 + b < B) ? p.state[(int64_t)(b0 + b) * CHI + k] : 0.0f;
  }
  if (tid < BT) lam[tid] = (p.mode == 0 && b0 + tid < B) ? p.lam[b0 + tid] : 0.0;
  __syncthreads();

  const int nsteps = p.t_end - p.t_begin;
  for (int q = 0; q < nsteps; ++q) {
    const int t = p.mode == 0 ? p.t_begin + q : p.t_end - 1 - q;
    const int site = p.half == 0 ? t : p.n - 1 - t;
    // forward on the left and adjoint on the right read the core as
    // L[k=a, s, j=c]; the other two read it transposed, L[k=c, s, j=a]
    const bool natural = (p.half == 0) == (p.mode == 0);
    const int Da = p.bond[site], Dc = p.bond[site + 1];
    const int Din = natural ? Da : Dc, Dout = natural ? Dc : Da;
    const float* __restrict__ A = p.core[site];
    for (int i = tid; i < CHI * 2 * CHI; i += NT) {
      const int j = i % CHI, s = (i / CHI) & 1, k = i / (2 * CHI);
      float v = 0.0f;
      if (k < Din && j < Dout) v = natural ? __ldg(A + ((int64_t)k * 2 + s) * Dc + j) : __ldg(A + ((int64_t)j * 2 + s) * Dc + k);
      Ls[i] = v;
    }
    if (tid < BT) {
      const float x = (b0 + tid < B) ? __ldg(p.pixels + (int64_t)(b0 + tid) * p.n + site) : 0.0f;
      phi[tid] = cospif(0.5f * x);
      phi[BT + tid] = sinpif(0.5f * x);
      if (p.mode == 1) scl[tid] = (b0 + tid < B) ? p.sc[(int64_t)t * B + b0 + tid] : 1.0f;
    }
    if (p.mode == 0 && p.store && ((t - p.store_base) % p.store_every) == 0) {
      float* dst = p.store + (int64_t)((t - p.store_base) / p.store_every) * B * CHI;
      for (int i = tid; i < BT * CHI; i += NT) {
        const int b = i / CHI, k = i % CHI;
        if (b0 + b < B) dst[(int64_t)(b0 + b) * CHI + k] = S[b * SR + k];
      }
    }
    __syncthreads();
    if (p.mode == 1) {
      // operands of dL for this step: Phi_s(x_b) g'_b[k] / scale_b; the left
      // half stores them as [b][s][k], the right half as [b][k][s]
      float* dst = p.xout + (int64_t)(t - p.t_begin) * B * 2 * CHI;
      for (int i = tid; i < BT * 2 * CHI; i += NT) {
        const int b = i / (2 * CHI), r = i % (2 * CHI);
        if (b0 + b >= B) continue;
        int s, k;
        if (p.half == 0) { s = r / CHI; k = r % CHI; }
        else { k = r >> 1; s = r & 1; }
        dst[(int64_t)(b0 + b) * 2 * CHI + r] = phi[s * BT + b] * S[b * SR + k] / scl[b];
      }
    }

    float acc0[4][4], acc1[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { acc0[i][j] = 0.0f; acc1[i][j] = 0.0f; }
    for (int k = 0; k < Din; ++k) {
      float sv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) sv[i] = S[(bq * 4 + i) * SR + k];
      const float4 l0 = *reinterpret_cast<const float4*>(Ls + (k * 2 + 0) * CHI + jq * 4);
      const float4 l1 = *reinterpret_cast<const float4*>(Ls + (k * 2 + 1) * CHI + jq * 4);
      const float a0[4] = {l0.x, l0.y, l0.z, l0.w}, a1[4] = {l1.x, l1.y, l1.z, l1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc0[i][j] = fmaf(sv[i], a0[j], acc0[i][j]);
          acc1[i][j] = fmaf(sv[i], a1[j], acc1[i][j]);
        }
    }
    float out[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int b = bq * 4 + i;
      const float f0 = phi[b], f1 = phi[BT + b];
#pragma unroll
      for (int j = 0; j < 4; ++j) out[i][j] = f0 * acc0[i][j] + f1 * acc1[i][j];
    }
    if (p.mode == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float m = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) m = fmaxf(m, fabsf(out[i][j]));
#pragma unroll
        for (int o = GQ / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const float sc = m > 0.0f ? m : 1.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) out[i][j] = out[i][j] / sc;
        const int b = bq * 4 + i;
        if (jq == 0) {
          lam[b] += (double)logf(sc);  // float32 log, float64 running sum
          if (b0 + b < B) p.sc[(int64_t)t * B + b0 + b] = sc;
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float sc = scl[bq * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) out[i][j] = out[i][j] / sc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) S[(bq * 4 + i) * SR + jq * 4 + j] = out[i][j];
    __syncthreads();
  }
  for (int i = tid; i < BT * CHI; i += NT) {
    const int b = i / CHI, k = i % CHI;
    if (b0 + b < B) p.state[(int64_t)(b0 + b) * CHI + k] = S[b * SR + k];
  }
  if (p.mode == 0 && tid < BT && b0 + tid < B) p.lam[b0 + tid] = lam[tid];
}

template <int CHI>
size_t sweep_smem() {
  return sizeof(float) * (2 * CHI * CHI + BT * (CHI + 1) + 3 * BT + 2) + sizeof(double) * BT;
}

template <int CHI>
int launch_sweep_chi(const SweepParams& p, cudaStream_t s) {
  const size_t smem = sweep_smem<CHI>();
  static std::atomic<uint64_t> attr{0};
  if (!smem_limit_once((const void*)cls_sweep_simt<CHI>, smem, &attr)) return TN_ERR_CUDA;
  cls_sweep_simt<CHI><<<(p.batch + BT - 1) / BT, 2 * CHI, smem, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int launch_sweep(int chi, const SweepParams& p, cudaStream_t s) {
  if (p.t_end <= p.t_begin) return TN_OK;
  if (chi == 32) return launch_sweep_chi<32>(p, s);
  if (chi == 64) return launch_sweep_chi<64>(p, s);
  return launch_sweep_chi<128>(p, s);
}

// ------------------------------------------------------------- label core
// The label core C[a, s, l, c] meets the two half-chain vectors vL, vR:
//   ftilde_b[l] = sum_{a,s} vL_b[a] Phi_s(x_b) G_b[a, s, l],  G_b[a, s, l] = sum_c C[a, s, l, c] vR_b[c],
// with G one float32 contraction over c for the whole batch. Its adjoint,
// for d_b = dLoss/dftilde_b and H_b[a, s, l] = vL_b[a] Phi_s(x_b) d_b[l]:
//   gL_b[a] = sum_{s,l} d_b[l] Phi_s(x_b) G_b[a, s, l],
//   gR_b[c] = sum_{a,s,l} H_b[a, s, l] C[a, s, l, c]   (a contraction over (a, s, l)),
//   dC[a, s, l, c] = sum_b H_b[a, s, l] vR_b[c]         (a contraction over b).
constexpr int LABEL_MAXL = 16;

struct LabelParams {
  int32_t n, batch, ls, L, chi, DL, DR;
  const float* pixels;  // [batch, n]
  const float* vL;      // [batch, chi]
  const double* lamL;
  const double* lamR;
  const float* G;       // [batch, DL, 2, L]
  float* ftilde;        // [batch, L]
  double* log_scale;    // [batch]
  const float* dft;     // adjoint: [batch, L]
  float* gL;            // adjoint: [batch, chi] (zero past DL)
  float* H;             // adjoint: [batch, DL, 2, L]
};

// One warp per sample: ftilde_b[l] = sum_{a,s} vL_b[a] Phi_s G_b[a, s, l].
__global__ void __launch_bounds__(256) cls_label_reduce(const __grid_constant__ LabelParams p) {
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= p.batch) return;
  const float x = __ldg(p.pixels + (int64_t)b * p.n + p.ls);
  const float ph[2] = {cospif(0.5f * x), sinpif(0.5f * x)};
  const float* vL = p.vL + (int64_t)b * p.chi;
  const float* G = p.G + (int64_t)b * p.DL * 2 * p.L;
  float acc[LABEL_MAXL];
#pragma unroll
  for (int l = 0; l < LABEL_MAXL; ++l) acc[l] = 0.0f;
  for (int as = lane; as < p.DL * 2; as += 32) {
    const float w = vL[as >> 1] * ph[as & 1];
#pragma unroll
    for (int l = 0; l < LABEL_MAXL; ++l)
      if (l < p.L) acc[l] = fmaf(w, G[(int64_t)as * p.L + l], acc[l]);
  }
#pragma unroll
  for (int l = 0; l < LABEL_MAXL; ++l)
    for (int o = 16; o > 0; o >>= 1) acc[l] += __shfl_xor_sync(0xffffffffu, acc[l], o);
  if (lane < p.L) {
    float v = acc[0];
#pragma unroll
    for (int l = 1; l < LABEL_MAXL; ++l)
      if (lane == l) v = acc[l];
    p.ftilde[(int64_t)b * p.L + lane] = v;
  }
  if (lane == 0) p.log_scale[b] = p.lamL[b] + p.lamR[b];
}

// One warp per sample: gL_b and H_b.
__global__ void __launch_bounds__(256) cls_label_adjoint(const __grid_constant__ LabelParams p) {
  const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= p.batch) return;
  const float x = __ldg(p.pixels + (int64_t)b * p.n + p.ls);
  const float ph[2] = {cospif(0.5f * x), sinpif(0.5f * x)};
  const float* vL = p.vL + (int64_t)b * p.chi;
  const float* G = p.G + (int64_t)b * p.DL * 2 * p.L;
  float* H = p.H + (int64_t)b * p.DL * 2 * p.L;
  const float* d = p.dft + (int64_t)b * p.L;
  for (int a = lane; a < p.chi; a += 32) {
    float acc = 0.0f;
    if (a < p.DL)
      for (int s = 0; s < 2; ++s)
        for (int l = 0; l < p.L; ++l) {
          const int64_t i = ((int64_t)a * 2 + s) * p.L + l;
          acc = fmaf(d[l] * ph[s], G[i], acc);
          H[i] = vL[a] * ph[s] * d[l];
        }
    p.gL[(int64_t)b * p.chi + a] = acc;
  }
}

// dst[b, c] = src[b, c] for c < D, 0 for D <= c < chi.
__global__ void cls_pad_rows(const float* __restrict__ src, int D, float* __restrict__ dst, int batch, int chi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)batch * chi) return;
  const int64_t b = i / chi;
  const int c = (int)(i % chi);
  dst[i] = c < D ? src[b * D + c] : 0.0f;
}

// Loss head: one CTA of 1024 threads, samples strided over the threads; the
// softmax of the normalised scores (|z| <= 1) in float32, the norm and the
// batch sum in float64, reduced in a fixed order (deterministic).
constexpr int LOSS_THREADS = 1024;
__global__ void __launch_bounds__(LOSS_THREADS)
cls_loss_kernel(const float* __restrict__ ft, const int64_t* __restrict__ y, int batch, int L, double* loss,
                float* dft) {
  __shared__ double red[LOSS_THREADS];
  double acc = 0.0;
  for (int b = threadIdx.x; b < batch; b += LOSS_THREADS) {
    const float* f = ft + (int64_t)b * L;
    double nrm = 0.0;
    for (int l = 0; l < L; ++l) nrm += (double)f[l] * f[l];
    nrm = sqrt(nrm);
    const float inv = nrm > 0.0 ? (float)(1.0 / nrm) : 0.0f;
    float z[LABEL_MAXL], pz[LABEL_MAXL], zmax = -3.0e38f;
    for (int l = 0; l < L; ++l) {
      z[l] = f[l] * inv;
      zmax = fmaxf(zmax, z[l]);
    }
    float se = 0.0f;
    for (int l = 0; l < L; ++l) {
      pz[l] = expf(z[l] - zmax);
      se += pz[l];
    }
    const int64_t yb = y[b];
    acc += (double)(zmax + logf(se) - z[yb]);
    if (dft) {
      float zg = 0.0f;
      const float ise = 1.0f / se;
      for (int l = 0; l < L; ++l) {
        pz[l] = pz[l] * ise - (l == yb ? 1.0f : 0.0f);
        zg += z[l] * pz[l];
      }
      const float sc = inv / (float)batch;
      for (int l = 0; l < L; ++l) dft[(int64_t)b * L + l] = (pz[l] - z[l] * zg) * sc;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = LOSS_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / batch;
}

// First vector of each half-chain: e_0 (bond 1 at the chain's ends), log-scale 0.
__global__ void cls_init_state(float* state, double* lam, int batch, int chi) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)batch * chi) state[i] = (i % chi) == 0 ? 1.0f : 0.0f;
  if (i < batch) lam[i] = 0.0;
}

// ----------------------------------------------------------------- layout
// Workspace of one classifier. The forward leaves the half-chain vectors,
// their log-scales, the per-step scales and the kept vectors here for the
// backward.
struct ClsLayout {
  int n, ls, L, batch, chi, ck, ntiles;
  int T[2];        // steps per half
  int nck[2];      // kept vectors per half
  int seg_len;     // steps per backward segment
  float* state[2];
  double* lam[2];
  float* ckpt[2];
  float* sc[2];
  float* g[2];
  float* replay[2];     // running vector of a segment's recomputation [batch][chi]
  double* replay_lam[2];
  // float32 path
  float* seg;      // recomputed vectors of one segment [seg_len][batch][chi]
  float* X;        // [seg_len][batch][2 chi]
  uint8_t* plan_ws;  // every segment's grouped plan, one region each
  size_t plan_bytes;
  int plan_count;
  // tensor-core path
  uint8_t* fimg[2];  // forward core images per half
  uint8_t* aimg[2];  // adjoint core images per half
  uint8_t* vseg[2];  // bf16 vector tiles of one segment per half
  float* grad[2];    // [t][chi][2 chi] accumulated core gradients per half
  // label core
  float* labG;     // [batch][DL][2][L]
  float* labH;     // [batch][DL][2][L]
  float* gR;       // [batch][DR]
  size_t bytes;
};

int chi_of(const tn_mps* W) {
  int64_t c = 1;
  for (int i = 0; i <= W->n; ++i) c = std::max(c, W->bond[i]);
  if (c <= 32) return 32;
  if (c <= 64) return 64;
  return 128;
}

ClsLayout cls_layout(uint8_t* base, const tn_mps* W, int ls, int L, int batch, int ck) {
  ClsLayout w;
  memset(&w, 0, sizeof(w));
  w.n = W->n;
  w.ls = ls;
  w.L = L;
  w.batch = batch;
  w.chi = chi_of(W);
  w.ck = ck;
  w.ntiles = (batch + CLS_TILE - 1) / CLS_TILE;
  w.T[0] = ls;
  w.T[1] = W->n - 1 - ls;
  const int cke = ck > 0 ? ck : 1;
  for (int h = 0; h < 2; ++h) w.nck[h] = ck > 0 ? (w.T[h] + cke - 1) / cke : 0;
  const int Tmax = std::max(w.T[0], w.T[1]);
  w.seg_len = ck <= 1 ? std::max(Tmax, 1) : ck;
  size_t off = 0;
  auto take = [&](size_t b) { uint8_t* p = base ? base + off : nullptr; off += align256(b); return p; };
  const int chi = w.chi;
  const size_t vec = sizeof(float) * (size_t)batch * chi;
  const bool bwd = ck > 0;
  for (int h = 0; h < 2; ++h) {
    w.state[h] = reinterpret_cast<float*>(take(vec));
    w.lam[h] = reinterpret_cast<double*>(take(sizeof(double) * (size_t)batch));
    w.ckpt[h] = reinterpret_cast<float*>(take(vec * (size_t)w.nck[h]));
    w.sc[h] = reinterpret_cast<float*>(take(sizeof(float) * (size_t)batch * std::max(w.T[h], 1)));
    w.g[h] = reinterpret_cast<float*>(take(bwd ? vec : 0));
    w.replay[h] = reinterpret_cast<float*>(take(bwd ? vec : 0));
    w.replay_lam[h] = reinterpret_cast<double*>(take(bwd ? sizeof(double) * (size_t)batch : 0));
  }
  // float32 backward: recomputed vectors and gradient operands of a segment,
  // and one grouped plan per segment (descriptors, split results to zero and
  // the unit map: each spec at most 2 x 1 output tiles of 128 (2 chi <= 256)
  // times ceil(batch / 2048) k ranges)
  w.seg = reinterpret_cast<float*>(take(bwd && ck > 1 ? vec * (size_t)w.seg_len : 0));
  w.X = reinterpret_cast<float*>(take(bwd ? 2 * vec * (size_t)w.seg_len : 0));
  const size_t units_per_spec = 2 * (size_t)((batch + 64 * MAX_SLABS_PER_UNIT - 1) / (64 * MAX_SLABS_PER_UNIT));
  w.plan_bytes = bwd ? align256(sizeof(ContractDesc) * (size_t)w.seg_len) + align256(sizeof(ZeroRange) * (size_t)w.seg_len) +
                           align256(sizeof(int32_t) * (size_t)w.seg_len * units_per_spec)
                     : 0;
  w.plan_count = bwd ? (w.T[0] + w.seg_len - 1) / w.seg_len + (w.T[1] + w.seg_len - 1) / w.seg_len : 0;
  w.plan_ws = take(w.plan_bytes * (size_t)w.plan_count);
  // tensor-core path (sized for the split BF16x3 images, the larger)
  for (int h = 0; h < 2; ++h) {
    w.fimg[h] = take(cls_fwd_image_bytes(chi, 1) * (size_t)w.T[h]);
    w.aimg[h] = take(bwd ? cls_adj_image_bytes(chi, 1) * (size_t)w.T[h] : 0);
    w.vseg[h] = take(bwd ? cls_vtile_bytes(chi, 1) * (size_t)w.ntiles * (size_t)std::min(w.seg_len, std::max(w.T[h], 1)) : 0);
    w.grad[h] = reinterpret_cast<float*>(take(bwd ? sizeof(float) * (size_t)w.T[h] * chi * 2 * chi : 0));
  }
  const int64_t DL = W->bond[ls], DR = W->bond[ls + 1];
  const size_t lab = sizeof(float) * (size_t)batch * (size_t)(DL * 2 * L);
  w.labG = reinterpret_cast<float*>(take(lab));
  w.labH = reinterpret_cast<float*>(take(bwd ? lab : 0));
  w.gR = reinterpret_cast<float*>(take(bwd ? sizeof(float) * (size_t)batch * DR : 0));
  w.bytes = off;
  return w;
}

int check_classifier(const tn_mps* W, int ls, int L, const float* pixels, int batch) {
  if (!W || !W->bond || !W->cores || !pixels || batch < 0) return TN_ERR_ARG;
  if (W->n < 2 || W->n > CLS_MAXN || ls < 0 || ls >= W->n || L < 1 || L > LABEL_MAXL) return TN_ERR_ARG;
  if (W->d != 2) return TN_ERR_UNSUPPORTED;
  if (W->bond[0] != 1 || W->bond[W->n] != 1) return TN_ERR_SHAPE;
  for (int i = 0; i < W->n; ++i) {
    if (!W->cores[i] || W->bond[i + 1] < 1) return TN_ERR_ARG;
    if (W->bond[i + 1] > CLS_MAXCHI) return TN_ERR_UNSUPPORTED;
  }
  return TN_OK;
}

SweepParams sweep_params(const tn_mps* W, const ClsLayout& w, const float* pixels, int half, int mode) {
  SweepParams p;
  memset(&p, 0, sizeof(p));
  p.n = W->n;
  p.batch = w.batch;
  p.half = half;
  p.mode = mode;
  for (int i = 0; i <= W->n; ++i) p.bond[i] = (int32_t)W->bond[i];
  for (int i = 0; i < W->n; ++i) p.core[i] = W->cores[i];
  p.pixels = pixels;
  p.state = w.state[half];
  p.lam = w.lam[half];
  p.sc = w.sc[half];
  p.store_every = 1;
  return p;
}

// Both halves' cores packed into the tensor-core images of one kind.
int pack_images(const tn_mps* W, const ClsLayout& w, int split, int adjoint, cudaStream_t s) {
  ClsPackParams pp;
  memset(&pp, 0, sizeof(pp));
  pp.n = W->n;
  pp.chi = w.chi;
  pp.split = split;
  pp.adjoint = adjoint;
  pp.T[0] = w.T[0];
  pp.T[1] = w.T[1];
  for (int i = 0; i <= W->n; ++i) pp.bond[i] = (int32_t)W->bond[i];
  for (int i = 0; i < W->n; ++i) pp.core[i] = W->cores[i];
  for (int h = 0; h < 2; ++h) pp.images[h] = adjoint ? w.aimg[h] : w.fimg[h];
  pp.step_bytes = adjoint ? cls_adj_image_bytes(w.chi, split) : cls_fwd_image_bytes(w.chi, split);
  return cls_pack(pp, s);
}

ClsTcParams tc_params(const tn_mps* W, const ClsLayout& w, const float* pixels) {
  ClsTcParams q;
  memset(&q, 0, sizeof(q));
  q.n = W->n;
  q.batch = w.batch;
  q.ntiles = w.ntiles;
  q.store_every = 1;
  q.half_site[0] = 0;
  q.half_dir[0] = 1;
  q.half_site[1] = W->n - 1;
  q.half_dir[1] = -1;
  q.pixels = pixels;
  for (int h = 0; h < 2; ++h) {
    q.sc[h] = w.sc[h];
    q.t_end[h] = w.T[h];
  }
  q.status = status_word();
  return q;
}

tn_tensor strided(float* p, int rank, const int64_t* shape, const int64_t* stride) {
  tn_tensor t;
  memset(&t, 0, sizeof(t));
  t.data = p;
  t.rank = rank;
  t.dtype = TN_F32;
  for (int i = 0; i < rank; ++i) {
    t.shape[i] = shape[i];
    t.stride[i] = stride[i];
  }
  return t;
}

LabelParams label_params(const tn_mps* W, const ClsLayout& w, const float* pixels) {
  LabelParams lp;
  memset(&lp, 0, sizeof(lp));
  lp.n = W->n;
  lp.batch = w.batch;
  lp.ls = w.ls;
  lp.L = w.L;
  lp.chi = w.chi;
  lp.DL = (int)W->bond[w.ls];
  lp.DR = (int)W->bond[w.ls + 1];
  lp.pixels = pixels;
  lp.vL = w.state[0];
  lp.lamL = w.lam[0];
  lp.lamR = w.lam[1];
  lp.G = w.labG;
  return lp;
}

// The label core's contractions: float32 for an FP32 classifier; the split
// BF16X3 tensor-core contraction for BF16 / BF16X3 (relative error ~2^-16 of
// |A||B| per element, below either mode's own sweep error, at a fraction of
// the float32 kernel's time).
int label_prec(int prec) { return prec == TN_PREC_FP32 ? TN_PREC_FP32 : TN_PREC_BF16X3; }

// G[b, a, s, l] = sum_c vR[b, c] C[a, s, l, c].
int label_G(const tn_mps* W, const ClsLayout& w, int prec, cudaStream_t s) {
  const int64_t DL = W->bond[w.ls], DR = W->bond[w.ls + 1], B = w.batch, L = w.L;
  const int64_t shv[2] = {B, DR}, stv[2] = {w.chi, 1};
  const int64_t shc[4] = {DL, 2, L, DR}, stc[4] = {0, 0, 0, 0};
  const int64_t shg[4] = {B, DL, 2, L}, stg[4] = {0, 0, 0, 0};
  tn_tensor tv = strided(w.state[1], 2, shv, stv);
  tn_tensor tc = strided(const_cast<float*>(W->cores[w.ls]), 4, shc, stc);
  tn_tensor tg = strided(w.labG, 4, shg, stg);
  const int lv[1] = {1}, lc[1] = {3};
  return contract_internal(&tv, lv, &tc, lc, 1, &tg, label_prec(prec), s);
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

int tn_mps_classify_loss(const float* ftilde, const int64_t* labels, int batch, int n_labels, double* loss,
                         float* dftilde, void* stream) {
  if (!ftilde || !labels || !loss || batch < 1 || n_labels < 1 || n_labels > LABEL_MAXL) return TN_ERR_ARG;
  cls_loss_kernel<<<1, LOSS_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(ftilde, labels, batch, n_labels, loss,
                                                                             dftilde);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

size_t tn_mps_classify_workspace_bytes(const tn_mps* W, int label_site, int n_labels, int batch, int ckpt_every) {
  if (!W || !W->bond || W->n < 2 || label_site < 0 || label_site >= W->n || batch < 0 || ckpt_every < 0) return 0;
  return cls_layout(nullptr, W, label_site, n_labels, batch, ckpt_every).bytes;
}

int tn_mps_classify(const tn_mps* W, int label_site, int n_labels, const float* pixels, int batch, int prec,
                    int ckpt_every, float* ftilde, double* log_scale, void* workspace, size_t ws_bytes,
                    void* stream) {
  int rc = check_classifier(W, label_site, n_labels, pixels, batch);
  if (rc != TN_OK) return rc;
  if (!ftilde || !log_scale || ckpt_every < 0) return TN_ERR_ARG;
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  if (batch == 0) return TN_OK;
  ClsLayout w = cls_layout(static_cast<uint8_t*>(workspace), W, label_site, n_labels, batch, ckpt_every);
  if (!workspace || ws_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nvec = (int64_t)batch * w.chi;
  for (int h = 0; h < 2; ++h) {
    cls_init_state<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(w.state[h], w.lam[h], batch, w.chi);
    if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
  }
  if (prec == TN_PREC_FP32) {
    for (int h = 0; h < 2; ++h) {
      SweepParams p = sweep_params(W, w, pixels, h, 0);
      p.t_begin = 0;
      p.t_end = w.T[h];
      if (ckpt_every > 0) {
        p.store = w.ckpt[h];
        p.store_every = ckpt_every;
        p.store_base = 0;
      }
      if ((rc = launch_sweep(w.chi, p, s)) != TN_OK) return rc;
    }
  } else {
    // both half-chains in one tcgen05 launch
    const int split = prec == TN_PREC_BF16X3;
    if ((rc = pack_images(W, w, split, 0, s)) != TN_OK) return rc;
    ClsTcParams q = tc_params(W, w, pixels);
    for (int h = 0; h < 2; ++h) {
      q.state[h] = w.state[h];
      q.lam[h] = w.lam[h];
      q.images[h] = w.fimg[h];
      if (ckpt_every > 0) q.store[h] = w.ckpt[h];
    }
    q.store_every = ckpt_every > 0 ? ckpt_every : 1;
    if ((rc = cls_fwd_tc_launch(w.chi, split, q, s)) != TN_OK) return rc;
  }
  if ((rc = label_G(W, w, prec, s)) != TN_OK) return rc;
  LabelParams lp = label_params(W, w, pixels);
  lp.ftilde = ftilde;
  lp.log_scale = log_scale;
  cls_label_reduce<<<(unsigned)((batch + 7) / 8), 256, 0, s>>>(lp);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int tn_mps_classify_backward(const tn_mps* W, int label_site, int n_labels, const float* pixels, int batch,
                             int prec, int ckpt_every, const float* dftilde, float* const* dcores,
                             void* workspace, size_t ws_bytes, void* stream) {
  int rc = check_classifier(W, label_site, n_labels, pixels, batch);
  if (rc != TN_OK) return rc;
  if (!dftilde || !dcores || ckpt_every < 1) return TN_ERR_ARG;
  for (int i = 0; i < W->n; ++i)
    if (!dcores[i]) return TN_ERR_ARG;
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16 && prec != TN_PREC_BF16X3) return TN_ERR_ARG;
  ClsLayout w = cls_layout(static_cast<uint8_t*>(workspace), W, label_site, n_labels, batch, ckpt_every);
  if (!workspace || ws_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int chi = w.chi, n = W->n, ls = label_site, L = n_labels;
  const int split = prec == TN_PREC_BF16X3;
  if (prec != TN_PREC_FP32 && !cls_adj_tc_supported(chi, split)) return TN_ERR_UNSUPPORTED;
  if (batch == 0) {
    for (int i = 0; i < n; ++i) {
      const int64_t e = W->bond[i] * 2 * W->bond[i + 1] * (i == ls ? L : 1);
      if (cudaMemsetAsync(dcores[i], 0, sizeof(float) * (size_t)e, s) != cudaSuccess) return TN_ERR_CUDA;
    }
    return TN_OK;
  }

  // label core: the adjoints entering both half-chains, and dC
  {
    if ((rc = label_G(W, w, prec, s)) != TN_OK) return rc;
    LabelParams lp = label_params(W, w, pixels);
    lp.dft = dftilde;
    lp.gL = w.g[0];
    lp.H = w.labH;
    cls_label_adjoint<<<(unsigned)((batch + 7) / 8), 256, 0, s>>>(lp);
    if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
    const int64_t B = batch, DL = lp.DL, DR = lp.DR;
    const int64_t shh[4] = {B, DL, 2, L}, sth[4] = {0, 0, 0, 0};
    const int64_t shc[4] = {DL, 2, L, DR}, stc[4] = {0, 0, 0, 0};
    const int64_t shr[2] = {B, DR}, str[2] = {0, 0};
    const int64_t shv[2] = {B, DR}, stv[2] = {chi, 1};
    tn_tensor th = strided(w.labH, 4, shh, sth);
    tn_tensor tc = strided(const_cast<float*>(W->cores[ls]), 4, shc, stc);
    tn_tensor tr = strided(w.gR, 2, shr, str);
    const int lh[3] = {1, 2, 3}, lc[3] = {0, 1, 2};
    if ((rc = contract_internal(&th, lh, &tc, lc, 3, &tr, label_prec(prec), s)) != TN_OK) return rc;
    const int64_t nvec = B * chi;
    cls_pad_rows<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(w.gR, (int)DR, w.g[1], batch, chi);
    if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
    tn_tensor tv = strided(w.state[1], 2, shv, stv);
    tn_tensor td = strided(dcores[ls], 4, shc, stc);
    const int l0[1] = {0};
    if ((rc = contract_internal(&th, l0, &tv, l0, 1, &td, label_prec(prec), s)) != TN_OK) return rc;
  }

  const int seg = ckpt_every <= 1 ? std::max(std::max(w.T[0], w.T[1]), 1) : ckpt_every;
  int nseg[2];
  for (int h = 0; h < 2; ++h) nseg[h] = (w.T[h] + seg - 1) / seg;
  const int rounds = std::max(nseg[0], nseg[1]);
  // segment of half h handled in round k (segments run from the label core outwards)
  auto seg_range = [&](int h, int k, int* t0, int* t1) {
    const int sg = nseg[h] - 1 - k;
    if (sg < 0) {
      *t0 = *t1 = 0;
      return false;
    }
    *t0 = sg * seg;
    *t1 = std::min(w.T[h], *t0 + seg);
    return true;
  };
  const size_t vbytes = sizeof(float) * (size_t)batch * chi;

  if (prec != TN_PREC_FP32) {
    // tcgen05: per round, one launch recomputes both halves' segments (their
    // bf16 vector tiles kept for the gradient products) and one launch runs
    // both adjoint segments, accumulating every step's core gradient
    if ((rc = pack_images(W, w, split, 0, s)) != TN_OK) return rc;
    if ((rc = pack_images(W, w, split, 1, s)) != TN_OK) return rc;
    for (int h = 0; h < 2; ++h)
      if (w.T[h] > 0 &&
          cudaMemsetAsync(w.grad[h], 0, sizeof(float) * (size_t)w.T[h] * chi * 2 * chi, s) != cudaSuccess)
        return TN_ERR_CUDA;
    for (int k = 0; k < rounds; ++k) {
      ClsTcParams f = tc_params(W, w, pixels);
      ClsTcParams a = tc_params(W, w, pixels);
      for (int h = 0; h < 2; ++h) {
        int t0, t1;
        seg_range(h, k, &t0, &t1);
        f.t_begin[h] = a.t_begin[h] = t0;
        f.t_end[h] = a.t_end[h] = t1;
        if (t1 > t0 && cudaMemcpyAsync(w.replay[h], w.ckpt[h] + (int64_t)(t0 / ckpt_every) * batch * chi, vbytes,
                                       cudaMemcpyDeviceToDevice, s) != cudaSuccess)
          return TN_ERR_CUDA;
        f.state[h] = w.replay[h];
        f.lam[h] = w.replay_lam[h];
        f.vseg[h] = w.vseg[h];
        f.images[h] = w.fimg[h];
        a.state[h] = w.g[h];
        a.vseg[h] = w.vseg[h];
        a.images[h] = w.aimg[h];
        a.grad[h] = w.grad[h];
      }
      if ((rc = cls_fwd_tc_launch(chi, split, f, s)) != TN_OK) return rc;
      if ((rc = cls_adj_tc_launch(chi, split, a, s)) != TN_OK) return rc;
    }
    ClsScatterParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.n = n;
    sp.chi = chi;
    sp.T[0] = w.T[0];
    sp.T[1] = w.T[1];
    for (int i = 0; i <= n; ++i) sp.bond[i] = (int32_t)W->bond[i];
    for (int i = 0; i < n; ++i) sp.dcore[i] = dcores[i];
    sp.grad[0] = w.grad[0];
    sp.grad[1] = w.grad[1];
    return cls_scatter_grad(sp, s);
  }

  // float32: per half and segment (from the label core outwards) the
  // recomputed vectors, the adjoint sweep writing the gradient operands, and
  // one grouped tensordot over the batch for the segment's cores. The
  // segments' plans are built and uploaded before the first sweep.
  struct SegPlan {
    int h, t0, t1;
    const float* vecs;
    tn_group_plan* plan;
    uint8_t* ws;
  };
  std::vector<SegPlan> plans;
  auto destroy_all = [&]() {
    for (auto& sp : plans)
      if (sp.plan) tn_group_plan_destroy(sp.plan);
  };
  for (int h = 0; h < 2; ++h)
    for (int k = 0; k < nseg[h]; ++k) {
      int t0, t1;
      seg_range(h, k, &t0, &t1);
      const float* vecs = ckpt_every <= 1 ? w.ckpt[h] + (int64_t)t0 * batch * chi : w.seg;
      std::vector<tn_contract_spec> specs((size_t)(t1 - t0));
      for (int t = t0; t < t1; ++t) {
        const int site = h == 0 ? t : n - 1 - t;
        const int64_t Da = W->bond[site], Dc = W->bond[site + 1];
        tn_contract_spec& sp = specs[(size_t)(t - t0)];
        memset(&sp, 0, sizeof(sp));
        float* v = const_cast<float*>(vecs) + (int64_t)(t - t0) * batch * chi;
        float* x = w.X + (int64_t)(t - t0) * batch * 2 * chi;
        const int64_t shd[3] = {Da, 2, Dc}, std0[3] = {0, 0, 0};
        sp.C = strided(dcores[site], 3, shd, std0);
        sp.nshared = 1;
        if (h == 0) {
          // dW[a, s, c] = sum_b v_b[a] X_b[s, c]
          const int64_t shv[2] = {batch, Da}, stv[2] = {chi, 1};
          const int64_t shx[3] = {batch, 2, Dc}, stx[3] = {2 * chi, chi, 1};
          sp.A = strided(v, 2, shv, stv);
          sp.B = strided(x, 3, shx, stx);
        } else {
          // dW[a, s, c] = sum_b X_b[a, s] v_b[c]
          const int64_t shx[3] = {batch, Da, 2}, stx[3] = {2 * chi, 2, 1};
          const int64_t shv[2] = {batch, Dc}, stv[2] = {chi, 1};
          sp.A = strided(x, 3, shx, stx);
          sp.B = strided(v, 2, shv, stv);
        }
      }
      SegPlan sp{h, t0, t1, vecs, nullptr, w.plan_ws + (size_t)plans.size() * w.plan_bytes};
      if ((rc = group_plan_create_ex(specs.data(), (int)specs.size(), TN_PREC_FP32, false, &sp.plan)) != TN_OK) {
        destroy_all();
        return rc;
      }
      plans.push_back(sp);
      if ((rc = tn_group_plan_upload(sp.plan, sp.ws, w.plan_bytes, s)) != TN_OK) {
        destroy_all();
        return rc;
      }
    }
  for (const SegPlan& sp : plans) {
    const int h = sp.h, t0 = sp.t0, t1 = sp.t1;
    if (ckpt_every > 1) {
      // recompute the segment from its kept vector, keeping the vector
      // entering every step; the replay rewrites the same per-step scales
      if (cudaMemcpyAsync(w.replay[h], w.ckpt[h] + (int64_t)(t0 / ckpt_every) * batch * chi, vbytes,
                          cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        destroy_all();
        return TN_ERR_CUDA;
      }
      SweepParams p = sweep_params(W, w, pixels, h, 0);
      p.state = w.replay[h];
      p.lam = w.replay_lam[h];
      p.t_begin = t0;
      p.t_end = t1;
      p.store = w.seg;
      p.store_every = 1;
      p.store_base = t0;
      if ((rc = launch_sweep(chi, p, s)) != TN_OK) break;
    }
    // adjoint steps t1-1 .. t0: g <- adjoint step, X[t - t0] <- gradient operands
    SweepParams p = sweep_params(W, w, pixels, h, 1);
    p.state = w.g[h];
    p.t_begin = t0;
    p.t_end = t1;
    p.xout = w.X;
    if ((rc = launch_sweep(chi, p, s)) != TN_OK) break;
    if ((rc = tn_group_plan_run(sp.plan, sp.ws, w.plan_bytes, s)) != TN_OK) break;
  }
  destroy_all();
  return rc;
}

}  // extern "C"
