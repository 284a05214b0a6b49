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
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(cls_sweep_simt<CHI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return TN_ERR_CUDA;
    attr = true;
  }
  cls_sweep_simt<CHI><<<(p.batch + BT - 1) / BT, 2 * CHI, smem, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int launch_sweep(int chi, const SweepParams& p, cudaStream_t s);

// The tensor-core images of one mode for both half-chains.
int pack_images(const tn_mps* W, const struct ClsLayout& w, int mode, cudaStream_t s);

// A sweep on the float32 kernel (prec FP32) or the tcgen05 kernel (else).
int run_sweep(int prec, const struct ClsLayout& w, const SweepParams& p, cudaStream_t s);

int launch_sweep(int chi, const SweepParams& p, cudaStream_t s) {
  if (p.t_end <= p.t_begin) return TN_OK;
  if (chi == 32) return launch_sweep_chi<32>(p, s);
  if (chi == 64) return launch_sweep_chi<64>(p, s);
  return launch_sweep_chi<128>(p, s);
}

// ------------------------------------------------------------- label core
struct LabelParams {
  int32_t n, batch, ls, L, chi, DL, DR;
  const float* C;       // (DL, 2, L, DR)
  const float* pixels;  // [batch, n]
  const float* vL;      // [batch, chi]
  const float* vR;
  const double* lamL;
  const double* lamR;
  float* ftilde;        // [batch, L]
  double* log_scale;    // [batch]
  const float* dft;     // adjoint: [batch, L]
  float* gL;            // adjoint: [batch, chi]
  float* gR;
  float* Y;             // adjoint: [batch, 2, L, DR]
};

constexpr int LABEL_MAXL = 16;

__global__ void __launch_bounds__(128) cls_label_fwd(const __grid_constant__ LabelParams p) {
  const int b = blockIdx.x, tid = threadIdx.x;
  __shared__ float red[LABEL_MAXL][128 / 32];
  const float x = p.pixels[(int64_t)b * p.n + p.ls];
  const float ph[2] = {cospif(0.5f * x), sinpif(0.5f * x)};
  const float* vL = p.vL + (int64_t)b * p.chi;
  const float* vR = p.vR + (int64_t)b * p.chi;
  float acc[LABEL_MAXL];
  for (int l = 0; l < LABEL_MAXL; ++l) acc[l] = 0.0f;
  for (int as = tid; as < p.DL * 2; as += blockDim.x) {
    const int a = as >> 1, s = as & 1;
    const float w = vL[a] * ph[s];
    for (int l = 0; l < p.L; ++l) {
      const float* Cr = p.C + ((int64_t)as * p.L + l) * p.DR;
      float t = 0.0f;
      for (int c = 0; c < p.DR; ++c) t = fmaf(Cr[c], vR[c], t);
      acc[l] = fmaf(w, t, acc[l]);
    }
  }
  for (int l = 0; l < p.L; ++l) {
    float v = acc[l];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[l][tid >> 5] = v;
  }
  __syncthreads();
  if (tid < p.L) {
    float v = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[tid][w];
    p.ftilde[(int64_t)b * p.L + tid] = v;
  }
  if (tid == 0) p.log_scale[b] = p.lamL[b] + p.lamR[b];
}

// Adjoint of the label core for one sample: gL[a] = sum_{s,l,c} d_l Phi_s C[a,s,l,c] vR[c],
// gR[c] = sum_{a,s,l} d_l vL[a] Phi_s C[a,s,l,c], Y[s,l,c] = d_l Phi_s vR[c].
__global__ void __launch_bounds__(128) cls_label_bwd(const __grid_constant__ LabelParams p) {
  const int b = blockIdx.x, tid = threadIdx.x;
  const float x = p.pixels[(int64_t)b * p.n + p.ls];
  const float ph[2] = {cospif(0.5f * x), sinpif(0.5f * x)};
  const float* vL = p.vL + (int64_t)b * p.chi;
  const float* vR = p.vR + (int64_t)b * p.chi;
  const float* d = p.dft + (int64_t)b * p.L;
  for (int a = tid; a < p.chi; a += blockDim.x) {
    float acc = 0.0f;
    if (a < p.DL)
      for (int s = 0; s < 2; ++s)
        for (int l = 0; l < p.L; ++l) {
          const float* Cr = p.C + (((int64_t)a * 2 + s) * p.L + l) * p.DR;
          float t = 0.0f;
          for (int c = 0; c < p.DR; ++c) t = fmaf(Cr[c], vR[c], t);
          acc = fmaf(d[l] * ph[s], t, acc);
        }
    p.gL[(int64_t)b * p.chi + a] = acc;
  }
  for (int c = tid; c < p.chi; c += blockDim.x) {
    float acc = 0.0f;
    if (c < p.DR)
      for (int a = 0; a < p.DL; ++a)
        for (int s = 0; s < 2; ++s) {
          const float w = vL[a] * ph[s];
          for (int l = 0; l < p.L; ++l) acc = fmaf(w * d[l], p.C[(((int64_t)a * 2 + s) * p.L + l) * p.DR + c], acc);
        }
    p.gR[(int64_t)b * p.chi + c] = acc;
  }
  for (int i = tid; i < 2 * p.L * p.DR; i += blockDim.x) {
    const int c = i % p.DR, l = (i / p.DR) % p.L, s = i / (p.DR * p.L);
    p.Y[(int64_t)b * 2 * p.L * p.DR + i] = d[l] * ph[s] * vR[c];
  }
}

// Loss head: one CTA, samples strided over its threads, float64 partial sums
// reduced in a fixed order.
__global__ void __launch_bounds__(256)
cls_loss_kernel(const float* __restrict__ ft, const int64_t* __restrict__ y, int batch, int L, double* loss,
                float* dft) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int b = threadIdx.x; b < batch; b += blockDim.x) {
    const float* f = ft + (int64_t)b * L;
    double nrm = 0.0;
    for (int l = 0; l < L; ++l) nrm += (double)f[l] * f[l];
    nrm = sqrt(nrm);
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    double z[LABEL_MAXL], pz[LABEL_MAXL], zmax = -1e300;
    for (int l = 0; l < L; ++l) {
      z[l] = f[l] * inv;
      zmax = fmax(zmax, z[l]);
    }
    double se = 0.0;
    for (int l = 0; l < L; ++l) {
      pz[l] = exp(z[l] - zmax);
      se += pz[l];
    }
    const int64_t yb = y[b];
    acc += zmax + log(se) - z[yb];
    if (dft) {
      double zg = 0.0;
      for (int l = 0; l < L; ++l) {
        pz[l] = pz[l] / se - (l == yb ? 1.0 : 0.0);
        zg += z[l] * pz[l];
      }
      for (int l = 0; l < L; ++l) dft[(int64_t)b * L + l] = (float)((pz[l] - z[l] * zg) * inv / batch);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
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
struct ClsLayout {
  int n, ls, L, batch, chi, ck;
  int T[2];        // steps per half
  int nck[2];      // kept vectors per half
  int seg_len;     // steps per backward segment
  float* state[2];
  double* lam[2];
  float* ckpt[2];
  float* sc[2];
  float* g[2];
  float* seg;      // recomputed vectors of one segment [seg_len][batch][chi]
  float* replay;   // running vector of the segment replay [batch][chi]
  float* X;        // [seg_len][batch][2 chi]
  float* Y;        // [batch][2][L][chi]
  uint8_t* plan_ws;
  uint8_t* img[2][2];  // bf16 core images per half and mode (tensor-core sweeps)
  size_t img_bytes;
  size_t plan_bytes;
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
  w.n = W->n;
  w.ls = ls;
  w.L = L;
  w.batch = batch;
  w.chi = chi_of(W);
  w.ck = ck;
  w.T[0] = ls;
  w.T[1] = W->n - 1 - ls;
  const int cke = ck > 0 ? ck : 1;
  for (int h = 0; h < 2; ++h) w.nck[h] = ck > 0 ? (w.T[h] + cke - 1) / cke : 0;
  const int Tmax = std::max(w.T[0], w.T[1]);
  w.seg_len = ck <= 1 ? std::max(Tmax, 1) : ck;
  size_t off = 0;
  auto take = [&](size_t b) { uint8_t* p = base ? base + off : nullptr; off += align256(b); return p; };
  const size_t vec = sizeof(float) * (size_t)batch * w.chi;
  for (int h = 0; h < 2; ++h) {
    w.state[h] = reinterpret_cast<float*>(take(vec));
    w.lam[h] = reinterpret_cast<double*>(take(sizeof(double) * (size_t)batch));
    w.ckpt[h] = reinterpret_cast<float*>(take(vec * (size_t)w.nck[h]));
    w.sc[h] = reinterpret_cast<float*>(take(sizeof(float) * (size_t)batch * std::max(w.T[h], 1)));
    w.g[h] = reinterpret_cast<float*>(take(vec));
  }
  const bool bwd = ck > 0;
  w.seg = reinterpret_cast<float*>(take(bwd && ck > 1 ? vec * (size_t)w.seg_len : 0));
  w.replay = reinterpret_cast<float*>(take(bwd && ck > 1 ? vec : 0));
  w.X = reinterpret_cast<float*>(take(bwd ? 2 * vec * (size_t)w.seg_len : 0));
  w.Y = reinterpret_cast<float*>(take(bwd ? sizeof(float) * (size_t)batch * 2 * L * w.chi : 0));
  // a segment's grouped plan: descriptors, split results to zero, and the
  // unit map (each spec: at most 2 x 1 output tiles of 128 (2 chi <= 256)
  // times ceil(batch / 2048) k ranges)
  const size_t units_per_spec = 2 * (size_t)((batch + 64 * MAX_SLABS_PER_UNIT - 1) / (64 * MAX_SLABS_PER_UNIT));
  w.plan_bytes = bwd ? align256(sizeof(ContractDesc) * (size_t)w.seg_len) + align256(sizeof(ZeroRange) * (size_t)w.seg_len) +
                           sizeof(int32_t) * (size_t)w.seg_len * units_per_spec
                     : 0;
  w.plan_ws = take(w.plan_bytes);
  w.img_bytes = cls_image_bytes(w.chi);
  for (int h = 0; h < 2; ++h)
    for (int m = 0; m < 2; ++m) w.img[h][m] = take(w.img_bytes * (size_t)w.T[h]);
  w.bytes = off;
  return w;
}

int pack_images(const tn_mps* W, const ClsLayout& w, int mode, cudaStream_t s) {
  for (int h = 0; h < 2; ++h) {
    ClsPackParams pp;
    memset(&pp, 0, sizeof(pp));
    pp.n = W->n;
    pp.half = h;
    pp.mode = mode;
    pp.chi = w.chi;
    pp.kpad = w.chi < 64 ? 64 : w.chi;
    pp.img_bytes = w.img_bytes;
    for (int i = 0; i <= W->n; ++i) pp.bond[i] = (int32_t)W->bond[i];
    for (int i = 0; i < W->n; ++i) pp.core[i] = W->cores[i];
    pp.images = w.img[h][mode];
    int rc = cls_pack(pp, w.T[h], s);
    if (rc != TN_OK) return rc;
  }
  return TN_OK;
}

int run_sweep(int prec, const ClsLayout& w, const SweepParams& p, cudaStream_t s) {
  if (prec == TN_PREC_FP32) return launch_sweep(w.chi, p, s);
  ClsTcParams q;
  memset(&q, 0, sizeof(q));
  q.n = p.n;
  q.batch = p.batch;
  q.half = p.half;
  q.mode = p.mode;
  q.t_begin = p.t_begin;
  q.t_end = p.t_end;
  q.store_every = p.store_every;
  q.store_base = p.store_base;
  q.pixels = p.pixels;
  q.state = p.state;
  q.lam = p.lam;
  q.store = p.store;
  q.sc = p.sc;
  q.xout = p.xout;
  q.images = w.img[p.half][p.mode];
  q.status = status_word();
  return cls_sweep_tc_launch(w.chi, q, s);
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

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

int tn_mps_classify_loss(const float* ftilde, const int64_t* labels, int batch, int n_labels, double* loss,
                         float* dftilde, void* stream) {
  if (!ftilde || !labels || !loss || batch < 1 || n_labels < 1 || n_labels > LABEL_MAXL) return TN_ERR_ARG;
  cls_loss_kernel<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(ftilde, labels, batch, n_labels, loss, dftilde);
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
  if (prec != TN_PREC_FP32 && prec != TN_PREC_BF16) return TN_ERR_UNSUPPORTED;
  if (batch == 0) return TN_OK;
  ClsLayout w = cls_layout(static_cast<uint8_t*>(workspace), W, label_site, n_labels, batch, ckpt_every);
  if (!workspace || ws_bytes < w.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nvec = (int64_t)batch * w.chi;
  if (prec != TN_PREC_FP32 && (rc = pack_images(W, w, 0, s)) != TN_OK) return rc;
  for (int h = 0; h < 2; ++h) {
    cls_init_state<<<(unsigned)((nvec + 255) / 256), 256, 0, s>>>(w.state[h], w.lam[h], batch, w.chi);
    SweepParams p = sweep_params(W, w, pixels, h, 0);
    p.t_begin = 0;
    p.t_end = w.T[h];
    if (ckpt_every > 0) {
      p.store = w.ckpt[h];
      p.store_every = ckpt_every;
      p.store_base = 0;
    }
    if ((rc = run_sweep(prec, w, p, s)) != TN_OK) return rc;
  }
  LabelParams lp;
  memset(&lp, 0, sizeof(lp));
  lp.n = W->n;
  lp.batch = batch;
  lp.ls = label_site;
  lp.L = n_labels;
  lp.chi = w.chi;
  lp.DL = (int)W->bond[label_site];
  lp.DR = (int)W->bond[label_site + 1];
  lp.C = W->cores[label_site];
  lp.pixels = pixels;
  lp.vL = w.state[0];
  lp.vR = w.state[1];
  lp.lamL = w.lam[0];
  lp.lamR = w.lam[1];
  lp.ftilde = ftilde;
  lp.log_scale = log_scale;
  cls_label_fwd<<<batch, 128, 0, s>>>(lp);
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
  if (batch == 0) {
    for (int i = 0; i < n; ++i) {
      const int64_t e = W->bond[i] * 2 * W->bond[i + 1] * (i == ls ? L : 1);
      if (cudaMemsetAsync(dcores[i], 0, sizeof(float) * (size_t)e, s) != cudaSuccess) return TN_ERR_CUDA;
    }
    return TN_OK;
  }
  const int dprec = prec == TN_PREC_FP32 ? TN_PREC_FP32 : prec;
  // reduced precisions run the sweeps on the tensor cores (bf16 operands)
  const int sprec = prec == TN_PREC_FP32 ? TN_PREC_FP32 : TN_PREC_BF16;
  if (sprec != TN_PREC_FP32) {
    if ((rc = pack_images(W, w, 0, s)) != TN_OK) return rc;
    if ((rc = pack_images(W, w, 1, s)) != TN_OK) return rc;
  }

  // label core: adjoints entering both half-chains, and dC = sum_b vL_b (x) Y_b
  LabelParams lp;
  memset(&lp, 0, sizeof(lp));
  lp.n = n;
  lp.batch = batch;
  lp.ls = ls;
  lp.L = L;
  lp.chi = chi;
  lp.DL = (int)W->bond[ls];
  lp.DR = (int)W->bond[ls + 1];
  lp.C = W->cores[ls];
  lp.pixels = pixels;
  lp.vL = w.state[0];
  lp.vR = w.state[1];
  lp.dft = dftilde;
  lp.gL = w.g[0];
  lp.gR = w.g[1];
  lp.Y = w.Y;
  cls_label_bwd<<<batch, 128, 0, s>>>(lp);
  if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
  {
    const int64_t shv[2] = {batch, lp.DL}, stv[2] = {chi, 1};
    const int64_t shy[4] = {batch, 2, L, lp.DR}, sty[4] = {2 * L * lp.DR, L * lp.DR, lp.DR, 1};
    const int64_t shc[4] = {lp.DL, 2, L, lp.DR}, stc[4] = {0, 0, 0, 0};
    tn_tensor tv = strided(w.state[0], 2, shv, stv);
    tn_tensor ty = strided(w.Y, 4, shy, sty);
    tn_tensor tc = strided(dcores[ls], 4, shc, stc);
    const int l0[1] = {0};
    if ((rc = contract_internal(&tv, l0, &ty, l0, 1, &tc, dprec, s)) != TN_OK) return rc;
  }

  // each half-chain: segments from the label core outwards
  for (int h = 0; h < 2; ++h) {
    const int T = w.T[h];
    if (T == 0) continue;
    const int seg = ckpt_every <= 1 ? T : ckpt_every;
    const int nseg = (T + seg - 1) / seg;
    for (int sg = nseg - 1; sg >= 0; --sg) {
      const int t0 = sg * seg, t1 = std::min(T, t0 + seg);
      const float* vecs;  // vectors entering steps t0..t1-1, [t - t0][batch][chi]
      if (ckpt_every <= 1) {
        vecs = w.ckpt[h] + (int64_t)t0 * batch * chi;
      } else {
        // recompute the segment from its kept vector, keeping the vector
        // entering every step; the replay rewrites the same per-step scales
        // (and the internal log-scale, which the backward does not read)
        if (cudaMemcpyAsync(w.replay, w.ckpt[h] + (int64_t)sg * batch * chi, sizeof(float) * (size_t)batch * chi,
                            cudaMemcpyDeviceToDevice, s) != cudaSuccess)
          return TN_ERR_CUDA;
        SweepParams p = sweep_params(W, w, pixels, h, 0);
        p.state = w.replay;
        p.t_begin = t0;
        p.t_end = t1;
        p.store = w.seg;
        p.store_every = 1;
        p.store_base = t0;
        if ((rc = run_sweep(sprec, w, p, s)) != TN_OK) return rc;
        vecs = w.seg;
      }
      // adjoint steps t1-1 .. t0: g <- adjoint step, X[t - t0] <- gradient operands
      SweepParams p = sweep_params(W, w, pixels, h, 1);
      p.state = w.g[h];
      p.t_begin = t0;
      p.t_end = t1;
      p.xout = w.X;
      if ((rc = run_sweep(sprec, w, p, s)) != TN_OK) return rc;
      // core gradients of the segment: one grouped tensordot over the batch
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
      tn_group_plan* plan = nullptr;
      if ((rc = group_plan_create_ex(specs.data(), (int)specs.size(), dprec, false, &plan)) != TN_OK) return rc;
      rc = tn_group_plan_upload(plan, w.plan_ws, w.plan_bytes, s);
      if (rc == TN_OK) rc = tn_group_plan_run(plan, w.plan_ws, w.plan_bytes, s);
      tn_group_plan_destroy(plan);
      if (rc != TN_OK) return rc;
    }
  }
  return TN_OK;
}

}  // extern "C"
