// The L-separate-MPS classifier (Sec. IV.A: one MPS per label; the score of
// label l is the overlap of the image's product state with MPS l). Each MPS is
// swept by the single-MPS classifier with one label (its middle core read as a
// (D, 2, 1, D') label core), each into its own slice of the workspace so the
// backward finds every MPS's checkpoints; a combine kernel then brings the L
// scores to one per-sample log-scale: f_l = ftilde_l e^(Lambda_l) =
// ftilde[b, l] e^(Lambda'), Lambda' = max_l Lambda_l, so the loss head of the
// label-core classifier applies unchanged. The backward scales dLoss/dftilde
// back to each MPS's own log-scale and runs that MPS's adjoint sweep.
#include <math.h>

#include <mutex>
#include <vector>

#include "tn_internal.h"

namespace tn {
namespace {

constexpr int SEP_MAX = 64;  // MPS per call

// ftilde[b, l] = ft_each[l][b] e^(lam_each[l][b] - max_l lam_each[l][b])
__global__ void cls_sep_combine(const float* __restrict__ ft_each, const double* __restrict__ lam_each, int batch,
                                int nl, float* __restrict__ ftilde, double* __restrict__ log_scale) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double m = lam_each[b];
  for (int l = 1; l < nl; ++l) m = fmax(m, lam_each[(int64_t)l * batch + b]);
  for (int l = 0; l < nl; ++l)
    ftilde[(int64_t)b * nl + l] =
        (float)((double)ft_each[(int64_t)l * batch + b] * exp(lam_each[(int64_t)l * batch + b] - m));
  log_scale[b] = m;
}

// d[b] = dftilde[b, l] e^(lam_each[l][b] - max_l' lam_each[l'][b]): the
// gradient with respect to MPS l's own ftilde
__global__ void cls_sep_scale(const float* __restrict__ dftilde, const double* __restrict__ lam_each, int batch,
                              int nl, int l, float* __restrict__ d) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double m = lam_each[b];
  for (int k = 1; k < nl; ++k) m = fmax(m, lam_each[(int64_t)k * batch + b]);
  d[b] = (float)((double)dftilde[(int64_t)b * nl + l] * exp(lam_each[(int64_t)l * batch + b] - m));
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

// The MPS are independent: their sweeps run on SEP_STREAMS library-owned
// streams of the current device (created once, non-blocking), forked from
// and joined back into the caller's stream by events, so that several
// sweeps (each a few dozen CTAs at batch 4096) share the GPU.
constexpr int SEP_STREAMS = 8;
std::mutex g_sep_lock;
int g_sep_device = -1;
cudaStream_t g_sep_streams[SEP_STREAMS];

// Streams for the current device, or null (then everything runs on the
// caller's stream) if they cannot be made or belong to another device.
cudaStream_t* sep_streams() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> g(g_sep_lock);
  if (g_sep_device == -1) {
    for (int i = 0; i < SEP_STREAMS; ++i)
      if (cudaStreamCreateWithFlags(&g_sep_streams[i], cudaStreamNonBlocking) != cudaSuccess) {
        for (int j = 0; j < i; ++j) cudaStreamDestroy(g_sep_streams[j]);
        g_sep_device = -2;
        return nullptr;
      }
    g_sep_device = dev;
  }
  return g_sep_device == dev ? g_sep_streams : nullptr;
}

// Runs body(l, stream) for every MPS: on the side streams when there are
// several MPS, with the caller's stream waiting for all of them at the end.
template <class F>
int run_forked(int nl, cudaStream_t caller, F body) {
  cudaStream_t* side = nl > 1 ? sep_streams() : nullptr;
  if (!side) {
    for (int l = 0; l < nl; ++l) {
      const int rc = body(l, caller);
      if (rc != TN_OK) return rc;
    }
    return TN_OK;
  }
  const int ns = nl < SEP_STREAMS ? nl : SEP_STREAMS;
  cudaEvent_t fork = nullptr, join[SEP_STREAMS] = {};
  auto done = [&](int rc) {
    if (fork) cudaEventDestroy(fork);
    for (int i = 0; i < ns; ++i)
      if (join[i]) cudaEventDestroy(join[i]);
    return rc;
  };
  if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventRecord(fork, caller) != cudaSuccess)
    return done(TN_ERR_CUDA);
  for (int i = 0; i < ns; ++i)
    if (cudaStreamWaitEvent(side[i], fork, 0) != cudaSuccess) return done(TN_ERR_CUDA);
  int rc = TN_OK;
  for (int l = 0; l < nl && rc == TN_OK; ++l) rc = body(l, side[l % ns]);
  // join even after an error, so the caller's stream never runs ahead of work in flight
  for (int i = 0; i < ns; ++i)
    if (cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(join[i], side[i]) != cudaSuccess || cudaStreamWaitEvent(caller, join[i], 0) != cudaSuccess)
      return done(TN_ERR_CUDA);
  return done(rc);
}

// Workspace: one single-MPS classifier workspace per MPS, then ftilde,
// log-scale and the scaled gradient of every MPS.
struct SepLayout {
  std::vector<size_t> off, bytes;
  size_t ft_off, lam_off, d_off, total;
};

int sep_layout(const tn_mps* Ws, int nl, int batch, int ckpt_every, SepLayout* o) {
  if (!Ws || nl < 1 || nl > SEP_MAX || batch < 0 || ckpt_every < 0) return TN_ERR_ARG;
  o->off.clear();
  o->bytes.clear();
  size_t at = 0;
  for (int l = 0; l < nl; ++l) {
    const tn_mps& W = Ws[l];
    if (!W.bond || W.n < 2) return TN_ERR_ARG;
    const size_t b = tn_mps_classify_workspace_bytes(&W, W.n / 2, 1, batch, ckpt_every);
    if (b == 0 && batch > 0) return TN_ERR_ARG;
    o->off.push_back(at);
    o->bytes.push_back(b);
    at += al256(b);
  }
  o->ft_off = at;
  o->lam_off = o->ft_off + al256(sizeof(float) * (size_t)nl * (size_t)batch);
  o->d_off = o->lam_off + al256(sizeof(double) * (size_t)nl * (size_t)batch);
  o->total = o->d_off + al256(sizeof(float) * (size_t)nl * (size_t)(batch > 0 ? batch : 1));
  return TN_OK;
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

size_t tn_mps_classify_separate_workspace_bytes(const tn_mps* Ws, int n_mps, int batch, int ckpt_every) {
  SepLayout lay;
  return sep_layout(Ws, n_mps, batch, ckpt_every, &lay) == TN_OK ? lay.total : 0;
}

int tn_mps_classify_separate(const tn_mps* Ws, int n_mps, const float* pixels, int batch, int prec, int ckpt_every,
                             float* ftilde, double* log_scale, void* workspace, size_t ws_bytes, void* stream) {
  SepLayout lay;
  int rc = sep_layout(Ws, n_mps, batch, ckpt_every, &lay);
  if (rc != TN_OK) return rc;
  for (int l = 1; l < n_mps; ++l)
    if (Ws[l].n != Ws[0].n) return TN_ERR_SHAPE;
  if (batch == 0) return TN_OK;  // no samples: nothing to write (the pointers may be null)
  if (!ftilde || !log_scale || !pixels) return TN_ERR_ARG;
  if (!workspace || ws_bytes < lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;
  uint8_t* base = static_cast<uint8_t*>(workspace);
  float* ft_each = reinterpret_cast<float*>(base + lay.ft_off);
  double* lam_each = reinterpret_cast<double*>(base + lay.lam_off);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  rc = run_forked(n_mps, s, [&](int l, cudaStream_t sl) {
    return tn_mps_classify(&Ws[l], Ws[l].n / 2, 1, pixels, batch, prec, ckpt_every, ft_each + (int64_t)l * batch,
                           lam_each + (int64_t)l * batch, base + lay.off[(size_t)l], lay.bytes[(size_t)l], sl);
  });
  if (rc != TN_OK) return rc;
  cls_sep_combine<<<(batch + 127) / 128, 128, 0, s>>>(ft_each, lam_each, batch, n_mps, ftilde, log_scale);
  return cudaGetLastError() == cudaSuccess ? TN_OK : TN_ERR_CUDA;
}

int tn_mps_classify_separate_backward(const tn_mps* Ws, int n_mps, const float* pixels, int batch, int prec,
                                      int ckpt_every, const float* dftilde, float* const* dcores, void* workspace,
                                      size_t ws_bytes, void* stream) {
  SepLayout lay;
  int rc = sep_layout(Ws, n_mps, batch, ckpt_every, &lay);
  if (rc != TN_OK) return rc;
  if (!dcores || ckpt_every < 1) return TN_ERR_ARG;
  if (batch > 0 && (!dftilde || !pixels)) return TN_ERR_ARG;
  for (int l = 1; l < n_mps; ++l)
    if (Ws[l].n != Ws[0].n) return TN_ERR_SHAPE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (batch == 0) {  // no samples: every gradient is zero
    int64_t first = 0;
    for (int l = 0; l < n_mps; ++l) {
      for (int i = 0; i < Ws[l].n; ++i) {
        if (!dcores[first + i]) return TN_ERR_ARG;
        const size_t e = (size_t)(Ws[l].bond[i] * 2 * Ws[l].bond[i + 1]);
        if (cudaMemsetAsync(dcores[first + i], 0, sizeof(float) * e, s) != cudaSuccess) return TN_ERR_CUDA;
      }
      first += Ws[l].n;
    }
    return TN_OK;
  }
  if (!workspace || ws_bytes < lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255)) return TN_ERR_WORKSPACE;
  uint8_t* base = static_cast<uint8_t*>(workspace);
  double* lam_each = reinterpret_cast<double*>(base + lay.lam_off);
  float* d = reinterpret_cast<float*>(base + lay.d_off);
  std::vector<int64_t> first((size_t)n_mps, 0);  // dcores: the cores of MPS 0, then of MPS 1, ...
  for (int l = 1; l < n_mps; ++l) first[(size_t)l] = first[(size_t)l - 1] + Ws[l - 1].n;
  return run_forked(n_mps, s, [&](int l, cudaStream_t sl) {
    float* dl = d + (int64_t)l * batch;
    cls_sep_scale<<<(batch + 127) / 128, 128, 0, sl>>>(dftilde, lam_each, batch, n_mps, l, dl);
    if (cudaGetLastError() != cudaSuccess) return (int)TN_ERR_CUDA;
    return tn_mps_classify_backward(&Ws[l], Ws[l].n / 2, 1, pixels, batch, prec, ckpt_every, dl,
                                    dcores + first[(size_t)l], base + lay.off[(size_t)l], lay.bytes[(size_t)l], sl);
  });
}

}  // extern "C"
