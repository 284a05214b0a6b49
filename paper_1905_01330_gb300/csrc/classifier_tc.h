// Internal interface of the tcgen05 classifier sweeps (classifier_tc.cu).
#pragma once

#include "tn_internal.h"

namespace tn {

constexpr int CLS_TC_MAXN = 1024;

// Packs the cores of steps 0 .. steps-1 of one half-chain into bf16 K-major
// images (see classifier_tc.cu).
struct ClsPackParams {
  int32_t n, half, mode, chi, kpad;
  int32_t pad;
  size_t img_bytes;
  int32_t bond[CLS_TC_MAXN + 1];
  const float* core[CLS_TC_MAXN];
  uint8_t* images;
};

// One tcgen05 sweep of a half-chain over steps [t_begin, t_end) (forward
// mode 0 in increasing order, adjoint mode 1 in decreasing order).
struct ClsTcParams {
  int32_t n, batch, half, mode, t_begin, t_end, store_every, store_base;
  const float* pixels;   // [batch, n]
  float* state;          // [batch, chi] in/out
  double* lam;           // [batch] forward log-scale in/out
  float* store;          // forward: kept vectors [slot][batch][chi] (or null)
  float* sc;             // [t][batch] per-step scales
  float* xout;           // adjoint: [t - t_begin][batch][2 chi]
  const uint8_t* images; // packed cores of this half and mode, indexed by step
  int* status;
};

size_t cls_image_bytes(int chi);
int cls_pack(const ClsPackParams& p, int steps, cudaStream_t s);
int cls_sweep_tc_launch(int chi, const ClsTcParams& p, cudaStream_t s);

}  // namespace tn
