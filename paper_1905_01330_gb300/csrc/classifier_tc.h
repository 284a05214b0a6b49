// Internal interface of the tcgen05 classifier sweeps (classifier_tc.cu).
#pragma once

#include "tn_internal.h"

namespace tn {

constexpr int CLS_TC_MAXN = 1024;
constexpr int CLS_TILE = 128;  // samples per tile (the MMA's M, one TMEM lane each)

// Bytes of the packed bf16 images of one step (hi, or hi and lo when split):
// the forward image (rows (s, j), K = the incoming bond k) and the adjoint
// image (rows k, K = (s, j)).
size_t cls_fwd_image_bytes(int chi, int split);
size_t cls_adj_image_bytes(int chi, int split);
// Bytes of one tile's bf16 sweep-vector image (the forward's MMA operand).
size_t cls_vtile_bytes(int chi, int split);

// Packs the cores of both half-chains into the images of one kind
// (adjoint = 0: forward images, 1: adjoint images), steps 0 .. T[h]-1 of
// half h (half 0: sites 0 .. ls-1; half 1: sites n-1 .. ls+1).
struct ClsPackParams {
  int32_t n, chi, split, adjoint;
  int32_t T[2];
  int32_t bond[CLS_TC_MAXN + 1];
  const float* core[CLS_TC_MAXN];
  uint8_t* images[2];  // per half, indexed by step
  size_t step_bytes;
};
int cls_pack(const ClsPackParams& p, cudaStream_t s);

// One launch sweeps both half-chains: CTA (half, tile) runs the steps
// [t_begin[h], t_end[h]) of its half (forward in increasing, adjoint in
// decreasing order) for its 128 samples.
struct ClsTcParams {
  int32_t n, batch, ntiles;
  int32_t t_begin[2], t_end[2];
  // forward: keep the float32 vector entering step t in
  // store[h][(t - store_base[h]) / store_every] when (t - store_base[h]) %
  // store_every == 0
  int32_t store_every;
  int32_t store_base[2];
  int32_t half_site[2];   // site of step 0: 0 (left) and n - 1 (right)
  int32_t half_dir[2];    // site of step t = half_site + half_dir * t
  const float* pixels;    // [batch, n]
  float* state[2];        // [batch, chi] in/out (forward: v, adjoint: g)
  double* lam[2];         // forward: [batch] log-scale in/out
  float* store[2];        // forward: kept float32 vectors (or null)
  float* sc[2];           // [t][batch] per-step scales (forward writes, adjoint reads)
  uint8_t* vseg[2];       // forward: bf16 vector images of the steps of this launch (or null);
                          // adjoint: the same, read: [t - t_begin][tile]
  const uint8_t* images[2];  // packed cores of this launch's kind, indexed by step
  float* grad[2];         // adjoint: [t][chi][2 chi] float32 core gradients, accumulated
  int* status;
};
int cls_fwd_tc_launch(int chi, int split, const ClsTcParams& p, cudaStream_t s);
int cls_adj_tc_launch(int chi, int split, const ClsTcParams& p, cudaStream_t s);
// Whether the tcgen05 adjoint supports this (chi, split): its staging must
// fit in shared memory.
bool cls_adj_tc_supported(int chi, int split);

// dcores[site] from the accumulated per-step gradients (both halves).
struct ClsScatterParams {
  int32_t n, chi;
  int32_t T[2];
  int32_t bond[CLS_TC_MAXN + 1];
  float* dcore[CLS_TC_MAXN];
  const float* grad[2];
};
int cls_scatter_grad(const ClsScatterParams& p, cudaStream_t s);

}  // namespace tn
