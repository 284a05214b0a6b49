// Host-side validation and planning of pairwise contractions: the GEMM view
// of a tensordot (edge flattening, Sec. III.B.2) with per-leg strides.
#include <string.h>

#include "tn_internal.h"

namespace tn {

static bool row_major_strides(const tn_tensor* t, int64_t* st) {
  bool all_zero = true;
  for (int i = 0; i < t->rank; ++i)
    if (t->stride[i] != 0) all_zero = false;
  int64_t s = 1;
  for (int i = t->rank - 1; i >= 0; --i) {
    st[i] = all_zero ? s : t->stride[i];
    s *= t->shape[i];
  }
  return all_zero;
}

static int check_tensor(const tn_tensor* t) {
  if (!t) return TN_ERR_ARG;
  if (t->rank < 0 || t->rank > TN_MAX_RANK) return TN_ERR_ARG;
  if (t->dtype != TN_F32) return TN_ERR_UNSUPPORTED;
  int64_t n = 1;
  for (int i = 0; i < t->rank; ++i) {
    if (t->shape[i] < 0) return TN_ERR_ARG;
    if (t->stride[i] < 0) return TN_ERR_UNSUPPORTED;
    n *= t->shape[i];
  }
  if (n > 0 && !t->data) return TN_ERR_ARG;
  return TN_OK;
}

int plan_contract(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                  int nshared, const tn_tensor* C, ContractDesc* d) {
  int rc;
  if ((rc = check_tensor(A)) != TN_OK) return rc;
  if ((rc = check_tensor(B)) != TN_OK) return rc;
  if ((rc = check_tensor(C)) != TN_OK) return rc;
  if (nshared < 0 || nshared > A->rank || nshared > B->rank) return TN_ERR_ARG;
  if (nshared > 0 && (!legsA || !legsB)) return TN_ERR_ARG;
  bool useda[TN_MAX_RANK] = {false}, usedb[TN_MAX_RANK] = {false};
  for (int j = 0; j < nshared; ++j) {
    const int la = legsA[j], lb = legsB[j];
    if (la < 0 || la >= A->rank || lb < 0 || lb >= B->rank) return TN_ERR_ARG;
    if (useda[la] || usedb[lb]) return TN_ERR_ARG;
    useda[la] = usedb[lb] = true;
    if (A->shape[la] != B->shape[lb]) return TN_ERR_SHAPE;  // connect needs matching dims
  }
  int64_t sa[TN_MAX_RANK], sb[TN_MAX_RANK], sc[TN_MAX_RANK];
  row_major_strides(A, sa);
  row_major_strides(B, sb);
  row_major_strides(C, sc);

  memset(d, 0, sizeof(*d));
  d->A = static_cast<const float*>(A->data);
  d->B = static_cast<const float*>(B->data);
  d->C = static_cast<float*>(C->data);

  // result legs: A's free legs then B's free legs
  int nout = 0;
  int64_t M = 1, N = 1, K = 1;
  for (int p = 0; p < A->rank; ++p) {
    if (useda[p]) continue;
    if (nout >= C->rank || C->shape[nout] != A->shape[p]) return TN_ERR_SHAPE;
    d->mdim[d->nm] = (int32_t)A->shape[p];
    d->mstr[d->nm] = sa[p];
    d->nm++;
    M *= A->shape[p];
    nout++;
  }
  for (int p = 0; p < B->rank; ++p) {
    if (usedb[p]) continue;
    if (nout >= C->rank || C->shape[nout] != B->shape[p]) return TN_ERR_SHAPE;
    d->ndim[d->nn] = (int32_t)B->shape[p];
    d->nstr[d->nn] = sb[p];
    d->nn++;
    N *= B->shape[p];
    nout++;
  }
  if (nout != C->rank) return TN_ERR_SHAPE;
  // the result is written row-major and dense
  {
    int64_t s = 1;
    for (int i = C->rank - 1; i >= 0; --i) {
      if (C->shape[i] > 1 && sc[i] != s) return TN_ERR_UNSUPPORTED;
      s *= C->shape[i];
    }
  }

  // shared legs: keep the caller's pairing; put innermost the pair holding
  // the unit-stride leg of the larger operand (B when N > M, else A), else
  // that of the other one, so k runs of the operand with more bytes are
  // contiguous
  int order[TN_MAX_RANK];
  for (int j = 0; j < nshared; ++j) order[j] = j;
  if (nshared > 1) {
    int best_a = -1, best_b = -1;
    int64_t bs_a = INT64_MAX, bs_b = INT64_MAX;
    for (int j = 0; j < nshared; ++j) {
      if (A->shape[legsA[j]] > 1 && sa[legsA[j]] < bs_a) { bs_a = sa[legsA[j]]; best_a = j; }
      if (B->shape[legsB[j]] > 1 && sb[legsB[j]] < bs_b) { bs_b = sb[legsB[j]]; best_b = j; }
    }
    const bool prefer_b = N > M;
    int best;
    if (prefer_b) best = (bs_b == 1 || bs_a != 1) ? best_b : best_a;
    else best = (bs_a == 1 || bs_b != 1) ? best_a : best_b;
    if (best < 0) best = best_a >= 0 ? best_a : best_b;
    if (best >= 0) {
      int w = 0;
      for (int j = 0; j < nshared; ++j)
        if (j != best) order[w++] = j;
      order[w] = best;
    }
  }
  for (int jj = 0; jj < nshared; ++jj) {
    const int j = order[jj];
    d->kdim[jj] = (int32_t)A->shape[legsA[j]];
    d->kstrA[jj] = sa[legsA[j]];
    d->kstrB[jj] = sb[legsB[j]];
    K *= A->shape[legsA[j]];
  }
  d->nk = nshared;
  if (M >= (1ll << 31) || N >= (1ll << 31) || K >= (1ll << 31)) return TN_ERR_UNSUPPORTED;
  d->M = M;
  d->N = N;
  d->K = K;

  // loader mapping per operand: walk the direction whose innermost leg has the
  // smaller stride with consecutive threads
  const int64_t big = INT64_MAX;
  const int64_t a_k = d->nk ? d->kstrA[d->nk - 1] : big;
  const int64_t b_k = d->nk ? d->kstrB[d->nk - 1] : big;
  const int64_t a_m = d->nm ? d->mstr[d->nm - 1] : big;
  const int64_t b_n = d->nn ? d->nstr[d->nn - 1] : big;
  d->a_kfast = (a_k < a_m) ? 1 : 0;
  d->b_kfast = (b_k < b_n) ? 1 : 0;

  // the kernels address operands with 32-bit element offsets
  int64_t span_a = 0, span_b = 0;
  for (int p = 0; p < A->rank; ++p) span_a += (A->shape[p] > 0 ? A->shape[p] - 1 : 0) * sa[p];
  for (int p = 0; p < B->rank; ++p) span_b += (B->shape[p] > 0 ? B->shape[p] - 1 : 0) * sb[p];
  if (span_a >= (1ll << 31) || span_b >= (1ll << 31)) return TN_ERR_UNSUPPORTED;
  d->splits = 1;
  d->k_per_split = K;
  return TN_OK;
}

void plan_units(ContractDesc* d, int64_t min_units) {
  d->tiles_m = (int32_t)((d->M + TC_BM - 1) / TC_BM);
  d->tiles_n = (int32_t)((d->N + TC_BN - 1) / TC_BN);
  const int64_t slabs = (d->K + 63) / 64;
  const int64_t tiles = (int64_t)d->tiles_m * d->tiles_n;
  int64_t splits = (slabs + MAX_SLABS_PER_UNIT - 1) / MAX_SLABS_PER_UNIT;
  if (min_units > tiles * splits) {
    const int64_t want = (min_units + tiles - 1) / tiles;
    const int64_t cap = slabs / 4 > 1 ? slabs / 4 : 1;
    if (want > splits) splits = want < cap ? want : cap;
  }
  if (splits < 1) splits = 1;
  const int64_t per = (slabs + splits - 1) / splits;
  d->splits = (int32_t)((slabs + per - 1) / per);
  d->k_per_split = per * 64;
}

// Units of the packed GEMM: no shared-memory table bounds its k range, so a
// spec with many output tiles keeps each tile's whole k range in one unit (up
// to 512 slabs: no zeroing pass, no atomics); a spec with few tiles is still
// cut into 32-slab ranges so its work spreads over the SMs. long_k = false
// keeps the 32-slab ranges everywhere (a schedule the autotuner may pick).
void plan_units_packed(ContractDesc* d, bool long_k) {
  plan_units(d, 1);
  const int64_t tiles = (int64_t)d->tiles_m * d->tiles_n;
  if (!long_k || tiles < 16) return;
  const int64_t slabs = (d->K + 63) / 64;
  const int64_t per = slabs < 512 ? slabs : 512;
  d->splits = (int32_t)((slabs + per - 1) / per);
  d->k_per_split = per * 64;
}

}  // namespace tn
