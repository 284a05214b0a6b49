// Grouped contraction staged from and to host memory: the end-to-end form of
// the grouped tensordot, for operands that start in (pinned) host memory and
// results that must end there. The specs are cut into chunks of consecutive
// specs of about equal bytes, each with its own group plan; a run pipelines
// the chunks over three library-owned streams -- chunk c's operands go host ->
// device while chunk c - 1 is contracted and chunk c - 2's results go device
// -> host -- so both copy directions and the kernels overlap.
#include <string.h>

#include <algorithm>
#include <vector>

#include "tn_internal.h"

struct tn_staged_plan {
  struct Chunk {
    tn_group_plan* plan;
    size_t lo_in, hi_in, lo_out, hi_out;  // byte ranges of dev_in / dev_out
    size_t list_off, list_bytes;          // its work lists in the workspace
  };
  std::vector<Chunk> chunks;
  size_t packed_off = 0, total = 0;  // one packed region shared by the chunk plans
  const uint8_t* dev_in = nullptr;
  uint8_t* dev_out = nullptr;
  cudaStream_t streams[3] = {nullptr, nullptr, nullptr};  // h2d, compute, d2h
  std::vector<cudaEvent_t> ready, done;                    // per chunk
  cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
  double flops = 0.0;
};

namespace {

// Byte range [lo, hi) of tensor t inside the buffer at base (bytes long);
// false when it lies (partly) outside.
bool tensor_span(const tn_tensor& t, const uint8_t* base, size_t bytes, size_t* lo, size_t* hi) {
  int64_t n = 1;
  for (int i = 0; i < t.rank; ++i) n *= t.shape[i];
  const uint8_t* p = static_cast<const uint8_t*>(t.data);
  if (n == 0) {
    *lo = *hi = p >= base ? (size_t)(p - base) : 0;
    return true;
  }
  if (p < base) return false;
  // extent in elements: row-major when every stride is 0 (tn_tensor's default)
  bool all_zero = true;
  for (int i = 0; i < t.rank; ++i) all_zero = all_zero && t.stride[i] == 0;
  int64_t span = 1;
  if (all_zero) {
    span = n;
  } else {
    for (int i = 0; i < t.rank; ++i) span += (t.shape[i] - 1) * t.stride[i];
  }
  *lo = (size_t)(p - base);
  *hi = *lo + (size_t)span * sizeof(float);
  return *hi <= bytes;
}

void destroy_impl(tn_staged_plan* p) {
  if (!p) return;
  for (auto& c : p->chunks) tn_group_plan_destroy(c.plan);
  for (cudaEvent_t e : p->ready)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : p->done)
    if (e) cudaEventDestroy(e);
  if (p->fork) cudaEventDestroy(p->fork);
  for (int i = 0; i < 3; ++i) {
    if (p->join[i]) cudaEventDestroy(p->join[i]);
    if (p->streams[i]) cudaStreamDestroy(p->streams[i]);
  }
  delete p;
}

}  // namespace

extern "C" {

int tn_chunk_bounds(const double* weights, int n, int chunks, int* bounds, int* nbounds) {
  if (n < 0 || chunks < 1 || !bounds || !nbounds || (n > 0 && !weights)) return TN_ERR_ARG;
  std::vector<double> cum((size_t)n);
  double acc = 0.0;
  for (int i = 0; i < n; ++i) {
    acc += weights[i];
    cum[(size_t)i] = acc;
  }
  int m = 0;
  bounds[m++] = 0;
  for (int k = 1; k < chunks; ++k) {
    const double t = acc * k / chunks;
    // first item whose running weight reaches t
    const int j = (int)(std::lower_bound(cum.begin(), cum.end(), t) - cum.begin());
    // candidates: strictly after the previous boundary, at most one past j, before the end
    int lo = std::max(bounds[m - 1] + 1, j), hi = std::min(j + 2, n);
    if (lo >= hi && bounds[m - 1] + 1 < n) {
      lo = bounds[m - 1] + 1;
      hi = lo + 1;
    }
    if (lo < hi) {
      int best = lo;
      for (int b = lo + 1; b < hi; ++b)
        if (std::abs(cum[(size_t)b - 1] - t) < std::abs(cum[(size_t)best - 1] - t)) best = b;
      bounds[m++] = best;
    }
  }
  bounds[m++] = n;
  *nbounds = m;
  return TN_OK;
}

int tn_staged_plan_create(const tn_contract_spec* specs, int nspecs, int prec, const void* dev_in, size_t in_bytes,
                          void* dev_out, size_t out_bytes, int chunks, tn_staged_plan** plan) {
  if (!plan) return TN_ERR_ARG;
  *plan = nullptr;
  if (nspecs < 0 || (nspecs > 0 && !specs) || chunks < 1 || !dev_in || !dev_out) return TN_ERR_ARG;
  tn_staged_plan* p = new (std::nothrow) tn_staged_plan();
  if (!p) return TN_ERR_ARG;
  p->dev_in = static_cast<const uint8_t*>(dev_in);
  p->dev_out = static_cast<uint8_t*>(dev_out);
  // chunk by the bytes each spec moves
  std::vector<double> w((size_t)nspecs);
  std::vector<size_t> lo_in((size_t)nspecs), hi_in((size_t)nspecs), lo_out((size_t)nspecs), hi_out((size_t)nspecs);
  for (int i = 0; i < nspecs; ++i) {
    size_t la, ha, lb, hb, lc, hc;
    if (!tensor_span(specs[i].A, p->dev_in, in_bytes, &la, &ha) ||
        !tensor_span(specs[i].B, p->dev_in, in_bytes, &lb, &hb) ||
        !tensor_span(specs[i].C, p->dev_out, out_bytes, &lc, &hc)) {
      destroy_impl(p);
      return TN_ERR_ARG;
    }
    lo_in[(size_t)i] = std::min(la, lb);
    hi_in[(size_t)i] = std::max(ha, hb);
    lo_out[(size_t)i] = lc;
    hi_out[(size_t)i] = hc;
    w[(size_t)i] = (double)(ha - la) + (double)(hb - lb) + (double)(hc - lc);
  }
  std::vector<int> bounds((size_t)chunks + 1);
  int nb = 0;
  int rc = tn_chunk_bounds(w.data(), nspecs, chunks, bounds.data(), &nb);
  if (rc != TN_OK) {
    destroy_impl(p);
    return rc;
  }
  size_t off = 0, packed = 0, prev_in = 0, prev_out = 0;
  for (int c = 0; c + 1 < nb; ++c) {
    const int b0 = bounds[(size_t)c], b1 = bounds[(size_t)c + 1];
    if (b1 <= b0) continue;
    tn_staged_plan::Chunk ch;
    ch.lo_in = *std::min_element(lo_in.begin() + b0, lo_in.begin() + b1);
    ch.hi_in = *std::max_element(hi_in.begin() + b0, hi_in.begin() + b1);
    ch.lo_out = *std::min_element(lo_out.begin() + b0, lo_out.begin() + b1);
    ch.hi_out = *std::max_element(hi_out.begin() + b0, hi_out.begin() + b1);
    // each chunk owns one range of each buffer: the tensors lie in spec order
    if (ch.lo_in < prev_in || ch.lo_out < prev_out) {
      destroy_impl(p);
      return TN_ERR_ARG;
    }
    prev_in = ch.hi_in;
    prev_out = ch.hi_out;
    ch.plan = nullptr;
    if ((rc = tn_group_plan_create(specs + b0, b1 - b0, prec, &ch.plan)) != TN_OK) {
      destroy_impl(p);
      return rc;
    }
    ch.list_off = off;
    ch.list_bytes = tn::group_plan_list_bytes(ch.plan);
    off += tn::align256(ch.list_bytes);
    packed = std::max(packed, tn::group_plan_packed_bytes(ch.plan));
    p->flops += tn_group_plan_flops(ch.plan);
    p->chunks.push_back(ch);
  }
  p->packed_off = off;
  p->total = off + tn::align256(packed);
  // library streams and events (on the current device)
  for (int i = 0; i < 3; ++i)
    if (cudaStreamCreateWithFlags(&p->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming) != cudaSuccess) {
      destroy_impl(p);
      return TN_ERR_CUDA;
    }
  if (cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess) {
    destroy_impl(p);
    return TN_ERR_CUDA;
  }
  p->ready.assign(p->chunks.size(), nullptr);
  p->done.assign(p->chunks.size(), nullptr);
  for (size_t c = 0; c < p->chunks.size(); ++c)
    if (cudaEventCreateWithFlags(&p->ready[c], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->done[c], cudaEventDisableTiming) != cudaSuccess) {
      destroy_impl(p);
      return TN_ERR_CUDA;
    }
  *plan = p;
  return TN_OK;
}

int tn_staged_plan_chunks(const tn_staged_plan* plan) { return plan ? (int)plan->chunks.size() : 0; }

double tn_staged_plan_flops(const tn_staged_plan* plan) { return plan ? plan->flops : 0.0; }

int tn_staged_plan_set_schedule(tn_staged_plan* plan, int cls, int tile_width, int long_k, int store16) {
  if (!plan) return TN_ERR_ARG;
  for (auto& c : plan->chunks) {
    const int rc = tn_group_plan_set_schedule(c.plan, cls, tile_width, long_k, store16);
    if (rc != TN_OK) return rc;
  }
  return TN_OK;
}

size_t tn_staged_plan_workspace_bytes(const tn_staged_plan* plan) { return plan ? plan->total : 0; }

int tn_staged_plan_upload(const tn_staged_plan* plan, void* workspace, size_t bytes, void* stream) {
  if (!plan) return TN_ERR_ARG;
  if (plan->total > 0 && (!workspace || bytes < plan->total || (reinterpret_cast<uintptr_t>(workspace) & 255)))
    return TN_ERR_WORKSPACE;
  uint8_t* base = static_cast<uint8_t*>(workspace);
  for (const auto& c : plan->chunks) {
    const int rc = tn::group_plan_upload_shared(c.plan, base + c.list_off, c.list_bytes, base + plan->packed_off,
                                                static_cast<cudaStream_t>(stream));
    if (rc != TN_OK) return rc;
  }
  return TN_OK;
}

int tn_staged_plan_run(const tn_staged_plan* plan, void* workspace, size_t bytes, const void* host_in,
                       void* host_out, void* stream) {
  if (!plan || !host_in || !host_out) return TN_ERR_ARG;
  if (plan->total > 0 && (!workspace || bytes < plan->total || (reinterpret_cast<uintptr_t>(workspace) & 255)))
    return TN_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStream_t h2d = plan->streams[0], comp = plan->streams[1], d2h = plan->streams[2];
  uint8_t* base = static_cast<uint8_t*>(workspace);
  const uint8_t* hin = static_cast<const uint8_t*>(host_in);
  uint8_t* hout = static_cast<uint8_t*>(host_out);
  // fork: the library streams start after the caller's earlier work
  if (cudaEventRecord(plan->fork, s) != cudaSuccess) return TN_ERR_CUDA;
  for (int i = 0; i < 3; ++i)
    if (cudaStreamWaitEvent(plan->streams[i], plan->fork, 0) != cudaSuccess) return TN_ERR_CUDA;
  for (size_t c = 0; c < plan->chunks.size(); ++c) {
    const auto& ch = plan->chunks[c];
    if (ch.hi_in > ch.lo_in &&
        cudaMemcpyAsync(const_cast<uint8_t*>(plan->dev_in) + ch.lo_in, hin + ch.lo_in, ch.hi_in - ch.lo_in,
                        cudaMemcpyHostToDevice, h2d) != cudaSuccess)
      return TN_ERR_CUDA;
    if (cudaEventRecord(plan->ready[c], h2d) != cudaSuccess || cudaStreamWaitEvent(comp, plan->ready[c], 0) !=
                                                                    cudaSuccess)
      return TN_ERR_CUDA;
    const int rc = tn::group_plan_run_shared(ch.plan, base + ch.list_off, ch.list_bytes, comp);
    if (rc != TN_OK) return rc;
    if (cudaEventRecord(plan->done[c], comp) != cudaSuccess || cudaStreamWaitEvent(d2h, plan->done[c], 0) !=
                                                                   cudaSuccess)
      return TN_ERR_CUDA;
    if (ch.hi_out > ch.lo_out &&
        cudaMemcpyAsync(hout + ch.lo_out, plan->dev_out + ch.lo_out, ch.hi_out - ch.lo_out, cudaMemcpyDeviceToHost,
                        d2h) != cudaSuccess)
      return TN_ERR_CUDA;
  }
  // join: the caller's stream waits for the last copy and kernel
  for (int i = 0; i < 3; ++i)
    if (cudaEventRecord(plan->join[i], plan->streams[i]) != cudaSuccess ||
        cudaStreamWaitEvent(s, plan->join[i], 0) != cudaSuccess)
      return TN_ERR_CUDA;
  return TN_OK;
}

void tn_staged_plan_destroy(tn_staged_plan* plan) { destroy_impl(plan); }

}  // extern "C"
