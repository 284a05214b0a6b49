// Node splitting (Sec. III.B "Node Splitting", Appendix A "Saving Memory"):
// the node read as a matrix (rows over the left legs, columns over the right
// legs, each group in the order given, last leg fastest), decomposed by the
// one-sided Jacobi SVD of Hestenes (1958) in float32, truncated, and written
// out as U sqrt(S) and sqrt(S) V^T (split_node) or U, S, V^T (full SVD).
//
// One-sided Jacobi orthogonalises the columns of a working matrix W (L x r,
// column-major, r = min(M, N) columns of length L = max(M, N): the matrix
// view itself when M >= N, else its transpose) by plane rotations of column
// pairs, accumulating the rotations in V (r x r, starting from I). A sweep
// visits every pair once, in r - 1 rounds of r / 2 disjoint pairs (the circle
// method of round-robin scheduling), one kernel per round (a CUDA graph per
// sweep) and one CTA per pair. At convergence W = U S and the matrix (or its transpose) is W V^T:
// the singular values are the column norms of W.
#include <math.h>
#include <string.h>

#include <vector>

#include "tn_internal.h"

namespace tn {
namespace {

constexpr int SVD_THREADS = 256;
constexpr int SVD_MAX_SWEEPS = 40;
constexpr int SVD_CACHE = 8;  // register-held entries per thread and column

// The node's matrix view: element (i, j) at A + loff(i) + roff(j).
struct SplitView {
  const float* A;
  int64_t M, N;
  int32_t nl, nr;
  int32_t wide;  // M < N: W holds the transpose
  int32_t pad;
  int32_t ldim[TN_MAX_RANK], rdim[TN_MAX_RANK];
  int64_t lstr[TN_MAX_RANK], rstr[TN_MAX_RANK];
};

__device__ __forceinline__ int64_t leg_offset(int64_t idx, int n, const int32_t* dim, const int64_t* str) {
  int64_t off = 0;
  for (int p = n - 1; p >= 0; --p) {
    const int64_t d = dim[p];
    off += (idx % d) * str[p];
    idx /= d;
  }
  return off;
}

// W[w] for every w = row + L * col (coalesced writes), V = I.
__global__ void svd_gather(SplitView v, float* __restrict__ W, float* __restrict__ V, int64_t L, int64_t r) {
  const int64_t total = L * r, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += stride) {
    const int64_t row = w % L, col = w / L;
    const int64_t i = v.wide ? col : row, j = v.wide ? row : col;
    W[w] = v.A[leg_offset(i, v.nl, v.ldim, v.lstr) + leg_offset(j, v.nr, v.rdim, v.rstr)];
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += stride)
    V[e] = (e % r == e / r) ? 1.0f : 0.0f;
}

// Sum of three per-thread values over the CTA, in double across warps.
__device__ __forceinline__ void block_sum3(float& a, float& b, float& c, double* out) {
  __shared__ double part[SVD_THREADS / 32][3];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    part[warp][0] = a;
    part[warp][1] = b;
    part[warp][2] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int w = 0; w < SVD_THREADS / 32; ++w) {
      s0 += part[w][0];
      s1 += part[w][1];
      s2 += part[w][2];
    }
    out[0] = s0;
    out[1] = s1;
    out[2] = s2;
  }
}

// Pair `k` of round `t` over rp (even) slots: slot 0 stays, the others
// rotate by one position per round, and position k meets position rp-1-k.
__device__ __forceinline__ int circle_slot(int pos, int t, int rp) {
  return pos == 0 ? 0 : 1 + (pos - 1 + t) % (rp - 1);
}

// One round: CTA k rotates column pair k so that the two columns of W become
// orthogonal (Hestenes): with a = |w_p|^2, b = |w_q|^2, g = w_p . w_q and
// zeta = (b - a) / 2g, t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1 / sqrt(1 + t^2), s = c t, the pair becomes (c w_p - s w_q, s w_p +
// c w_q); V's columns p and q take the same rotation. Pairs already
// orthogonal to within tol (|g| <= tol sqrt(ab)) are left alone; the others
// are counted in *rotations.
__global__ void __launch_bounds__(SVD_THREADS)
svd_round(float* __restrict__ W, float* __restrict__ V, int64_t L, int r, int rp, int t, float tol,
          int* __restrict__ rotations) {
  const int k = blockIdx.x;
  const int p = circle_slot(k, t, rp), q = circle_slot(rp - 1 - k, t, rp);
  if (p >= r || q >= r) return;  // the dummy slot of an odd r
  float* wp = W + (int64_t)p * L;
  float* wq = W + (int64_t)q * L;
  float* vp = V + (int64_t)p * r;
  float* vq = V + (int64_t)q * r;
  // columns of up to SVD_CACHE * SVD_THREADS entries stay in registers
  // between the dot products and the rotation; V's two columns are loaded
  // with W's, so their latency overlaps the reduction
  const bool cached = L <= (int64_t)SVD_CACHE * SVD_THREADS;
  const bool vcached = r <= SVD_CACHE * SVD_THREADS;
  float xs[SVD_CACHE], ys[SVD_CACHE], us[SVD_CACHE], ts[SVD_CACHE];
  if (vcached) {
#pragma unroll
    for (int u = 0; u < SVD_CACHE; ++u) {
      const int i = threadIdx.x + u * SVD_THREADS;
      us[u] = i < r ? vp[i] : 0.0f;
      ts[u] = i < r ? vq[i] : 0.0f;
    }
  }
  float a = 0.0f, b = 0.0f, g = 0.0f;
  if (cached) {
#pragma unroll
    for (int u = 0; u < SVD_CACHE; ++u) {
      const int64_t i = threadIdx.x + (int64_t)u * SVD_THREADS;
      xs[u] = i < L ? wp[i] : 0.0f;
      ys[u] = i < L ? wq[i] : 0.0f;
      a = fmaf(xs[u], xs[u], a);
      b = fmaf(ys[u], ys[u], b);
      g = fmaf(xs[u], ys[u], g);
    }
  } else {
    for (int64_t i = threadIdx.x; i < L; i += SVD_THREADS) {
      const float x = wp[i], y = wq[i];
      a = fmaf(x, x, a);
      b = fmaf(y, y, b);
      g = fmaf(x, y, g);
    }
  }
  __shared__ double sums[3];
  __shared__ float rot[2];
  __shared__ int skip;
  block_sum3(a, b, g, sums);
  if (threadIdx.x == 0) {
    // the angle in float64: with float32 c and s from float32 arithmetic the
    // rounding of c^2 + s^2 is biased and the column norms drift by ~1e-4
    // over the ~10^4 rotations a column of a 1000-column matrix takes
    const double al = sums[0], be = sums[1], ga = sums[2];
    const bool go = al > 0.0 && be > 0.0 && fabs(ga) > (double)tol * sqrt(al) * sqrt(be);
    if (go) {
      const double z = (be - al) / (2.0 * ga);
      const double tt = (z >= 0.0 ? 1.0 : -1.0) / (fabs(z) + sqrt(1.0 + z * z));
      const double c = 1.0 / sqrt(1.0 + tt * tt);
      rot[0] = (float)c;
      rot[1] = (float)(c * tt);
      atomicAdd(rotations, 1);
    }
    skip = go ? 0 : 1;
  }
  __syncthreads();
  if (skip) return;
  const float c = rot[0], s = rot[1];
  if (cached) {
#pragma unroll
    for (int u = 0; u < SVD_CACHE; ++u) {
      const int64_t i = threadIdx.x + (int64_t)u * SVD_THREADS;
      if (i < L) {
        wp[i] = c * xs[u] - s * ys[u];
        wq[i] = s * xs[u] + c * ys[u];
      }
    }
  } else {
    for (int64_t i = threadIdx.x; i < L; i += SVD_THREADS) {
      const float x = wp[i], y = wq[i];
      wp[i] = c * x - s * y;
      wq[i] = s * x + c * y;
    }
  }
  if (vcached) {
#pragma unroll
    for (int u = 0; u < SVD_CACHE; ++u) {
      const int i = threadIdx.x + u * SVD_THREADS;
      if (i < r) {
        vp[i] = c * us[u] - s * ts[u];
        vq[i] = s * us[u] + c * ts[u];
      }
    }
  } else {
    for (int i = threadIdx.x; i < r; i += SVD_THREADS) {
      const float x = vp[i], y = vq[i];
      vp[i] = c * x - s * y;
      vq[i] = s * x + c * y;
    }
  }
}

// sigma[j] = |W[:, j]| (CTA j).
__global__ void __launch_bounds__(SVD_THREADS)
svd_norms(const float* __restrict__ W, int64_t L, float* __restrict__ sigma) {
  const float* w = W + (int64_t)blockIdx.x * L;
  float a = 0.0f, z0 = 0.0f, z1 = 0.0f;
  for (int64_t i = threadIdx.x; i < L; i += SVD_THREADS) a = fmaf(w[i], w[i], a);
  __shared__ double sums[3];
  block_sum3(a, z0, z1, sums);
  if (threadIdx.x == 0) sigma[blockIdx.x] = (float)sqrt(sums[0]);
}

// order[c] = index of the c-th largest singular value (ties by index; a NaN
// sorts last), sorted[c] its value: the rank of j is the number of values
// before it in that strict order, so the ranks are a permutation.
__global__ void svd_sort(const float* __restrict__ sigma, int r, int32_t* __restrict__ order,
                         float* __restrict__ sorted) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= r) return;
  const float sj = isnan(sigma[j]) ? -1.0f : sigma[j];
  int rank = 0;
  for (int i = 0; i < r; ++i) {
    const float si = isnan(sigma[i]) ? -1.0f : sigma[i];
    rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
  }
  order[rank] = j;
  sorted[rank] = sigma[j];
}

// The outputs for the k kept values. Columns of W give singular vectors
// scaled by sigma (w_j = sigma_j u_j), columns of V unit ones. Left (M x k,
// row-major): W's columns when M >= N, else V's; right (k x N, row-major):
// the other one. absorb: both sides carry sqrt(sigma) (split_node), else
// neither (full SVD). A W column of a zero singular value has no direction:
// its vector is written as zeros (not completed to an orthonormal basis).
__global__ void svd_write(const float* __restrict__ W, const float* __restrict__ V, const int32_t* __restrict__ order,
                          const float* __restrict__ sorted, int64_t M, int64_t N, int64_t L, int r, int k,
                          int wide, int absorb, float* __restrict__ U, float* __restrict__ S, float* __restrict__ Vt,
                          float* __restrict__ dropped) {
  const int64_t nl = M * k, nr = (int64_t)k * N, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t e = t0; e < nl + nr; e += stride) {
    const bool left = e < nl;
    const int64_t f = left ? e : e - nl;
    const int c = left ? (int)(f % k) : (int)(f / N);
    const int64_t i = left ? f / k : f % N;  // row of the left node, column of the right one
    const int j = min(max(order[c], 0), r - 1);
    const float sg = sorted[c];
    const bool from_w = left != (wide != 0);  // left from W iff M >= N
    float x;
    if (from_w) {
      const float sc = sg > 0.0f ? (absorb ? 1.0f / sqrtf(sg) : 1.0f / sg) : 0.0f;
      x = W[(int64_t)j * L + i] * sc;
    } else {
      x = V[(int64_t)j * r + i] * (absorb ? sqrtf(fmaxf(sg, 0.0f)) : 1.0f);
    }
    if (left)
      U[f] = x;
    else
      Vt[f] = x;
  }
  for (int64_t c = t0; c < r; c += stride) {
    if (c < k && S) S[c] = sorted[c];
    if (c >= k && dropped) dropped[c - k] = sorted[c];
  }
}

static size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

struct SplitLayout {
  SplitView v;
  int64_t L, r;
  size_t w_off, v_off, sig_off, ord_off, sorted_off, cnt_off, total;
};

static int plan_split(const tn_tensor* A, const int* left, int nleft, const int* right, int nright,
                      SplitLayout* out) {
  if (!A || A->rank < 0 || A->rank > TN_MAX_RANK || nleft < 0 || nright < 0 || nleft + nright != A->rank)
    return TN_ERR_ARG;
  if ((nleft > 0 && !left) || (nright > 0 && !right)) return TN_ERR_ARG;
  if (A->dtype != TN_F32) return TN_ERR_UNSUPPORTED;
  int seen[TN_MAX_RANK] = {0};
  for (int i = 0; i < nleft + nright; ++i) {
    const int leg = i < nleft ? left[i] : right[i - nleft];
    if (leg < 0 || leg >= A->rank || seen[leg]) return TN_ERR_ARG;
    seen[leg] = 1;
  }
  bool all_zero = true;
  for (int i = 0; i < A->rank; ++i) {
    if (A->shape[i] < 0) return TN_ERR_ARG;
    if (A->stride[i] < 0) return TN_ERR_UNSUPPORTED;
    if (A->stride[i] != 0) all_zero = false;
  }
  int64_t st[TN_MAX_RANK];
  int64_t s = 1;
  for (int i = A->rank - 1; i >= 0; --i) {
    st[i] = all_zero ? s : A->stride[i];
    s *= A->shape[i];
  }
  SplitLayout& o = *out;
  memset(&o, 0, sizeof(o));
  o.v.A = static_cast<const float*>(A->data);
  o.v.nl = nleft;
  o.v.nr = nright;
  o.v.M = o.v.N = 1;
  for (int i = 0; i < nleft; ++i) {
    o.v.ldim[i] = (int32_t)A->shape[left[i]];
    o.v.lstr[i] = st[left[i]];
    o.v.M *= A->shape[left[i]];
  }
  for (int i = 0; i < nright; ++i) {
    o.v.rdim[i] = (int32_t)A->shape[right[i]];
    o.v.rstr[i] = st[right[i]];
    o.v.N *= A->shape[right[i]];
  }
  for (int i = 0; i < A->rank; ++i)
    if (A->shape[i] > 0x7FFFFFFF) return TN_ERR_UNSUPPORTED;
  o.v.wide = o.v.M < o.v.N ? 1 : 0;
  o.L = o.v.wide ? o.v.N : o.v.M;
  o.r = o.v.wide ? o.v.M : o.v.N;
  if (o.r > 0x3FFFFFFF) return TN_ERR_UNSUPPORTED;
  if (o.r > 0 && !o.v.A) return TN_ERR_ARG;
  o.w_off = 0;
  o.v_off = al256(sizeof(float) * (size_t)(o.L * o.r));
  o.sig_off = o.v_off + al256(sizeof(float) * (size_t)(o.r * o.r));
  o.ord_off = o.sig_off + al256(sizeof(float) * (size_t)o.r);
  o.sorted_off = o.ord_off + al256(sizeof(int32_t) * (size_t)o.r);
  o.cnt_off = o.sorted_off + al256(sizeof(float) * (size_t)o.r);
  o.total = o.cnt_off + 256;
  return TN_OK;
}

static unsigned grid_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 64 ? 152 * 64 : b));
}

}  // namespace
}  // namespace tn

using namespace tn;

extern "C" {

int64_t tn_split_truncation(const float* sigma_desc, int64_t r, int64_t max_singular_values,
                            double max_truncation_err) {
  if (r <= 0 || !sigma_desc) return 0;
  int64_t k = r;
  if (max_truncation_err >= 0.0) {
    double dropped = 0.0;
    while (k > 0 && dropped + (double)sigma_desc[k - 1] <= max_truncation_err) {
      dropped += (double)sigma_desc[k - 1];
      --k;
    }
  }
  if (max_singular_values > 0 && k > max_singular_values) k = max_singular_values;
  return k < 1 ? 1 : k;
}

size_t tn_split_node_workspace_bytes(const tn_tensor* A, const int* left, int nleft, const int* right, int nright) {
  SplitLayout lay;
  if (plan_split(A, left, nleft, right, nright, &lay) != TN_OK) return 0;
  return lay.total;
}

int tn_split_node(const tn_tensor* A, const int* left, int nleft, const int* right, int nright,
                  int64_t max_singular_values, double max_truncation_err, int absorb, float* U, float* S,
                  float* Vt, float* dropped, int64_t* kept, int32_t* sweeps, void* workspace, size_t ws_bytes,
                  void* stream) {
  SplitLayout lay;
  int rc = plan_split(A, left, nleft, right, nright, &lay);
  if (rc != TN_OK) return rc;
  if (!kept) return TN_ERR_ARG;
  *kept = 0;
  if (sweeps) *sweeps = 0;
  if (lay.r == 0) return TN_OK;
  if (!U || !Vt || (!absorb && !S)) return TN_ERR_ARG;
  if (!workspace || ws_bytes < lay.total || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return TN_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint8_t* base = static_cast<uint8_t*>(workspace);
  float* W = reinterpret_cast<float*>(base + lay.w_off);
  float* V = reinterpret_cast<float*>(base + lay.v_off);
  float* sigma = reinterpret_cast<float*>(base + lay.sig_off);
  int32_t* order = reinterpret_cast<int32_t*>(base + lay.ord_off);
  float* sorted = reinterpret_cast<float*>(base + lay.sorted_off);
  int* counter = reinterpret_cast<int*>(base + lay.cnt_off);
  const int64_t L = lay.L;
  const int r = (int)lay.r, rp = r + (r & 1);
  svd_gather<<<grid_for(L * lay.r, 256), 256, 0, s>>>(lay.v, W, V, L, lay.r);
  if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
  // off-diagonal threshold: a few times the float32 rounding of a length-L dot product
  const float tol = 4.0f * sqrtf((float)L) * 5.9604645e-8f;
  // one sweep = a CUDA graph: the counter reset, then the r - 1 rounds in
  // order (built once per call, launched once per sweep)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  };
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return TN_ERR_CUDA;
  {
    cudaGraphNode_t prev = nullptr, node = nullptr;
    cudaMemsetParams mp;
    memset(&mp, 0, sizeof(mp));
    mp.dst = counter;
    mp.value = 0;
    mp.elementSize = sizeof(int);
    mp.width = 1;
    mp.height = 1;
    if (cudaGraphAddMemsetNode(&prev, graph, nullptr, 0, &mp) != cudaSuccess) {
      cleanup();
      return TN_ERR_CUDA;
    }
    float* w_arg = W;
    float* v_arg = V;
    int64_t l_arg = L;
    int r_arg = r, rp_arg = rp;
    float tol_arg = tol;
    int* c_arg = counter;
    for (int t = 0; t < rp - 1; ++t) {
      int t_arg = t;
      void* args[] = {&w_arg, &v_arg, &l_arg, &r_arg, &rp_arg, &t_arg, &tol_arg, &c_arg};
      cudaKernelNodeParams kp;
      memset(&kp, 0, sizeof(kp));
      kp.func = reinterpret_cast<void*>(svd_round);
      kp.gridDim = dim3((unsigned)(rp / 2));
      kp.blockDim = dim3(SVD_THREADS);
      kp.kernelParams = args;
      if (cudaGraphAddKernelNode(&node, graph, &prev, 1, &kp) != cudaSuccess) {
        cleanup();
        return TN_ERR_CUDA;
      }
      prev = node;
    }
  }
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
    cleanup();
    return TN_ERR_CUDA;
  }
  int done = 0, used = 0;
  for (int sw = 0; sw < SVD_MAX_SWEEPS && !done; ++sw) {
    int host_count = -1;
    if (cudaGraphLaunch(exec, s) != cudaSuccess ||
        cudaMemcpyAsync(&host_count, counter, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      cleanup();
      return TN_ERR_CUDA;
    }
    ++used;
    done = host_count == 0;
  }
  cleanup();
  if (sweeps) *sweeps = done ? used : -used;
  svd_norms<<<r, SVD_THREADS, 0, s>>>(W, L, sigma);
  svd_sort<<<(r + 255) / 256, 256, 0, s>>>(sigma, r, order, sorted);
  if (cudaGetLastError() != cudaSuccess) return TN_ERR_CUDA;
  std::vector<float> host_sorted((size_t)r);
  if (cudaMemcpyAsync(host_sorted.data(), sorted, sizeof(float) * (size_t)r, cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TN_ERR_CUDA;
  const int64_t k = tn_split_truncation(host_sorted.data(), r, max_singular_values, max_truncation_err);
  svd_write<<<grid_for((lay.v.M + lay.v.N) * k + r, 256), 256, 0, s>>>(W, V, order, sorted, lay.v.M, lay.v.N, L,
                                                                        r, (int)k, lay.v.wide, absorb ? 1 : 0, U, S, Vt,
                                                                        dropped);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return TN_ERR_CUDA;
  *kept = k;
  return TN_OK;
}

}  // extern "C"
