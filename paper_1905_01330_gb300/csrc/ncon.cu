// ncon planning (Appendix B): turns a labelled network into the sequence of
// pairwise contractions and traces that evaluates it, and the permutation of
// the last result's legs into the output order. Host code only: the steps run
// as tn_contract calls (a trace as a contraction with the identity).
//
// Labels >= 0 are edges (two legs each: of two tensors, or a trace on one),
// labels < 0 dangling legs -1, -2, ... of the result. Edges are taken in
// con_order (default ascending); an edge between two tensors contracts every
// edge those two share at once (contract_between, Sec. III.B.2), the result
// holding the first tensor's free legs then the second's and going to the end
// of the operand list; tensors still unconnected at the end are joined by
// outer products (Sec. III.B.5) in list order.
#include <string.h>

#include <algorithm>
#include <vector>

#include "tn_internal.h"

namespace {

struct Operand {
  int id;                      // 0..n-1 inputs, n + s the result of step s
  std::vector<int> labels;
  std::vector<int64_t> dims;
};

int find_leg(const Operand& o, int label, int from = 0) {
  for (size_t p = (size_t)from; p < o.labels.size(); ++p)
    if (o.labels[p] == label) return (int)p;
  return -1;
}

}  // namespace

extern "C" int tn_ncon_plan(int n, const int* ranks, const int64_t* dims, const int* labels, const int* con_order,
                            int n_order, const int* out_order, int n_out, tn_ncon_step* steps, int max_steps,
                            int* n_steps, int* out_perm, int* out_rank) {
  if (n <= 0 || !ranks || !n_steps || !out_perm || !out_rank || n_order < 0 || n_out < 0) return TN_ERR_ARG;
  std::vector<Operand> ops;
  int total = 0;
  for (int t = 0; t < n; ++t) {
    if (ranks[t] < 0 || ranks[t] > TN_MAX_RANK) return TN_ERR_ARG;
    total += ranks[t];
  }
  if (total > 0 && (!dims || !labels)) return TN_ERR_ARG;
  // labels: edges twice with equal dims, dangling legs -1 .. -k once each
  std::vector<int> edge_labels, open_labels;
  std::vector<std::pair<int, int64_t>> seen;  // (label, dim) of every leg
  for (int t = 0, off = 0; t < n; off += ranks[t], ++t) {
    Operand o;
    o.id = t;
    for (int p = 0; p < ranks[t]; ++p) {
      if (dims[off + p] < 0) return TN_ERR_ARG;
      o.labels.push_back(labels[off + p]);
      o.dims.push_back(dims[off + p]);
      seen.push_back({labels[off + p], dims[off + p]});
    }
    ops.push_back(o);
  }
  std::sort(seen.begin(), seen.end());
  for (size_t i = 0; i < seen.size();) {
    size_t j = i;
    while (j < seen.size() && seen[j].first == seen[i].first) ++j;
    const int lab = seen[i].first;
    const size_t cnt = j - i;
    if (lab >= 0) {
      if (cnt != 2) return TN_ERR_ARG;
      if (seen[i].second != seen[i + 1].second) return TN_ERR_SHAPE;
      edge_labels.push_back(lab);
    } else {
      if (cnt != 1) return TN_ERR_ARG;
      open_labels.push_back(lab);
    }
    i = j;
  }
  std::sort(open_labels.begin(), open_labels.end(), [](int a, int b) { return a > b; });
  for (size_t i = 0; i < open_labels.size(); ++i)
    if (open_labels[i] != -(int)i - 1) return TN_ERR_ARG;
  if ((int)open_labels.size() > TN_MAX_RANK) return TN_ERR_UNSUPPORTED;
  std::vector<int> order;
  if (n_order > 0) {
    if (!con_order) return TN_ERR_ARG;
    order.assign(con_order, con_order + n_order);
    std::vector<int> sorted_order = order;
    std::sort(sorted_order.begin(), sorted_order.end());
    if (sorted_order != edge_labels) return TN_ERR_ARG;
  } else {
    if (!edge_labels.empty()) order = edge_labels;
  }
  std::vector<int> out;
  if (n_out > 0) {
    if (!out_order) return TN_ERR_ARG;
    out.assign(out_order, out_order + n_out);
    std::vector<int> sorted_out = out;
    std::sort(sorted_out.begin(), sorted_out.end(), [](int a, int b) { return a > b; });
    if (sorted_out != open_labels) return TN_ERR_ARG;
  } else {
    out = open_labels;
  }

  int ns = 0;
  std::vector<char> done_edge;  // indexed by position in edge_labels
  done_edge.assign(edge_labels.size(), 0);
  auto mark_done = [&](int lab) {
    const size_t k = (size_t)(std::lower_bound(edge_labels.begin(), edge_labels.end(), lab) - edge_labels.begin());
    done_edge[k] = 1;
  };
  auto is_done = [&](int lab) {
    const size_t k = (size_t)(std::lower_bound(edge_labels.begin(), edge_labels.end(), lab) - edge_labels.begin());
    return done_edge[k] != 0;
  };
  auto emit = [&](tn_ncon_step st, Operand res) -> int {
    if (res.labels.size() > TN_MAX_RANK) return TN_ERR_UNSUPPORTED;
    st.rank = (int32_t)res.labels.size();
    for (size_t p = 0; p < res.dims.size(); ++p) st.shape[p] = res.dims[p];
    if (steps) {
      if (ns >= max_steps) return TN_ERR_ARG;
      steps[ns] = st;
    }
    res.id = n + ns;
    ++ns;
    ops.push_back(res);
    return TN_OK;
  };
  for (int lab : order) {
    if (is_done(lab)) continue;
    std::vector<size_t> where;
    for (size_t i = 0; i < ops.size(); ++i)
      if (find_leg(ops[i], lab) >= 0) where.push_back(i);
    tn_ncon_step st;
    memset(&st, 0, sizeof(st));
    Operand res;
    if (where.size() == 1) {  // a trace on one tensor
      const Operand a = ops[where[0]];
      const int i = find_leg(a, lab), j = find_leg(a, lab, i + 1);
      st.a = a.id;
      st.b = -1;
      st.nshared = 1;
      st.legs_a[0] = i;
      st.legs_b[0] = j;
      for (size_t p = 0; p < a.labels.size(); ++p)
        if ((int)p != i && (int)p != j) {
          res.labels.push_back(a.labels[p]);
          res.dims.push_back(a.dims[p]);
        }
      ops.erase(ops.begin() + (long)where[0]);
      mark_done(lab);
    } else {
      const Operand a = ops[where[0]], b = ops[where[1]];
      st.a = a.id;
      st.b = b.id;
      std::vector<char> a_shared(a.labels.size(), 0), b_shared(b.labels.size(), 0);
      for (size_t p = 0; p < a.labels.size(); ++p) {
        const int x = a.labels[p];
        if (x < 0) continue;
        const int q = find_leg(b, x);
        if (q < 0) continue;
        if (st.nshared >= TN_MAX_RANK) return TN_ERR_UNSUPPORTED;
        st.legs_a[st.nshared] = (int32_t)p;
        st.legs_b[st.nshared] = q;
        ++st.nshared;
        a_shared[p] = 1;
        b_shared[(size_t)q] = 1;
        mark_done(x);
      }
      for (size_t p = 0; p < a.labels.size(); ++p)
        if (!a_shared[p]) {
          res.labels.push_back(a.labels[p]);
          res.dims.push_back(a.dims[p]);
        }
      for (size_t p = 0; p < b.labels.size(); ++p)
        if (!b_shared[p]) {
          res.labels.push_back(b.labels[p]);
          res.dims.push_back(b.dims[p]);
        }
      ops.erase(ops.begin() + (long)where[1]);
      ops.erase(ops.begin() + (long)where[0]);
    }
    const int rc = emit(st, res);
    if (rc != TN_OK) return rc;
  }
  while (ops.size() > 1) {  // unconnected pieces: outer products in list order
    tn_ncon_step st;
    memset(&st, 0, sizeof(st));
    const Operand a = ops[0], b = ops[1];
    st.a = a.id;
    st.b = b.id;
    Operand res;
    res.labels = a.labels;
    res.dims = a.dims;
    res.labels.insert(res.labels.end(), b.labels.begin(), b.labels.end());
    res.dims.insert(res.dims.end(), b.dims.begin(), b.dims.end());
    ops.erase(ops.begin(), ops.begin() + 2);
    // the product goes to the front, so the next piece joins it in list order
    const int rc = emit(st, res);
    if (rc != TN_OK) return rc;
    Operand last = ops.back();
    ops.pop_back();
    ops.insert(ops.begin(), last);
  }
  const Operand& fin = ops[0];
  for (size_t i = 0; i < out.size(); ++i) out_perm[i] = find_leg(fin, out[i]);
  *out_rank = (int)out.size();
  *n_steps = ns;
  return TN_OK;
}
