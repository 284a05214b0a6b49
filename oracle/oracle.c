/*
 * Oracle for the tensor-network contraction path -- TEST INFRASTRUCTURE ONLY.
 * See oracle.h for the contract and the list of pins. Plain nested loops in
 * float64; OpenMP only splits independent outputs (result elements, samples)
 * across threads and never changes any summation order.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXR 16

static int64_t prod(const int64_t* v, int n) {
  int64_t p = 1;
  for (int i = 0; i < n; ++i) p *= v[i];
  return p;
}

/* Row-major strides of a shape. */
static void strides_of(const int64_t* sh, int r, int64_t* st) {
  int64_t s = 1;
  for (int i = r - 1; i >= 0; --i) {
    st[i] = s;
    s *= sh[i];
  }
}

/* ------------------------------------------------------------------------ */
/* Tensordot: Sec. III.A.3 (standard edge = numpy tensordot) and III.B.4      */
/* (contract_between flattens all shared edges into one, then contracts).     */
/* ------------------------------------------------------------------------ */
int or_tensordot(const double* A, int ra, const int64_t* sha, const int* legsa,
                 const double* B, int rb, const int64_t* shb, const int* legsb,
                 int k, double* C) {
  if (ra < 0 || rb < 0 || ra > OR_MAXR || rb > OR_MAXR || k < 0 || k > ra || k > rb) return -1;
  int useda[OR_MAXR] = {0}, usedb[OR_MAXR] = {0};
  for (int j = 0; j < k; ++j) {
    if (legsa[j] < 0 || legsa[j] >= ra || legsb[j] < 0 || legsb[j] >= rb) return -1;
    if (useda[legsa[j]] || usedb[legsb[j]]) return -1;
    if (sha[legsa[j]] != shb[legsb[j]]) return -1; /* "if the dimensions match" */
    useda[legsa[j]] = 1;
    usedb[legsb[j]] = 1;
  }
  int64_t sta[OR_MAXR], stb[OR_MAXR];
  strides_of(sha, ra, sta);
  strides_of(shb, rb, stb);

  /* Output legs: A's free legs in A's order, then B's free legs in B's order. */
  int nout = 0;
  int64_t odim[2 * OR_MAXR], ostride_in[2 * OR_MAXR];
  int oside[2 * OR_MAXR];
  for (int p = 0; p < ra; ++p)
    if (!useda[p]) { odim[nout] = sha[p]; ostride_in[nout] = sta[p]; oside[nout] = 0; ++nout; }
  for (int p = 0; p < rb; ++p)
    if (!usedb[p]) { odim[nout] = shb[p]; ostride_in[nout] = stb[p]; oside[nout] = 1; ++nout; }
  int64_t ncount = prod(odim, nout);

  /* Shared legs in the order given by legsa. */
  int64_t kdim[OR_MAXR], ksa[OR_MAXR], ksb[OR_MAXR];
  for (int j = 0; j < k; ++j) {
    kdim[j] = sha[legsa[j]];
    ksa[j] = sta[legsa[j]];
    ksb[j] = stb[legsb[j]];
  }
  int64_t kcount = prod(kdim, k);

#pragma omp parallel for schedule(static)
  for (int64_t o = 0; o < ncount; ++o) {
    /* Decode the output index (last leg fastest) into base offsets in A and B. */
    int64_t rem = o, offa = 0, offb = 0;
    for (int q = nout - 1; q >= 0; --q) {
      int64_t idx = rem % odim[q];
      rem /= odim[q];
      if (oside[q] == 0) offa += idx * ostride_in[q];
      else offb += idx * ostride_in[q];
    }
    /* Odometer over the shared indices, last shared leg fastest. */
    double acc = 0.0;
    for (int64_t t = 0; t < kcount; ++t) {
      int64_t r2 = t, ka = 0, kb = 0;
      for (int j = k - 1; j >= 0; --j) {
        int64_t idx = r2 % kdim[j];
        r2 /= kdim[j];
        ka += idx * ksa[j];
        kb += idx * ksb[j];
      }
      acc += A[offa + ka] * B[offb + kb];
    }
    C[o] = acc;
  }
  return 0;
}

/* Trace edge, Sec. III.A.3: sum over the diagonal of legs l1 and l2. */
int or_trace(const double* A, int r, const int64_t* sh, int l1, int l2, double* out) {
  if (r < 2 || r > OR_MAXR || l1 == l2 || l1 < 0 || l2 < 0 || l1 >= r || l2 >= r) return -1;
  if (sh[l1] != sh[l2]) return -1;
  int64_t st[OR_MAXR];
  strides_of(sh, r, st);
  int64_t odim[OR_MAXR], ost[OR_MAXR];
  int no = 0;
  for (int p = 0; p < r; ++p)
    if (p != l1 && p != l2) { odim[no] = sh[p]; ost[no] = st[p]; ++no; }
  int64_t n = prod(odim, no);
  for (int64_t o = 0; o < n; ++o) {
    int64_t rem = o, off = 0;
    for (int q = no - 1; q >= 0; --q) {
      off += (rem % odim[q]) * ost[q];
      rem /= odim[q];
    }
    double acc = 0.0;
    for (int64_t i = 0; i < sh[l1]; ++i) acc += A[off + i * st[l1] + i * st[l2]];
    out[o] = acc;
  }
  return 0;
}

/* Divide v[0..n) by its max-abs entry (if nonzero) and add log(max) to *lg. */
static void rescale(double* v, int64_t n, double* lg) {
  double m = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double a = fabs(v[i]);
    if (a > m) m = a;
  }
  if (m > 0.0) {
    for (int64_t i = 0; i < n; ++i) v[i] /= m;
    *lg += log(m);
  }
}

/* ------------------------------------------------------------------------ */
/* MPS inner product <bra|ket> (MPS network, Sec. II): left environment        */
/* E_i[b,b'] = sum_{a,a',s} E_{i-1}[a,a'] bra_i[a,s,b] ket_i[a',s,b'], done    */
/* as T[a,s,b'] = sum_a' E[a,a'] ket[a',s,b'], then E'[b,b'] =                */
/* sum_{a,s} bra[a,s,b] T[a,s,b'].                                              */
/* ------------------------------------------------------------------------ */
int or_mps_inner(int n, int d, const int64_t* bond_bra, const double* const* bra,
                 const int64_t* bond_ket, const double* const* ket,
                 double* value, double* log_scale) {
  if (n < 1 || d < 1) return -1;
  if (bond_bra[0] != 1 || bond_ket[0] != 1 || bond_bra[n] != 1 || bond_ket[n] != 1) return -1;
  int64_t maxd = 1;
  for (int i = 0; i <= n; ++i) {
    if (bond_bra[i] > maxd) maxd = bond_bra[i];
    if (bond_ket[i] > maxd) maxd = bond_ket[i];
  }
  double* E = (double*)calloc((size_t)(maxd * maxd), sizeof(double));
  double* E2 = (double*)calloc((size_t)(maxd * maxd), sizeof(double));
  double* T = (double*)calloc((size_t)(maxd * d * maxd), sizeof(double));
  if (!E || !E2 || !T) { free(E); free(E2); free(T); return -1; }
  E[0] = 1.0;
  double lg = 0.0;
  for (int i = 0; i < n; ++i) {
    const int64_t Da = bond_bra[i], Db = bond_bra[i + 1], Dak = bond_ket[i], Dbk = bond_ket[i + 1];
    const double* Ab = bra[i];
    const double* Ak = ket[i];
#pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < Da; ++a)
      for (int s = 0; s < d; ++s)
        for (int64_t bk = 0; bk < Dbk; ++bk) {
          double acc = 0.0;
          for (int64_t ak = 0; ak < Dak; ++ak) acc += E[a * Dak + ak] * Ak[(ak * d + s) * Dbk + bk];
          T[(a * d + s) * Dbk + bk] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < Db; ++b)
      for (int64_t bk = 0; bk < Dbk; ++bk) {
        double acc = 0.0;
        for (int64_t a = 0; a < Da; ++a)
          for (int s = 0; s < d; ++s) acc += Ab[(a * d + s) * Db + b] * T[(a * d + s) * Dbk + bk];
        E2[b * Dbk + bk] = acc;
      }
    double* t = E; E = E2; E2 = t;
    rescale(E, Db * Dbk, &lg);
  }
  *value = E[0];
  *log_scale = lg;
  free(E); free(E2); free(T);
  return 0;
}

/* Brute force: psi(s_1..s_N) = A_1[s_1] A_2[s_2] ... A_N[s_N] (1x1 at the end). */
int or_mps_state(int n, int d, const int64_t* bond, const double* const* cores, double* psi) {
  if (n < 1 || d < 1 || bond[0] != 1 || bond[n] != 1) return -1;
  /* cur[(prefix index) * D_i + b], prefix over s_1..s_i with s_1 most significant */
  int64_t count = 1;
  double* cur = (double*)malloc(sizeof(double));
  if (!cur) return -1;
  cur[0] = 1.0;
  for (int i = 0; i < n; ++i) {
    const int64_t Da = bond[i], Db = bond[i + 1];
    double* nxt = (double*)malloc(sizeof(double) * (size_t)(count * d * Db));
    if (!nxt) { free(cur); return -1; }
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < count; ++p)
      for (int s = 0; s < d; ++s)
        for (int64_t b = 0; b < Db; ++b) {
          double acc = 0.0;
          for (int64_t a = 0; a < Da; ++a) acc += cur[p * Da + a] * cores[i][(a * d + s) * Db + b];
          nxt[(p * d + s) * Db + b] = acc;
        }
    free(cur);
    cur = nxt;
    count *= d;
  }
  memcpy(psi, cur, sizeof(double) * (size_t)count);
  free(cur);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* <psi|H|psi> by the MPO left-environment sweep, three steps per site:       */
/*  (i)   T1[w,a',s,b]  = sum_a L[a,w,a'] A[a,s,b]                              */
/*  (ii)  T2[w',s',a',b] = sum_{w,s} T1[w,a',s,b] W[w,w',s,s']                  */
/*  (iii) L'[b,w',b']   = sum_{a',s'} T2[w',s',a',b] A[a',s',b']                 */
/* ------------------------------------------------------------------------ */
int or_mpo_expect(int n, int d, const int64_t* bond, const double* const* cores,
                  const int64_t* wbond, const double* const* W,
                  double* value, double* log_scale) {
  if (n < 1 || d < 1 || bond[0] != 1 || bond[n] != 1 || wbond[0] != 1 || wbond[n] != 1) return -1;
  int64_t maxd = 1, maxw = 1;
  for (int i = 0; i <= n; ++i) {
    if (bond[i] > maxd) maxd = bond[i];
    if (wbond[i] > maxw) maxw = wbond[i];
  }
  size_t nl = (size_t)(maxd * maxw * maxd), nt = (size_t)(maxw * maxd * d * maxd);
  double* L = (double*)calloc(nl, sizeof(double));
  double* L2 = (double*)calloc(nl, sizeof(double));
  double* T1 = (double*)calloc(nt, sizeof(double));
  double* T2 = (double*)calloc(nt, sizeof(double));
  if (!L || !L2 || !T1 || !T2) { free(L); free(L2); free(T1); free(T2); return -1; }
  L[0] = 1.0;
  double lg = 0.0;
  for (int i = 0; i < n; ++i) {
    const int64_t Da = bond[i], Db = bond[i + 1], wa = wbond[i], wb = wbond[i + 1];
    const double* A = cores[i];
    const double* Wi = W[i];
    /* (i) */
#pragma omp parallel for schedule(static)
    for (int64_t w = 0; w < wa; ++w)
      for (int64_t ak = 0; ak < Da; ++ak)
        for (int s = 0; s < d; ++s)
          for (int64_t b = 0; b < Db; ++b) {
            double acc = 0.0;
            for (int64_t a = 0; a < Da; ++a) acc += L[(a * wa + w) * Da + ak] * A[(a * d + s) * Db + b];
            T1[((w * Da + ak) * d + s) * Db + b] = acc;
          }
    /* (ii) */
#pragma omp parallel for schedule(static)
    for (int64_t w2 = 0; w2 < wb; ++w2)
      for (int s2 = 0; s2 < d; ++s2)
        for (int64_t ak = 0; ak < Da; ++ak)
          for (int64_t b = 0; b < Db; ++b) {
            double acc = 0.0;
            for (int64_t w = 0; w < wa; ++w)
              for (int s = 0; s < d; ++s)
                acc += T1[((w * Da + ak) * d + s) * Db + b] * Wi[((w * wb + w2) * d + s) * d + s2];
            T2[((w2 * d + s2) * Da + ak) * Db + b] = acc;
          }
    /* (iii) */
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < Db; ++b)
      for (int64_t w2 = 0; w2 < wb; ++w2)
        for (int64_t bk = 0; bk < Db; ++bk) {
          double acc = 0.0;
          for (int64_t ak = 0; ak < Da; ++ak)
            for (int s2 = 0; s2 < d; ++s2)
              acc += T2[((w2 * d + s2) * Da + ak) * Db + b] * A[(ak * d + s2) * Db + bk];
          L2[(b * wb + w2) * Db + bk] = acc;
        }
    double* t = L; L = L2; L2 = t;
    rescale(L, Db * wb * Db, &lg);
  }
  *value = L[0];
  *log_scale = lg;
  free(L); free(L2); free(T1); free(T2);
  return 0;
}

/* H = -J sum Z_i Z_{i+1} - h sum X_i on a dense state; bit (n-1-i) of the
 * basis index is site i's spin, 0 -> Z = +1. */
double or_tfim_energy_dense(int n, double J, double h, const double* psi) {
  const int64_t dim = (int64_t)1 << n;
  double e = 0.0;
#pragma omp parallel for reduction(+ : e) schedule(static)
  for (int64_t x = 0; x < dim; ++x) {
    double diag = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
      int zi = ((x >> (n - 1 - i)) & 1) ? -1 : 1;
      int zj = ((x >> (n - 2 - i)) & 1) ? -1 : 1;
      diag += -J * zi * zj;
    }
    double hpsi = diag * psi[x];
    for (int i = 0; i < n; ++i) hpsi += -h * psi[x ^ ((int64_t)1 << (n - 1 - i))];
    e += psi[x] * hpsi;
  }
  return e;
}

/* ------------------------------------------------------------------------ */
/* MPS classifier, Sec. IV.A.                                                 */
/* ------------------------------------------------------------------------ */
static void feature(double p, double* phi) {
  /* local feature map Phi(p) = (cos(pi p / 2), sin(pi p / 2)) */
  phi[0] = cos(M_PI * p / 2.0);
  phi[1] = sin(M_PI * p / 2.0);
}

/* Per-sample forward state kept for the gradient. */
typedef struct {
  double** vl;  /* vl[i]: normalised left vector after sites 0..i-1 (size D_i), i = 0..ls */
  double* lamv; /* lamv[i]: its log-scale */
  double** ur;  /* ur[i]: normalised right vector after sites i..n-1 (size D_i), i = ls+1..n */
  double* lamu;
} fwd_state;

static int max_bond(int n, const int64_t* bond) {
  int64_t m = 1;
  for (int i = 0; i <= n; ++i)
    if (bond[i] > m) m = bond[i];
  return (int)m;
}

/* Sweeps one sample; if st != NULL, keeps every intermediate vector. */
static void classify_one(int n, const int64_t* bond, const double* const* cores, int ls, int L,
                         const double* x, double* ft, double* lam, fwd_state* st) {
  const int md = max_bond(n, bond);
  double* v = (double*)calloc((size_t)md, sizeof(double));
  double* v2 = (double*)calloc((size_t)md, sizeof(double));
  double lv = 0.0, lu = 0.0, phi[2];
  v[0] = 1.0;
  if (st) { memcpy(st->vl[0], v, sizeof(double)); st->lamv[0] = 0.0; }
  /* left half: v'[b] = sum_{a,s} v[a] phi_s A[a,s,b] */
  for (int i = 0; i < ls; ++i) {
    const int64_t Da = bond[i], Db = bond[i + 1];
    feature(x[i], phi);
    for (int64_t b = 0; b < Db; ++b) {
      double acc = 0.0;
      for (int64_t a = 0; a < Da; ++a)
        for (int s = 0; s < 2; ++s) acc += v[a] * phi[s] * cores[i][(a * 2 + s) * Db + b];
      v2[b] = acc;
    }
    double* t = v; v = v2; v2 = t;
    rescale(v, Db, &lv);
    if (st) { memcpy(st->vl[i + 1], v, sizeof(double) * (size_t)Db); st->lamv[i + 1] = lv; }
  }
  /* right half: u'[a] = sum_{s,b} A[a,s,b] phi_s u[b] */
  double* u = (double*)calloc((size_t)md, sizeof(double));
  double* u2 = (double*)calloc((size_t)md, sizeof(double));
  u[0] = 1.0;
  if (st) { memcpy(st->ur[n], u, sizeof(double)); st->lamu[n] = 0.0; }
  for (int i = n - 1; i > ls; --i) {
    const int64_t Da = bond[i], Db = bond[i + 1];
    feature(x[i], phi);
    for (int64_t a = 0; a < Da; ++a) {
      double acc = 0.0;
      for (int s = 0; s < 2; ++s)
        for (int64_t b = 0; b < Db; ++b) acc += cores[i][(a * 2 + s) * Db + b] * phi[s] * u[b];
      u2[a] = acc;
    }
    double* t = u; u = u2; u2 = t;
    rescale(u, Da, &lu);
    if (st) { memcpy(st->ur[i], u, sizeof(double) * (size_t)Da); st->lamu[i] = lu; }
  }
  /* label core: f_l = sum_{a,s,b} v[a] C[a,s,l,b] phi_s u[b] */
  {
    const int64_t Da = bond[ls], Db = bond[ls + 1];
    feature(x[ls], phi);
    for (int l = 0; l < L; ++l) {
      double acc = 0.0;
      for (int64_t a = 0; a < Da; ++a)
        for (int s = 0; s < 2; ++s)
          for (int64_t b = 0; b < Db; ++b)
            acc += v[a] * cores[ls][((a * 2 + s) * L + l) * Db + b] * phi[s] * u[b];
      ft[l] = acc;
    }
  }
  *lam = lv + lu;
  free(v); free(v2); free(u); free(u2);
}

int or_classify(int n, const int64_t* bond, const double* const* cores, int label_site, int L,
                const double* pixels, int batch, double* ftilde, double* lam) {
  if (n < 1 || label_site < 0 || label_site >= n || L < 1 || batch < 0) return -1;
  if (bond[0] != 1 || bond[n] != 1) return -1;
#pragma omp parallel for schedule(dynamic, 4)
  for (int b = 0; b < batch; ++b)
    classify_one(n, bond, cores, label_site, L, pixels + (int64_t)b * n, ftilde + (int64_t)b * L,
                 lam + b, NULL);
  return 0;
}

/* Loss of one sample from its scores ftilde (the scale exp(lam) cancels in
 * z = f / ||f||): CE(softmax(z), y) = logsumexp(z) - z_y. If dz != NULL,
 * writes dLoss/dftilde (for the unit-weight sample) into dz. */
static double sample_loss(const double* ft, int L, int64_t y, double* dft) {
  double nrm = 0.0;
  for (int l = 0; l < L; ++l) nrm += ft[l] * ft[l];
  nrm = sqrt(nrm);
  double z[64], p[64];
  double zmax = -1e300;
  for (int l = 0; l < L; ++l) {
    z[l] = ft[l] / nrm;
    if (z[l] > zmax) zmax = z[l];
  }
  double se = 0.0;
  for (int l = 0; l < L; ++l) { p[l] = exp(z[l] - zmax); se += p[l]; }
  for (int l = 0; l < L; ++l) p[l] /= se;
  double loss = zmax + log(se) - z[y];
  if (dft) {
    /* g_z = softmax(z) - onehot(y);  dL/dftilde = (g_z - z (z . g_z)) / ||ftilde|| */
    double gz[64], zg = 0.0;
    for (int l = 0; l < L; ++l) {
      gz[l] = p[l] - (l == y ? 1.0 : 0.0);
      zg += z[l] * gz[l];
    }
    for (int l = 0; l < L; ++l) dft[l] = (gz[l] - z[l] * zg) / nrm;
  }
  return loss;
}

int or_classify_loss(int n, const int64_t* bond, const double* const* cores, int label_site, int L,
                     const double* pixels, int batch, const int64_t* labels, double* loss) {
  if (L > 64 || batch < 1) return -1;
  double* ft = (double*)malloc(sizeof(double) * (size_t)batch * L);
  double* lam = (double*)malloc(sizeof(double) * (size_t)batch);
  int rc = or_classify(n, bond, cores, label_site, L, pixels, batch, ft, lam);
  if (rc == 0) {
    double acc = 0.0;
    for (int b = 0; b < batch; ++b) acc += sample_loss(ft + (int64_t)b * L, L, labels[b], NULL);
    *loss = acc / batch;
  }
  free(ft); free(lam);
  return rc;
}

/* Analytic gradient. With v_i = vl_i exp(lamv_i) the true left vectors and
 * u_i = ur_i exp(lamu_i) the true right vectors, and f = ftilde exp(Lam):
 *   dLoss/df = exp(-Lam) delta,  delta = dLoss/dftilde as if ftilde were f;
 *   dLoss/dv_{ls} = exp(-lamv_ls) g,  g[a] = sum_l delta_l sum_{s,b} C[a,s,l,b] phi_s ur[b];
 *   going left, g_{i}[a] = exp(lamv_i - lamv_{i+1}) sum_{s,c} A_i[a,s,c] phi_s g_{i+1}[c],
 *   and dA_i[a,s,c] += exp(lamv_i - lamv_{i+1}) vl_i[a] phi_s g_{i+1}[c];
 * mirrored on the right; dC[a,s,l,b] += delta_l vl_ls[a] phi_s ur_{ls+1}[b]. */
int or_classify_grad(int n, const int64_t* bond, const double* const* cores, int label_site, int L,
                     const double* pixels, int batch, const int64_t* labels,
                     double* loss, double* const* dcores) {
  if (n < 1 || label_site < 0 || label_site >= n || L < 1 || L > 64 || batch < 1) return -1;
  if (bond[0] != 1 || bond[n] != 1) return -1;
  const int ls = label_site;
  const int md = max_bond(n, bond);
  int64_t csize[4096];
  if (n > 4096) return -1;
  for (int i = 0; i < n; ++i) {
    csize[i] = bond[i] * 2 * bond[i + 1] * (i == ls ? L : 1);
    memset(dcores[i], 0, sizeof(double) * (size_t)csize[i]);
  }
  double total = 0.0;
  const double invb = 1.0 / batch;
  /* Samples are independent; each thread accumulates into private gradients. */
#pragma omp parallel reduction(+ : total)
  {
    double** dloc = (double**)malloc(sizeof(double*) * (size_t)n);
    for (int i = 0; i < n; ++i) dloc[i] = (double*)calloc((size_t)csize[i], sizeof(double));
    fwd_state st;
    st.vl = (double**)malloc(sizeof(double*) * (size_t)(n + 1));
    st.ur = (double**)malloc(sizeof(double*) * (size_t)(n + 1));
    st.lamv = (double*)calloc((size_t)(n + 1), sizeof(double));
    st.lamu = (double*)calloc((size_t)(n + 1), sizeof(double));
    for (int i = 0; i <= n; ++i) {
      st.vl[i] = (double*)calloc((size_t)md, sizeof(double));
      st.ur[i] = (double*)calloc((size_t)md, sizeof(double));
    }
    double* g = (double*)calloc((size_t)md, sizeof(double));
    double* g2 = (double*)calloc((size_t)md, sizeof(double));
    double ft[64], dft[64], lam, phi[2];
#pragma omp for schedule(dynamic, 4)
    for (int bi = 0; bi < batch; ++bi) {
      const double* x = pixels + (int64_t)bi * n;
      classify_one(n, bond, cores, ls, L, x, ft, &lam, &st);
      total += sample_loss(ft, L, labels[bi], dft) * invb;
      for (int l = 0; l < L; ++l) dft[l] *= invb;
      const double* vl = st.vl[ls];
      const double* ur = st.ur[ls + 1];
      const int64_t Dl = bond[ls], Dr = bond[ls + 1];
      const double* C = cores[ls];
      feature(x[ls], phi);
      /* label core gradient */
      for (int64_t a = 0; a < Dl; ++a)
        for (int s = 0; s < 2; ++s)
          for (int l = 0; l < L; ++l)
            for (int64_t b = 0; b < Dr; ++b)
              dloc[ls][((a * 2 + s) * L + l) * Dr + b] += dft[l] * vl[a] * phi[s] * ur[b];
      /* left side */
      for (int64_t a = 0; a < Dl; ++a) {
        double acc = 0.0;
        for (int s = 0; s < 2; ++s)
          for (int l = 0; l < L; ++l)
            for (int64_t b = 0; b < Dr; ++b) acc += dft[l] * C[((a * 2 + s) * L + l) * Dr + b] * phi[s] * ur[b];
        g[a] = acc;
      }
      for (int i = ls - 1; i >= 0; --i) {
        const int64_t Da = bond[i], Db = bond[i + 1];
        const double f = exp(st.lamv[i] - st.lamv[i + 1]);
        feature(x[i], phi);
        for (int64_t a = 0; a < Da; ++a)
          for (int s = 0; s < 2; ++s)
            for (int64_t c = 0; c < Db; ++c) dloc[i][(a * 2 + s) * Db + c] += f * st.vl[i][a] * phi[s] * g[c];
        for (int64_t a = 0; a < Da; ++a) {
          double acc = 0.0;
          for (int s = 0; s < 2; ++s)
            for (int64_t c = 0; c < Db; ++c) acc += cores[i][(a * 2 + s) * Db + c] * phi[s] * g[c];
          g2[a] = f * acc;
        }
        double* t = g; g = g2; g2 = t;
      }
      /* right side: h[b] = dLoss/du_{ls+1} without its scale */
      feature(x[ls], phi);
      for (int64_t b = 0; b < Dr; ++b) {
        double acc = 0.0;
        for (int64_t a = 0; a < Dl; ++a)
          for (int s = 0; s < 2; ++s)
            for (int l = 0; l < L; ++l) acc += dft[l] * vl[a] * C[((a * 2 + s) * L + l) * Dr + b] * phi[s];
        g[b] = acc;
      }
      for (int i = ls + 1; i < n; ++i) {
        const int64_t Da = bond[i], Db = bond[i + 1];
        const double f = exp(st.lamu[i + 1] - st.lamu[i]);
        feature(x[i], phi);
        for (int64_t a = 0; a < Da; ++a)
          for (int s = 0; s < 2; ++s)
            for (int64_t c = 0; c < Db; ++c) dloc[i][(a * 2 + s) * Db + c] += f * g[a] * phi[s] * st.ur[i + 1][c];
        for (int64_t c = 0; c < Db; ++c) {
          double acc = 0.0;
          for (int64_t a = 0; a < Da; ++a)
            for (int s = 0; s < 2; ++s) acc += g[a] * phi[s] * cores[i][(a * 2 + s) * Db + c];
          g2[c] = f * acc;
        }
        double* t = g; g = g2; g2 = t;
      }
    }
#pragma omp critical
    for (int i = 0; i < n; ++i)
      for (int64_t e = 0; e < csize[i]; ++e) dcores[i][e] += dloc[i][e];
    for (int i = 0; i < n; ++i) free(dloc[i]);
    free(dloc);
    for (int i = 0; i <= n; ++i) { free(st.vl[i]); free(st.ur[i]); }
    free(st.vl); free(st.ur); free(st.lamv); free(st.lamu); free(g); free(g2);
  }
  *loss = total;
  return 0;
}
