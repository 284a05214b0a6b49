/*
 * Oracle for the tensor-network contraction path -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously correct FP64 CPU implementations of what the GPU
 * library computes. Only the tests, the smoke check and the bench's CPU
 * baseline use it; the library never links, loads or calls it, and it shares
 * no code with the library. Every array is dense row-major float64.
 *
 * Parity pins (checked by the CPU tests against mathematics, not against
 * this file): the elementary contractions of Sec. II (inner, matrix-vector,
 * matrix-matrix products and the trace), the ones(2).ones(2) = 2 example of
 * the edge-contraction subsection, the Hadamard chain of the connect
 * subsection, the outer-product shape rule, the ncon example of Appendix B,
 * flatten-then-contract equal to contract-then-trace, contraction-order
 * independence, brute-force 2^N state vectors, unit norm of left-canonical
 * MPS, transverse-field Ising closed forms, the identity-core closed form of
 * the classifier, and central finite differences of the classifier loss.
 */
#ifndef TN_ORACLE_H
#define TN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Pairwise tensordot (standard edges, Sec. III.A.3; contract_between, III.B.4):
 * C[free A legs in A's order, free B legs in B's order] =
 *   sum over shared indices of A[...] B[...], legsA[j] paired with legsB[j].
 * k = 0 gives the outer product (III.B.5). Returns 0, or -1 on bad arguments. */
int or_tensordot(const double* A, int ra, const int64_t* sha, const int* legsa,
                 const double* B, int rb, const int64_t* shb, const int* legsb,
                 int k, double* C);

/* Trace edge (III.A.3): sum_i A[.., i, .., i, ..] over legs l1 != l2 of equal
 * dim; the result keeps the other legs in order. Returns 0 or -1. */
int or_trace(const double* A, int r, const int64_t* sh, int l1, int l2, double* out);

/* <bra|ket> of two open-boundary MPS with cores (D_{i-1}, d, D_i) by the
 * left-to-right transfer sweep; E is rescaled by its max-abs entry after each
 * site. Result = value * exp(log_scale). Returns 0 or -1. */
int or_mps_inner(int n, int d, const int64_t* bond_bra, const double* const* bra,
                 const int64_t* bond_ket, const double* const* ket,
                 double* value, double* log_scale);

/* Brute-force state vector psi[s_1 .. s_N] (s_1 most significant, d^N entries)
 * of an MPS with D_0 = D_N = 1. Returns 0 or -1. */
int or_mps_state(int n, int d, const int64_t* bond, const double* const* cores, double* psi);

/* <psi|H|psi> for an MPS psi and an MPO H with cores W (w_{i-1}, w_i, s, s'),
 * w_0 = w_N = 1, by the left environment sweep L[a, w, a'] (a on the bra, a'
 * on the ket) in three steps per site. Result = value * exp(log_scale). */
int or_mpo_expect(int n, int d, const int64_t* bond, const double* const* cores,
                  const int64_t* wbond, const double* const* W,
                  double* value, double* log_scale);

/* <psi|H|psi> with H = -J sum_i Z_i Z_{i+1} - h sum_i X_i (open chain) applied
 * to a dense 2^n state vector (s_1 most significant; Z|0> = |0>). */
double or_tfim_energy_dense(int n, double J, double h, const double* psi);

/* MPS classifier (Sec. IV.A): feature map Phi(p) = (cos(pi p/2), sin(pi p/2)),
 * score_l = <Phi(x)|W_l>. W has n cores (D_{i-1}, 2, D_i), except the core at
 * label_site with shape (D, 2, L, D'). Outputs per sample the scores as
 * ftilde[b, l] * exp(lam[b]). Returns 0 or -1. */
int or_classify(int n, const int64_t* bond, const double* const* cores, int label_site, int L,
                const double* pixels, int batch, double* ftilde, double* lam);

/* Loss and gradient of the classifier: z = f / ||f||_2 per sample,
 * loss = mean_b CE(softmax(z_b), y_b). dcores has the cores' shapes. */
int or_classify_grad(int n, const int64_t* bond, const double* const* cores, int label_site, int L,
                     const double* pixels, int batch, const int64_t* labels,
                     double* loss, double* const* dcores);

/* Loss only (same definition), for finite differences. */
int or_classify_loss(int n, const int64_t* bond, const double* const* cores, int label_site, int L,
                     const double* pixels, int batch, const int64_t* labels, double* loss);

#ifdef __cplusplus
}
#endif
#endif
