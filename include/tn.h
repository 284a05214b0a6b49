/*
 * tn.h -- C ABI of the GB300 tensor-network contraction library (libtn.so).
 *
 * The library contracts tensor networks edge by edge on one NVIDIA GB300
 * (sm_103a): a pairwise tensordot of two nodes over their shared legs
 * (TensorNetwork paper, Sec. III.A.3 "Standard Edges" and III.B.4
 * "contract_between", which flattens all edges between two nodes into one
 * before contracting, Sec. III.B.2), driven along matrix product state (MPS)
 * chains (Sec. II, Fig. 3a) as environment sweeps, and the MPS image
 * classifier of Sec. IV.A.
 *
 * Conventions shared by every entry point
 *  - All tensor data pointers are DEVICE pointers owned by the caller; the
 *    library never frees or keeps them. Scalars documented as "device" are
 *    device pointers too. Host arrays (shapes, leg lists, pointer tables) are
 *    read during the call only.
 *  - Dense float32 tensors, strides in elements. A tensor whose strides are
 *    all zero is read as row-major contiguous.
 *  - Legs are 0-based (the paper's a[0], get_edge(0)).
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *    default stream). A nonzero return means nothing was launched. Errors
 *    raised inside a kernel (a bounded wait that expired) are recorded in a
 *    device status word, read and cleared by tn_sync_status().
 *  - No entry point allocates device memory: scratch space is a caller
 *    buffer whose size the matching *_workspace_bytes call returns.
 */
#ifndef TN_H
#define TN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TN_MAX_RANK 8

/* Status codes. */
enum {
  TN_OK = 0,
  TN_ERR_ARG = 1,         /* null pointer, rank > 8, leg out of range or repeated, bad count */
  TN_ERR_SHAPE = 2,       /* paired legs differ in dimension (the paper's "if the dimensions
                             match", Sec. II), or an output shape that is not the result's */
  TN_ERR_UNSUPPORTED = 3, /* valid request outside what the kernels implement (dtype, layout) */
  TN_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  TN_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired (kernel returned early) */
  TN_ERR_WORKSPACE = 6    /* workspace missing, misaligned (256 B) or too small */
};

/* Element types. */
enum { TN_F32 = 0 };

/* Arithmetic of a contraction. Inputs and outputs stay float32 in memory. */
enum {
  TN_PREC_FP32 = 0,  /* float32 FMA on the CUDA cores */
  TN_PREC_BF16 = 1,  /* operands rounded to bfloat16 (nearest-even), float32
                        accumulation on the tcgen05 tensor cores */
  TN_PREC_BF16X3 = 2 /* split bfloat16: x = hi + lo with hi = bf16(x),
                        lo = bf16(x - hi); A*B ~ Ahi*Bhi + Ahi*Blo + Alo*Bhi,
                        all three on tcgen05 into one float32 accumulator */
};

/* A dense tensor (a node's array, Sec. III.A.2). */
typedef struct tn_tensor {
  void* data;                     /* device pointer */
  int32_t rank;                   /* 0 .. TN_MAX_RANK; rank 0 is a scalar */
  int32_t dtype;                  /* TN_F32 */
  int64_t shape[TN_MAX_RANK];     /* dims; entries past rank ignored */
  int64_t stride[TN_MAX_RANK];    /* element strides, or all zero for row-major */
} tn_tensor;

/* Fills t as a row-major float32 tensor. Returns TN_OK or TN_ERR_ARG. */
int tn_tensor_init(tn_tensor* t, void* data, int rank, const int64_t* shape);

/* ------------------------------------------------------------------------ */
/* Pairwise tensordot (Sec. III.A.3, III.B.4; numpy tensordot semantics)     */
/* ------------------------------------------------------------------------ */
/*
 * C[f_A..., f_B...] = sum over the shared legs of A[...] * B[...], where leg
 * legsA[j] of A is connected to leg legsB[j] of B (j < nshared). The result's
 * legs are A's free legs in A's order followed by B's free legs in B's order;
 * nshared = 0 is the outer product (Sec. III.B.5). All shared legs are merged
 * into one contraction index (edge flattening, Sec. III.B.2) without moving
 * data: leg permutations are folded into the kernels' operand gathers, so no
 * transposed copy is ever made.
 *   A, B   input tensors (float32, any strides)
 *   legsA, legsB  host arrays of nshared leg indices (may be NULL if nshared = 0)
 *   C      output tensor: float32, row-major contiguous, shape as above; it
 *          must not overlap A or B
 *   prec   TN_PREC_FP32 / TN_PREC_BF16 / TN_PREC_BF16X3
 * Errors: TN_ERR_ARG, TN_ERR_SHAPE, TN_ERR_UNSUPPORTED, TN_ERR_CUDA.
 */
int tn_contract(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                int nshared, const tn_tensor* C, int prec, void* stream);

/*
 * tn_contract with scratch space: BF16 / BF16X3 contractions then run as two
 * launches, a pack of both operands into bf16 blocks (in `workspace`) and the
 * warp-specialised tcgen05 GEMM that reads them (the path of the grouped
 * launch; much faster on large contractions than tn_contract's single-pass
 * kernel, which converts every operand tile once per output tile). Both
 * launches take their lists by value, so the call can be captured in a graph.
 *   workspace: DEVICE scratch, 256-byte aligned, at least
 *     tn_contract_workspace_bytes() bytes (0 for FP32 and empty contractions),
 *     or NULL to run tn_contract's kernels.
 * Errors: as tn_contract, plus TN_ERR_WORKSPACE (misaligned or too small).
 */
size_t tn_contract_workspace_bytes(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB,
                                   int nshared, const tn_tensor* C, int prec);
int tn_contract_ws(const tn_tensor* A, const int* legsA, const tn_tensor* B, const int* legsB, int nshared,
                   const tn_tensor* C, int prec, void* workspace, size_t bytes, void* stream);

/* One pairwise contraction of a grouped launch. */
typedef struct tn_contract_spec {
  tn_tensor A, B, C;
  int32_t nshared;
  int32_t legsA[TN_MAX_RANK];
  int32_t legsB[TN_MAX_RANK];
} tn_contract_spec;

/*
 * Grouped contraction: many tensordots of uneven shapes in one persistent
 * launch. A plan validates and lays out the specs once (host), its device
 * work list is uploaded into a caller workspace, and each run launches one
 * kernel over all output tiles, largest contractions first.
 *   tn_group_plan_create: specs (host array, read during the call), prec;
 *     returns TN_OK and *plan, or the first spec's error (*plan = NULL).
 *   tn_group_plan_workspace_bytes: device bytes the plan's work list needs.
 *   tn_group_plan_upload: copies the work list into `workspace` (device,
 *     256-byte aligned, at least the size above) on `stream`, from host
 *     lists that a captured copy could not replay: on a stream being
 *     captured into a CUDA graph it returns TN_ERR_UNSUPPORTED (upload
 *     before capturing; tn_group_plan_run itself only launches).
 *   tn_group_plan_run: launches the contractions; `workspace` must hold the
 *     uploaded work list (uploads and runs are ordered on the stream).
 *   tn_group_plan_destroy: frees the host plan (never device memory).
 * Errors: as tn_contract, plus TN_ERR_WORKSPACE.
 */
typedef struct tn_group_plan tn_group_plan;
int tn_group_plan_create(const tn_contract_spec* specs, int nspecs, int prec, tn_group_plan** plan);
size_t tn_group_plan_workspace_bytes(const tn_group_plan* plan);
int tn_group_plan_upload(const tn_group_plan* plan, void* workspace, size_t bytes, void* stream);
int tn_group_plan_run(const tn_group_plan* plan, void* workspace, size_t bytes, void* stream);
void tn_group_plan_destroy(tn_group_plan* plan);
/*
 * Grouped contraction that allocates nothing: the same results as a plan's
 * create + upload + run, computed by the single-pass grouped kernels (the
 * tcgen05 kernel for BF16 / BF16X3, the SIMT kernel for FP32; not the pack +
 * GEMM launches or the small-first-operand FP32 kernel a plan may choose, so
 * speed and rounding order can differ from a plan's), with the work list kept
 * in a fixed 4 MiB array inside the library instead of a caller workspace. (The
 * paper has no counterpart; this is a convenience of the library.) It is for
 * callers that must not call cudaMalloc: code whose device memory all belongs
 * to another framework's pool, where an extra cudaMalloc can exceed the
 * pool's budget and synchronises the device, and code on a latency-bound path
 * that may only launch kernels.
 *   specs, nspecs, prec: as tn_group_plan_create; at most 4096 specs, and
 *     the work list (464 bytes per spec, 16 per split result, 4 per work
 *     unit: one 128x128 output tile over at most 2048 shared indices) must
 *     fit in the 4 MiB array; larger requests return TN_ERR_UNSUPPORTED and
 *     launch nothing.
 *   The first call on a device looks up the array's device address there
 *   (cudaGetSymbolAddress). A call on a stream that is being captured into a
 *   CUDA graph returns TN_ERR_UNSUPPORTED and enqueues nothing: the work list
 *   is copied from host staging arrays that the next call overwrites, so a
 *   captured copy would replay another call's work list.
 *   Every GPU that loads libtn.so holds the array until the process exits.
 *   All calls share the array: calls whose work overlaps on the GPU (other
 *   streams or host threads) race on it; calls on one stream are ordered.
 *   The work list goes to the array in three copies from the library's
 *   pageable host staging arrays; a copy from pageable memory may block the
 *   calling thread until the stream's earlier work has finished.
 * Errors: as tn_group_plan_create, plus TN_ERR_UNSUPPORTED (too large, or
 * the stream is capturing) and TN_ERR_CUDA.
 */
int tn_contract_grouped_static(const tn_contract_spec* specs, int nspecs, int prec, void* stream);

/* Total floating-point work (2 M N K summed over specs) and algorithmic bytes
 * (|A| + |B| + |C| float32 elements summed over specs) of a plan. */
double tn_group_plan_flops(const tn_group_plan* plan);
double tn_group_plan_bytes(const tn_group_plan* plan);
/* Kernel launches one tn_group_plan_run makes: [a zeroing kernel, when some
 * results are accumulated over split k ranges] [the pack kernel, for BF16 /
 * BF16X3 plans] and the contraction kernel -- for BF16 / BF16X3 plans the
 * GEMM on packed operands and / or, for BF16 contractions whose narrower
 * operand has at most 64 rows, a fused GEMM that reads the wider operand as
 * float32 and rounds it to bf16 in shared memory (it is read by exactly one
 * work unit, so it is never packed): the TMA one, which loads each tile of
 * it as one box of a tensor map over its legs (the leg permutation done by
 * the copy), when the operand is in device memory with a unit-stride last
 * free or shared leg, at most five legs longer than 1 and 16-byte strides,
 * else the one whose warps copy it element-wise through offset tables. */
int tn_group_plan_launches(const tn_group_plan* plan);
/* Runs launch `index` (0 .. launches-1) of that sequence alone, so each can
 * be timed by itself; running them all in order is one tn_group_plan_run.
 * Errors: TN_ERR_ARG (index out of range), as tn_group_plan_run. */
int tn_group_plan_run_launch(const tn_group_plan* plan, void* workspace, size_t bytes, int index, void* stream);
/* "zero", "pack", "gemm" (packed bf16 blocks), "gemm_fused" (wider operand
 * copied through offset tables and rounded inside the GEMM), "gemm_tma"
 * (wider operand loaded in tensor-map boxes and rounded inside the GEMM) or
 * "contract" (single-pass kernel) for launch `index`; NULL when out of
 * range. */
const char* tn_group_plan_launch_name(const tn_group_plan* plan, int index);
/* Algorithmic bytes of launch `index`: what it must move at the least, each
 * operand element read once and each result written once -- zero: 4 B per
 * zeroed result; pack: 4 B read + 2 B (BF16) or 4 B (BF16X3, hi and lo)
 * written per packed operand element; gemm: 2 B (4 B) per packed operand
 * element + 4 B per result; gemm_fused and gemm_tma: 4 B per element of the
 * float32 operand + 2 B per packed element + 4 B per result; contract: 4 B per
 * operand element and per result. -1 when `index` is out of range. */
double tn_group_plan_launch_bytes(const tn_group_plan* plan, int index);
/*
 * Autotuner of a BF16 / BF16X3 plan's GEMM schedule (the paper has no
 * counterpart; its contractions run through TensorFlow). The contractions
 * fall in three classes, tuned one after the other: 0 thin (fewer than 128
 * rows on one side), 1 short shared index (K <= 512), 2 the rest. For each
 * class the candidates are the output tile width (128 or 64 rows of the
 * narrower operand per tile, and for BF16 classes 1 and 2 also 256: each
 * block of the wider operand then feeds 256 result columns), the
 * epilogue's tensor-memory read shape (one
 * row per thread, or 16-lane x 256-bit blocks whose stores cover whole
 * 32-byte sectors), and, for class 2, whether a contraction with at least 16
 * output tiles keeps each tile's whole k range in one work unit or cuts it
 * into 2048-long ranges accumulated with atomics. Each candidate runs on the
 * device with the plan's own operands (one warm-up run, two timed with CUDA
 * events) and the fastest is kept; the choice is also stored in a host-side
 * cache inside the library, keyed by precision and the contractions' shapes,
 * from which later plans of the same shapes start.
 *   workspace: the plan's workspace (any schedule fits it); on return the
 *     plan is uploaded there with the chosen schedule.
 *   The call runs the contractions (results are written, correctly, several
 *   times) and synchronises `stream`; it cannot be captured in a graph.
 *   FP32 plans have nothing to tune: TN_OK, nothing launched.
 * Errors: as tn_group_plan_run.
 */
int tn_group_plan_autotune(tn_group_plan* plan, void* workspace, size_t bytes, void* stream);
/* The schedule a plan runs for class `cls` (0, 1, 2 as above): the output
 * tile width (64, 128 or 256), whether long k ranges are kept whole, and whether
 * the epilogue reads 16-lane x 256-bit blocks. Errors: TN_ERR_ARG. */
int tn_group_plan_schedule(const tn_group_plan* plan, int cls, int* tile_width, int* long_k, int* store16);
/* Sets that schedule by hand (tile_width 64, 128, or 256 for BF16 plans);
 * the plan must be uploaded again before its next run. FP32 plans ignore it.
 * Errors: TN_ERR_ARG, TN_ERR_UNSUPPORTED (256 on a BF16X3 plan). */
int tn_group_plan_set_schedule(tn_group_plan* plan, int cls, int tile_width, int long_k, int store16);

/*
 * A grouped contraction staged from and to HOST memory: the end-to-end form
 * of the plan above, for operands that start in host memory and results
 * that must end there. (The paper's contractions start and end in the
 * backend's memory; this is a convenience of the library.)
 *   specs: as tn_group_plan_create; every A and B a view into the device
 *     buffer dev_in (in_bytes long), every C a view into dev_out (out_bytes),
 *     laid out in spec order (a later spec's tensors never start before an
 *     earlier spec's end), so each run of consecutive specs owns one byte
 *     range of each buffer.
 *   chunks: the specs are cut into at most this many runs of about equal
 *     bytes (tn_chunk_bounds), each with its own group plan.
 *   tn_staged_plan_create: host validation and planning; creates three
 *     non-blocking streams and two events per chunk on the current device
 *     (released by _destroy).
 *   tn_staged_plan_set_schedule: tn_group_plan_set_schedule on every chunk's
 *     plan (before _upload).
 *   tn_staged_plan_workspace_bytes / _upload: one DEVICE workspace (256-byte
 *     aligned) holding every chunk plan's work lists and one packed region
 *     they share (they run one after another); upload on `stream`.
 *   tn_staged_plan_run: host_in (HOST, laid out like dev_in; pinned for the
 *     copies to overlap) and host_out (HOST, laid out like dev_out). Chunk c's
 *     byte range of host_in is copied to dev_in on one library stream while
 *     chunk c - 1 is contracted on a second and chunk c - 2's range of
 *     dev_out goes to host_out on a third; the library streams start after
 *     `stream`'s earlier work and `stream` waits for all of them, so host_out
 *     is complete once `stream` is. Runs of one plan must not overlap (one
 *     host thread, one stream at a time): they share its streams and events.
 *     The run only launches and copies, so it can be captured in a CUDA
 *     graph (host_in / host_out must then outlive the graph).
 * Errors: as tn_group_plan_create and _run, plus TN_ERR_ARG when a tensor
 * lies outside its buffer or the layout is not in spec order.
 */
typedef struct tn_staged_plan tn_staged_plan;
int tn_staged_plan_create(const tn_contract_spec* specs, int nspecs, int prec, const void* dev_in, size_t in_bytes,
                          void* dev_out, size_t out_bytes, int chunks, tn_staged_plan** plan);
int tn_staged_plan_chunks(const tn_staged_plan* plan);
double tn_staged_plan_flops(const tn_staged_plan* plan);
int tn_staged_plan_set_schedule(tn_staged_plan* plan, int cls, int tile_width, int long_k, int store16);
size_t tn_staged_plan_workspace_bytes(const tn_staged_plan* plan);
int tn_staged_plan_upload(const tn_staged_plan* plan, void* workspace, size_t bytes, void* stream);
int tn_staged_plan_run(const tn_staged_plan* plan, void* workspace, size_t bytes, const void* host_in,
                       void* host_out, void* stream);
void tn_staged_plan_destroy(tn_staged_plan* plan);
/* Cuts n items with the given (host) weights into at most `chunks` runs of
 * consecutive items of about equal total weight: bounds (HOST, room for
 * chunks + 1 ints) receives the run boundaries 0 = b_0 < b_1 < ... = n (0, 0
 * for n = 0), *nbounds their count. Boundary k goes where the running weight
 * comes closest to k/chunks of the total, strictly after the previous one and
 * before the end; a run never splits an item, so heavy items make fewer,
 * unequal runs. Host only. Errors: TN_ERR_ARG. */
int tn_chunk_bounds(const double* weights, int n, int chunks, int* bounds, int* nbounds);

/* ------------------------------------------------------------------------ */
/* Matrix product states and operators (Sec. II, Fig. 3a)                    */
/* ------------------------------------------------------------------------ */
/* An open-boundary MPS: n rank-3 cores, core i of shape (bond[i], d,
 * bond[i+1]) row-major float32 on the device, bond[0] = bond[n] = 1. The
 * bond array and the pointer table are host memory. */
typedef struct tn_mps {
  int32_t n;
  int32_t d;
  const int64_t* bond;
  float* const* cores;
} tn_mps;

/* An MPO: n rank-4 cores W_i of shape (w[i], w[i+1], d, d) row-major float32
 * on the device, index order (left bond, right bond, bra s, ket s'),
 * w[0] = w[n] = 1. */
typedef struct tn_mpo {
  int32_t n;
  int32_t d;
  const int64_t* bond;
  float* const* cores;
} tn_mpo;

/*
 * <bra|ket> of two MPS with the same n and d, by the left-to-right transfer
 * sweep E_i[b,b'] = sum_{a,a',s} E_{i-1}[a,a'] bra_i[a,s,b] ket_i[a',s,b'],
 * done per site as two contractions (T = E.ket_i over a', then
 * E' = bra_i.T over a and s). After every site E is divided by its
 * largest magnitude and the natural log of that factor is added, in float64,
 * to a running log-scale, so long chains neither overflow nor underflow.
 *   result: DEVICE pointer to 2 doubles, written as {value, log_scale} with
 *           <bra|ket> = value * exp(log_scale).
 *   prec:   arithmetic of the two contractions per site. Chains whose bonds
 *           are all <= 64 run in one CTA in float32 (environment kept in
 *           shared memory across sites) whatever prec says; longer bonds run
 *           each contraction through the tcgen05 (BF16, BF16X3) or float32
 *           kernels of tn_contract.
 *   workspace: DEVICE scratch of tn_mps_inner_workspace_bytes() bytes,
 *           256-byte aligned (may be NULL when that size is 0).
 * Errors: TN_ERR_ARG (null, n < 1, bonds not matching, edge bonds != 1,
 * cores missing), TN_ERR_WORKSPACE, TN_ERR_CUDA.
 */
size_t tn_mps_inner_workspace_bytes(const tn_mps* bra, const tn_mps* ket);
int tn_mps_inner(const tn_mps* bra, const tn_mps* ket, int prec, void* workspace, size_t ws_bytes,
                 double* result, void* stream);

/*
 * <psi|H|psi> and <psi|psi> for an MPS psi and an MPO H (same n and d), by the
 * left environment sweep L[w, a, a'] (w the MPO bond, a the bra bond, a' the
 * ket bond), three contractions per site:
 *   (i)   T1[w, a', s, b]   = sum_a      L[w, a, a'] psi_i[a, s, b]
 *   (ii)  T2[w', s', a', b] = sum_{w, s} W_i[w, w', s, s'] T1[w, a', s, b]
 *   (iii) L'[w', b, b']     = sum_{a',s'} T2[w', s', a', b] psi_i[a', s', b']
 * (i) and (iii) use `prec`, (ii) (contraction length w*d) runs in float32.
 * <psi|psi> is carried in the same sweep as one more MPO channel (the MPO
 * extended by a channel that maps to itself with the identity operator);
 * after every site the environment is scaled by 2^-e, e the binary exponent
 * of its largest magnitude (applied exactly, in the next site's step (ii)),
 * and e ln 2 is added to the float64 log-scale shared by both results.
 * The MPO's bonds must satisfy (bond + 1) * d <= 32, n <= 1024 and
 * (bond + 1) * D * d * D < 2^31 for the largest MPS bond D (else
 * TN_ERR_UNSUPPORTED).
 * Launch forms (results the same up to the order of float32 sums):
 *   - BF16 / BF16X3 with (bond + 1) * d <= 8 on every MPO bond, n <= 512 and
 *     D <= 512: ONE persistent cooperative launch for the whole chain (one
 *     CTA per SM, the sites' GEMM (i) / step (ii) / GEMM (iii) phases
 *     separated by device-wide barriers; the cores packed to bf16 once per
 *     call, step (ii) and GEMM (iii) writing the next contraction's packed
 *     operand). Its barriers are bounded: on expiry TN_ERR_TIMEOUT is
 *     recorded in the status word (tn_sync_status) and the launch ends.
 *   - BF16 / BF16X3 otherwise with (bond + 1) * d <= 8: four launches per
 *     site (a pack of L and the core, the GEMM of (i), step (ii) written
 *     straight into (iii)'s packed operand, the GEMM of (iii)).
 *   - FP32 and wider MPOs: three contractions, a float32 step (ii) and a
 *     max-abs pass per site.
 *   result: DEVICE pointer to 4 doubles {e_value, e_log_scale, n_value,
 *           n_log_scale}: <psi|H|psi> = e_value * exp(e_log_scale) and
 *           <psi|psi> = n_value * exp(n_log_scale); the energy per the
 *           normalised state is their ratio.
 *   workspace: DEVICE scratch of tn_mps_expect_workspace_bytes() bytes
 *           (for chains with bonds <= 512 it includes room for every
 *           site's core packed once per call, as the persistent form needs).
 * Errors: as tn_mps_inner, plus TN_ERR_UNSUPPORTED.
 */
size_t tn_mps_expect_workspace_bytes(const tn_mps* psi, const tn_mpo* H);
int tn_mps_expect(const tn_mps* psi, const tn_mpo* H, int prec, void* workspace, size_t ws_bytes,
                  double* result, void* stream);

/*
 * tn_mps_expect for a batch of `count` MPS sharing one MPO (same n and d for
 * all; bond dimensions may differ from state to state). Each site step runs
 * as grouped launches over the whole batch ((i), (ii), (iii) and one max-abs
 * pass, the norm carried as an extra MPO channel as in tn_mps_expect), so a
 * sweep is a fixed number of launches per site whatever the batch size.
 *   psis:   HOST array of `count` chains.
 *   result: DEVICE pointer to 4*count doubles, {e_value, e_log_scale,
 *           n_value, n_log_scale} per state, as tn_mps_expect.
 *   workspace: DEVICE scratch of tn_mps_expect_grouped_workspace_bytes()
 *           bytes, 256-byte aligned: the environments and intermediates of
 *           every state plus the uploaded launch tables. The call uploads
 *           those tables (host -> device copies on `stream`) and then
 *           launches; on a stream being captured into a CUDA graph it
 *           returns TN_ERR_UNSUPPORTED (as does _plan below; _run only
 *           launches).
 * Errors: as tn_mps_expect, plus TN_ERR_ARG when count < 1 or the states
 * differ in length or physical dimension.
 */
size_t tn_mps_expect_grouped_workspace_bytes(const tn_mps* psis, int count, const tn_mpo* H, int prec);
int tn_mps_expect_grouped(const tn_mps* psis, int count, const tn_mpo* H, int prec, void* workspace,
                          size_t ws_bytes, double* result, void* stream);

/*
 * tn_mps_expect_grouped in two parts, for a batch evaluated many times:
 * _plan builds the host layout of the sweep (per site the grouped work lists
 * of steps (i) and (iii), the step (ii) descriptors, the max-abs tables) in
 * `workspace` and uploads its tables on `stream` (host -> device copies from
 * pageable memory); _run only launches (one extended-MPO build, per site two
 * grouped contractions, one grouped float32 step and one max-abs pass, then
 * the finisher) and writes `result` as tn_mps_expect_grouped does. The plan
 * keeps the device pointers of the states' and the MPO's cores and the
 * workspace (which must stay allocated and unused by others); the values
 * behind them are read at every run. Errors: as tn_mps_expect_grouped;
 * _run: TN_ERR_ARG (null plan or result), TN_ERR_CUDA. Plans are not
 * thread-safe; runs of one plan on different streams race on its workspace.
 */
typedef struct tn_expect_plan tn_expect_plan;
int tn_mps_expect_grouped_plan(const tn_mps* psis, int count, const tn_mpo* H, int prec, void* workspace,
                               size_t ws_bytes, tn_expect_plan** plan, void* stream);
int tn_mps_expect_grouped_run(const tn_expect_plan* plan, double* result, void* stream);
void tn_mps_expect_grouped_destroy(tn_expect_plan* plan);

/* ------------------------------------------------------------------------ */
/* MPS image classifier (Sec. IV.A)                                          */
/* ------------------------------------------------------------------------ */
/*
 * Scores of a batch of greyscale images under one MPS W with a label leg:
 * pixel p of image b is encoded by the local feature map
 * Phi(p) = (cos(pi p / 2), sin(pi p / 2)), and score_l(b) is the inner
 * product of the product state of the n encoded pixels with W_l, the MPS
 * obtained by fixing the label leg to l. W has n cores of shape
 * (bond[i], 2, bond[i+1]) except the label core at `label_site`, of shape
 * (bond[ls], 2, n_labels, bond[ls+1]); every bond <= 128, d = 2.
 * The sweep runs from both ends towards the label core: the left vector after
 * sites 0..ls-1 and the right vector after sites n-1..ls+1 (each step
 * v' = sum_s Phi_s(x_i) v.W_i[:, s, :]) are rescaled per sample after every
 * site (float32 path: divided by their largest magnitude; tensor-core paths:
 * multiplied by 2^-e, e the binary exponent of that magnitude, exactly), the
 * logs of the factors summed in float64, and met at the label core (a
 * contraction over the batch: float32 for TN_PREC_FP32, the split BF16X3
 * tensor-core contraction for the BF16 / BF16X3 modes).
 *   pixels:  DEVICE [batch, n] float32, row-major.
 *   ftilde:  DEVICE [batch, n_labels] float32; log_scale: DEVICE [batch]
 *            float64. score_l(b) = ftilde[b, l] * exp(log_scale[b]).
 *   prec:    TN_PREC_FP32 (float32 on the CUDA cores), TN_PREC_BF16 (bf16
 *            operands, float32 accumulation on tcgen05) or TN_PREC_BF16X3
 *            (split bf16 operands, hi*hi + lo*hi + hi*lo); both half-chains
 *            run in one launch, bonds padded to chi in {32, 64, 128}.
 *   ckpt_every: the forward keeps the per-sample sweep vector every
 *            ckpt_every sites (1 = every site) for the backward pass, which
 *            recomputes the vectors in between; 0 keeps none (no backward).
 *   workspace: DEVICE scratch of tn_mps_classify_workspace_bytes(); it holds
 *            the forward's state for tn_mps_classify_backward.
 * Errors: TN_ERR_ARG, TN_ERR_SHAPE (bonds or label core inconsistent),
 * TN_ERR_UNSUPPORTED (bond > 128, d != 2),
 * TN_ERR_WORKSPACE, TN_ERR_CUDA.
 */
size_t tn_mps_classify_workspace_bytes(const tn_mps* W, int label_site, int n_labels, int batch,
                                       int ckpt_every);
int tn_mps_classify(const tn_mps* W, int label_site, int n_labels, const float* pixels, int batch,
                    int prec, int ckpt_every, float* ftilde, double* log_scale, void* workspace,
                    size_t ws_bytes, void* stream);

/*
 * Gradient of a loss with respect to every core, given dLoss/dftilde
 * (DEVICE [batch, n_labels] float32) for a loss that depends on the scores
 * only through their direction f / ||f|| (so log_scale carries no gradient),
 * e.g. cross-entropy of softmax(f / ||f||). Must follow tn_mps_classify on
 * the same W, pixels, batch and workspace with ckpt_every >= 1. Per site i,
 * with v the normalised sweep vector entering i and g the adjoint of the
 * vector leaving it,
 *   dW_i[a, s, c] = sum_b v_b[a] Phi_s(x_bi) g_b[c] / scale_bi,
 *   g_b <- sum_{s,c} W_i[a, s, c] Phi_s(x_bi) g_b[c] / scale_bi,
 * done per checkpoint segment: TN_PREC_BF16 / TN_PREC_BF16X3 run one launch
 * that recomputes both halves' segments and one adjoint launch that also
 * accumulates every step's dW (the products over the segment's samples on
 * tcgen05, float32 reductions into a workspace buffer, then one scatter);
 * TN_PREC_FP32 runs the float32 adjoint sweep and one grouped tensordot over
 * the batch per segment (their plans built and uploaded in the call, so the
 * FP32 backward returns TN_ERR_UNSUPPORTED on a stream being captured into a
 * CUDA graph; BF16 / BF16X3 only launch).
 *   dcores: host table of n DEVICE pointers, each shaped like its core
 *           (overwritten).
 *   prec:   arithmetic of the sweeps and of the gradient products (the label
 *           core's contractions run in float32 for TN_PREC_FP32, split BF16X3
 *           otherwise). TN_PREC_BF16X3 needs chi <=
 *           64 (its staging at chi = 128 does not fit in shared memory).
 * Errors: as tn_mps_classify, plus TN_ERR_UNSUPPORTED for TN_PREC_BF16X3 at
 * chi = 128. The gradient reductions are float32 atomics: results agree
 * between runs to rounding, not bit for bit.
 */
int tn_mps_classify_backward(const tn_mps* W, int label_site, int n_labels, const float* pixels,
                             int batch, int prec, int ckpt_every, const float* dftilde,
                             float* const* dcores, void* workspace, size_t ws_bytes, void* stream);

/*
 * Loss head of the classifier: with z_b = ftilde_b / ||ftilde_b||_2 (equal
 * to f_b / ||f_b||, so the log-scale drops out),
 *   loss = (1 / batch) sum_b [ logsumexp(z_b) - z_b[label_b] ],
 *   dftilde_b = (g_b - z_b (z_b . g_b)) / (batch ||ftilde_b||),
 *   g_b = softmax(z_b) - onehot(label_b).
 *   ftilde: DEVICE [batch, n_labels] float32; labels: DEVICE [batch] int64 in
 *   [0, n_labels); loss: DEVICE float64 scalar; dftilde: DEVICE [batch,
 *   n_labels] float32 (may be NULL). The mean is reduced in a fixed order
 *   (deterministic). Errors: TN_ERR_ARG, TN_ERR_CUDA.
 */
int tn_mps_classify_loss(const float* ftilde, const int64_t* labels, int batch, int n_labels,
                         double* loss, float* dftilde, void* stream);

/*
 * Failure-path check (the paper has no counterpart): launches one small
 * kernel whose threads wait, with the bounded wait every kernel of the
 * library uses, on an mbarrier that nothing completes, giving up after
 * limit_ns nanoseconds of wall time (clamped to 10 ms .. 2 s). The kernel
 * then records TN_ERR_TIMEOUT in the device status word and returns
 * normally, so tn_sync_status() reports it and the context stays usable.
 * Errors: TN_ERR_CUDA (launch failed).
 */
int tn_check_wait_timeout(uint64_t limit_ns, void* stream);
/* Failure-path check of the persistent energy sweep's device-wide barrier: a
 * two-CTA cooperative launch in which one CTA leaves without arriving, so the
 * other's bounded wait gives up after limit_ns (clamped to 10 ms .. 2 s) and
 * records TN_ERR_TIMEOUT in the status word. counter: 4 bytes of DEVICE memory
 * the barrier counts in (zeroed here, on `stream`). No GPU fault is involved;
 * the context stays usable. Errors: TN_ERR_ARG, TN_ERR_CUDA. */
int tn_check_grid_barrier_timeout(uint64_t limit_ns, void* counter, void* stream);

/* ------------------------------------------------------------------------ */
/* Classifier with one MPS per label (Sec. IV.A)                              */
/* ------------------------------------------------------------------------ */
/*
 * n_mps MPS of n sites each (cores (D_{i-1}, 2, D_i), D_0 = D_n = 1, D <= 128,
 * bonds may differ between the MPS): the score of label l for image b is the
 * overlap of the image's product state phi(x_b) = (x) (cos pi x/2, sin pi x/2)
 * with MPS l. Output as for tn_mps_classify: f[b, l] = ftilde[b, l] *
 * exp(log_scale[b]) (ftilde [batch, n_mps] float32, log_scale [batch]
 * float64, one log-scale per sample shared by its labels), so
 * tn_mps_classify_loss applies unchanged. Each MPS is swept as a one-label
 * classifier (its middle core n/2 read as the label core (D, 2, 1, D')) in
 * its own part of the workspace; prec TN_PREC_FP32 or TN_PREC_BF16 as for
 * tn_mps_classify. The backward takes dLoss/dftilde [batch, n_mps] and the
 * forward's workspace (same ckpt_every >= 1) and writes the gradients of
 * every core: dcores[l * n + i] is core i of MPS l (device, the core's
 * shape). Workspace: tn_mps_classify_separate_workspace_bytes (256-B
 * aligned). Errors: TN_ERR_ARG (counts, null pointers, n_mps > 64),
 * TN_ERR_SHAPE (the MPS differ in length, or bonds as in tn_mps_classify),
 * TN_ERR_UNSUPPORTED, TN_ERR_WORKSPACE, TN_ERR_CUDA.
 */
size_t tn_mps_classify_separate_workspace_bytes(const tn_mps* Ws, int n_mps, int batch, int ckpt_every);
int tn_mps_classify_separate(const tn_mps* Ws, int n_mps, const float* pixels, int batch, int prec, int ckpt_every,
                             float* ftilde, double* log_scale, void* workspace, size_t ws_bytes, void* stream);
int tn_mps_classify_separate_backward(const tn_mps* Ws, int n_mps, const float* pixels, int batch, int prec,
                                      int ckpt_every, const float* dftilde, float* const* dcores, void* workspace,
                                      size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Node splitting (Sec. III.B "Node Splitting", Appendix A "Saving Memory")  */
/* ------------------------------------------------------------------------ */
/*
 * Splits node A by the singular value decomposition of its matrix view: rows
 * run over the legs `left` (in that order, last fastest), columns over the
 * legs `right`; left and right together name every leg of A exactly once.
 * With M = prod of the left dims, N = prod of the right dims and
 * r = min(M, N), A = U S V^T with S descending. The new bond keeps k <= r
 * singular values:
 *  - max_truncation_err >= 0: the smallest values are dropped while the sum
 *    of the dropped ones stays <= max_truncation_err (Appendix A); < 0: none;
 *  - max_singular_values > 0: at most that many are kept; <= 0: no cap;
 *  - with both, the smaller count; at least one value is always kept.
 * Outputs (device, row-major, written for the k kept values; size them for
 * r): U_out holds M x k -- the left node, shape (left dims..., k); Vt_out
 * holds k x N -- the right node, shape (k, right dims...). absorb = 1
 * (split_node): U sqrt(S) and sqrt(S) V^T. absorb = 0 (split_node_full_svd):
 * U and V^T, and S_out (k values) the diagonal of the singular-value node.
 * S_out (optional when absorb = 1) gets the k kept values, dropped_out
 * (optional) the r - k dropped ones, both descending. *kept (host) = k;
 * *sweeps (host, optional) = Jacobi sweeps used, negative if the sweep limit
 * (40) was reached before every column pair was orthogonal.
 *
 * Arithmetic: float32 one-sided Jacobi (Hestenes) on the r columns of
 * length max(M, N), the rotation angles computed in float64; singular values
 * are column norms. The singular vectors of a zero singular value on the
 * longer side (columns of U when M >= N, rows of V^T when M < N) are zeros. Workspace: tn_split_node_workspace_bytes (256-B
 * aligned). Unlike the other entry points this call synchronises `stream`
 * (once per sweep and before the outputs, whose shapes depend on k).
 * Errors: TN_ERR_ARG (legs not a partition of A's, null outputs or kept),
 * TN_ERR_UNSUPPORTED (dtype, negative strides, r >= 2^30), TN_ERR_WORKSPACE,
 * TN_ERR_CUDA. An empty node (r = 0) returns TN_OK with k = 0.
 */
size_t tn_split_node_workspace_bytes(const tn_tensor* A, const int* left, int nleft, const int* right, int nright);
int tn_split_node(const tn_tensor* A, const int* left, int nleft, const int* right, int nright,
                  int64_t max_singular_values, double max_truncation_err, int absorb, float* U_out, float* S_out,
                  float* Vt_out, float* dropped_out, int64_t* kept, int32_t* sweeps, void* workspace,
                  size_t ws_bytes, void* stream);
/* The truncation rule alone (host): how many of the r singular values
 * sigma_desc (descending, host array) tn_split_node keeps. */
int64_t tn_split_truncation(const float* sigma_desc, int64_t r, int64_t max_singular_values,
                            double max_truncation_err);

/* ------------------------------------------------------------------------ */
/* ncon (Appendix B): planning a labelled network into pairwise steps        */
/* ------------------------------------------------------------------------ */
/*
 * n tensors; tensor t has ranks[t] legs with dims and labels given in
 * tensor order (concatenated). A label >= 0 is an edge: exactly two legs,
 * of equal dimension (on two tensors, or twice on one -- a trace). A label
 * < 0 is a dangling leg of the result; -1, -2, ... each appear once. Edges
 * are taken in con_order (n_order labels, each edge once; n_order = 0:
 * ascending). An edge between two tensors contracts every edge the two share
 * in one step (contract_between, Sec. III.B.2); its result holds the first
 * tensor's free legs, then the second's (tensordot order), and joins the end
 * of the operand list (inputs first, in order; a step consumes its operands).
 * An edge on one tensor is a trace step (b = -1, legs_a[0] and legs_b[0] both
 * legs of a). Tensors still unconnected at the end are joined by outer
 * products (nshared = 0) in list order. out_perm[i] is the leg of the last
 * result (or of the single input when there are no steps) that becomes
 * output leg i, the output legs ordered as out_order (n_out labels; 0:
 * -1, -2, ...); *out_rank = number of dangling legs.
 * steps may be NULL to count them (*n_steps); otherwise max_steps bounds
 * the array (at most the number of edges plus n - 1 are needed).
 * Host only: no device memory is touched. Errors: TN_ERR_ARG (labels,
 * orders, counts), TN_ERR_SHAPE (an edge's two legs differ in dimension),
 * TN_ERR_UNSUPPORTED (an intermediate or the result above rank 8).
 */
typedef struct tn_ncon_step {
  int32_t a, b;                 /* operands: input t is t, step s's result is n + s; b = -1: a trace of a */
  int32_t nshared;              /* leg pairs legs_a[j] (of a) <-> legs_b[j] (of b; of a for a trace) */
  int32_t rank;                 /* rank of the step's result */
  int32_t legs_a[TN_MAX_RANK];
  int32_t legs_b[TN_MAX_RANK];
  int64_t shape[TN_MAX_RANK];   /* the result's shape */
} tn_ncon_step;
int tn_ncon_plan(int n, const int* ranks, const int64_t* dims, const int* labels, const int* con_order, int n_order,
                 const int* out_order, int n_out, tn_ncon_step* steps, int max_steps, int* n_steps, int* out_perm,
                 int* out_rank);

/* Device status word: returns the first kernel-side error since the last
 * call (TN_OK if none) after synchronising `stream`, and clears it. */
int tn_sync_status(void* stream);

/* Human-readable name of a status code (static string). */
const char* tn_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
