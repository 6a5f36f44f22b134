/*
 * kerdock.h -- C ABI of the GB300 (sm_103a) Kerdock fast sparsifying transform.
 *
 * Method: Fuchs, Gross, Krahmer, Kueng, Mixon, "Sketching with Kerdock's
 * crayons: fast sparsifying transforms for arbitrary linear maps"
 * (arXiv 2105.05879).  Problem 1 (Sec. 1.1): preprocess an arbitrary
 * A in R^{m x n} so that h_eps(Ax), the entrywise eps-hard threshold of Ax,
 * is fast to compute for every unit x whose Ax is (nearly) s-sparse.
 * Algorithm 1 gives the two halves this library implements:
 *
 *   kerdock_preprocess  -- the preprocessing step: the representation
 *                          {A s_l : l in [L]} in the d/2+1 real mutually
 *                          unbiased Kerdock bases, by sign flips and fast
 *                          Walsh-Hadamard transforms of the rows of A (Lemma 6).
 *   kerdock_apply       -- the streaming step: draw N = JK indices l_j,
 *                          y_j = (A s_{l_j})(s_{l_j}^T x), median of means over
 *                          K batches of J (Theorem 3), top-S of |mu|, exact
 *                          A_S x, output entries with |value| >= eps.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - d = 2^k is the smallest power of FOUR with d >= n (Lemma 6 needs k even;
 *    Algorithm 1's "power of 2" is read as "power of 4").  Supported:
 *    1 <= n <= 4096, 1 <= m <= 4096 with m == n checked by the caller's
 *    workload only (m != n is accepted).
 *  - Bases b in [0, d/2) are the Kerdock bases of the field elements with
 *    integer code b in GF(2^(k-1)) (Prop. 5; polynomial basis, irreducible
 *    polynomials t+1, t^3+t+1, t^5+t^2+1, t^7+t+1, t^9+t^4+1, t^11+t^2+1;
 *    basis of V = (t^0,0),...,(t^(k-2),0),(0,1)).  Basis d/2 is the identity.
 *    Sample index l = b*d + w, L = d*(d/2+1).  s_l = sqrt(d) Pi u_l with
 *    u_{M,w}(p) = 2^(-k/2) (-1)^(Q_M(p) + w.p) (Eq. "definition of vectors")
 *    and Pi the projection onto the first n coordinates (Algorithm 1).
 *  - Representation layout in device memory: R[b][w][i] = (A s_{b,w})_i,
 *    i contiguous, row stride ldr = m rounded up to a multiple of 8 elements
 *    (entries i in [m, ldr) are written as 0).  Element type float32 or
 *    bfloat16 (round-to-nearest-even of the float32 result).
 *  - Sampling: sample j of query q uses z = SplitMix64 output function applied
 *    to seed + 0x9E3779B97F4A7C15 * (q*N + j + 1) (mod 2^64) and
 *    l = floor(z * L / 2^64).  Batch k holds samples j in [kJ, (k+1)J).
 *  - Median of an even number K of batch means is the mean of the two middle
 *    values (Sec. 4: K = 2 gives the plain mean).  Top-S ties go to the
 *    smaller index.  The threshold is inclusive: |v| >= eps (Sec. 1.1).
 *  - Memory ownership: the library never allocates device memory.  The
 *    caller allocates the representation, the table buffer, inputs, outputs
 *    and (optional) workspace and keeps them alive while a plan uses them.
 *    A plan owns only host metadata.
 *  - Streams: every launch goes to the stream given to kerdock_plan_bind (or
 *    kerdock_set_stream).  Calls are asynchronous; results are ready after
 *    the stream is synchronised (kerdock_sync does that and also reports any
 *    device-side error recorded by the kernels).
 *  - Errors: every call returns KERDOCK_OK (0) or a negative KERDOCK_ERR_*.
 *    No exception crosses the ABI.  Arguments are validated on the host
 *    before anything is launched; a failing call launches nothing.
 *  - Threading: a plan must not be used from two host threads at once.
 */
#ifndef KERDOCK_H
#define KERDOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KERDOCK_OK 0
#define KERDOCK_ERR_INVALID_ARG (-1)      /* null pointer, bad size, bad value */
#define KERDOCK_ERR_UNSUPPORTED (-2)      /* sizes outside the supported range */
#define KERDOCK_ERR_NOT_BOUND (-3)        /* plan has no device buffers yet */
#define KERDOCK_ERR_NOT_PREPROCESSED (-4) /* apply before preprocess */
#define KERDOCK_ERR_CAPACITY (-5)         /* a caller buffer is too small */
#define KERDOCK_ERR_CUDA (-6)             /* a CUDA runtime call failed */
#define KERDOCK_ERR_DEVICE_TIMEOUT (-7)   /* a bounded device-side wait gave up */
#define KERDOCK_ERR_ALIGNMENT (-8)        /* a device pointer is not 16-byte aligned */

#define KERDOCK_F32 0  /* representation stored as float32 */
#define KERDOCK_BF16 1 /* representation stored as bfloat16 */

/* kerdock_apply flags */
#define KERDOCK_FLAG_FULL_OUTPUT 1 /* return all S refined entries, unthresholded
                                      ("we would not discard this information",
                                      Sec. 1.1) */

typedef struct kerdock_plan_s* kerdock_plan_t;

typedef struct {
  int64_t m, n;        /* A is m x n */
  int32_t k;           /* d = 2^k */
  int32_t dtype;       /* KERDOCK_F32 / KERDOCK_BF16 */
  int64_t d;           /* padded dimension, a power of four */
  int64_t num_bases;   /* d/2 + 1 */
  int64_t L;           /* design size d*(d/2+1) */
  int64_t ldr;         /* representation row stride in elements */
  int32_t J, K, S;     /* batch size, number of batches, candidate-set size */
  int32_t reserved;
  size_t repr_bytes;   /* bytes the caller must provide for R */
  size_t table_bytes;  /* bytes the caller must provide for the tables */
} kerdock_plan_info_t;

/* Create a plan for an m x n matrix.  dtype: KERDOCK_F32 or KERDOCK_BF16.
 * J >= 1, 1 <= K <= 32, 1 <= S; S is clamped to m.  N = J*K <= 2^24.
 * Host only (no CUDA call).  *plan is set to NULL on failure. */
int kerdock_plan_create(kerdock_plan_t* plan, int64_t m, int64_t n, int32_t dtype,
                        int32_t J, int32_t K, int32_t S);

/* Fill *info.  Host only. */
int kerdock_plan_info(kerdock_plan_t plan, kerdock_plan_info_t* info);

/* Attach caller-owned device memory and a CUDA stream (cudaStream_t passed
 * as void*; NULL = legacy default stream).  repr_dev needs info.repr_bytes
 * bytes, table_dev info.table_bytes bytes; both 256-byte aligned.  Builds the
 * Kerdock sign tables D_b on the device (step (i) of Lemma 6: one bit
 * Q_{M_b}(p) per (b, p), computed from the GF(2^(k-1)) construction of
 * Prop. 5; stored twice, in p order for the preprocessing and transposed by
 * p mod 32 for the coefficient step) and clears the device status word,
 * asynchronously on the stream. */
int kerdock_plan_bind(kerdock_plan_t plan, void* repr_dev, size_t repr_bytes,
                      void* table_dev, size_t table_bytes, void* stream);

/* Change the stream later launches of this plan go to. */
int kerdock_set_stream(kerdock_plan_t plan, void* stream);

/* Preprocessing step of Algorithm 1 / Lemma 6.  A_dev: m x n float32,
 * row-major with leading dimension lda >= n (elements).  Writes the whole
 * representation R.  The plan remembers (A_dev, lda): kerdock_apply reads
 * rows of A for the exact refinement A_S x, so A_dev must stay valid and
 * unchanged while the plan is applied. */
int kerdock_preprocess(kerdock_plan_t plan, const float* A_dev, int64_t lda);

/* Bytes of device workspace kerdock_apply needs for q queries (may be 0). */
size_t kerdock_apply_workspace_bytes(kerdock_plan_t plan, int64_t q);

/* Streaming step of Algorithm 1 for q queries.
 *   X_dev     q x n float32 row-major, leading dimension ldx >= n.  Used as
 *             given: the guarantees of Theorem 3 assume unit-norm x.
 *   eps       threshold (> 0 unless KERDOCK_FLAG_FULL_OUTPUT).
 *   seed      sampling seed (see the sampling convention above).
 *   out_idx   q x S int32, out_val q x S float32 (row r of query q at
 *             offset q*S + r): the kept (index, value) pairs in ascending
 *             index order; out_count[q] = how many were kept (<= S).
 *             Entries past out_count[q] are left unspecified.
 *   ws_dev    workspace of kerdock_apply_workspace_bytes(plan, q) bytes
 *             (NULL allowed when that is 0).
 * q = 0 is a valid no-op. */
int kerdock_apply(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                  float eps, uint64_t seed, int32_t flags, int32_t* out_idx,
                  float* out_val, int32_t* out_count, void* ws_dev, size_t ws_bytes);

/* Same as kerdock_apply, and additionally writes, when the pointer is not
 * NULL: mu_out (q x m float32) the median-of-means estimate mu (Theorem 3),
 * ells_out (q x N int64) the drawn indices l_j, coef_out (q x N float32)
 * the coefficients s_{l_j}^T x.  For parity tests. */
int kerdock_apply_debug(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                        float eps, uint64_t seed, int32_t flags, int32_t* out_idx,
                        float* out_val, int32_t* out_count, void* ws_dev, size_t ws_bytes,
                        float* mu_out, int64_t* ells_out, float* coef_out);

/* Allocation-free variant of kerdock_apply (the paper has no counterpart:
 * this is an integration aid).  It is for callers that cannot allocate
 * device memory -- code running while a stream is captured into a CUDA
 * graph, real-time or embedded hosts with a device-memory budget fixed at
 * start-up, plugin hosts that own the allocator -- and so cannot provide the
 * workspace kerdock_apply may need.  Same arguments, results and ordering
 * as kerdock_apply without the workspace; the batch-mean scratch lives in a
 * 16 MiB array inside the library instead, which every GPU that loads the
 * library keeps until the process exits.
 *   - Limit: 8 * K * ldr * min(q, number of SMs) bytes must not exceed
 *     16 MiB; larger calls return KERDOCK_ERR_CAPACITY and launch nothing
 *     (e.g. with K = 2 and m = 4096 on a 152-SM GPU it fits; K = 16 with
 *     m = 1024 does not unless q <= 128).
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before
 *     any stream capture.
 *   - All calls share the one array: calls that overlap on the GPU (other
 *     streams, other plans) race with each other.  Nothing in it needs to
 *     be cleared between calls.
 *   - The current device must be the plan's device (KERDOCK_ERR_INVALID_ARG
 *     otherwise).  The looked-up address belongs to the device's current
 *     context: do not use this entry point after cudaDeviceReset in the
 *     same process.
 *   - It calls no cudaMalloc, cudaFree or allocating library routine. */
int kerdock_apply_noalloc(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                          float eps, uint64_t seed, int32_t flags, int32_t* out_idx,
                          float* out_val, int32_t* out_count);

/* ------------------------------------------------------------------------
 * Batches: queries over any mix of plans (sizes, representation types,
 * sparsities) answered by one persistent launch, optionally replayed from a
 * captured CUDA graph.  (Serving form of Algorithm 1's streaming step.)
 * ------------------------------------------------------------------------ */
#define KERDOCK_BATCH_GRAPH 1 /* capture the launch into a CUDA graph (needs a non-NULL stream) */

typedef struct {
  kerdock_plan_t plan;  /* a bound, preprocessed plan on the current device */
  const float* x;       /* device pointer to this query's n floats */
  int32_t J, K;         /* batch size and number of batches of the median of means (K <= 32) */
  int32_t S;            /* candidate-set size, 1 <= S <= m (Sec. 4 uses S = 10 s) */
  int32_t flags;        /* KERDOCK_FLAG_FULL_OUTPUT or 0 */
  float eps;            /* threshold (> 0 unless full output) */
  int32_t reserved;
  uint64_t seed;        /* sampling seed */
  int64_t index;        /* the q of the sampling convention (sample j uses counter index*J*K + j) */
  int32_t* out_idx;     /* device, S int32: kept indices, ascending */
  float* out_val;       /* device, S float32: their values */
  int32_t* out_count;   /* device, one int32: how many were kept */
} kerdock_query_t;

typedef struct kerdock_batch_s* kerdock_batch_t;

/* Device workspace bytes kerdock_batch_create needs for this list (0 on
 * invalid input). */
size_t kerdock_batch_workspace_bytes(const kerdock_query_t* queries, int64_t count);

/* Validate the queries, deal them to the CTAs plan by plan (plans in
 * decreasing row size; each plan's queries longest first onto the
 * least-loaded CTA by estimated cost, loads carried over), so that all CTAs
 * work through one representation at a time; upload descriptors and schedule into
 * ws_dev (256-byte aligned, caller-owned, kept alive with the batch), and --
 * with KERDOCK_BATCH_GRAPH -- capture the launch into a CUDA graph.
 * Synchronises the stream once (the upload).  Every plan must stay bound and
 * preprocessed while the batch exists; x and the outputs are read/written at
 * every launch. */
int kerdock_batch_create(kerdock_batch_t* batch, const kerdock_query_t* queries, int64_t count,
                         void* ws_dev, size_t ws_bytes, void* stream, int32_t options);

/* Run the batch (graph replay or plain launch), asynchronously. */
int kerdock_batch_launch(kerdock_batch_t batch);

/* Set the query kernel's ring geometry for this batch: ring_kb KiB of shared
 * memory for representation rows and crows rows per ring chunk (1, 2, 4 or
 * 8; 0 = default for either); re-captures the graph.  A geometry whose ring
 * holds too few chunks for the kernel's coefficient warps is refused with
 * KERDOCK_ERR_UNSUPPORTED. */
int kerdock_batch_set_tuning(kerdock_batch_t batch, int32_t ring_kb, int32_t crows);

/* Re-deal the queries to the CTAs by the caller's cost estimates: cost[i]
 * (any unit, finite, >= 0) for the i-th query of the creation list, count
 * the list's length.  The schedule is made as at creation (plan by plan,
 * longest first onto the least-loaded CTA), where the estimate is the
 * query's gathered and refined bytes.  Results do not depend on the schedule (every query runs
 * whole on one CTA, its samples in counter order).  Synchronises the stream
 * once (the upload); INVALID_ARG on a wrong count or a negative, infinite or
 * NaN cost. */
int kerdock_batch_set_costs(kerdock_batch_t batch, const double* cost, int64_t count);

/* Test entry (host only, no device work): the schedule kerdock_batch_create
 * makes for count queries over grid CTAs, where plan_ids[i] identifies query
 * i's plan (any value, equal for queries of one plan), row_bytes[i] is that
 * plan's representation row size and cost[i] the query's estimated cost.
 * Plans in decreasing row size (ties: first appearance), each plan's queries
 * longest first (ties: list order) onto the least-loaded CTA (ties: lowest
 * index), loads carried from plan to plan.  order_out: count int32, the
 * queries CTA by CTA; cta_start_out: grid + 1 int64.  INVALID_ARG for a NULL
 * pointer, count < 1, grid < 1 or a negative, infinite or NaN cost. */
int kerdock_debug_batch_schedule(const void* const* plan_ids, const uint32_t* row_bytes,
                                 const double* cost, int64_t count, int32_t grid,
                                 int32_t* order_out, int64_t* cta_start_out);

/* CTAs of the batch's launch (one per SM, at most one per query); 0 for a
 * null batch. */
int32_t kerdock_batch_ctas(kerdock_batch_t batch);

/* Set the schedule explicitly: CTA c (0 <= c < ctas) runs the queries
 * order[cta_start[c] .. cta_start[c+1]-1] in that sequence (indices into the
 * creation list).  order is a permutation of 0..count-1, cta_start has
 * ctas + 1 non-decreasing entries from 0 to count, 1 <= ctas <=
 * kerdock_batch_ctas(batch); CTAs from ctas on get no queries.  Both arrays
 * are host memory, copied.  Results do not depend on the schedule.
 * Synchronises the stream once; INVALID_ARG on any violation. */
int kerdock_batch_set_schedule(kerdock_batch_t batch, const int32_t* order,
                               const int64_t* cta_start, int32_t ctas);

/* Autotuner: time reps launches of every candidate geometry (ring 64/96/128/
 * 160 KiB x 1/2/4/8 rows per chunk), keep the fastest and report it. */
int kerdock_batch_tune(kerdock_batch_t batch, int32_t reps, int32_t* ring_kb, int32_t* crows,
                       float* best_ms);

/* Synchronise the batch's stream and report a recorded device error. */
int kerdock_batch_sync(kerdock_batch_t batch);

int kerdock_batch_destroy(kerdock_batch_t batch);

/* Ring geometry of a plan's kerdock_apply (0 = default); and the autotuner
 * that times kerdock_apply with each candidate and keeps the fastest. */
int kerdock_plan_set_tuning(kerdock_plan_t plan, int32_t ring_kb, int32_t crows);
int kerdock_plan_tune(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx, float eps,
                      uint64_t seed, int32_t* out_idx, float* out_val, int32_t* out_count,
                      void* ws_dev, size_t ws_bytes, int32_t reps, int32_t* ring_kb,
                      int32_t* crows, float* best_ms);

/* ------------------------------------------------------------------------
 * Learned proposal (a project form, not in the paper): a three-layer
 * perceptron in bfloat16 (FP32 accumulation on tensor cores) maps a cheap
 * sketch mu (a plan with small J, K) to one score per output index; the top
 * scores replace the top-|mu| candidates of Algorithm 1's refinement step.
 *   H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Z = H2 W3^T + b3 (+ skip X),
 * trained with binary cross-entropy on logits (positive weight w+) and AdamW.
 * ------------------------------------------------------------------------ */
typedef struct kerdock_mlp_s* kerdock_mlp_t;

/* in_dim, hidden, out_dim even; max_batch rows per forward/backward call. */
int kerdock_mlp_create(kerdock_mlp_t* mlp, int32_t in_dim, int32_t hidden, int32_t out_dim,
                       int32_t max_batch);
/* Input transform of the features: X = bf16(feat_scale * f) (LINEAR, the
 * default) or X = bf16(feat_scale * |f|) (ABS: only sketch magnitudes). */
#define KERDOCK_MLP_INPUT_LINEAR 0
#define KERDOCK_MLP_INPUT_ABS 1
int kerdock_mlp_set_input(kerdock_mlp_t mlp, int32_t mode);
/* Residual logits Z = H2 W3^T + b3 + skip * X (in_dim == out_dim): with W3,
 * b3 zero the network starts from the plain ranking by the features. */
int kerdock_mlp_set_skip(kerdock_mlp_t mlp, float skip);

/* Device bytes for the state (FP32 master weights, gradients, AdamW moments,
 * bfloat16 weight copies) and for the activations of max_batch rows. */
int kerdock_mlp_sizes(kerdock_mlp_t mlp, size_t* state_bytes, size_t* work_bytes,
                      int64_t* param_count);
int kerdock_mlp_bind(kerdock_mlp_t mlp, void* state_dev, size_t state_bytes, void* work_dev,
                     size_t work_bytes, void* stream);
/* Device pointers of the FP32 parameters and gradients (layout W1, b1, W2,
 * b2, W3, b3, row-major; offsets[7] receives the 6 start offsets and the end).
 * After writing parameters directly call kerdock_mlp_sync_weights. */
int kerdock_mlp_pointers(kerdock_mlp_t mlp, float** params, float** grads, int64_t* offsets);
int kerdock_mlp_sync_weights(kerdock_mlp_t mlp);
/* Weights U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from the SplitMix64 counter hash,
 * zero biases and moments. */
int kerdock_mlp_init(kerdock_mlp_t mlp, uint64_t seed);
/* logits (B x out_dim FP32) for features feat_scale * feats (B x in_dim FP32). */
int kerdock_mlp_forward(kerdock_mlp_t mlp, const float* feats, int32_t B, float feat_scale,
                        float* logits);
/* Forward + backward for labels (B x out_dim, 0/1): fills the gradients and
 * the loss (read with kerdock_mlp_loss). */
int kerdock_mlp_backward(kerdock_mlp_t mlp, const float* feats, const float* labels, int32_t B,
                         float feat_scale, float pos_weight);
int kerdock_mlp_loss(kerdock_mlp_t mlp, float* loss_host);
/* One AdamW step (decoupled weight decay) on all parameters. */
int kerdock_mlp_adamw(kerdock_mlp_t mlp, float lr, float beta1, float beta2, float eps,
                      float weight_decay);
int kerdock_mlp_destroy(kerdock_mlp_t mlp);

/* Refinement from scores: for each of q queries take the S indices with the
 * largest scores (q x m FP32, ties to the smaller index), compute a_i^T x
 * exactly (Algorithm 1's last step) and keep |value| >= eps (all S with
 * KERDOCK_FLAG_FULL_OUTPUT).  Outputs as kerdock_apply with capacity S. */
int kerdock_refine_scores(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                          const float* scores, int32_t S, float eps, int32_t flags,
                          int32_t* out_idx, float* out_val, int32_t* out_count);

/* A second plan over the same bound and preprocessed representation with
 * other J, K, S (e.g. a cheap sketch setting).  The clone shares the source's
 * device memory and stream; the source must outlive it. */
int kerdock_plan_clone(kerdock_plan_t* out, kerdock_plan_t src, int32_t J, int32_t K, int32_t S);

/* Algorithm 1's streaming step for q queries that share one sample set: the
 * N = JK indices kerdock_apply draws for query 0 serve every query of the
 * batch (each query is still Algorithm 1 with N uniform samples, so Theorem 3
 * holds per query; failures of different queries become dependent).  The
 * coefficients X S^T and the batch means C_k R_k / J run as tensor-core
 * products (bfloat16 operands split hi + lo, float32 accumulation), then the
 * median, top-S of |mu|, exact refinement and threshold as kerdock_apply.
 * Outputs as kerdock_apply.  ws: device memory of
 * kerdock_apply_shared_workspace_bytes(plan, q) bytes, 256-byte aligned.
 * Errors as kerdock_apply; CAPACITY when ws is smaller than asked. */
size_t kerdock_apply_shared_workspace_bytes(kerdock_plan_t plan, int64_t q);
int kerdock_apply_shared(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                         float eps, uint64_t seed, int32_t flags, int32_t* out_idx,
                         float* out_val, int32_t* out_count, void* ws, size_t ws_bytes);

/* The first half of kerdock_apply_shared: the scores it ranks, without the
 * selection and refinement.  scores[r * m + i] = |mu_r[i]|, where mu_r is
 * Theorem 3's estimate for query r with the shared sample set: the entrywise
 * median over the K batch means (the mean of the two middle ones for even K)
 * of c_j R[l_j] / J (Algorithm 1's streaming step).  scores: device, q * m
 * float32, 16-byte aligned, caller-owned.  ws as kerdock_apply_shared.
 * kerdock_refine_scores(plan, X, q, ldx, scores, S, eps, flags, ...) on these
 * scores gives kerdock_apply_shared's outputs.  Errors as
 * kerdock_apply_shared; ALIGNMENT for a misaligned scores. */
int kerdock_apply_shared_scores(kerdock_plan_t plan, const float* X_dev, int64_t q, int64_t ldx,
                                uint64_t seed, float* scores, void* ws, size_t ws_bytes);

/* Parameters with a guarantee (Theorem 3 with gamma = (eps - delta)/2, as
 * the argument around Algorithm 1 asks of mu): J = ceil(4 e^2 a^2 / gamma^2)
 * and K = ceil(2 ln(m / eta)), where a = max_i ||a_i|| (||A||_{2->inf}).
 * Then for unit x with Ax in Sigma(A, s, delta), ||mu - Ax||_inf < gamma with
 * probability >= 1 - eta.  Host only; no plan needed.
 * Errors: INVALID_ARG unless a > 0, eps > delta >= 0, 0 < eta <= 1, m >= 1;
 * UNSUPPORTED when K exceeds the library's 32 batches or J*K its sample
 * limit (J and K are still written). */
int kerdock_theory_parameters(double a_row_norm_max, double eps, double delta, double eta,
                              int64_t m, int32_t* J, int32_t* K);

/* ------------------------------------------------------------------------
 * FP64 checks of a preprocessed representation against A, on the GPU (the
 * precision form keeps float64 for these checks only).  Both read the plan's
 * A (the matrix given to kerdock_preprocess) and the device representation;
 * both are asynchronous on the plan's stream and allocate nothing.
 * ------------------------------------------------------------------------ */

/* Reconstruction (Lemma 6 read backwards: W W = d I, so the slab T_b = A Pi
 * D_b W gives back A Pi D_b = T_b W / d).  For each basis b in [b0, b0 + nb)
 * err_dev[b - b0] receives, in float64,
 *     max over i < ldr, p < d of | (1/d) (T_b W)[i][p] (-1)^{Q_b(p)} - Apad[i][p] |
 * (for the identity basis b = d/2: | R[d/2][p][i] / sqrt(d) - Apad[i][p] |),
 * where Apad[i][p] = A[i][p] for i < m, p < n and 0 elsewhere (padding
 * columns p >= n and padding rows i in [m, ldr) must come back as 0).
 * err_dev: nb doubles, device, 8-byte aligned (overwritten).
 * Errors: INVALID_ARG for a NULL pointer, b0 < 0, nb < 1, b0 + nb > d/2 + 1 or
 * a current device other than the plan's; NOT_BOUND, NOT_PREPROCESSED;
 * UNSUPPORTED for nb > 65535 (check in pieces); ALIGNMENT. */
int kerdock_check_reconstruction(kerdock_plan_t plan, int64_t b0, int64_t nb, double* err_dev);

/* Tight frame (Prop. 2 through the design: each basis is orthonormal, so
 * sum_w s_{b,w} s_{b,w}^T = d I_n and sum_{l in bases} R[l] <R[l], y> =
 * nb d A A^T y; over all d/2 + 1 bases this is sum_j B_j B_j^T = (d/2+1) I).
 * For P probe vectors y_p (Y_dev: P x m float64, row-major, 1 <= P <= 4):
 *     frame_dev[p][i] = sum over rows l = (b, w), b in [b0, b0 + nb), of
 *                       R[l][i] <R[l], y_p>            (float64 accumulation)
 *     ref_dev[p][i]   = nb d (A A^T y_p)_i             (float64, from A)
 * frame_dev and ref_dev: P x m doubles, device, 8-byte aligned (overwritten).
 * The residual frame - ref is zero for an exact representation.
 * Errors as kerdock_check_reconstruction, and INVALID_ARG for P outside
 * [1, 4]. */
int kerdock_check_tight_frame(kerdock_plan_t plan, const double* Y_dev, int32_t P, int64_t b0,
                              int64_t nb, double* frame_dev, double* ref_dev);

/* Synchronise the plan's stream and report the first error any kernel of
 * this plan recorded in the device status word (then clear it). */
int kerdock_sync(kerdock_plan_t plan);

/* Copy the device sign table to host memory: (d/2) rows of max(4, d/32)
 * uint32 words (rows padded to 16 bytes); bit (p mod 32) of word p/32 of row
 * b is Q_{M_b}(p) for p < d, and padding bits are 0.
 * Synchronises the stream. */
int kerdock_debug_signs(kerdock_plan_t plan, uint32_t* host_out, size_t host_words);

/* Test of the failure path: a one-warp kernel waits, at most max_polls
 * mbarrier polls, on a phase nothing completes, then records
 * KERDOCK_ERR_DEVICE_TIMEOUT in the plan's status word and returns (no trap,
 * no hang).  The next kerdock_sync reports it and clears it. */
int kerdock_debug_wait_timeout(kerdock_plan_t plan, int32_t max_polls);

/* Test of the query kernel's own failure path: later kerdock_apply /
 * kerdock_apply_noalloc launches of this plan give up a wait after max_polls
 * unsuccessful mbarrier polls (0 restores the default of 2^22).  With a tiny
 * limit the waits run out during normal operation: every role of the kernel
 * stops, the CTA waits (boundedly) for the row copies it issued, and
 * KERDOCK_ERR_DEVICE_TIMEOUT is recorded for kerdock_sync; outputs of such a
 * launch are unspecified.  Host only. */
int kerdock_debug_set_poll_limit(kerdock_plan_t plan, uint32_t max_polls);

/* Test entry for the library's bfloat16 tensor-core product (the products of
 * the learned network and of kerdock_apply_shared).  Plane z of C (float32,
 * device, row pitch ldc >= N, plane z at C + z * M * ldc) receives
 *   C_z[m][n] = sum over k in slice z of A(m, k) B(n, k),
 * with A(m, k) at A[m * sAm + k * sAk] and B(n, k) at B[n * sBn + k * sBk]
 * (bfloat16, device).  kc = 0 sums the whole K into plane 0; kc > 0 (a
 * multiple of 64) cuts K into ceil(K / kc) slices of kc.  Two k-major operands
 * (unit k stride, row pitch a multiple of 8 elements, 16-byte aligned base)
 * run on tcgen05, other layouts with 16-byte rows on the cp.async kernel, the
 * rest on the element-wise kernel.  Enqueued on `stream` (NULL: the default
 * stream); KERDOCK_ERR_INVALID_ARG for M, N or K < 1, ldc < N, kc < 0 or not a
 * multiple of 64, or a NULL pointer. */
int kerdock_debug_gemm(const void* A, int64_t sAm, int64_t sAk, const void* B, int64_t sBn,
                            int64_t sBk, int32_t M, int32_t N, int32_t K, int32_t kc, float* C,
                            int64_t ldc, void* stream);

/* Destroy a plan (host metadata only; NULL is accepted). */
int kerdock_plan_destroy(kerdock_plan_t plan);

/* Static, human-readable text for an error code. */
const char* kerdock_strerror(int code);

/* Library version as major*10000 + minor*100 + patch. */
int kerdock_version(void);

#ifdef __cplusplus
}
#endif
#endif /* KERDOCK_H */
