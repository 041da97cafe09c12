/*
 * qaoa.h -- C ABI of the GB300 (sm_103a) QAOA statevector library.
 *
 * The library evaluates the p-round QAOA expectation of arXiv 2312.06451
 * (JuliQAOA), Eq. 1,
 *
 *     |beta,gamma> = e^{-i b_p H_M} e^{-i g_p H_C} ... e^{-i b_1 H_M} e^{-i g_1 H_C} |psi_0>,
 *     <C>          = <beta,gamma| C |beta,gamma>                        (Sec. 1)
 *
 * over a cost vector C(x) precomputed on the feasible set (Sec. 2.1), with
 * either the transverse-field mixer H_M = sum_i X_i applied as per-qubit
 * rotations (Sec. 2.1 Eq. 2, Sec. 2.2) or a constrained mixer applied through
 * a stored eigendecomposition H_M = V D V^-1 (Sec. 2.1, Sec. 2.2), and the
 * gradient of <C> with respect to all 2p angles (Sec. 2.3, Sec. 4).
 *
 * Conventions shared by every call
 *   - Qubit i is bit i of the basis-state index x (bit 0 = least significant).
 *   - A state is an array of complex64 amplitudes stored as interleaved
 *     float pairs (re, im), one per feasible basis state, in increasing x.
 *   - Angles are float64 in the order of Listing 1:
 *     [beta_1, ..., beta_p, gamma_1, ..., gamma_p]; gradients use the same order.
 *   - Round k applies the phase separator with gamma_k first, then the mixer
 *     with beta_k (Eq. 1).
 *   - The default initial state is the uniform superposition over the feasible
 *     set: 2^{-n/2} on all 2^n states, or 1/sqrt(D) on the D Hamming-weight-k
 *     states (Sec. 3, default of simulate()).
 *   - To minimise instead of maximise, negate the cost vector (Sec. 3).
 *
 * Memory ownership
 *   Pointers named d_* are device memory owned by the caller; the library never
 *   frees or retains them past the call.  Pointers without the prefix are host
 *   memory.  Scratch (work states, per-round checkpoints, reduction partials,
 *   launch descriptors) belongs to the context: it is allocated on first need,
 *   grown when a larger problem arrives, reused across calls (Sec. 2.2: memory
 *   is pre-allocated and re-used) and freed by qaoa_destroy().
 *
 * Errors
 *   Every call returns a qaoa_status.  Nothing aborts, traps or prints.  On a
 *   non-OK status, qaoa_last_error() gives a one-line description.  Arguments
 *   are validated (sizes, dtypes, p >= 1, finite angles, a device-memory
 *   estimate) before any kernel is launched.  A CUDA error from a launch or a
 *   copy is reported as QAOA_ERR_CUDA with the CUDA error string.
 *
 * Streams
 *   All work is issued on the stream given to qaoa_create().  Calls that take
 *   host result pointers synchronise that stream before returning; the batched
 *   call only enqueues work and writes device results, so it can be captured
 *   into a CUDA graph by the caller after one warm-up call has sized the
 *   context's scratch.
 */
#ifndef QAOA_GB300_H
#define QAOA_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QAOA_OK = 0,
    QAOA_ERR_INVALID = 1,     /* bad argument (size, dtype, pointer, angle) */
    QAOA_ERR_OOM = 2,         /* device memory for the scratch is not available */
    QAOA_ERR_CUDA = 3,        /* a CUDA runtime call failed */
    QAOA_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    QAOA_ERR_UNSUPPORTED = 5  /* valid request outside what this build implements */
} qaoa_status;

typedef struct qaoa_ctx qaoa_ctx;

/* Cost-vector element types. */
enum {
    QAOA_COST_F32 = 0, /* float32 cost values */
    QAOA_COST_U8 = 1   /* integer costs 0..255 stored as uint8 */
};

/* Built-in cost functions (Sec. 2.1 and Sec. 3).
 *   MAXCUT : C(x) = #{edges (u,v) : x_u != x_v}                    (Listing 1)
 *   WMAXCUT: C(x) = sum over edges of w_uv [x_u != x_v]
 *   SK     : C(x) = sum_{i<j} J_ij z_i z_j, z_i = 1 - 2 x_i; an arbitrary user
 *            cost, which the paper allows for any function of x (Sec. 3).
 *   DKS    : densest k-subgraph, C(x) = #{edges (u,v) : x_u = x_v = 1} on the
 *            Hamming-weight-k states (Sec. 2.1, Listing 2).
 *   KVC    : max k-vertex cover, C(x) = #{edges (u,v) : x_u = 1 or x_v = 1} on
 *            the Hamming-weight-k states (Sec. 2.1). */
enum {
    QAOA_PROBLEM_MAXCUT = 0,
    QAOA_PROBLEM_WMAXCUT = 1,
    QAOA_PROBLEM_SK = 2,
    QAOA_PROBLEM_DKS = 3,
    QAOA_PROBLEM_KVC = 4
};

/* Mixer kinds. */
enum {
    QAOA_MIXER_X = 0,     /* H_M = sum_i X_i on all 2^n states (Sec. 2.1, Eq. 2) */
    QAOA_MIXER_EIGEN = 1, /* H_M = V diag(lambda) V^T on D feasible states (Sec. 2.1) */
    QAOA_MIXER_X_MA = 2,  /* multi-angle QAOA (Sec. 3: one mixer per qubit per layer,
                             each with its own angle): round k applies
                             e^{-i beta_{k,q} X_q} to every qubit q.  An angle set is
                             p (n + 1) values [beta_{1,0..n-1}, ..., beta_{p,0..n-1},
                             gamma_1..gamma_p]; gradients use the same layout. */
    QAOA_MIXER_EIGEN_SYM = 4, /* an XY mixer (ring or clique) on the D weight-k states
                             through the eigendecompositions of its cyclic-shift
                             blocks (see qaoa_xy_block_hamiltonians): d_V holds the
                             block eigenvector matrices V_b back to back (each
                             D_b x D_b float32, row-major, eigenvectors as columns),
                             d_lambda the D float64 eigenvalues block after block,
                             k the Hamming weight.  Same results as QAOA_MIXER_EIGEN
                             with the full V, at about 2/n of its product work. */
    QAOA_MIXER_X_GENERAL = 3, /* a sum of products of Pauli X (Sec. 2.1),
                             f(X) = sum_S c_|S| prod_{i in S} X_i on all 2^n states,
                             given by its Hadamard-basis eigenvalues: d_lambda holds
                             n + 1 float64 values d_w = sum_k c_k K_k(w) (K_k the
                             Krawtchouk polynomial); d_w = [w = 0] is the Grover
                             mixer |+><+|.  Angles and gradients as for X. */
    QAOA_MIXER_GROVER = 5    /* the Grover mixer H_M = |u><u| (Sec. 2.4), u the uniform
                             superposition over the dim states the cost vector lists
                             (all 2^n, the binom(n, k) weight-k states, or any other
                             feasible set), applied as the rank-one update
                             e^{-i b H_M} phi = phi + (e^{-i b} - 1) <u|phi> u: one
                             streaming pass per round and direction.  dim >= 1; n is
                             informational; d_V, d_lambda, k, id unused.  d_init,
                             when given, must be 16-byte aligned.  Angles and
                             gradients as for X.  Gradient runs keep p + 1 state
                             vectors when they fit (QAOA_CKPT_ROUND or _PASS), else
                             two (QAOA_CKPT_NONE: each adjoint pass also undoes the
                             forward round on the state). */
};

/* Hadamard-basis weights of a general X mixer (Sec. 2.1: a mixer written as a
 * sum of products of Pauli X is diagonal after H^n, with the diagonal
 * precomputed): for f(X) = sum_{k=0..kmax} c_k sum_{|S| = k} prod_{i in S} X_i
 * on n qubits, d[w] = sum_k c_k K_k(w) for w = 0..n, K_k(w) the Krawtchouk
 * polynomial (the value of sum_{|S|=k} prod Z_i on a weight-w state).  These
 * are the n + 1 values a QAOA_MIXER_X_GENERAL mixer's d_lambda holds.
 *   c  host, kmax + 1 float64 coefficients (c[0] multiplies the identity)
 *   d  host output, n + 1 float64
 * 1 <= n <= 62, 0 <= kmax <= n; otherwise QAOA_ERR_INVALID.  Host-only; no
 * context or device is needed. */
qaoa_status qaoa_x_mixer_weights(int n, int kmax, const double *c, double *d);

/* Precision of the dense eigenbasis products for QAOA_MIXER_EIGEN. */
enum {
    QAOA_GEMM_FP32_SIMT = 0, /* complex64 CUDA-core products, fp32 accumulate */
    QAOA_GEMM_3XTF32 = 1,    /* tensor cores, tf32 hi/lo split, 3 products */
    QAOA_GEMM_BF16X3 = 2     /* tensor cores, bf16 hi/lo split, 3 products */
};

/* Problem description for qaoa_cost_precompute (all pointers host memory).
 *   n      qubits (1..34 unconstrained, 2..40 constrained)
 *   k      Hamming weight of the feasible states for DKS, else -1
 *   m      edge count; edges holds 2m vertex indices (u_0, v_0, u_1, ...)
 *   weights m float32 weights (WMAXCUT only)
 *   J      n*n float32 row-major couplings (SK only; entries with i < j used) */
typedef struct {
    int kind;
    int n;
    int k;
    int m;
    const int32_t *edges;
    const float *weights;
    const float *J;
} qaoa_problem;

/* Mixer description.
 *   kind   one of QAOA_MIXER_*
 *   n      qubits
 *   dim    feasible-set size: 2^n for the X mixers, D for EIGEN / EIGEN_SYM
 *   d_V    EIGEN: D x D float32, row-major, real orthogonal eigenvectors as
 *          columns (H_M V = V diag(lambda)); EIGEN_SYM: the block matrices
 *   d_lambda EIGEN, EIGEN_SYM: D float64 eigenvalues; X_GENERAL: n + 1 float64
 *          weights
 *   gemm_precision EIGEN, EIGEN_SYM: one of QAOA_GEMM_*
 *   k      EIGEN_SYM: Hamming weight of the feasible states (else ignored)
 *   id     EIGEN, EIGEN_SYM: 0, or a caller-chosen id of this (d_V, d_lambda)
 *          pair.  The products use V in padded (and, for 3xTF32, split) copies.
 *          With id 0 every call rebuilds them from d_V / d_lambda; with an id
 *          the context builds them once and keeps them for every later call
 *          with that id, so the caller must give a new id whenever the
 *          contents change (device addresses alone are not enough: freed
 *          memory is reused). */
typedef struct {
    int kind;
    int n;
    int64_t dim;
    const float *d_V;
    const double *d_lambda;
    int gemm_precision;
    int k;
    uint64_t id;
} qaoa_mixer;

/* ------------------------------------------------------------- context */

/* Create a context bound to CUDA device `device` and the stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns all
 * scratch memory and the error text. */
qaoa_status qaoa_create(qaoa_ctx **ctx, int device, void *cuda_stream);

/* Free every scratch allocation and the context.  NULL is ignored. */
void qaoa_destroy(qaoa_ctx *ctx);

/* Text of the last error on this context ("" if none).  Valid until the next
 * call on the context. */
const char *qaoa_last_error(const qaoa_ctx *ctx);

/* Bytes of device scratch the context currently holds. */
int64_t qaoa_scratch_bytes(const qaoa_ctx *ctx);

/* ------------------------------------------------------- pre-computation */

/* Cost vector over the feasible set (Sec. 2.1: C(x) is computed once, stored
 * for every feasible x and re-used by every evaluation).
 *   d_cost      device output, dim elements of cost_dtype
 *   cost_dtype  QAOA_COST_U8 (integer costs; fails with QAOA_ERR_INVALID if a
 *               value can exceed 255) or QAOA_COST_F32
 *   dim         2^n for unconstrained problems, binom(n,k) for DKS
 * SK with couplings on the 2^-20 grid (|J| < 8) is summed exactly in integers
 * and rounded once to float32; other couplings are summed in float64. */
qaoa_status qaoa_cost_precompute(qaoa_ctx *ctx, const qaoa_problem *prob, void *d_cost,
                                 int cost_dtype, int64_t dim);

/* The binom(n,k) Hamming-weight-k basis states in increasing integer order
 * (Sec. 2.1 feasible subspace; Sec. 2.4 orders them as Gosper's hack does).
 * d_states: device output, dim uint64 values. */
qaoa_status qaoa_dicke_states(qaoa_ctx *ctx, int n, int k, uint64_t *d_states, int64_t dim);

/* Dense ring mixer H_M = sum_i (X_i X_{i+1} + Y_i Y_{i+1}), ring read as
 * periodic, restricted to the Hamming-weight-k states (Sec. 2.1), written
 * row-major into d_H (dim x dim float64, device).  Its eigendecomposition
 * gives the d_V / d_lambda of a QAOA_MIXER_EIGEN mixer. */
qaoa_status qaoa_ring_hamiltonian(qaoa_ctx *ctx, int n, int k, double *d_H, int64_t dim);

/* Dense clique XY mixer sum_{i<j} (X_i X_j + Y_i Y_j) on the Hamming-weight-k
 * states (Sec. 2.1), the matrix whose eigendecomposition a QAOA_MIXER_EIGEN
 * mixer stores.  Element (a, b) = 2 when states a and b differ by exchanging
 * one set and one clear bit, else 0.  d_H: device, dim x dim float64,
 * row-major, dim = C(n, k), 2 <= n <= 40.  Synchronous. */
qaoa_status qaoa_clique_hamiltonian(qaoa_ctx *ctx, int n, int k, double *d_H, int64_t dim);

/* XY mixers on the weight-k states, block by block (Sec. 2.1 constrained
 * mixers; Sec. 2.2: the products with the stored eigendecomposition dominate
 * their cost).  The ring and clique mixers commute with the cyclic shift of
 * the qubits, so in a real basis of shift momenta they split into
 * floor(n/2) + 1 blocks (momenta m and n - m share one real block).  This
 * call gives the blocks' sizes and, when H is not NULL, the dense block
 * matrices in that basis, whose eigendecompositions make a
 * QAOA_MIXER_EIGEN_SYM mixer.
 *   mixer     QAOA_XY_RING or QAOA_XY_CLIQUE (the matrices of
 *             qaoa_ring_hamiltonian / qaoa_clique_hamiltonian)
 *   n, k      2 <= n <= 32, 0 <= k <= n, C(n, k) <= 65536
 *   n_blocks  in: capacity of block_dim; out: the number of (non-empty) blocks
 *   block_dim host output, the sizes D_b (sum = C(n, k)); NULL to query
 *             n_blocks only
 *   H         host output, sum of D_b^2 float64: block b row-major after the
 *             blocks before it; NULL to skip
 * Host-only (no context or device).  QAOA_ERR_INVALID on bad arguments or a
 * too-small capacity. */
enum { QAOA_XY_RING = 0, QAOA_XY_CLIQUE = 1 };
qaoa_status qaoa_xy_block_hamiltonians(int mixer, int n, int k, int *n_blocks, int64_t *block_dim, double *H);

/* ----------------------------------------------------------- simulation */

/* <C> of Eq. 1 for one angle set.
 *   d_cost, cost_dtype  cost vector over the mixer's feasible set
 *   d_init  device complex64 initial state (mixer->dim amplitudes) or NULL for
 *           the uniform superposition (Sec. 3, initial_state)
 *   p       rounds (>= 1); angles: host, 2p float64 (p (n + 1) for QAOA_MIXER_X_MA);
 *           E: host output.
 * Synchronous on the context stream. */
qaoa_status qaoa_expectation(qaoa_ctx *ctx, const void *d_cost, int cost_dtype,
                             const qaoa_mixer *mixer, const void *d_init, int p,
                             const double *angles, double *E);

/* How the adjoint sweep gets back the forward states it needs. */
enum {
    QAOA_CKPT_NONE = 0,  /* undo each round on psi as well (2 state vectors) */
    QAOA_CKPT_ROUND = 1, /* keep the state at every round boundary (p + 1 vectors) */
    QAOA_CKPT_PASS = 2   /* keep the output of every forward pass (X mixer: about
                            p * ceil(n / 12) + 1 vectors); the adjoint then writes
                            only lambda.  Eigenbasis mixers treat it as ROUND. */
};

/* <C> and its 2p partial derivatives by one forward and one adjoint
 * (reverse) sweep (Sec. 2.3, Sec. 4: the gradient for a constant multiple of
 * one evaluation).  grad: host output, 2p float64 in the angle order.
 *   ckpt  one of QAOA_CKPT_* (any other value is QAOA_ERR_INVALID). */
qaoa_status qaoa_gradient(qaoa_ctx *ctx, const void *d_cost, int cost_dtype,
                          const qaoa_mixer *mixer, const void *d_init, int p,
                          const double *angles, double *E, double *grad, int ckpt);

/* One batched job: n_sets angle sets evaluated on one cost vector and mixer.
 *   d_angles  device, n_sets x 2p float64 (row = one angle set; p (n + 1) for
 *             QAOA_MIXER_X_MA)
 *   d_E       device output, n_sets float64
 *   d_grad    device output, n_sets rows like d_angles (ignored unless want_grad)
 *   d_init    device initial state shared by all sets, or NULL */
typedef struct {
    const void *d_cost;
    int cost_dtype;
    const qaoa_mixer *mixer;
    int p;
    int n_sets;
    const double *d_angles;
    double *d_E;
    double *d_grad;
    const void *d_init;
} qaoa_job;

/* Many angle sets of many problem instances (of uneven size) in one enqueued
 * sequence of launches, for the angle-finding outer loop (Sec. 2.3) that
 * calls the simulator many times.  Asynchronous: results land in the jobs'
 * device buffers when the context stream reaches them.  Scratch is sized by
 * the first call with a given job list; after that the same call enqueues no
 * allocation and may be captured in a CUDA graph.  Fails with QAOA_ERR_OOM
 * before launching anything when the scratch would not fit. */
qaoa_status qaoa_expectation_batched(qaoa_ctx *ctx, int n_jobs, const qaoa_job *jobs,
                                     int want_grad);

/* The same batched evaluation with the angles and results in host memory, for
 * an angle-finding loop (Sec. 2.3) that proposes angles on the host and reads
 * <C> (and the gradients) back every iteration.  One call copies every job's
 * angles to device staging held by the context, enqueues the batched
 * launches, copies the results back and returns after the context stream has
 * finished (synchronous).
 *   h_angles  host, n_sets x 2p float64 (p (n + 1) for QAOA_MIXER_X_MA), read
 *   h_E       host output, n_sets float64
 *   h_grad    host output, n_sets rows like h_angles (ignored unless want_grad)
 *   d_cost, mixer, d_init  device data as in qaoa_job
 * Pinned host memory (cudaMallocHost, or a pinned tensor) gives asynchronous
 * copies; pageable memory works at a lower rate.  The caller keeps ownership of
 * every buffer; the call retains none of them.  Staging grows when a call
 * needs more and is reused afterwards, so repeating a call with the same job
 * shapes enqueues no allocation and re-uses the launch plan.  Errors: the
 * checks of qaoa_expectation_batched, plus QAOA_ERR_INVALID for NULL host
 * pointers or a capturing stream; a device-side error word raised by the
 * launches is returned after the synchronisation (QAOA_ERR_INVALID for a
 * non-finite angle, QAOA_ERR_TIMEOUT for a bounded wait that gave up). */
typedef struct {
    const void *d_cost;
    int cost_dtype;
    const qaoa_mixer *mixer;
    int p;
    int n_sets;
    const double *h_angles;
    double *h_E;
    double *h_grad;
    const void *d_init;
} qaoa_host_job;

qaoa_status qaoa_expectation_batched_host(qaoa_ctx *ctx, int n_jobs, const qaoa_host_job *jobs,
                                          int want_grad);

/* Checkpointing used by qaoa_expectation_batched gradients (default
 * QAOA_CKPT_PASS).  Per unit the planner steps down PASS -> ROUND -> NONE
 * when one angle set's scratch would not fit in free device memory. */
qaoa_status qaoa_set_checkpointing(qaoa_ctx *ctx, int mode);

/* Cap on the device memory a call may plan for state scratch (work states,
 * checkpoints and eigenbasis state matrices), in bytes; negative = no cap
 * beyond the device's free memory.  Planning happens on the host before any
 * launch: an angle set whose states cannot fit under the cap even without
 * checkpoints makes the call fail with QAOA_ERR_OOM, launching nothing; the
 * context stays usable.  Lets a caller share the device with other work, and
 * lets tests drive the refusal without exhausting the device.  Host-only. */
qaoa_status qaoa_set_state_limit(qaoa_ctx *ctx, int64_t bytes);

/* ------------------------------------------ X-mixer pass schedule tuning */

/* Schedule of the transverse-field mixer passes for one qubit count and cost
 * dtype.  Every pass applies the rotations of 12 qubits (Sec. 2.2: the mixer
 * is a sequence of single-qubit operations, so any grouping gives the same
 * state): qubits 0..11 in contiguous tiles, then the higher qubits in chunks,
 * each gathered from runs of 2^c contiguous amplitudes, c = 12 - chunk >= cmin.
 *   cmin    4..8 (shortest run 2^cmin amplitudes; 4 = one 128-byte line)
 *   split   0 equal chunks, 1 full chunks first, 2 remainder first
 *   nbuf_bwd_contig / nbuf_bwd_gather  1 or 2 tile buffers per CTA in the
 *           adjoint passes (1: two CTAs per SM; 2: one CTA per SM)
 *   ms      time of the tuning run that chose it (output only)
 * The schedule changes the rounding order only. */
typedef struct {
    int n;
    int cost_dtype;
    int cmin;
    int split;
    int nbuf_bwd_contig;
    int nbuf_bwd_gather;
    double ms;
} qaoa_xtune;

/* The pass groups a schedule gives (host-only; touches no device).  Writes up
 * to max (c, lo) pairs: pass j keeps qubits 0..c_j-1 contiguous and gathers
 * qubits lo_j..lo_j+11-c_j.  Returns the pass count, or -1 for n outside
 * 13..32, cmin outside 4..8 or split outside 0..2. */
int qaoa_pass_schedule(int n, int cmin, int split, int *c, int *lo, int max);

/* Autotuner: times forward (+ adjoint when want_grad) sweeps of p rounds
 * (1..8) on the caller's cost vector for every schedule with the fewest
 * passes, then the adjoint buffer choices, on the context stream, and keeps
 * the fastest for (n, cost_dtype) in the context; out (may be NULL) receives
 * it.  Angles are fixed internal values; results of the runs are discarded.
 * Synchronous.  Uses the context's scratch like a gradient call of p rounds. */
qaoa_status qaoa_autotune_x(qaoa_ctx *ctx, const void *d_cost, int cost_dtype, int n, int p,
                            int want_grad, qaoa_xtune *out);
/* Set (e.g. restore a saved tuning) or read the schedule used for
 * (t->n, t->cost_dtype).  Without a stored entry the default is cmin 4,
 * split 0, one adjoint buffer. */
qaoa_status qaoa_set_xtune(qaoa_ctx *ctx, const qaoa_xtune *t);
qaoa_status qaoa_get_xtune(qaoa_ctx *ctx, int n, int cost_dtype, qaoa_xtune *out);

/* ------------------------------------------ Grover mixer on degeneracies */

/* Degeneracies of an integer cost over the feasible set (Sec. 2.4): with the
 * Grover mixer H_G = |u><u| (u the uniform superposition over the feasible
 * set) and the uniform initial state, all states of equal cost keep equal
 * amplitudes, so the QAOA needs only the distinct values and their counts.
 *   prob      MAXCUT with k = -1 over all 2^n states (n <= 44), or DKS / KVC
 *             over the Hamming-weight-k states (n <= 128, C(n, k) <= 2^44)
 *   d_counts  device, n_bins int64: zeroed, then d_counts[c] = number of
 *             feasible states with cost c; n_bins must exceed the largest
 *             possible cost (the edge count; for DKS at most k(k-1)/2) and be
 *             at most 4096
 * Synchronous on the context stream.  Valid input never yields a cost outside
 * [0, n_bins); the kernel checks it anyway and reports QAOA_ERR_CUDA. */
qaoa_status qaoa_cost_degeneracy(qaoa_ctx *ctx, const qaoa_problem *prob, int64_t *d_counts, int n_bins);

/* <C> (and, when d_grad != NULL, all 2p derivatives) of QAOA with the Grover
 * mixer and the uniform initial state, for n_sets angle sets, from the
 * degeneracies d_counts[0..n_bins) of the cost values 0..n_bins-1 (as written
 * by qaoa_cost_degeneracy; other integer costs may be counted by the caller).
 *   d_angles  device, n_sets x 2p float64 [beta_1..beta_p, gamma_1..gamma_p]
 *   d_E       device output, n_sets float64
 *   d_grad    device output, n_sets x 2p float64, or NULL
 *   p         1 .. 1024 rounds
 * Float64 throughout (the reduced vector holds one amplitude per value).
 * Asynchronous on the context stream; a non-finite angle gives NaN results. */
qaoa_status qaoa_grover_batched(qaoa_ctx *ctx, const int64_t *d_counts, int n_bins, int p, int n_sets,
                                const double *d_angles, double *d_E, double *d_grad);

/* ------------------------------------------------ allocation-free variant */

/* <C> (and, when d_grad != NULL, its 2p derivatives) for one angle set of a
 * small problem, n <= 12 qubits and p <= 96 rounds, with the transverse-field
 * mixer and the uniform initial state -- without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (a host that owns and pre-partitions all device
 * memory, code running where allocation after start-up is forbidden).
 *
 *   d_cost      device cost vector, 2^n elements of cost_dtype (16-byte aligned)
 *   d_angles    device, 2p float64 in the usual order
 *   d_E         device output, 1 float64
 *   d_grad      device output, 2p float64, or NULL for the expectation only
 *   cuda_stream the stream to run on (NULL = legacy default stream)
 *
 * Scratch (coefficients, phase tables, launch descriptors, an error word) is a
 * fixed 256 KiB file-scope device array that every device loading the library
 * keeps until exit; sizes beyond n = 12 or p = 96 are rejected with
 * QAOA_ERR_INVALID.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) once and keeps it; make that first call
 * before any stream capture, and do not call the entry point on a device after
 * cudaDeviceReset there (the array may then sit at another address).  The
 * caller must pass buffers of the stated sizes: they are not checked.  The call is synchronous on cuda_stream.  All calls share the one
 * array: calls that overlap on the GPU (other threads or streams) race, so
 * serialise them.  No other context or state is needed.  A non-finite angle
 * returns QAOA_ERR_INVALID; a CUDA failure QAOA_ERR_CUDA. */
qaoa_status qaoa_gradient_small_noalloc(const void *d_cost, int cost_dtype, int n, int p,
                                        const double *d_angles, double *d_E, double *d_grad,
                                        void *cuda_stream);

/* ------------------------------------------------------------- diagnostics */

/* Runs the library's bounded device-side wait (the one every TMA / mbarrier
 * wait of the kernels uses) on a barrier that nothing ever completes.  The
 * wait gives up after one second of GPU time, the kernel records it
 * in the context's error word and returns, and the call reports
 * QAOA_ERR_TIMEOUT; the context and the device stay usable.  For tests of the
 * failure path; the paper has no counterpart.  Synchronous. */
qaoa_status qaoa_check_bounded_wait(qaoa_ctx *ctx);

/* ------------------------------------------------------------ measurement */

/* Per-kernel-family launch statistics, collected when profiling is on: each
 * launch is bracketed by CUDA events on the context stream and its algorithmic
 * bytes (the bytes the method must move: state reads and writes and cost
 * reads, no scratch) are added up. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
    double algo_bytes;  /* HBM-bound kernels: bytes the method must move */
    double algo_flops;  /* contractions: useful floating-point operations */
} qaoa_kernel_stat;

qaoa_status qaoa_set_profiling(qaoa_ctx *ctx, int enable);
/* Fills up to max entries; returns the number of kernel families (or -1). */
int qaoa_kernel_stats(qaoa_ctx *ctx, qaoa_kernel_stat *out, int max);
void qaoa_reset_stats(qaoa_ctx *ctx);
/* Kernel launches issued by this context since creation or the last reset. */
int64_t qaoa_launch_count(const qaoa_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* QAOA_GB300_H */
