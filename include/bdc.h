/*
 * bdc.h -- C ABI of the B300 Blahut-Arimoto engine for the finite-length
 * binary deletion channel BDC_d (inputs {0,1}^n, outputs {0,1}^{<=n}).
 *
 * The operation (paper Sec. 2.3, in the log2 form of Sec. 3): for an input
 * distribution p over {0,1}^n,
 *     q(y)  = sum_x p(x) W(y|x),   W(y|x) = Count(y,x) d^(n-|y|) (1-d)^|y|
 *     D_x   = sum_y W(y|x) log2(W(y|x)/q(y))
 *     lower = log2 sum_x p(x) 2^{D_x}      upper = max_x D_x
 *     p    <- p 2^{D} / sum_x p 2^{D}
 * where Count(y,x) is the number of times y appears as a subsequence of x
 * (Sec. 2.2).  C_n(d)/n is an upper bound on the deletion-channel capacity
 * C(d) (Sec. 2.2, first lemma); upper is a valid upper bound on C_n(d) for
 * every p (the dual/minimax bound; certified in FP64 by bdc_certify_upper).
 *
 * Encoding: x in {0,1}^n is the integer whose most significant of n bits is
 * x_0 (lexicographic order = numeric order).  An output y of length k has the
 * code (1<<k)|y; codes lie in [1, 2^(n+1)), code 1 is the empty output and
 * slot 0 of every code-indexed array is unused (0).  Logs are base 2 (Sec. 2.1).
 *
 * Memory: the library never allocates device memory on the engine path.  The
 * caller allocates one device workspace of bdc_workspace_bytes() and binds it
 * with a CUDA stream; every kernel runs on that stream, in stream order.
 * Host pointers are read or written before the call returns.  Calls on one
 * engine must not overlap.  Errors are returned as bdc_status codes; no C++
 * exception crosses the ABI; bdc_last_error() gives a thread-local message.
 */
#ifndef BDC_H
#define BDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BDC_OK = 0,
    BDC_EINVAL = -1,      /* bad argument (sizes, ranges, NULL) */
    BDC_ENOMEM = -2,      /* workspace too small */
    BDC_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
    BDC_ETIMEOUT = -4,    /* a bounded device wait gave up */
    BDC_ENONFINITE = -5,  /* a NaN/Inf reached a reduction */
    BDC_ENOTBOUND = -6,   /* no workspace bound yet */
    BDC_ECHECK = -7       /* an index check of the checked build (compiled with -DBDC_CHECKS) failed: the
                             kernel recorded it in the instance status and skipped the access */
} bdc_status;

enum { BDC_FP32 = 0, BDC_FP64 = 1 };       /* precision of the iteration */
enum { BDC_SWEEP = 0, BDC_LITERAL = 1 };   /* algorithm of the iteration */

typedef struct bdc_engine bdc_engine;

typedef struct {
    /* Replace D by its mean over the complement/reversal orbit of x before
     * every p update (Appendix A: the iterates are orbit-invariant in exact
     * arithmetic; this removes rounding drift).  Default 1. */
    int symmetrize;
    /* Capture one iteration of all instances in a CUDA graph and replay it.
     * Default 1. */
    int use_graph;
    /* Iterations per graph launch when use_graph (default 8).  The host reads
     * the per-instance stop flags after each launch. */
    int chunk;
    /* Floor applied to the per-length output marginal before its log in BA
     * iterations (both precisions; keeps log2 finite if p underflowed in
     * FP32; 0 = no floor).  The certificate never floors.  Default 1e-30. */
    double q_floor;
    /* Weight of the uniform input mixed into p before certification, so the
     * certified output distribution is positive everywhere.  Default 2^-30. */
    double certify_mix;
    /* Row-sweep length n2 and column tile width override for the sweep
     * schedule (0 = automatic; a negative n2 selects the streaming schedule,
     * one global-memory pass per input symbol, which is what the automatic
     * choice is for FP64 at n >= 27, where no shared-memory tile split
     * exists). */
    int sched_n2_fp32, sched_w_fp32, sched_n2_fp64, sched_w_fp64;
    /* Reserve the buffers of the literal (enumeration) path.  Default 1. */
    int enable_literal;
    /* While p is complement-invariant (true for BA iterates from a uniform
     * start, Appendix A), compute only half of every sweep and mirror the
     * rest.  Default 1. */
    int use_half;
    /* Bit mask: run the first forward / last adjoint steps of a sweep tile
     * in registers (identical arithmetic, fewer shared-memory passes) in the
     * forward rows pass (1), the adjoint rows pass (2), and, in BA iterations,
     * the forward (4) and adjoint (8) columns passes, where the tile shape
     * allows.  Default 15; 0 keeps every step in shared memory. */
    int use_regsteps;
    /* Where the register-resident column kernels apply (bits 4 and 8 of
     * use_regsteps), run each BA iteration's boundary in one pass: the adjoint
     * columns pass of iteration t also applies the update and runs the
     * forward columns pass of t+1.  The orbit mean of D is then not taken
     * each iteration (the iterates are plain BA iterates, up to rounding);
     * the orbit mean of p is taken whenever the state is read, so p read back
     * is exactly orbit-invariant.  Default 1. */
    int fuse_update;
    /* In that one-pass boundary kernel (FP32, complement half mode, column
     * tiles of 4, n1 >= 9), load the tile with the Tensor Memory Accelerator
     * (cp.async.bulk.tensor) instead of per-thread loads: same values, same
     * arithmetic, bit-identical results.  Default 0: a tile column is 16
     * bytes per row, so each box is 256 separate 16-byte rows, and on B300
     * the per-thread 16-byte loads fill the tile faster (n = 24: 0.124 ms per
     * launch against 0.147 ms with TMA). */
    int use_tma;
    /* Polls of that kernel's wait for its TMA tile before it gives up, sets
     * BDC_ETIMEOUT for the instance, waits (bounded) for its copies still in
     * flight and returns.  0: the default, 2^22 polls (about a second); a
     * negative value: no poll at all, so the wait gives up at once (for
     * tests of the timeout path).  The wait for the copies in flight always
     * uses the default bound. */
    int tma_wait_polls;
} bdc_options;

/* Fill *opt with the defaults above. */
void bdc_default_options(bdc_options *opt);

/* --- lifecycle ---------------------------------------------------------- */

/* Create an engine for input length n (1 <= n <= 28) and nd >= 1 deletion
 * probabilities d[0..nd) in [0,1] (copied).  opt may be NULL (defaults).
 * Runs no kernel.  *out is owned by the caller (bdc_destroy). */
bdc_status bdc_create(int n, const double *d, int nd, const bdc_options *opt, bdc_engine **out);

/* Create an engine for a length-mixture deletion channel: instance z
 * outputs a length-k subsequence of x, chosen uniformly among the C(n,k)
 * choices of positions (so W(y|x) = b_k Count(y,x) / C(n,k) for |y| = k),
 * with k drawn from the distribution b[z][0..n] (host [nb][n+1], finite,
 * non-negative, positive sum; normalised here, copied).  b = the unit vector
 * at k is the exact deletion channel BDC_{n,k} of Sec. 2.2 (capacity
 * C_{n,k}); b_k = C(n,k) d^(n-k) (1-d)^k is BDC_d itself.  Every other call
 * works as for bdc_create, except that dF/dd of bdc_dual_bound is not
 * defined (BDC_EINVAL).  Errors: BDC_EINVAL. */
bdc_status bdc_create_lengths(int n, const double *b, int nb, const bdc_options *opt, bdc_engine **out);

/* Bytes of device workspace the engine needs (0 on NULL). */
size_t bdc_workspace_bytes(const bdc_engine *eng);

/* Bind a caller-owned device workspace (>= bdc_workspace_bytes, 256-byte
 * aligned) and a cudaStream_t (NULL = legacy default stream).  The engine
 * does not own the memory and must not outlive it.  Runs the d-free
 * precompute (orbit representatives; per representative x and length k the
 * number of distinct subsequences N_{x,k} and S_k(x) = sum count*log2(count),
 * Sec. 4.1 and Appendix A), the per-d entropy term, and sets p to uniform
 * (Sec. 2.3).  Synchronous. */
bdc_status bdc_bind(bdc_engine *eng, void *dev_workspace, size_t bytes, void *cuda_stream);

/* Free the host-side engine object (not the workspace). */
void bdc_destroy(bdc_engine *eng);

/* --- iteration ---------------------------------------------------------- */

/* Run up to max_iters BA iterations (Sec. 2.3) on every instance, in the
 * given precision (BDC_FP32 / BDC_FP64) and algorithm (BDC_SWEEP: factorised
 * forward/adjoint sweeps over all 2^n inputs; BDC_LITERAL: per-input
 * subsequence enumeration and per-output supersequence enumeration on orbit
 * representatives, Sec. 3-5 and Appendix A; FP64 only).  Iteration t uses p_t
 * and q_t for its bounds; an instance stops after the iteration whose gap
 * upper-lower is < gap_tol_bits (pass a negative value to never stop), and
 * its p then holds the updated input.  lower/upper/iters_done are host
 * arrays of nd (may be NULL): the bounds of the last iteration run and the
 * iterations run by this call.  Iterations continue from the current p. */
bdc_status bdc_ba_iterate(bdc_engine *eng, int max_iters, double gap_tol_bits, int precision, int impl,
                          double *lower, double *upper, int *iters_done);

/* Build, without running it, the CUDA graph that bdc_ba_iterate replays for
 * this precision and algorithm (use_graph = 1 and a non-NULL stream; a no-op
 * otherwise), so that the graph's capture and instantiation, a host-side cost
 * of milliseconds, happen before the first timed call.  Converts the state to
 * that precision like bdc_ba_iterate; advances no iteration.  Errors:
 * BDC_EINVAL (bad precision/algorithm), BDC_ECUDA (capture failed). */
bdc_status bdc_prepare(bdc_engine *eng, int precision, int impl);

/* A batch iterates several bound engines (different n, each with its own d
 * values) from one CUDA graph: every engine's iterations are captured on a
 * stream forked from their common stream, so small instances run
 * concurrently.  Engines must share one non-default stream and must not be
 * used elsewhere while the batch iterates.  Iterations run in multiples of
 * `chunk` (per launch of the graph); each instance still stops on its own
 * gap.  Results are read per engine (bdc_get_history, bdc_certify_upper). */
typedef struct bdc_batch bdc_batch;
bdc_status bdc_batch_create(bdc_engine *const *engines, int count, int chunk, bdc_batch **out);
/* Sweep path only.  *iters_launched = iterations the graph ran (a multiple of
 * chunk, at least max_iters unless every instance stopped earlier). */
bdc_status bdc_batch_iterate(bdc_batch *batch, int max_iters, double gap_tol_bits, int precision,
                             int *iters_launched);
void bdc_batch_destroy(bdc_batch *batch);

/* Copy the per-iteration bound history of instance inst (the last
 * min(len, 8192) iterations since bdc_bind or bdc_set_p) into host arrays;
 * returns the number of entries written in *count. */
bdc_status bdc_get_history(bdc_engine *eng, int inst, double *lower, double *upper, int len, int *count);

/* D_x for every instance and every x, in double precision, into the caller's
 * device array D_dev [nd][2^n].  q_dev NULL: q from the current p (computed
 * in `precision`); otherwise q_dev is a device array [nd][2^(n+1)] of the
 * given precision (float or double), indexed by code, any positive values
 * (it is normalised internally: D uses q/sum q). */
bdc_status bdc_divergence(bdc_engine *eng, const void *q_dev, int precision, double *D_dev);

/* Certified upper bound on C_n(d) per instance, in FP64 with an explicit
 * rounding-error margin (the dual bound max_x D(W_x || q/sum q) holds for
 * every positive q).  q_dev NULL: q is the FP64 output marginal of the
 * current p mixed with certify_mix of the uniform input; otherwise a device
 * array [nd][2^(n+1)] of doubles (positive at every code).  Host arrays of
 * nd: upper (the certified bound, rounded up), margin (the added rounding
 * margin, bits), lower (FP64 Blahut lower bound of the current p; NaN when
 * q_dev is given).  Any may be NULL.  When every instance's mixed input is
 * exactly complement-invariant (checked on the device; true for BA iterates
 * from a complement-invariant start) and the FP64 schedule splits, the two
 * FP64 sweeps compute half of the values and mirror the rest (use_half = 0
 * turns this off); the bound is the same.  Errors: BDC_ENONFINITE (a NaN or
 * Inf in the given q, or a non-finite bound), BDC_EINVAL (a given q that is
 * not positive at every code); the values of the other instances are valid. */
bdc_status bdc_certify_upper(bdc_engine *eng, const double *q_dev, double *upper, double *margin, double *lower);

/* --- state access (caller-owned host buffers, copied) -------------------- */

/* p of every instance, normalised, host [nd][2^n]. */
bdc_status bdc_get_p(bdc_engine *eng, double *p_host);
/* Set p of every instance from host [nd][2^n] (non-negative, positive sum;
 * normalised here).  Clears the bound history.  A p that is not invariant
 * under complement (and reversal) switches off the half-sweep mode (and the
 * orbit mean of D, and the literal path, which then returns BDC_EINVAL). */
bdc_status bdc_set_p(bdc_engine *eng, const double *p_host);
/* Output marginal q of the current p, host [nd][2^(n+1)] by code, computed in
 * the given precision. */
bdc_status bdc_get_q(bdc_engine *eng, int precision, double *q_host);
/* Output marginal q of the current p computed by the literal path (FP64:
 * for each output class representative y, the sum over its supersequences
 * x of p(x) Count(y,x), Sec. 5 and Appendix A), host [nd][2^(n+1)] by code,
 * normalised like bdc_get_q.  Needs enable_literal and an orbit-invariant p
 * (else BDC_EINVAL).  Switches the engine to the literal representation of
 * p, like a literal iteration. */
bdc_status bdc_get_q_literal(bdc_engine *eng, double *q_host);
/* d-free precompute of representative r (0 <= r < number of reps): its
 * input string, orbit size, N_{x,k} and S_k for k = 0..n (host arrays of
 * n+1). */
bdc_status bdc_get_rep_stats(bdc_engine *eng, int64_t r, uint64_t *x, int *orbit, uint64_t *N_k, double *S_k);
/* Number of orbit representatives of {0,1}^n. */
int64_t bdc_num_reps(const bdc_engine *eng);
/* Save / restore p and the iteration count to a file (binary; the channel,
 * d values or length weights, is stored and must match on load). */
bdc_status bdc_save(bdc_engine *eng, const char *path);
bdc_status bdc_load(bdc_engine *eng, const char *path);

/* --- smoothed dual bound and its adjoint ---------------------------------- */

/* Number of output orbit classes (strings of every length up to n under
 * complement and reversal, Appendix A). */
int64_t bdc_num_output_classes(const bdc_engine *eng);
/* Class index of every code, host int64 [2^(n+1)] (slot 0 = -1). */
bdc_status bdc_output_classes(bdc_engine *eng, int64_t *cls_host);

/* F = tau log2 sum_x 2^{D_x(q)/tau} for instance inst, with q the softmax of
 * theta over output classes (theta_dev: device array of num_output_classes
 * in `precision`).  Gradients (computed by forward and adjoint sweeps, never
 * storing W): grad_theta_dev (device, same type and length as theta; may be
 * NULL) and *grad_d = dF/dd at fixed theta (may be NULL; needs 0 < d < 1).
 * *F and *max_D (max_x D_x, the bound itself) are host doubles. */
bdc_status bdc_dual_bound(bdc_engine *eng, int inst, const void *theta_dev, double tau, int precision,
                          double *F, double *max_D, void *grad_theta_dev, double *grad_d);

/* q = softmax of theta over output classes, written for every code into the
 * caller's device array q_dev (doubles [2^(n+1)], slot 0 = 0), e.g. to
 * certify an optimised q with bdc_certify_upper (one instance: pass a
 * q_dev of nd rows when nd > 1).  theta_dev as in bdc_dual_bound. */
bdc_status bdc_softmax_classes(bdc_engine *eng, int inst, const void *theta_dev, int precision, double *q_dev);

/* Logits of an output distribution over classes: theta_dev[r] = ln max(q(c_r),
 * floor) for the representative code c_r of every output class r (q_dev:
 * device doubles [2^(n+1)] by code, orbit-invariant and normalised; theta_dev:
 * device array of num_output_classes in `precision`).  softmax over classes
 * of the result is q again (the inverse of bdc_softmax_classes), e.g. to
 * start the dual-bound optimisation from a BA output marginal.  Synchronous.
 * Errors: BDC_EINVAL, BDC_ECUDA. */
bdc_status bdc_class_logits(bdc_engine *eng, const double *q_dev, double floor, int precision, void *theta_dev);

/* --- measurement --------------------------------------------------------- */

/* Number of kernels this engine has launched so far (kernels replayed inside
 * CUDA graphs included). */
int64_t bdc_launch_count(const bdc_engine *eng);

/* Run `reps` iterations without graphs, recording a CUDA event on the bound
 * stream after every stage (one kernel each), and return the mean time per
 * stage in milliseconds (stage_ms, host array of >= 32), the stage names as
 * a comma-separated list (names, host buffer of names_len bytes, may be
 * NULL) and the number of stages.  The iterations are real BA iterations:
 * they advance p like bdc_ba_iterate. */
bdc_status bdc_profile_iteration(bdc_engine *eng, int precision, int impl, int reps, double *stage_ms, char *names,
                                 int names_len, int *nstages);

/* Microbenchmarks of this device, run on cuda_stream and timed with CUDA
 * events (the peaks the sweep and walk kernels are measured against):
 * out[0] = FP32 FMA instructions per second / 1e12 (an add takes the same
 * pipe slot), out[1] = the same in FP64, out[2] = L2 read bandwidth in GB/s
 * (a 32 MiB buffer read over repeatedly), out[3] = shared-memory bandwidth
 * in TB/s (16-byte accesses), out[4] = number of SMs.  scratch_dev: device
 * buffer of at least 64 MiB, 16-byte aligned, caller-owned (overwritten).
 * Synchronous.  Errors: BDC_EINVAL, BDC_ECUDA. */
bdc_status bdc_measure_peaks(void *scratch_dev, size_t bytes, void *cuda_stream, double *out);

/* Schedule of the sweep in `precision`: input split n1 + n2 (n2 = 0: one
 * pass; n2 = -1: the streaming schedule) and the column tile width. */
bdc_status bdc_get_schedule(const bdc_engine *eng, int precision, int *n1, int *n2, int *width);

/* Autotune the sweep schedule of `precision` on this engine: time `reps`
 * forward + adjoint sweeps of every candidate split (n2 in [max(8, n-14),
 * 13 or 14]) and column width, keep the fastest (*best_ms = its time per
 * forward + adjoint pair).  With n2 > 0, set that schedule instead of
 * searching (e.g. from a cache).  The current p is kept (its pending update
 * is applied first); cached graphs are rebuilt on the next iteration. */
bdc_status bdc_autotune(bdc_engine *eng, int precision, int reps, int n2, int width, double *best_ms);

/* --- test hook ------------------------------------------------------------ */

/* For nx inputs x_dev[i] (device uint64) of length n <= 32: per input and
 * length k = 0..n the number of distinct subsequences (N_dev, device uint64
 * [nx][n+1]) and S_k = sum count*log2(count) over them (S_dev, device double
 * [nx][n+1], may be NULL); if nx == 1 and emb_dev != NULL, also the
 * embedding count of every code (device uint64 [2^(n+1)], zero where y is
 * not a subsequence).  Runs the same warp-cooperative enumeration as the
 * precompute, on `stream`.  Synchronous. */
bdc_status bdc_subseq_counts(int n, const uint64_t *x_dev, int64_t nx, uint64_t *N_dev, double *S_dev,
                             uint64_t *emb_dev, void *cuda_stream);

/* --- allocation-free variant ------------------------------------------------ */

/* Output marginal q(y) = sum_x p(x) W(y|x) of BDC_d for one d, computed by
 * the same forward sweep as the engine but without an engine, a workspace or
 * any device allocation.  It exists for callers that cannot allocate device
 * memory (inside someone else's stream capture, under a host framework that
 * owns all allocations, or under strict memory accounting); the paper has no
 * counterpart.  Its scratch lives in one fixed device array inside the
 * library (about 10.5 MB, held by every GPU that loads the library until the
 * process exits), so 1 <= n <= 18.  p_dev: device doubles [2^n]; q_dev:
 * device doubles [2^(n+1)] by code (slot 0 written 0).  Runs on cuda_stream
 * (NULL = legacy default stream) and returns without synchronising.  All
 * calls on a device share the array: calls that overlap on the GPU race, so
 * the caller orders them.  The first call on a device does a one-time
 * set-up (looks up the array's address, sets shared-memory limits) and must
 * come before any stream capture.  n > 18 or bad arguments: BDC_EINVAL. */
bdc_status bdc_output_marginal_static(int n, double d, const double *p_dev, double *q_dev, void *cuda_stream);

/* --- bound post-processing (host only, Sec. 6) ----------------------------- */

/* Lemma prob-vs-exact (Sec. 2.2): *Cn_d = sum_{k=1}^n C(n,k) d^(n-k)
 * (1-d)^k Cnk[k], an upper bound on C_n(d) when Cnk[k] >= C_{n,k} (host
 * array of n+1, index k; Cnk[0] unused).  Long double sum of non-negative
 * terms, rounded up.  1 <= n <= 64, 0 <= d <= 1.  Errors: BDC_EINVAL. */
bdc_status bdc_bound_prob_vs_exact(int n, double d, const double *Cnk, double *Cn_d);

/* Lemma worse-UB (Sec. 6): *Cnk = sum_{i=0}^s C(s,i) C(n-s,k-i) / C(n,k)
 * (Cs[i] + Cns[k-i]), an upper bound on C_{n,k} when Cs[i] >= C_{s,i}
 * (host [s+1]) and Cns[j] >= C_{n-s,j} (host [n-s+1]).  Terms with k-i
 * outside [0, n-s] have weight 0.  Rounded up.  2 <= n <= 64, 0 <= k <= n,
 * 1 <= s < n.  Errors: BDC_EINVAL. */
bdc_status bdc_bound_split(int n, int k, int s, const double *Cs, const double *Cns, double *Cnk);

/* Lemma convex (Sec. 6, Rahmati and Duman): C(d)/(1-d) <= C(d')/(1-d') for
 * every d in [d', 1].  From an upper bound C_dp on C(d'), writes *Cd >= C(d)
 * and *ratio >= C(d')/(1-d') (either may be NULL), rounded up.
 * Errors: BDC_EINVAL (d' outside [0,1), d outside [d',1], C_dp < 0). */
bdc_status bdc_bound_high_noise(double d_prime, double C_dp, double d, double *Cd, double *ratio);

/* Thread-local message of the last failing call on this thread. */
const char *bdc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BDC_H */
