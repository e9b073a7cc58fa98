/*
 * tc.h -- C ABI of a single-GPU (GB300, sm_103a) library for the (T) triples
 * correction of closed-shell, canonical-orbital CCSD(T).
 *
 * What is computed (Fajen, Kelly, Hohenstein, Martinez, "Accelerating CCSD(T)
 * on GPUs", arXiv 2512.01055, Implementation Details, Eqs. 1-5):
 *
 *   E_(T) = sum_{a>=b>=c} (2 - d_ab - d_bc) sum_{ijk} (W + V)_ijk^abc
 *           (4 W_ijk + W_jki + W_kij - 2 W_jik - 2 W_ikj - 2 W_kji)^abc / D_ijk^abc      (Eq. 1)
 *   W_ijk^abc = P_ijk^abc [ sum_f G_if^ab t_kj^cf - sum_l G_ij^al t_lk^bc ]                  (Eqs. 2, 5)
 *   V_ijk^abc = t_i^a G_jk^bc + t_j^b G_ik^ac + t_k^c G_ij^ab                                 (Eq. 3)
 *   D_ijk^abc = e_i + e_j + e_k - e_a - e_b - e_c                                             (Fig. 4)
 *
 * with G_pq^rs = (pr|qs) (Mulliken) real two-electron integrals.  The library
 * assumes the symmetries of real orbitals, (ia|bd) = (ia|db) and
 * t_ij^ab = t_ji^ba; it does not check them.
 *
 * Array conventions (all row-major, C-contiguous, IEEE binary64):
 *   eps  [o + v]         orbital energies, occupied first
 *   t1   [o][v]          t_i^a
 *   t2   [o][o][v][v]    t2[i][j][a][b] = t_ij^ab
 *   ovvv [o][v][v][v]    ovvv[i][a][b][d] = (ia|bd)
 *   ovoo [o][v][o][o]    ovoo[i][a][j][l] = (ia|jl)
 *   ovov [o][v][o][v]    ovov[i][a][j][b] = (ia|jb)
 * Indices: occupied i,j,k,l in [0,o); virtual a,b,c,d in [0,v).
 *
 * Ownership: the caller owns every array passed in.  Host arrays are copied
 * before tc_energy / tc_submit return; device arrays passed to tc_energy_dev
 * are read in place and must stay valid until that call returns.
 *
 * Errors: every entry point returns a tc_status; no exception, abort or
 * longjmp crosses this boundary.  The text of the last failure of a context is
 * available from tc_last_error.
 */
#ifndef TC_H
#define TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_ctx tc_ctx;

typedef enum {
  TC_OK = 0,
  TC_EINVAL = 1,       /* bad argument: o or v <= 0, NULL array, slices out of range ... */
  TC_ENOMEM = 2,       /* the job does not fit the HBM budget (refused before any work) */
  TC_ECUDA = 3,        /* a CUDA runtime call failed; see tc_last_error */
  TC_ENOTREADY = 4,    /* tc_poll: the job has not finished yet */
  TC_ETIMEOUT = 5,     /* tc_wait gave up, or a device-side wait hit its limit */
  TC_EBUSY = 6,        /* the request queue is full */
  TC_ECANCELLED = 7,   /* the job was cancelled */
  TC_EINTERNAL = 8     /* a device-side consistency check failed */
} tc_status;

typedef enum {
  TC_FP64 = 0,         /* W built with FP64 tensor-core (DMMA) tiles, FP64 everywhere */
  TC_SPLIT_BF16 = 1    /* W built from BF16 slices on tcgen05 tensor cores, FP32 accumulation;
                          V and the Eq. 1 bracket in FP32; D, 1/D, each point's quotient and
                          the sums over a work item in float pairs (~48 significant bits);
                          FP64 per triplet; compensated (Neumaier) FP64 total */
} tc_precision;

typedef struct {
  int device;                /* CUDA device ordinal */
  size_t hbm_budget_bytes;   /* device bytes the context may hold; 0 = 90% of free memory at init */
  int default_prec;          /* tc_precision used when a call passes prec < 0 */
  int default_slices;        /* BF16 slices per operand (2..4) used when a call passes slices <= 0 */
  int timeout_ms;            /* limit for tc_wait and for device-side waits; 0 = 60000 */
  int max_inflight;          /* serving: jobs admitted to the device at once (1..32; 0 = 16) */
  int max_queue;             /* serving: jobs waiting for admission before tc_submit says TC_EBUSY (0 = 4096) */
  int iteration_ms;          /* serving: target duration of one batched launch (0 = 50) */
} tc_options;

typedef struct {
  const double *ovvv;        /* [o][v][v][v] (ia|bd) */
  const double *ovoo;        /* [o][v][o][o] (ia|jl) */
  const double *ovov;        /* [o][v][o][v] (ia|jb) */
} tc_ints;

typedef struct {
  double e_t;                /* E_(T) in Eh */
  double seconds;            /* wall time of the call (tc_energy / tc_energy_dev) or of the job */
  double tflops_alg;         /* 2 (o^3 v^4 + o^4 v^3) / seconds / 1e12 */
  int prec;                  /* precision actually used */
  int slices;                /* BF16 slices per operand (0 for TC_FP64) */
  int o, v;
  double queue_seconds;      /* serving: time from tc_submit to the start of its GPU work */
  double kernel_seconds;     /* device time of the W/V/energy kernels (CUDA events on the call's stream):
                                FP64, the fused kernel; split path, all W-term and energy launches */
  double prep_seconds;       /* device time of the slicing / re-layout kernels (split path), else 0 */
  long long n_items;         /* energy work items (triplet x tile-orbit chunk) processed */
  int launches;              /* kernels this call launched */
  int reserved;
  double wterm_seconds;      /* device time of the kernels that form W: FP64, the fused kernel (= kernel_seconds);
                                split path, the W-term GEMM launches alone (blocking entry points only) */
  double e_t5;               /* E[5]_ST: the part of E_(T) from the V factor of Eq. 1, sum (V r3(W))/D with the
                                same weights; E[4] = e_t - e_t5 is the W r3(W)/D part (r3 is the bracket of Eq. 1) */
  double df_seconds;         /* tc_energy_df(_dev): device time of the integral assembly from the DF
                                factors (digit images + three tensor-core digit products), else 0 */
  int df_digits;             /* tc_energy_df(_dev): base-256 digits per factor value the assembly used
                                (1..7; 3 for factors on a 2^-20 grid), else 0 */
  int reserved2;
} tc_result;

/* Create a context on opt->device (opt may be NULL: device 0, defaults).
 * Allocates nothing large; device memory is reserved per job and reused. */
tc_status tc_init(tc_ctx **ctx, const tc_options *opt);

/* E_(T) from HOST arrays (Eqs. 1-5).  Blocking.  Copies the inputs to the
 * device, runs the hot path, returns E_(T) in out->e_t.  On the split path
 * t2, ovvv, ovoo and ovov are copied on a second stream in chunks of their
 * first (occupied) index, and each chunk is sliced just before the first
 * block of triplets that reads it, so from page-locked host arrays the copies
 * overlap the tensor-core work (pageable arrays work too, without the
 * overlap); prep_seconds then sums the slicing of all chunks, and
 * kernel_seconds includes the later chunks' slicing and any wait for their
 * copies.  No copy reads the caller's arrays after the call returns.
 * prec: tc_precision, or < 0 for the context default.  slices: 2..4 for
 * TC_SPLIT_BF16, <= 0 for the default; ignored for TC_FP64.
 * e_ijk (optional, may be NULL): host array [o][o][o] that receives the
 * weighted contribution of each occupied triplet i >= j >= k at [i][j][k]
 * (E_(T) is their sum); entries with i < j or j < k are set to 0. */
tc_status tc_energy(tc_ctx *ctx, int o, int v, const double *eps, const double *t1,
                    const double *t2, const tc_ints *ints, int prec, int slices,
                    double *e_ijk, tc_result *out);

/* Same as tc_energy with every array a DEVICE pointer (e.g. a PyTorch tensor's
 * data_ptr on ctx's device), read in place.  stream: a cudaStream_t (NULL =
 * legacy default stream) on which all work is enqueued; the call returns after
 * that work completes.  e_ijk_dev (optional): DEVICE array [o][o][o] as above. */
tc_status tc_energy_dev(tc_ctx *ctx, int o, int v, const double *eps, const double *t1,
                        const double *t2, const tc_ints *ints, int prec, int slices,
                        double *e_ijk_dev, void *stream, tc_result *out);

/* Same as tc_energy_dev with the integrals given as density-fitting (or
 * Cholesky) factors instead of integral arrays (Eq. 6 of the paper):
 *   B   DEVICE array [nq][o+v][o+v], B[Q][p][q] with occupied p, q first, so
 *       that (pq|rs) = sum_Q B[Q][p][q] B[Q][r][s] (Mulliken notation).
 *   nq  number of factors Q (> 0).
 * The library assembles (ia|bd), (ia|jl) and (ia|jb) on the device in its own
 * memory (grow-only, reused by later calls), then computes the energy as
 * tc_energy_dev.  Only B, eps, t1 and t2 cross from the caller.  The assembly
 * runs on the BF16 tensor cores as products of base-256 digits: each row of a
 * factor block is scaled by a power of two and its values split into up to 7
 * signed 8-bit digits; digit products are exact and summed exactly (integer
 * class sums), so an integral carries one final rounding.  Factors whose
 * values need at most 3 digits (e.g. values on a 2^-20 grid below 1 in
 * magnitude) give every integral exactly; general FP64 factors use 7 digits
 * and keep the digit pairs p + q <= 6, an error below 2^-45 of the largest
 * |B_pq^Q B_rs^Q| summed over Q.  The call synchronises the stream once (to
 * read the digit count).
 * out->df_seconds is the device time of the assembly; kernel_seconds and
 * wterm_seconds cover the energy as for tc_energy_dev.  Errors as
 * tc_energy_dev, plus TC_EINVAL for nq <= 0 or a NULL B, and TC_ENOMEM when
 * the assembled integrals do not fit the context's budget. */
tc_status tc_energy_df_dev(tc_ctx *ctx, int o, int v, int nq, const double *eps, const double *t1,
                           const double *t2, const double *B, int prec, int slices,
                           double *e_ijk_dev, void *stream, tc_result *out);

/* Same as tc_energy_df_dev with eps, t1, t2 and B as HOST arrays (copied to
 * the device, on the context's stream, before the call returns; the caller
 * keeps ownership).  e_ijk (optional): HOST array [o][o][o] as in tc_energy. */
tc_status tc_energy_df(tc_ctx *ctx, int o, int v, int nq, const double *eps, const double *t1,
                       const double *t2, const double *B, int prec, int slices, double *e_ijk,
                       tc_result *out);

/* Weighted contributions of selected occupied triplets (the i >= j >= k
 * regrouping of Eq. 1: E_(T) is the sum over all triplets).  Same inputs as
 * tc_energy_dev (DEVICE pointers, read in place).
 *   trip   HOST array [n][3] of (i, j, k) with o > i >= j >= k >= 0, any order,
 *          repeats allowed.
 *   e_out  HOST array [n]: e_out[m] receives the contribution of trip[m]
 *          (0 when i == j == k).
 * Uses: checking sampled triplets of a large job against a reference,
 * splitting one energy across devices or calls, resuming by triplet range.
 * out->e_t is the sum of e_out.  TC_EINVAL on an out-of-range or unordered
 * triplet (nothing is launched). */
tc_status tc_triplets_dev(tc_ctx *ctx, int o, int v, const double *eps, const double *t1,
                          const double *t2, const tc_ints *ints, int prec, int slices,
                          const int *trip, int n, double *e_out, void *stream, tc_result *out);

/* ------------------------------------------------------------------------
 * One energy over several devices or processes.  The paper hands each GPU a
 * batch of the work and scales the (T) step over GPUs (Implementation
 * Details; Results, Figs. 5-6).  Here the units are the occupied triplets
 * i >= j >= k of the regrouped Eq. 1 (all-equal ones excluded: their
 * contribution is exactly zero), which are independent of one another and
 * cost the same; rank r of W takes the contiguous range [n r / W, n (r+1) / W)
 * of their order (i, j, k) lexicographic.  Each rank needs all the inputs.
 * The only exchange is one gather of a (sum, compensation) pair per rank,
 * combined in rank order by tc_combine_parts, so every rank obtains the same
 * bits whatever the collective's own order.
 * ------------------------------------------------------------------------ */

/* First triplet (index in the order above) and number of triplets of rank
 * `rank` of `world` for o occupied orbitals.  Pure host arithmetic.
 * TC_EINVAL for o <= 0, world <= 0 or rank outside [0, world). */
tc_status tc_shard_range(int o, int rank, int world, long long *first, long long *count);

/* This rank's share of E_(T): inputs as tc_energy_dev (DEVICE pointers, read
 * in place, work on `stream`).  part: HOST array [2] that receives the
 * Neumaier-compensated sum of the range's triplet contributions, in order, as
 * (sum, compensation); out->e_t = part[0] + part[1].  A rank with an empty
 * range launches nothing and returns (0, 0).  Errors as tc_energy_dev, plus
 * TC_EINVAL for an invalid (rank, world). */
tc_status tc_energy_shard_dev(tc_ctx *ctx, int o, int v, const double *eps, const double *t1,
                              const double *t2, const tc_ints *ints, int prec, int slices, int rank,
                              int world, double *part, void *stream, tc_result *out);

/* (sum, compensation) of n host values x[0..n) in order (Neumaier): part[2].
 * The rank-local step of tc_energy_shard_dev, for callers that hold the
 * contributions themselves.  Pure host arithmetic. */
tc_status tc_sum_parts(const double *x, long long n, double *part);

/* E_(T) from the gathered pairs parts[n][2] of ranks 0 .. n-1: compensated
 * sum of the sums in rank order plus all compensations.  Pure host
 * arithmetic; the same inputs give the same bits on every rank. */
tc_status tc_combine_parts(const double *parts, int n, double *e_t);

/* ------------------------------------------------------------------------
 * Serving: many (T) jobs of uneven (o, v) and mixed precision on one device.
 *
 * tc_submit queues a job and returns at once.  A scheduler owned by the
 * context admits queued jobs while at most max_inflight are admitted and the
 * sum of their device footprints (inputs unless resident, work tables, BF16
 * images) stays within hbm_budget_bytes; admitted jobs are prepared on side
 * streams while others compute.  Computation proceeds in iterations of about
 * iteration_ms: each iteration is one persistent multi-job launch (replayed
 * from a CUDA graph) over a slice of the items of every ready job of one
 * precision group, the slices shared fairly, so a job submitted while others
 * run starts within an iteration and small jobs are not stuck behind large
 * ones.  A job's result does not depend on the other jobs it ran with.
 * ------------------------------------------------------------------------ */
#define TC_JOB_DEVICE_INPUTS 1   /* tc_job arrays are DEVICE pointers, kept valid and
                                    unchanged by the caller until the job completes */

typedef struct {
  int o, v;
  const double *eps, *t1, *t2;   /* layouts as for tc_energy */
  tc_ints ints;
  int prec;                      /* tc_precision, or < 0 for the context default */
  int slices;                    /* TC_SPLIT_BF16: 2..4, <= 0 for the default */
  int flags;                     /* 0: host arrays, copied before tc_submit returns;
                                    TC_JOB_DEVICE_INPUTS: resident device arrays, not copied */
  int nq;                        /* > 0: the integrals come from the density-fitting factors B
                                    (Eq. 6) and ints is ignored (may hold NULLs); 0: from ints */
  const double *B;               /* nq > 0: [nq][o+v][o+v] as for tc_energy_df, host or device per
                                    flags; the service assembles the integrals on the device when it
                                    admits the job (in the job's own memory, counted in its footprint) */
} tc_job;

/* Queue a job.  *ticket identifies it in tc_poll / tc_wait / tc_cancel.
 * TC_EINVAL bad job; TC_ENOMEM its footprint alone exceeds the budget;
 * TC_EBUSY the queue holds max_queue jobs already. */
tc_status tc_submit(tc_ctx *ctx, const tc_job *job, uint64_t *ticket);

/* TC_ENOTREADY while the job is queued or running.  Otherwise fills *out
 * (e_t; seconds = submit to completion; queue_seconds = submit to its first
 * iteration), releases the ticket and returns the job's status (TC_OK,
 * TC_ECANCELLED, or the error it failed with).  Unknown ticket: TC_EINVAL. */
tc_status tc_poll(tc_ctx *ctx, uint64_t ticket, tc_result *out);

/* As tc_poll, waiting up to timeout_ms (< 0: ctx timeout) for completion;
 * TC_ETIMEOUT if the job is still pending then (the ticket stays valid). */
tc_status tc_wait(tc_ctx *ctx, uint64_t ticket, int timeout_ms, tc_result *out);

/* Cancel a job that has not been admitted yet (TC_OK); TC_EBUSY once it is
 * admitted; TC_EINVAL unknown ticket. */
tc_status tc_cancel(tc_ctx *ctx, uint64_t ticket);

typedef struct {
  uint64_t submitted, completed, failed, cancelled;
  uint64_t queued, inflight;      /* now */
  uint64_t iterations, graph_launches, batched_jobs;   /* batched_jobs: sum over iterations of jobs per launch */
  size_t reserved_bytes;          /* device bytes held by admitted jobs now */
} tc_serve_stats;
tc_status tc_serve_stats_get(tc_ctx *ctx, tc_serve_stats *out);

/* Host-side fault injection for tests (nothing is faulted on the device):
 * TC_FAULT_ALLOC: the next admission behaves as if device allocation failed
 * (that job fails with TC_ENOMEM); TC_FAULT_STALL: the scheduler pauses for
 * param milliseconds before its next iteration. */
#define TC_FAULT_ALLOC 1
#define TC_FAULT_STALL 2
tc_status tc_inject_fault(tc_ctx *ctx, int kind, int param);

/* Size of the library's static device scratch array used by
 * tc_energy_dev_noalloc (held on every GPU that loads the library). */
#define TC_NOALLOC_SCRATCH_BYTES ((size_t)8 << 20)

/* FP64 E_(T) for callers that cannot allocate device memory.  The paper has
 * no counterpart; this entry point exists for code that runs where it may not
 * call cudaMalloc -- inside a host runtime that owns every device allocation
 * (fixed pools, embedded solvers, plugins), or where a new allocation could
 * fail or fragment memory mid-run.
 *
 * Same computation and input layouts as tc_energy_dev with prec = TC_FP64, but
 * no context: it runs on the current device and allocates nothing (no
 * cudaMalloc/cudaFree, no allocating library call).  Its scratch -- work
 * tables, partial sums, the work counter -- lives in one static device array
 * of TC_NOALLOC_SCRATCH_BYTES, shared by every call.
 *   e_t_dev    DEVICE pointer to one double that receives E_(T) (required).
 *   e_ijk_dev  optional DEVICE array [o][o][o] of per-triplet contributions.
 *   stream     cudaStream_t (NULL = legacy default stream).  The call only
 *              enqueues work; results are valid once that stream reaches them.
 *   errbuf     optional buffer (errlen bytes) for a message on failure.
 * Returns TC_ENOMEM, without enqueuing anything, when the job's scratch would
 * exceed TC_NOALLOC_SCRATCH_BYTES (roughly: more than ~2.5e5 tile orbits).
 * The first call on a device looks up the array's device address and sets
 * the kernel's shared-memory limit; make that call before any stream capture.
 * The address is then kept per device ordinal for the life of the process:
 * it belongs to the device's primary context (the one the CUDA runtime uses),
 * so call this with that context current and do not reset the device
 * (cudaDeviceReset) between calls.
 * Calls whose GPU work overlaps race on the shared array: serialise them. */
tc_status tc_energy_dev_noalloc(int o, int v, const double *eps, const double *t1,
                                const double *t2, const tc_ints *ints, double *e_t_dev,
                                double *e_ijk_dev, void *stream, char *errbuf, size_t errlen);

/* Device bytes a job of this shape and precision needs besides its inputs
 * (work tables, partial sums; split path also the BF16 operand images, FP32
 * copies and the W buffer of one block of triplets).  Pure host arithmetic. */
size_t tc_workspace_bytes(int o, int v, int prec, int slices);

/* Human-readable name of a status. */
const char *tc_status_str(tc_status s);

/* Text of the last failure recorded on ctx ("" if none). */
const char *tc_last_error(tc_ctx *ctx);

/* Release everything the context holds.  ctx may be NULL. */
void tc_finalize(tc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TC_H */
