/*
 * cn.h -- C ABI of the B300-native N-shaped partition Crank-Nicolson library
 * (libcn_b300.so).
 *
 * Method: Lutsyshyn, Navarrete, Bauer, "The N-shaped partition method: A novel
 * parallel implementation of the Crank Nicolson algorithm".
 *
 * One Crank-Nicolson step of the 1D TDSE  i d/dt psi = H(t) psi,
 * H = -1/2 d^2/dx^2 + V(x, t) on the grid x_j = x_min + j dx (j = 0..n-1,
 * psi = 0 outside, Sec. 4), is (Sec. 2, Eq. Cn_both_steps)
 *     d = T^dagger psi(t)            (explicit forward half-step, Eq. ForwardStep)
 *     T psi(t + dt) = d              (implicit backward half-step, Eq. BackwardStep)
 *     T = 1 + i dt/2 H(t + dt/2)
 * with the 3-point stencil: T_jj = 1 + i dt/2 (1/dx^2 + V_j),
 * T_{j,j+-1} = -i dt / (4 dx^2).  The tridiagonal solve is the N-shaped
 * partition method of Sec. 4 (Table 1: RD, JD, RU, JU, RS, SS), applied
 * recursively to its reduced system as in Eq. (iteration).
 *
 * Conventions for every entry point:
 *   - complex values are complex128: interleaved (re, im) IEEE doubles, 16 B
 *     per element (the layout of torch.complex128 / numpy complex128),
 *     contiguous, 16-byte aligned;
 *   - "device pointer" means memory the caller allocated on the CUDA device
 *     the plan was created on; the caller keeps ownership; the library never
 *     frees it;
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); device
 *     work is enqueued on it and the call returns without synchronising,
 *     except where stated; the kernels are launched with programmatic
 *     stream serialization, so one may be scheduled while the work before
 *     it in the stream still runs, but each waits on the device for that
 *     work to complete before it reads or writes any memory: the effects
 *     are in plain stream order;
 *   - argument errors are detected on the host before any work is enqueued
 *     and returned as a cn_status; nothing is enqueued then;
 *   - errors raised on the device (non-finite pivots, exhausted waits) are
 *     recorded in the plan's device status word and returned by
 *     cn_plan_status();
 *   - no function throws or aborts; a plan must not be used from two host
 *     threads at once, and calls that share a plan must be ordered on one
 *     stream (they share the plan's workspace).
 */
#ifndef CN_B300_H
#define CN_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cn_plan_s* cn_plan;
typedef struct cn_batch_s* cn_batch;

typedef enum {
    CN_OK = 0,
    CN_ERR_INVALID_ARG = 1,  /* bad size, pointer, alignment or descriptor field */
    CN_ERR_UNSUPPORTED = 2,  /* valid request this build does not implement      */
    CN_ERR_OOM = 3,          /* device workspace allocation failed               */
    CN_ERR_CUDA = 4,         /* a CUDA runtime call failed                       */
    CN_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out               */
    CN_ERR_NONFINITE = 6,    /* a pivot or result was zero / inf / NaN           */
    CN_ERR_BOUNDS = 7        /* debug build: an access outside every registered
                                buffer was caught and skipped (cn_debug_report)  */
} cn_status;

/* Static part Vs(x) of V(x, t) = Vs(x) + x E(t) (length-gauge field term). */
typedef enum {
    CN_POT_NONE = 0,         /* Vs = 0                                                     */
    CN_POT_ARRAY = 1,        /* Vs(x_j) = V0[j], V0 a device array of n doubles              */
    CN_POT_SOFTCOULOMB = 2,  /* Vs(x) = -1 / sqrt(x^2 + soft_s), regenerated on the fly      */
    CN_POT_COSSERIES = 3     /* Vs(x) = sum_{k=1..n_cos} cos_a[k-1] cos(2 pi k x / L)        */
} cn_pot_kind;

/* Arithmetic the solver runs in.  Inputs and outputs are complex128 in both. */
typedef enum {
    CN_ARITH_F64 = 0,        /* native IEEE binary64                                       */
    CN_ARITH_DF64 = 1        /* double-float: value = hi + lo, two binary32 words (~48-bit
                                significand; Dekker 1971, Joldes-Muller-Popescu 2017)        */
} cn_arith;

typedef struct {
    int64_t n;               /* grid points (unknowns), n >= 3                              */
    double dx, dt, x_min;    /* grid spacing, time step, first grid point                   */
    int32_t pot;             /* cn_pot_kind                                                  */
    int32_t n_cos;           /* CN_POT_COSSERIES: number of terms, 0..16                     */
    const double* V0;        /* CN_POT_ARRAY: device pointer, n doubles, read at every step  */
    double soft_s;           /* CN_POT_SOFTCOULOMB: softening s > 0                          */
    const double* cos_a;     /* CN_POT_COSSERIES: HOST pointer, n_cos doubles (copied)       */
    double L;                /* CN_POT_COSSERIES: period length                              */
    int32_t block;           /* rows per level-0 block (one GPU thread each): 3..32;
                                0 = default (8)                                              */
    int32_t arith;           /* cn_arith                                                     */
    int32_t flags;           /* CN_FLAG_* bits                                               */
    int32_t level_block;     /* rows per block on the reduced levels (Eq. iteration): 3..32;
                                0 = default (8)                                              */
    int32_t level1_block;    /* rows per block on level 1 alone: 3..32; 0 = level_block.  Lets
                                the largest reduced level fill whole waves of the GPU while
                                the small levels keep short serial chains                    */
} cn_desc;

/* cn_desc.flags: tabulate the static part of the diagonal, 2 + 2 dx^2 Vs(x_j),
 * once at plan creation (8 B per grid point of plan workspace, read by every
 * level-0 sweep) instead of regenerating it from x_j at every step.  Implied
 * for CN_POT_ARRAY and CN_POT_COSSERIES with CN_ARITH_DF64. */
#define CN_FLAG_COEFF_TABLE 1
/* cn_desc.flags: low-memory mode.  By default the level-0 reduction keeps, per
 * grid point, the explicit right-hand side and the elimination pivot (32 B of
 * plan workspace per point) so the substitution does not regenerate them and
 * updates psi in place.  With CN_FLAG_RECOMPUTE the substitution regenerates
 * both from psi instead, and the plan holds one n-point state buffer (16 B per
 * point) for the step ping-pong -- for grids whose 32 B per point do not fit. */
#define CN_FLAG_RECOMPUTE 2
/* cn_desc.flags: how the stages below level 0 are launched (see cn_plan_create):
 * one launch per stage and level (CN_FLAG_LEVEL_LAUNCHES) or all of them in one
 * persistent launch (CN_FLAG_PERSISTENT_LEVELS); not both.  Without either the
 * library picks per arithmetic the faster one on B300: the persistent launch for
 * CN_ARITH_F64, one launch per stage and level for CN_ARITH_DF64.  The results
 * are the same bits either way. */
#define CN_FLAG_LEVEL_LAUNCHES 4
#define CN_FLAG_PERSISTENT_LEVELS 8
/* cn_desc.flags: level 0 one thread per block whatever the blocks (the paper's
 * per-process serial elimination, Sec. 4.1; the partition study's model).  Without
 * it, a single system in store mode whose level-0 blocks are 64 .. 1024 rows long
 * and at most 4096 in number is reduced and substituted by one CTA per block (up
 * to four warps, two rows a thread or more), the recurrences as prefix scans
 * (cn_plan_info.level0_lanes threads, 32 .. 128): the same solution up to
 * rounding, at a fraction of the latency. */
#define CN_FLAG_SERIAL_BLOCKS 16

/* Create a plan for systems of size desc->n.  The N-shaped solve is nested
 * (Eq. iteration): level 0 is cut into blocks of desc->block rows, level 1 into
 * blocks of desc->level1_block rows (if nonzero), every other reduced level into
 * blocks of desc->level_block rows, until a level has at most 1024
 * rows; that system (the RS stage) is solved inside one CTA by cyclic
 * reduction.  The stages below level 0 -- the reductions of levels 1 .. L-1,
 * the RS stage and the substitutions back up -- run either as one launch per
 * stage and level or in ONE persistent cooperative launch (all its CTAs
 * resident at once, one per multiprocessor, stages separated by grid-wide
 * barriers bounded by a time limit: a barrier that gives up records
 * CN_ERR_TIMEOUT, see cn_plan_set_wait_limit), chosen by CN_FLAG_LEVEL_LAUNCHES /
 * CN_FLAG_PERSISTENT_LEVELS or per arithmetic; the persistent launch serves
 * single systems of this default hierarchy whose kernel can be resident, else
 * the per-level launches run.  Either way the results are the same bits.  Allocates the device workspace on the current device: the
 * reduced systems of every level (~80 B per row of level 1 and below), 32 B
 * per grid point of kept right-hand sides and pivots (16 B of state buffer
 * instead with CN_FLAG_RECOMPUTE), the optional coefficient table, a status
 * word.  On success *out owns it. */
cn_status cn_plan_create(const cn_desc* desc, cn_plan* out);

/* Create a plan with an explicit nesting depth and block sizes, for studying
 * the partition (Sec. 4.3: the single- and multiple-iteration time model and
 * Eq. optimal_nblocks / optimal-P-multistage; Fig. 2).  Level i, i = 0 ..
 * nlevels-1, is cut into blocks of blocks[i] rows (n_bl(i+1) = ceil((rows_i -
 * 1) / blocks[i]) parallel blocks, one thread each) and reduced; level
 * nlevels is solved by the serial RS stage whatever its size (one thread).
 *   nlevels: 1 .. CN_MAX_LEVELS - 1;
 *   blocks: host int32[nlevels], each 3 .. CN_LEVELS_MAX_BLOCK; a level-0 block
 *     longer than 32 rows takes a substitution that stages its values in
 *     device scratch instead of shared memory (the plan allocates it); the
 *     levels below substitute, at any block length, from the RD results their
 *     reductions keep in place of their rows;
 *   desc: as for cn_plan_create; desc->block, desc->level_block and
 *     desc->level1_block are ignored.
 * Returns CN_ERR_INVALID_ARG if some level i < nlevels has fewer than 3 rows,
 * and CN_ERR_UNSUPPORTED for CN_FLAG_RECOMPUTE with blocks[0] > 32.  The plan
 * is used with every cn_plan_* / cn_step* / cn_solve_tridiag / cn_adjoint_step
 * call like any other. */
#define CN_LEVELS_MAX_BLOCK 1048576
cn_status cn_plan_create_levels(const cn_desc* desc, int32_t nlevels, const int32_t* blocks, cn_plan* out);

/* Free the plan and its workspace (synchronises the device first).  NULL is a no-op. */
cn_status cn_plan_destroy(cn_plan plan);

/* nsteps Crank-Nicolson steps (Sec. 2) starting from psi_in (device,
 * complex128[n]); the result is written to psi_out (device, complex128[n]).
 * E_mid: device array of nsteps doubles, E_mid[k] = E(t0 + (k + 1/2) dt), the
 * field at the midpoint of step k (Sec. 2: T is built at t + dt/2); NULL
 * means E = 0.  psi_in may equal psi_out; psi_in is otherwise not modified.
 * nsteps = 0 copies psi_in to psi_out.  In store mode (blocks of at most 32
 * rows) the steps of one call pass psi on chip: each step's level-0
 * substitution and the next step's level-0 reduction run as one kernel, and
 * psi is written once, by the last step.  In binary64 a call of K steps and K
 * calls of one step give the same bits; in double-float psi keeps its
 * double-float form between the steps of a call instead of being rounded to
 * complex128, so the two agree to rounding.  Recompute mode and blocks longer
 * than 32 rows keep every step separate.  Asynchronous on `stream`;
 * device-side errors go to the plan status (cn_plan_status). */
cn_status cn_step(cn_plan plan, const void* psi_in, void* psi_out, const double* E_mid,
                  int64_t nsteps, void* stream);

/* As cn_step, but every step's result is kept: step k (k = 0 .. nsteps-1)
 * writes psi_{k+1} to states_out + k n (device, complex128[nsteps n], the
 * states back to back) -- what a backward pass that recomputes a segment of a
 * propagation needs.  psi_in must not overlap states_out (CN_ERR_INVALID_ARG).
 * In store mode the steps run as in cn_step's step loop (psi stays on chip
 * from one step to the next; the stored state is its complex128 rounding), so
 * states_out[nsteps-1] equals cn_step's result bitwise. */
cn_status cn_step_states(cn_plan plan, const void* psi_in, void* states_out, const double* E_mid,
                         int64_t nsteps, void* stream);

/* As cn_step, with psi_in, psi_out and E_mid in HOST memory (pageable or
 * pinned).  The host-to-device copies, the steps and the device-to-host copy
 * are enqueued on `stream`; the call synchronises the stream before it
 * returns, so psi_out is valid on return. */
cn_status cn_step_host(cn_plan plan, const void* psi_in_host, void* psi_out_host,
                       const double* E_mid_host, int64_t nsteps, void* stream);

/* Solve the general complex tridiagonal system T x = d (Sec. 4, Eq. algorithm)
 * by the N-shaped partition method: b = lower diagonal (b[j] = T[j][j-1],
 * b[0] ignored), a = diagonal, c = upper diagonal (c[j] = T[j][j+1], c[n-1]
 * ignored), d = right-hand side; all device complex128[n]; x = device
 * complex128[n] output (may alias d; must not alias b, a or c).  n must equal
 * the plan's n.  No pivoting: T must admit an unpivoted LU factorisation of
 * every block (true for the CN matrices and for diagonally dominant T). */
cn_status cn_solve_tridiag(cn_plan plan, const void* b, const void* a, const void* c,
                           const void* d, void* x, int64_t n, void* stream);

/* One step of the discrete adjoint of the CN recursion T_n psi_{n+1} = T_n^dagger psi_n
 * (Sec. 2; the paper has no adjoint: this is the hand-written backward pass for a
 * real loss L(psi_N) with the convention dL = 2 Re(lam^H dpsi)):
 *   mu      = (T_n^dagger)^{-1} lam_{n+1}      (N-shaped solve, Sec. 4)
 *   lam_n   = T_n mu                            (= 2 mu - lam_{n+1}, since T + T^dagger = 2)
 *   *dLdE  += dL/dE_n = dt Im( sum_j conj(mu_j) x_j (psi_n,j + psi_{n+1},j) )
 * psi_n, psi_np1, lam_np1: device complex128[n] (psi_n, psi_np1 the forward states of
 * step n); lam_n: device complex128[n] output, may alias lam_np1; E_mid: device pointer
 * to E(t_n + dt/2) (NULL: 0); dLdE: device double, accumulated (not overwritten).  The
 * plan allocates an n-point buffer for mu on its first adjoint call.  The sum is
 * formed in a fixed order: results are bitwise reproducible. */
cn_status cn_adjoint_step(cn_plan plan, const void* psi_n, const void* psi_np1, const void* lam_np1,
                          void* lam_n, const double* E_mid, double* dLdE, void* stream);

/* Piecewise-linear field from n_controls >= 2 samples u_c on the uniform nodes
 * t_c = c t_final / (n_controls - 1), clamped outside [0, t_final]:
 *   E_mid[k] = sum_c u_c hat_c(t0 + (k + 1/2) dt),  k = 0..nsteps-1,
 * and its transpose  grad_u[c] = sum_k dLdE[k] hat_c(t0 + (k + 1/2) dt)
 * (overwritten).  All arrays are device doubles. */
cn_status cn_field_from_controls(const double* u, int64_t n_controls, double t_final, double t0, double dt,
                                 int64_t nsteps, double* E_mid, void* stream);
cn_status cn_field_grad_to_controls(const double* dLdE, int64_t nsteps, double t_final, double t0, double dt,
                                    int64_t n_controls, double* grad_u, void* stream);

/* Static description of a plan: the nesting levels of its N-shaped solve
 * (Eq. iteration) and the kernels one step launches. */
#define CN_MAX_LEVELS 24
typedef struct {
    int64_t n;                           /* unknowns                                      */
    int32_t levels;                      /* reduced levels below level 0; level `levels`  */
                                         /* is solved by the RS stage (one CTA, cyclic    */
                                         /* reduction; serial for cn_plan_create_levels)  */
    int32_t launches_per_step;           /* kernels one single-step cn_step / one solve
                                            launches: 3 with the persistent launch below
                                            level 0, else 2 levels + 1; inside a cn_step of
                                            nsteps >= 2 in store mode a step launches one
                                            fewer, plus one substitution per call          */
    int64_t level_rows[CN_MAX_LEVELS];   /* rows of level 0 .. levels                     */
    int32_t level_block[CN_MAX_LEVELS];  /* rows per block of level 0 .. levels-1         */
    int64_t workspace_bytes;             /* device memory the plan holds                  */
    int32_t level0_lanes;                /* threads that reduce and substitute one level-0
                                            block: 1, or 32 .. 128 (a CTA, the recurrences
                                            as prefix scans) for few blocks of 64 .. 1024
                                            rows of one system in store mode               */
} cn_plan_info;
cn_status cn_plan_query(cn_plan plan, cn_plan_info* out);

/* Kernel timing for profiling.  While enabled, every kernel the plan launches
 * is bracketed by two CUDA events recorded on its stream.  cn_plan_profile_read
 * synchronises on the last event, then returns, per kernel class, the summed
 * elapsed milliseconds (ms[c]) and the number of launches (launches[c]) since
 * the previous read, and restarts the count.  Classes: 0 = level-0 reduction
 * (RD+JD+RU+JU), 1 = level-0 substitution (SS), 2 = reductions of levels >= 1,
 * 3 = substitutions of levels >= 1, 4 = RS stage, 5 = level-0 SS of one step
 * fused with the level-0 reduction of the next (cn_step with nsteps >= 2 in
 * store mode), 6 = the persistent launch of every stage below level 0 (classes
 * 2 .. 4 then stay empty).  cap = entries available in ms / launches (at most
 * 7 are written). */
#define CN_PROFILE_CLASSES 7
cn_status cn_plan_profile(cn_plan plan, int enable);
cn_status cn_plan_profile_read(cn_plan plan, double* ms, int64_t* launches, int32_t cap);

/* cn_solve_tridiag_noalloc: the tridiagonal solve of cn_solve_tridiag for
 * callers that cannot allocate device memory on their solve path (code under a
 * framework whose memory pool owns all device memory, or a latency-critical
 * loop where cudaMalloc / cudaFree would synchronise the device).  It takes no
 * plan and allocates nothing: the reduced systems of all nesting levels live
 * in one fixed 16 MiB device array inside the library, which every GPU that
 * loads the library holds until the process exits.  The paper has no
 * counterpart; this is a deployment variant of the same N-shaped solve.
 *   b, a, c, d, x, n: as for cn_solve_tridiag (device complex128[n]; x may
 *     alias d); n <= CN_NOALLOC_MAX_N, larger n returns CN_ERR_UNSUPPORTED
 *     before any work is enqueued;
 *   arith: CN_ARITH_F64 or CN_ARITH_DF64; blocks of 8 rows on every level;
 *   stream: as elsewhere; the call returns without synchronising.
 * Every call looks up the device address of the array on the current device
 * (cudaGetSymbolAddress), so a device reset between calls is harmless; the
 * first call on a device also loads the library's kernels there, so make that
 * first call before any stream capture.
 * Every call uses the same array: calls that may overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Each call writes every scratch word it reads, so nothing has to be cleared
 * between calls.  Zero or non-finite pivots are not reported through a
 * status word (there is no plan); they show up as non-finite values in x. */
#define CN_NOALLOC_MAX_N 1048576
cn_status cn_solve_tridiag_noalloc(const void* b, const void* a, const void* c, const void* d, void* x,
                                   int64_t n, int32_t arith, void* stream);

/* ---- Slabs of a sharded grid (Sec. 6.2, MPI implementation; Sec. 4.1.3, the
 * joint-line exchange).
 *
 * A grid of n points is split by joint lines J_0 = 0 < J_1 < ... < J_G = n - 1
 * into G slabs; slab r owns rows J_r .. J_{r+1} (both joint lines included)
 * and lives in one process / on one GPU.  One CN step of the whole grid is
 *   1. cn_slab_reduce on every slab: coefficients, explicit half-step and the
 *      N-shaped reduction of the slab's rows (Table 1, nested by Eq. iteration)
 *      down to its two edge rows, whose six values -- the slab's share of the
 *      joint-line system -- go to share_out;
 *   2. an all-gather of the G x 6 shares, in rank order (the only exchange:
 *      6 G complex values per step, whatever n; no halo);
 *   3. cn_slab_finish on every slab: the (G + 1)-row joint-line system solved
 *      redundantly (one CUDA thread, Thomas: the RS stage), then the slab's
 *      substitution (SS) at every level with its two support values.
 * A slab plan is a cn_plan: cn_plan_destroy, cn_plan_query, cn_plan_status,
 * cn_plan_profile and cn_plan_fill_workspace apply; cn_step, cn_step_states,
 * cn_step_host, cn_solve_tridiag and cn_adjoint_step return CN_ERR_UNSUPPORTED.
 * The slabs' joint values agree bitwise after every step (every rank solves the
 * same joint system in the same order). */
#define CN_SLAB_MAX 65536

/* Create the plan of slab `rank` (0 .. nslabs-1) of the grid desc describes
 * (desc->n: the WHOLE grid; x_min, the potential and every other field as for
 * cn_plan_create; CN_POT_ARRAY: desc->V0 is the whole grid's array, of which
 * the slab reads its rows).  joints: host int64[nslabs + 1], J_0 = 0 <
 * J_1 < ... < J_G = n - 1 with gaps of at least 2, or NULL for
 * J_r = floor(r (n - 1) / nslabs).  The slab's hierarchy is nested with
 * desc->block / level1_block / level_block until its two edge rows remain.
 * CN_FLAG_RECOMPUTE is not supported (CN_ERR_UNSUPPORTED at the first step).
 * Allocates the slab's workspace on the current device, as cn_plan_create
 * does, plus 32 (nslabs + 1) bytes for the joint-line solve. */
cn_status cn_slab_create(const cn_desc* desc, int32_t nslabs, int32_t rank, const int64_t* joints, cn_plan* out);

/* Rows of the whole grid the slab holds: *lo = J_rank, *hi = J_{rank+1};
 * the slab's local arrays have hi - lo + 1 complex128 entries. */
cn_status cn_slab_range(cn_plan slab, int64_t* lo, int64_t* hi);

/* Step part 1: psi_local (device complex128[hi - lo + 1]: the slab's rows,
 * both joint values included), E_mid (device pointer to E(t + dt/2); NULL:
 * 0) -> share_out (device complex128[6]: c, a, d of row J_rank and b, a, d of
 * row J_{rank+1}, the slab's share of the joint-line system after its
 * interior rows are eliminated).  The slab keeps what step part 2 needs;
 * psi_local is not written. */
cn_status cn_slab_reduce(cn_plan slab, const void* psi_local, const double* E_mid, void* share_out, void* stream);

/* Step part 2: shares (device complex128[6 nslabs], every slab's share_out in
 * rank order) -> psi_local_out (device complex128[hi - lo + 1], the slab's
 * rows after the step; may be the psi_local of part 1). */
cn_status cn_slab_finish(cn_plan slab, const void* shares, void* psi_local_out, void* stream);

/* Wait for the plan's stream work to finish (device synchronise) and return
 * the first device-side error recorded since the last call (then clear it). */
cn_status cn_plan_status(cn_plan plan);

/* The bounded waits of the persistent launch below level 0: every grid-wide
 * barrier gives up after timeout_ns nanoseconds (default 2e9), records
 * CN_ERR_TIMEOUT in the plan's status and lets the launch end; cn_plan_status
 * returns it and restores the barrier.  missing_ctas > 0 is a test hook: the
 * barriers then wait for that many CTAs beyond the launch, which never arrive,
 * so every barrier runs out (the results of such a step are not valid).
 * CN_ERR_INVALID_ARG for timeout_ns <= 0 or missing_ctas < 0. */
cn_status cn_plan_set_wait_limit(cn_plan plan, int64_t timeout_ns, int32_t missing_ctas);

/* Debugging aid (the check that stands in for a memory sanitizer): synchronise
 * the device, then fill every scratch buffer the plan owns with the byte value
 * `byte` (0..255; 0xFF makes every binary64 and binary32 word a NaN) -- the
 * kept right-hand sides and pivots, the reduced systems, CTA slots and
 * solutions of every nesting level, the long-block and serial-RS scratch, the
 * adjoint's mu buffer, the staging buffers of cn_step_host and a slab's
 * joint-solve scratch.  Not touched: the coefficient table and the per-system
 * tables built at creation, the status word, the adjoint's ticket counter and
 * the persistent launch's barrier words.  Since every call writes each
 * scratch word before it reads it, results after a fill are bitwise those
 * without it.  CN_ERR_INVALID_ARG for byte outside 0..255.  Synchronous. */
cn_status cn_plan_fill_workspace(cn_plan plan, int32_t byte);

/* ---- Batches: many independent systems of uneven sizes in one launch per stage.
 *
 * The paper solves one system at a time; a batch runs the same N-shaped solve
 * (Sec. 4, Table 1; nested as in Eq. iteration) over `nsys` independent CN
 * systems whose rows lie back to back in one complex128 array.  Every stage
 * of every nesting level is ONE launch for all systems: a thread finds its
 * system by binary search over the per-level block offsets, so the work of a
 * launch is balanced across systems of any size mix.  Launches per step:
 * 2 L + 1, with L the deepest system's level count.
 *
 * The systems share dx, dt, the potential kind, block sizes, arithmetic and
 * flags (from `common`; common->n, x_min and cos_a are ignored).  System s
 * has sizes[s] >= 3 rows, starts at row offset offsets[s] (cn_batch_offsets:
 * the prefix sum of sizes) and its grid is x_j = x_min[s] + j dx.
 *   x_min: host double[nsys], or NULL for x_min[s] = -floor(sizes[s]/2) dx;
 *   cos_a: host double[nsys * n_cos] (CN_POT_COSSERIES; row s = system s's
 *     coefficients), copied; the period is common->L when > 0, else the
 *     system's own length sizes[s] dx;
 *   CN_POT_ARRAY: common->V0 is a device double[sum of sizes], indexed like
 *     the state; read only during cn_batch_create.
 * The static diagonal part (2 + 2 dx^2 Vs) of every system is tabulated once
 * at creation.  Ownership, streams and errors: as for plans. */
cn_status cn_batch_create(const cn_desc* common, int64_t nsys, const int64_t* sizes, const double* x_min,
                          const double* cos_a, cn_batch* out);

/* Free the batch and its workspace (synchronises the device first).  NULL is a no-op. */
cn_status cn_batch_destroy(cn_batch batch);

/* offsets: host int64[nsys + 1]; receives the row offset of each system and,
 * last, the total row count (the length of the batch state). */
cn_status cn_batch_offsets(cn_batch batch, int64_t* offsets);

/* nsteps CN steps of every system, as cn_step: psi_in / psi_out are device
 * complex128[total rows] (may be equal); E_mid (device double[nsteps] or
 * NULL) is the field shared by all systems.  Enqueues a fixed launch
 * sequence with no host synchronisation and no allocation, so it may be
 * captured into a CUDA graph and replayed. */
cn_status cn_batch_step(cn_batch batch, const void* psi_in, void* psi_out, const double* E_mid, int64_t nsteps,
                        void* stream);

/* As cn_plan_status, for a batch. */
cn_status cn_batch_status(cn_batch batch);

/* As cn_plan_fill_workspace, for a batch. */
cn_status cn_batch_fill_workspace(cn_batch batch, int32_t byte);

/* Static description of a status code. */
const char* cn_status_string(cn_status s);

/* Library build information: "<version> sm_<arch>", with " debug" appended
 * in the CN_DEBUG build. */
const char* cn_version(void);

/* Name of the last CUDA runtime error (cudaGetErrorName) that a call of the
 * calling host thread turned into CN_ERR_CUDA or CN_ERR_OOM; "cudaSuccess" if
 * none.  The string is static. */
const char* cn_cuda_error_string(void);

/* Throughput of the current device's FP64 pipe, the denominator of the binary64
 * path's ALU roofline: independent chains of binary64 FMAs (*fma_per_s) and of
 * binary64 additions (*add_per_s) on every multiprocessor, in operations per
 * second of the whole device (best of five CUDA-event timings, about 20 ms of
 * GPU time).  Synchronises the device; allocates and frees a small buffer. */
cn_status cn_measure_fp64_rate(double* fma_per_s, double* add_per_s);

/* ---- The CN_DEBUG build (libcn_b300_debug.so; the stand-in for a memory
 * sanitizer).  Every global-memory load and store of the kernels is checked
 * against the extents of the buffers the enqueuing call may touch -- the
 * plan's workspace and the caller's arrays at the sizes the call implies --
 * registered by the host before the call's first launch.  An access outside
 * all of them is recorded (the first one: address and size) and skipped: a
 * load returns zero, a store is dropped.  Calls that share a stream see
 * their own registrations; the debug build is for tests, one stream at a time.
 *
 * cn_debug_report: synchronise the device, then return CN_ERR_BOUNDS and the
 * recorded access (*addr, *bytes; either may be NULL) if one was caught since
 * the previous report, and clear the record; CN_OK if none.  The default
 * build returns CN_ERR_UNSUPPORTED (nothing is checked there).
 * cn_debug_selftest: plant one access just outside a registered extent (inside
 * a live allocation, so nothing outside it is touched even if the check
 * failed) and return CN_OK if the checks caught and reported it;
 * CN_ERR_UNSUPPORTED in the default build. */
cn_status cn_debug_report(uint64_t* addr, uint64_t* bytes);
cn_status cn_debug_selftest(void);

#ifdef __cplusplus
}
#endif
#endif
