/*
 * dwf.h — C ABI of the GB300 (sm_103a) domain-wall fermion solver library (libdwf.so).
 *
 * Problem (Guo, Mawhinney, Tu, "Solving DWF Dirac Equation Using Multisplitting
 * Preconditioned Conjugate Gradient", arXiv:1804.08593):
 *   the domain-wall operator D is not Hermitian, so the solver runs conjugate gradient on the
 *   normal equations (Sec. 2.2, Eq. 3), here on the even sites after even-odd (Schur)
 *   preconditioning: A = Mpc^dag Mpc, A x = phi.  The multisplitting preconditioner of
 *   Sec. 2.1 (Eqs. 1-2) with a zero initial guess reduces to independent local solves
 *   A_s x_s = b_s on lattice blocks (Sec. 2.3, Eqs. 4-5); on one GPU the paper's node
 *   subdomains are lattice blocks solved concurrently.
 *
 * Operator conventions (standard Moebius domain-wall fermions; the paper does not print the
 * operator):
 *   D_W(-M5) = (4 - M5) - Dh/2,
 *   Dh psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu),
 *   (K psi)_s = P- psi_{s+1} + P+ psi_{s-1},  psi_{Ls} = -mf psi_0,  psi_{-1} = -mf psi_{Ls-1},
 *   D+ = b + c K,  D- = 1 - K,  D = D_W D+ + D-        (Shamir: b = 1, c = 0),
 *   M5op = (4 - M5) D+ + D-,
 *   Mpc  = M5op - 1/4 Dh_eo D+ M5op^-1 Dh_oe D+   (even sites).
 * Chiral gamma basis: gamma_5 = diag(1, 1, -1, -1); P+ = spins {0,1}, P- = spins {2,3}.
 * Boundary conditions: periodic in all four directions.
 *
 * Data layouts (all caller buffers are complex128 = two little-endian doubles, re then im):
 *   links  : [T][Z][Y][X][mu=x,y,z,t][3][3]     (row index first: U[a][b])
 *   even-half 5D field : [Ls][V/2][4][3]        (even sites x+y+z+t = 0 mod 2, lexicographic
 *                                                order x fastest)
 *   full 5D field      : [Ls][V][4][3]          (all sites, lexicographic, x fastest)
 *   force dS/dU        : same layout as links.
 * Every field pointer may be device memory or host memory (pageable or pinned); the library
 * detects which with cudaPointerGetAttributes and copies host buffers through its own device
 * workspace on the handle's stream.  Input and output must not alias.
 *
 * Ownership: the caller owns every buffer it passes; no call keeps a caller pointer after it
 * returns.  A handle owns its packed copies of the links, neighbour tables and workspace.
 * A handle is not thread safe: use one handle per host thread.
 *
 * Errors: every call returns a dwf_status; dwf_last_error() gives a thread-local message
 * describing the last failure.  No C++ exception crosses this interface.  Solver calls
 * write their statistics into *stats when stats is not NULL.
 *
 * Requirements: X, Y, Z, T even and >= 2; Ls in {4, 6, 8, 10, 12, 16} (kernels are
 * specialised per Ls); the device must be sm_103 (GB300).
 *
 * Launch variants: every operator stage exists in a few compiled variants (register budget,
 * grid shape, how links and neighbours are staged, how the fifth-dimension post matrices are
 * applied).  Per process, the first launches of each (stage kind, lattice size) that carry no
 * solver stop flag cycle through them timed with CUDA events, and the fastest is kept.  All
 * variants agree bit for bit except the tensor-core and recurrence forms of the 16-bit post
 * and the packed-float2 FP32 form (another rounding order), each within its precision's
 * tolerance.  Environment switches: DWF_STAGE_VARIANT=<i> forces
 * variant i; DWF_TUNE_LOG=1 prints each decision on stderr; DWF_POST=matrix|recurrence and
 * DWF_DISABLE_TC=1 (read by dwf_create) restrict the post forms; DWF_RU_DELTA overrides the
 * reliable-update threshold 0.1 of the mixed-precision solvers.
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dwf_ctx* dwf_t;

typedef enum {
  DWF_OK = 0,
  DWF_ERR_ARG = 1,            /* invalid argument (sizes, pointers, unsupported Ls, ...) */
  DWF_ERR_CUDA = 2,           /* a CUDA runtime call failed (message has the CUDA error)  */
  DWF_ERR_NOMEM = 3,          /* device allocation failed                                   */
  DWF_ERR_NOT_CONVERGED = 4,  /* maxit reached before the tolerance                         */
  DWF_ERR_BREAKDOWN = 5,      /* non-finite or non-positive curvature in a Krylov solver    */
  DWF_ERR_TIMEOUT = 6         /* a bounded device-side wait gave up                         */
} dwf_status;

/* Storage precision of the fields a kernel reads and writes.  FP32/FP16/BF16 kernels
 * accumulate in FP32; FP64 kernels in FP64.  FP16/BF16 fields carry one FP32 scale. */
typedef enum { DWF_F64 = 0, DWF_F32 = 1, DWF_F16 = 2, DWF_BF16 = 3 } dwf_prec;

/* Operators of dwf_apply. */
typedef enum {
  DWF_OP_M = 0,          /* full 5D D on a full field                        (Sec. 2.2) */
  DWF_OP_MDAG = 1,       /* D^dag on a full field                                       */
  DWF_OP_MPC = 2,        /* Mpc on an even-half field                                   */
  DWF_OP_MPC_DAG = 3,    /* Mpc^dag on an even-half field                               */
  DWF_OP_MDAGM = 4       /* A = Mpc^dag Mpc on an even-half field            (Eq. 3)    */
} dwf_op;

/* Solver statistics. */
typedef struct {
  int iterations;            /* outer (global) iterations: CG iterations or MSPCG outer   */
  int inner_iterations;      /* total local iterations per block summed over outer steps  */
  int reliable_updates;      /* FP64 true-residual recomputations                          */
  int operator_applications; /* applications of the full-lattice A = Mpc^dag Mpc           */
  double true_residual;      /* ||phi - A x|| / ||phi|| computed in FP64 at exit           */
  double seconds;            /* wall time of the call (device synchronised)                */
  double* history;           /* optional caller array: ||r_k||/||phi|| per outer iteration */
  int history_capacity;      /* length of history (0 = not recorded)                       */
  int history_len;           /* entries written                                            */
  /* optional caller array (dwf_cg only; history_capacity entries, history_len written):
   * <p_k, A p_k> / ||phi||^2 of CG iteration k.  With history it gives the CG coefficients
   * alpha_k = rho_k / <p_k, A p_k>, beta_k = rho_{k+1} / rho_k (rho_k = ||r_k||^2), i.e. the
   * Lanczos tridiagonal of A whose extreme eigenvalues estimate kappa(A).  Meaningful for an
   * uninterrupted CG sequence: prec = DWF_F64 (no reliable-update restarts). */
  double* curvature_history;
} dwf_stats;

/* Creates a handle for a lattice dims = {X, Y, Z, T} with Ls slices and operator parameters
 * (M5, mf, b, c) and packs the links (layout above).  stream is a cudaStream_t (NULL = the
 * legacy default stream); every kernel of this handle runs on it.
 * Sec. 2.2 (operator), Sec. 2.1 (decomposition of fields). */
dwf_status dwf_create(dwf_t* handle, const int dims[4], int Ls, double M5, double mf,
                      double b, double c, const void* links, void* stream);

/* Replaces the links (same layout, host or device; read during the call only, the caller
 * keeps them); packed copies of every precision are rebuilt before the next use.  For gauge
 * fields that change between solves, the ensemble-generation setting of Sec. 1.  Returns
 * DWF_ERR_ARG for a NULL argument, DWF_ERR_CUDA if the copy fails; synchronises the stream. */
dwf_status dwf_update_links(dwf_t handle, const void* links);

/* out = op(in), computed in precision prec (in is rounded to prec first; out is written back
 * in complex128).  Field layout per op: even-half for MPC/MPC_DAG/MDAGM, full for M/MDAG.
 * Sec. 2.2 (D, D^dag D), Eq. 3. */
dwf_status dwf_apply(dwf_t handle, dwf_op op, const void* in, void* out, dwf_prec prec);

/* Conjugate gradient on A x = phi (Eq. 3; the paper's unpreconditioned baseline, Sec. 3).
 * x holds the initial guess on entry (zero for the paper's setting) and the solution on
 * exit; tol is the target ||phi - A x|| / ||phi||.
 *   prec = DWF_F64 : plain FP64 CG.
 *   prec = DWF_F32 (or F16/BF16): CG in that precision with FP64 reliable updates (the
 *   true residual is recomputed in FP64 whenever the low-precision residual has dropped by
 *   delta = 0.1 since the last update), FP64 global dots and final residual check.
 * Returns DWF_ERR_NOT_CONVERGED if maxit iterations do not reach tol (x holds the last
 * iterate). */
dwf_status dwf_cg(dwf_t handle, const void* phi, void* x, double tol, int maxit,
                  dwf_prec prec, dwf_stats* stats);

/* Multisplitting preconditioned CG (Sec. 2.3).  The preconditioner is M = sum_s A_s
 * (Eq. 5) over lattice blocks of size block = {bx, by, bz, bt} (each dividing the lattice,
 * each even), applied as inner_iters local CG iterations per block from a zero guess
 * (Eq. 4, "local iterations"), all blocks at once with block-local dot products.
 * local_op selects A_s:
 *   DWF_LOCAL_DROP  : Mpc^dag Mpc with every hop across a block face removed;
 *   DWF_LOCAL_EXACT : P_s A P_s, the diagonal block of A itself (Eq. 5 as printed).
 * Precisions: inner = DWF_F16/BF16/F32/F64 (storage of the local solves), middle = DWF_F32
 * or DWF_F64 (outer preconditioned CG); with middle = F32 the FP64 true residual is
 * recomputed by reliable updates (delta = 0.1).  flexible != 0 uses the Polak-Ribiere beta
 * <z', r' - r>/<r, z>, otherwise Fletcher-Reeves <r', z'>/<r, z>.
 * x: initial guess must be zero (the routine starts from x = 0 and overwrites x). */
typedef enum { DWF_LOCAL_DROP = 0, DWF_LOCAL_EXACT = 1 } dwf_local_op;
dwf_status dwf_mspcg(dwf_t handle, const int block[4], int inner_iters, dwf_prec inner,
                     dwf_prec middle, dwf_local_op local_op, int flexible, const void* phi,
                     void* x, double tol, int maxit, dwf_stats* stats);

/* Stationary block iterations on A x = phi built from the same local solves (comparison
 * solvers of Sec. 1.2 and Sec. 2.1; the paper reports the multisplitting iteration itself to
 * converge slowly, Sec. 2.3, which is why it preconditions CG instead).  One sweep:
 *   colours = 1 : the multisplitting iteration of Eq. 2: every block solves its own equation
 *                 with the current solution outside it as the boundary value, all blocks at
 *                 once: x <- x + M^-1 (phi - A x), M the direct sum of the A_s (Eq. 5);
 *   colours = 2 : multiplicative Schwarz over the black-white checkerboard of blocks
 *                 (colour (b_x + b_y + b_z + b_t) mod 2 of the block coordinates b_mu): the
 *                 blocks of one colour solve, the residual is recomputed, then the other;
 *   colours = 16: the same over the 2^4 checkerboard (colour sum_mu 2^mu (b_mu mod 2)).
 * Each A_s^-1 is inner_iters local CG iterations from a zero guess in storage precision
 * `inner` (FP16/BF16 with a unit-RMS scale), local_op as in dwf_mspcg; the outer vectors and
 * the residual b - A x (recomputed after every colour) are FP64.  Stops when
 * ||phi - A x|| <= tol ||phi|| (tol = 0: run maxit sweeps) or after maxit sweeps
 * (DWF_ERR_NOT_CONVERGED); stats->iterations counts sweeps, history the relative residual
 * after each sweep.  x: initial guess must be zero (overwritten).  Returns DWF_ERR_ARG for
 * colours not in {1, 2, 16}, or a checkerboard whose block count in some direction is odd
 * and larger than one (the colouring would not alternate across the periodic boundary). */
dwf_status dwf_ms_solve(dwf_t handle, const int block[4], int inner_iters, dwf_prec inner,
                        dwf_local_op local_op, int colours, const void* phi, void* x,
                        double tol, int maxit, dwf_stats* stats);

/* Gradient of the pseudofermion action S = phi^dag (Mpc^dag Mpc)^-1 phi with respect to every
 * link, in the PyTorch complex convention dS/dRe U + i dS/dIm U (links layout).  X may be the
 * solution A^-1 phi (even-half, complex128) or NULL, in which case it is solved internally
 * with FP64 CG to tol.  The gradient kernel runs in FP64.
 * dS = -2 Re <Mpc X, dMpc X>, dMpc from the hopping terms of Mpc (Sec. 2.2). */
dwf_status dwf_force(dwf_t handle, const void* phi, const void* X, void* dSdU, double tol);

/* The pseudofermion action S = phi^dag (Mpc^dag Mpc)^-1 phi whose solves the paper speeds up
 * (Sec. 1), for a solution X (even-half complex128, host or device) or NULL (solved
 * internally with FP64 CG to tol).  Evaluated as Re(2 <phi, X> - ||Mpc X||^2), which equals S
 * at the exact solution and errs quadratically in the solve residual.  *S is a host double;
 * returns DWF_ERR_ARG for a NULL handle, phi or S. */
dwf_status dwf_action(dwf_t handle, const void* phi, const void* X, double tol, double* S);

/* One problem of a batched solve. */
typedef struct {
  int dims[4];
  int Ls;
  double M5, mf, b, c;
  const void* links;    /* complex128 links (device or host)                 */
  const void* phi;      /* complex128 even-half source                       */
  void* x;              /* complex128 even-half solution (overwritten)       */
} dwf_problem;

/* Solves n independent problems A_i x_i = phi_i (each its own lattice, Ls and masses) to tol
 * with FP32 CG and FP64 reliable updates (the CG of Eq. 3 per problem; batching many solves
 * has no counterpart in the paper).  All problems advance together: problems with the same
 * Ls share one concatenated site space, and a chunk of 16 CG steps of all of them is, per Ls
 * group, either one persistent cooperative kernel launch (five phases per step separated by
 * grid barriers with bounded waits) or five launches per step (stages A, B, A^dag, B^dag on
 * persistent grids, then the update), whichever the first chunks time faster (the choice is
 * kept for later calls on the same problem mix); the chosen chunks of all groups are captured
 * once as a CUDA graph and replayed, with the per-problem FP64 reliable updates between
 * replays.  stream: cudaStream_t.  per_solve (n entries,
 * nullable) receives each problem's statistics.  Fields are host or device; the call keeps
 * none of the caller's pointers.  Returns DWF_ERR_ARG for n <= 0, a bad tolerance, an
 * unsupported size or a NULL field, DWF_ERR_NOT_CONVERGED if some problem misses tol within
 * maxit steps, DWF_ERR_TIMEOUT if a bounded device-side wait gave up. */
dwf_status dwf_batch_solve(int n, const dwf_problem* problems, double tol, int maxit,
                           dwf_stats* per_solve, void* stream);

/* Per-kernel timing of one handle (instrumentation; no counterpart in the paper).  While
 * enabled, every kernel launch of the handle is bracketed by CUDA events on the handle's
 * stream and its algorithmic HBM bytes are recorded (reads of every input and write of every
 * output once, links once per site).  dwf_profile_read synchronises the stream, sums the
 * event times per kernel class and resets the counters. */
typedef struct {
  char name[48];              /* kernel class, e.g. "hop_f16_blocked"                     */
  int launches;
  double ms_total;            /* sum of event-measured launch durations                    */
  double bytes_total;         /* algorithmic bytes over all launches                       */
  double flops_total;         /* algorithmic flops (1320 per site-slice per hop)           */
} dwf_kernel_profile;
dwf_status dwf_profile_enable(dwf_t handle, int on);
dwf_status dwf_profile_read(dwf_t handle, dwf_kernel_profile* out, int capacity, int* n);

/* Size of the device array that dwf_mdagm_noalloc works in: 64 MiB per GPU, held for the
 * life of the process by every GPU that loads the library. */
#define DWF_NOALLOC_SCRATCH_BYTES (64u << 20)

/* A = Mpc^dag Mpc on an even-half field for callers that cannot allocate device memory when
 * they need the operator (a runtime that owns a fixed device budget, or code that must not
 * call cudaMalloc/cudaFree mid-run).  The paper has no counterpart: this entry point exists
 * for such callers only.  It creates no handle and calls no cudaMalloc, cudaFree or other
 * allocating routine: the links (complex128 [T][Z][Y][X][4][3][3]), in and out (complex128
 * [Ls][V/2][4][3]) are caller DEVICE buffers, and every intermediate (neighbour tables, packed
 * links, fifth-dimension matrices, packed and intermediate fields) lives in one static device
 * array of DWF_NOALLOC_SCRATCH_BYTES.  Lattices that need more return DWF_ERR_ARG with the
 * required size in dwf_last_error() (FP64 fits up to about 8^4 x Ls = 16, FP32 twice that).
 * The work is queued on stream (cudaStream_t, NULL = legacy default) and the call returns
 * without synchronising.  The first call on each device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress); make it before any stream capture.  All
 * calls share the array and leave their data in it, so calls that overlap on the GPU race. */
dwf_status dwf_mdagm_noalloc(const int dims[4], int Ls, double M5, double mf, double b,
                             double c, const void* links, const void* in, void* out,
                             dwf_prec prec, void* stream);

/* Per-handle options (failure detection; no counterpart in the paper).
 *   DWF_OPT_WAIT_LIMIT_US: time limit, in microseconds (1 .. 1e7), of every bounded device-side
 *     wait of the handle's kernels (TMA link staging, tensor-core completion); default 10 ms.
 *     A wait that runs out makes the call return DWF_ERR_TIMEOUT (its output is not valid);
 *     the handle stays usable.
 *   DWF_OPT_TEST_WAIT_PROBE: value != 0 makes every FP32/FP16/BF16 operator stage of the handle
 *     run its TMA link-staging variant without issuing the copies, so the wait on the
 *     copies' mbarrier cannot complete and runs out: the call returns DWF_ERR_TIMEOUT with
 *     nothing left in flight.  For tests of the timeout path only; FP64 stages (which have no
 *     such variant) fail with DWF_ERR_CUDA while it is set.
 * Returns DWF_ERR_ARG for a NULL handle, an unknown option or a value out of range. */
typedef enum { DWF_OPT_WAIT_LIMIT_US = 0, DWF_OPT_TEST_WAIT_PROBE = 1 } dwf_option;
dwf_status dwf_set_option(dwf_t handle, dwf_option option, double value);

/* Measures a peak arithmetic rate of the current device (measurement support for the
 * rooflines; no counterpart in the paper): which = 0 FP64 fused multiply-add (DFMA), 1 FP32
 * (FFMA).  Runs a short kernel of independent FMA chains on every SM, timed with CUDA events
 * on stream (cudaStream_t), and writes the rate in TFLOP/s (2 flops per FMA) to *tflops.  No
 * clock or power setting is touched.  Returns DWF_ERR_ARG for a bad `which` or NULL tflops. */
dwf_status dwf_measure_peak(int which, void* stream, double* tflops);

/* Thread-local description of the last error (never NULL). */
const char* dwf_last_error(void);

/* Frees the handle and everything it owns.  NULL is accepted. */
void dwf_destroy(dwf_t handle);

/* Library version string. */
const char* dwf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DWF_H */
