/*
 * rve.h -- C ABI of the batched fiber-network RVE solver (GB300, sm_103a).
 *
 * The library solves the microscale problem of an FE^2 analysis of fibrous
 * materials (arXiv 2306.09427): many independent representative volume
 * elements (RVEs), each a 3-D truss network whose boundary nodes follow the
 * macroscale deformation gradient F (affine boundary condition, Sec. 2,
 * Eq. affine-bc).  Each RVE is relaxed to static force equilibrium by
 * damped dynamic relaxation (Algorithm 2, Sec. 3.2) and homogenized to the
 * volume-averaged Cauchy stress
 *     sigma = (1/v) sum_e N_e (d_e (x) d_e) / |d_e|,   v = det(F) V0,
 * the fiber form of the average that follows Eq. hill-mandel.  The calls
 * are "batched" in the paper's sense (Sec. 4): they take a set of
 * deformation gradients and return the stresses (and tangents) of the whole
 * set at once.
 *
 * Fiber law: eps_G = (l^2/L0^2 - 1)/2, N = (EA/B)(exp(B eps_G) - 1), and
 * N = EA eps_G when B = 0.  Force of fiber e = (i, j) on node i is
 * N (x_j - x_i)/l.
 *
 * Conventions
 *  - Every function returns RVE_OK (0) or a negative RVE_E* code; the
 *    message of the last failure on the calling thread is rve_last_error().
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory on the batch's device (e.g. torch tensors' data_ptr()).
 *  - F is row-major: F[9k + 3i + j] = F_ij of item k.  sigma likewise
 *    (all 9 entries, symmetric).  dsigma/dF is [item][ij][kl]: 81 doubles
 *    per item, entry 9(3i+j) + (3k+l).
 *  - Device-pointer calls are asynchronous on `stream` (a cudaStream_t,
 *    NULL = legacy default stream); outputs are valid once the stream
 *    reaches that point.  The GPU work of each call on a batch starts after
 *    that of the batch's previous call, whatever streams they use (they
 *    share the batch's state).  The batch object is not thread safe:
 *    serialise calls on one batch.
 */
#ifndef RVE_H
#define RVE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define RVE_OK 0
#define RVE_EINVAL (-1)  /* bad argument or malformed network            */
#define RVE_ENOMEM (-2)  /* device or host allocation failed             */
#define RVE_ECUDA (-3)   /* a CUDA runtime call failed                   */
#define RVE_EADMIT (-4)  /* request exceeds a configured capacity        */

/* per-item status written by the solve calls */
#define RVE_STATUS_CONVERGED 0 /* residual test (and sigma_tol test) passed          */
#define RVE_STATUS_MAX_ITER 1  /* iteration cap hit; sigma is of the last iterate  */
#define RVE_STATUS_NONFINITE 2 /* residual became NaN/Inf; sigma is not meaningful */
#define RVE_STATUS_EMPTY 3     /* no free node left after pruning; sigma is exact
                                  (boundary-to-boundary fibers only), 0 iterations  */
#define RVE_STATUS_RUNNING 4   /* serving only: the wave ended before the solve did;
                                  the solve is parked on the device and resumes in
                                  the next wave (never returned by rve_server_poll) */

/* precision / execution path */
#define RVE_PREC_PLAIN_F64 0   /* one RVE at a time, several FP64 kernels per DR
                                  iteration, convergence tested on the host
                                  (the paper's naive approach, Sec. 4.3)         */
#define RVE_PREC_MIXED 1       /* batched fused kernel: FP32 forces and updates,
                                  FP64 residual norm and stress accumulation     */
#define RVE_PREC_BATCHED_F64 2 /* batched fused kernel, FP64 throughout         */

typedef struct rve_batch rve_batch; /* opaque, library owned */

/*
 * Solver options (Algorithm 2's tolerance, iteration cap and damping).
 *  tol          relative residual: converged when ||f_free||_2 <=
 *               max(tol * R_aff, 1e-16 * sum_e EA_e), R_aff the 2-norm of
 *               the fiber forces at the affine state x = F X.  Default 3e-7
 *               (sigma within 1e-4 of the converged value on the workloads
 *               tested; see sigma_tol for a direct stress criterion).
 *  max_iter     DR iteration cap (Algorithm 2's n_max).  Default 200000.
 *  check_every  residual test and damping update interval k (>= 1).
 *               Default 50.
 *  precision    RVE_PREC_*; default RVE_PREC_MIXED.
 *  warm_start   1: start each solve from the RVE's fluctuation h = x - F X
 *               left by its previous solve in the same precision (0 after
 *               create or rve_reset_state); 0: start from h = 0.  Default 0.
 *  damping      > 0: constant mass-proportional damping c (the paper's
 *               choice, Sec. 3.2); <= 0: c re-estimated every check_every
 *               iterations from a Rayleigh quotient.  Default 0.
 *  threads      threads per CTA for the batched kernels (0 = automatic).
 *  graphs       1: rve_solve (batched precisions, on a created stream -- the
 *               default streams cannot be captured) records its launch
 *               sequence as a CUDA graph on the first call with a given set
 *               of arguments and stream, and replays it on later calls with
 *               the same ones (e.g. the Newton iterations of a load step);
 *               at most 16 argument sets are kept; options or bin changes
 *               drop them.  Default 0.
 *  sigma_tol    > 0: also require the estimated remaining stress error to be
 *               <= sigma_tol at a check n: with rho = min(R_n / R_{n-2}, 0.95)
 *               the residual ratio over the last two check intervals,
 *               est = |sigma_n - sigma_{n-2}|_F / |sigma_n|_F * rho / (1 - rho),
 *               the remaining error of a geometrically converging sequence.
 *               It only adds a condition to the residual test and is skipped
 *               once the residual is below 1e-3 * sigma_tol * R_aff.
 *               <= 0 disables it.  Default 0 (off).
 *  damping_mode RVE_DAMP_VISCOUS (0): mass-proportional viscous damping as
 *               set by `damping`.  RVE_DAMP_KINETIC (1): kinetic damping,
 *               the other family of DR accelerations the paper names
 *               (Sec. 3.2): no viscous term; the kinetic energy sum m |v|^2
 *               of every step is tracked, and a step whose kinetic energy
 *               is below the previous step's went past a peak: it is taken
 *               back, the velocities are set to zero, and the motion
 *               restarts with the half step v = f/(2m).  Batched precisions only
 *               (RVE_EINVAL with RVE_PREC_PLAIN_F64).  Default 0.
 *  damping_scale  s in the adaptive damping c = s * 2 sqrt(lambda) (lambda
 *               the Rayleigh quotient of the last step's velocity, which
 *               sits above the slowest mode's eigenvalue).  Default 1.0;
 *               0.7 takes about 20 % fewer iterations on the uniform and
 *               uneven workloads, but one 16^3 network solved in FP64 to
 *               1e-10 with it stopped on a weakly unstable equilibrium.
 *               Must be in (0, 1]; 0 means the default.
 *  energy_check 1: the all-RVE solves (rve_solve) run the kernel variant
 *               with Algorithm 2's optional energy balance (Sec. 3.2, after
 *               Belytschko).  At every check it evaluates the stored energy
 *               of the active fibers exactly (8-point Gauss-Legendre of the
 *               axial force per fiber), so its change dW from the start; the
 *               kinetic energy K of the last half step; and from sums over
 *               the steps the kinetic energy lost to damping D and to the
 *               step cap C, and the work M of the fictitious mass changes.
 *               K + D + C - M equals the trapezoidal rule of the force work
 *               along the iterates, so the balance error
 *               |dW + K + D + C - M + v.f/2| / max(|dW|, K, D + C) (v.f/2
 *               the pending half step) is the quadrature error of the
 *               central-difference steps, the time-integration error the
 *               check exists to expose; the largest over the checks is kept.
 *               Read the records with rve_energy.  Batched precisions with
 *               viscous damping only (RVE_EINVAL otherwise); diagnostic, the
 *               iterates are those of the two-phase kernel.  Default 0.
 *  kernel       RVE_KERNEL_AUTO (0) or RVE_KERNEL_TWO_PHASE (1): the
 *               two-phase kernel (a fiber phase, then a node-centric CSR
 *               gather of the fiber forces; RVEs too large for one CTA's
 *               shared memory stream their fiber data from L2/HBM): the
 *               fastest on large batches.  RVE_KERNEL_NODE (2), for the
 *               viscous damping modes: RVEs that fit one CTA run the
 *               node-centric kernel (each thread owns free nodes and
 *               evaluates their incident fibers itself: one barrier per DR
 *               iteration, no fiber scratch; a fiber with two free ends is
 *               evaluated at both ends, with exactly opposite forces); larger
 *               RVEs of the mixed precision run on a thread-block cluster of
 *               2-8 CTAs that holds the whole RVE in distributed shared
 *               memory (lower latency per RVE, more SMs per RVE).  All
 *               compute Algorithm 2's iterates (Sec. 3.2); the force sums at a
 *               node are taken in other orders, so results differ at the
 *               rounding level.  Default 0.
 *  reserved_    must be 0.
 */
typedef struct rve_options {
  double tol;
  int32_t max_iter;
  int32_t check_every;
  int32_t precision;
  int32_t warm_start;
  double damping;
  int32_t threads;
  int32_t graphs;
  double sigma_tol;
  int32_t damping_mode;
  int32_t energy_check;
  double damping_scale;
  int32_t kernel;
  int32_t reserved_;
} rve_options;

#define RVE_DAMP_VISCOUS 0
#define RVE_DAMP_KINETIC 1
#define RVE_KERNEL_AUTO 0
#define RVE_KERNEL_TWO_PHASE 1
#define RVE_KERNEL_NODE 2

/* Fill *opt with the defaults above.  Never fails. */
void rve_options_default(rve_options* opt);

/*
 * Create a batch of n_rve networks (Algorithm 2 set-up: connectivity,
 * lumped mass data and upload to the device, done once per RVE; the
 * packed per-RVE offset layout is the paper's PackedView, Sec. 4.3).
 * All array arguments are HOST pointers and are copied; the caller keeps
 * ownership.
 *   device       CUDA device ordinal the batch lives on.
 *   node_off     n_rve+1 int64, node range of RVE r is [node_off[r], node_off[r+1]).
 *   X            3*N_total doubles, reference coordinates (row per node).
 *   fiber_off    n_rve+1 int64, fiber range of RVE r.
 *   conn         2*E_total int32, RVE-local node ids (0-based) of each fiber.
 *   L0, EA, B    E_total doubles each: rest length (> 0), axial stiffness
 *                (> 0), exponential nonlinearity (>= 0).
 *   is_boundary  N_total bytes, nonzero for nodes pinned to x = F X.
 *   V0           n_rve doubles, reference volume per RVE; NULL means the
 *                volume of each RVE's bounding box.
 *   opt          NULL for defaults.
 * Validation (RVE_EINVAL): offsets start at 0 and do not decrease, node
 * ids in range, no fiber joining a node to itself, finite coordinates,
 * the parameter ranges above, at least one boundary node in an RVE that
 * has fibers, at most 65534 free nodes and 32767 active fibers per RVE.
 * Pruning: free nodes with no fiber path to the boundary and free nodes
 * of degree <= 1 (repeatedly) are removed; their fibers carry no force at
 * equilibrium, so sigma is unchanged.
 * On success *out receives the batch; on failure *out is NULL.
 */
int rve_batch_create(rve_batch** out, int device, int64_t n_rve, const int64_t* node_off,
                     const double* X, const int64_t* fiber_off, const int32_t* conn,
                     const double* L0, const double* EA, const double* B,
                     const uint8_t* is_boundary, const double* V0, const rve_options* opt);

/* Replace the batch's options (validated as in create). */
int rve_set_options(rve_batch* b, const rve_options* opt);

/*
 * Solve every RVE of the batch (Algorithm 2 to convergence, then the
 * stress average after Eq. hill-mandel).
 *   F       device, 9*n_rve doubles, det F > 0 expected (det F <= 0 gives
 *           status RVE_STATUS_NONFINITE for that RVE).
 *   tol     <= 0 keeps the batch option; max_iter <= 0 likewise.
 *   sigma   device, 9*n_rve doubles (written).
 *   iters   device, n_rve int32 DR iterations performed (may be NULL).
 *   status  device, n_rve int32 RVE_STATUS_* (may be NULL).
 */
int rve_solve(rve_batch* b, const double* F, double tol, int32_t max_iter, double* sigma,
              int32_t* iters, int32_t* status, void* stream);

/*
 * Solve the m RVEs listed in ids (HOST array of distinct RVE indices) with
 * deformation gradients F[9k..] for ids[k]; outputs are indexed by k
 * (device arrays of m items).  Used by the serving loop.
 */
int rve_solve_subset(rve_batch* b, const int64_t* ids, int64_t m, const double* F, double tol,
                     int32_t max_iter, double* sigma, int32_t* iters, int32_t* status,
                     void* stream);

/*
 * End-to-end variant of rve_solve with HOST buffers: copies F to the
 * device, solves, copies sigma/iters/status back and synchronises.
 * iters/status may be NULL.
 */
int rve_solve_host(rve_batch* b, const double* F, double tol, int32_t max_iter, double* sigma,
                   int32_t* iters, int32_t* status);

/*
 * Allocation-free plain FP64 solve of RVE r of an existing batch.  The
 * paper has no counterpart; this call exists for callers that must not
 * allocate device memory while they solve (device memory carved up once at
 * start-up by a caching allocator or a fixed budget, where cudaMalloc may
 * fail or synchronise the whole device; loops whose latency limits forbid
 * allocator calls).  It runs the kernels of the RVE_PREC_PLAIN_F64 path
 * with their working buffers in a fixed scratch array compiled into the
 * library (about 2.3 MB held on every GPU that loads the library, until
 * the process exits), and calls no allocator: no cudaMalloc/cudaFree, no
 * library allocation.
 *   r         RVE index; its active fibers must not exceed
 *             RVE_NOALLOC_MAX_ACTIVE_FIBERS and its free nodes
 *             RVE_NOALLOC_MAX_FREE_NODES, else RVE_EINVAL with a message.
 *   F         device, 9 doubles; sigma device, 9 doubles;
 *   iters, status   device, one int32 each (may be NULL).
 *   tol <= 0, max_iter <= 0 keep the batch options.
 * Always starts from h = 0 and leaves the batch's warm-start state alone.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) for that device; make that first call before any
 * stream capture.  All calls, on any batch, share the one array.  The call
 * returns after the solve's last convergence check, but its stress and
 * finishing kernels are still queued on `stream` and read the array: a
 * second call on another stream, from this thread or any other, races with
 * them unless the caller orders the two (an event recorded on the first
 * call's stream and waited on by the second's, or a synchronisation of the
 * first call's stream).  Calls on one stream are ordered by the stream.
 */
#define RVE_NOALLOC_MAX_ACTIVE_FIBERS 16384
#define RVE_NOALLOC_MAX_FREE_NODES 8192
int rve_solve_plain_noalloc(rve_batch* b, int64_t r, const double* F, double tol, int32_t max_iter,
                            double* sigma, int32_t* iters, int32_t* status, void* stream);

/*
 * Energy records of the last rve_solve run with the option energy_check = 1,
 * on the given batched precision.  energy: DEVICE, 6 doubles per RVE:
 *   [0] dW   change of stored energy from the start state (<= 0 when relaxing)
 *   [1] K    kinetic energy of the last half step at the last check
 *   [2] D    kinetic energy lost to viscous damping
 *   [3] C    further kinetic energy lost (the step cap)
 *   [4] M    work of the fictitious mass changes
 *   [5] the largest relative balance error over the checks (option
 *        energy_check).
 * Asynchronous on stream.  RVE_EINVAL before any such solve.
 */
int rve_energy(rve_batch* b, int32_t precision, double* energy, void* stream);

/*
 * Stress and stress tangent: sigma(F) and the central-difference
 * derivative dsigma_ij/dF_kl = (sigma_ij(F + h E_kl) - sigma_ij(F - h E_kl)) / 2h,
 * E_kl = e_k (x) e_l, nine directions, i.e. 18 perturbed solves per RVE
 * batched in one launch and warm-started from the base solution (the
 * paper obtains its material stiffness from finite-difference microscale
 * solves, Sec. 3.2).  h <= 0 means 1e-4.
 *   F          device 9*n_rve; sigma device 9*n_rve; dsigma_dF device 81*n_rve;
 *   status     device n_rve (worst status over the 19 solves) or NULL.
 */
int rve_tangent(rve_batch* b, const double* F, double h, double tol, int32_t max_iter,
                double* sigma, double* dsigma_dF, int32_t* status, void* stream);

/*
 * The paper's material tangent (Sec. 3.2, Eqs. tensor_fd and
 * stiffness-push-forward): with F = R U, six forward-difference solves of
 * the second Piola-Kirchhoff stress Pi = J F^-1 sigma F^-T along the
 * probing directions T_p (the columns of the paper's Mandel matrix [T]),
 *   P_ij,p = (Pi_ij(R (U + h T_p)) - Pi_ij(F)) / h,
 * run as six solves per RVE in one launch per bin, warm-started from the
 * base solution (Pi depends on U only, so R (U + h T_p) probes U + h T_p);
 * [A] from [A][M][T] = [P] with M = dE/dU; and the spatial stiffness
 * C_mnpq = J^-1 F_mi F_nj A_ijrs F_pr F_qs.  Post-processing in FP64 on
 * the device, one thread per RVE.  h <= 0 means 1e-4.
 *   F       device 9*n_rve; sigma device 9*n_rve (stress at F);
 *   C       device 36*n_rve: the 6x6 Mandel matrix of C per RVE, row-major,
 *           index order (11, 22, 33, 23, 13, 12), shear rows and columns
 *           scaled by sqrt(2);
 *   status  device n_rve (worst over the 7 solves; RVE_STATUS_NONFINITE if
 *           [M][T] is singular) or NULL.
 * Needs RVE_PREC_MIXED or RVE_PREC_BATCHED_F64 (RVE_EINVAL otherwise).
 */
int rve_tangent_mandel(rve_batch* b, const double* F, double h, double tol, int32_t max_iter,
                       double* sigma, double* C, int32_t* status, void* stream);

/* Forget the warm-start state of the m RVEs in ids (HOST array); ids ==
 * NULL resets every RVE.  Synchronous. */
int rve_reset_state(rve_batch* b, const int64_t* ids, int64_t m);

/* Sizes after pruning, for throughput accounting. */
typedef struct rve_batch_info {
  int64_t n_rve;
  int64_t free_nodes;     /* sum over RVEs of free nodes kept            */
  int64_t active_fibers;  /* fibers with >= 1 free end (updated per DR iteration) */
  int64_t fixed_fibers;   /* boundary-to-boundary fibers (stress only)  */
  int64_t pruned_fibers;  /* fibers removed by pruning                  */
  int64_t n_bins;         /* size bins of the batched path               */
  int64_t device_bytes;   /* device memory held by the batch             */
} rve_batch_info;
int rve_batch_get_info(const rve_batch* b, rve_batch_info* info);

/*
 * Launch configuration of the batched path, per size bin.  Bins group RVEs
 * by footprint: resident bins (mode 0) hold a whole RVE in shared memory,
 * streamed bins (1, 2) read fiber data from L2/HBM, unless the mixed path
 * holds them in a thread-block cluster:
 *   kernel        which kernel runs the bin with the batch's options:
 *                 0 two-phase, 1 node-centric (one CTA per RVE),
 *                 2 node-centric over a cluster of `cluster` CTAs per RVE;
 *   cluster       CTAs per RVE of kernel 2 (0 otherwise);
 *   smem_bytes    dynamic shared memory per CTA of that kernel;
 *   exclusive     RVEs of the bin that a whole-batch solve (rve_solve,
 *                 rve_tangent) runs on SMs of their own, in a launch before
 *                 the rest of the bin (the costliest by the longest-first
 *                 order; 0: one launch);
 *   sorted        1 when a longest-first sort kernel precedes the bin's
 *                 launches.
 */
typedef struct rve_bin_info {
  int32_t n_rve, mode, threads, nodes_per_thread, ctas_per_sm, check_every;
  int64_t smem_bytes;
  int32_t kernel, cluster, exclusive, sorted;
} rve_bin_info;
/* Fill up to max entries for `precision` (RVE_PREC_MIXED or _BATCHED_F64);
 * returns the number of bins (0 before the first batched solve). */
int rve_batch_get_bins(const rve_batch* b, int32_t precision, int32_t max, rve_bin_info* out);

/*
 * Autotuner (the project's own; the paper fixes 512 threads per team,
 * Sec. 4.3): for every size bin of the batch's precision, time solves of
 * the bin's RVEs (cold start, deformation gradients F: device, 9 n_rve)
 * under each thread count its RVE sizes allow and check intervals 25, 50
 * and 100, best of `reps`, and keep the fastest configuration for the bin
 * (the tangent's bins follow).  Synchronous.  The RVEs' warm-start state is
 * left as after a solve.  ms_before / ms_after (may be NULL) receive the
 * summed bin times of the old and the chosen configurations.
 */
int rve_autotune(rve_batch* b, const double* F, int32_t reps, void* stream, double* ms_before,
                 double* ms_after);

/*
 * Launch timing of the fused DR kernel (measurement aid, Sec. 5's timings).
 * With on = 1, every launch of the fused solve kernel is bracketed by two
 * CUDA events recorded on the stream that launches it (the caller's stream,
 * or an internal side stream when several bins run concurrently), and
 * rve_solve is not captured into or replayed from a CUDA graph.  Every call
 * clears the record; launches of all later calls (solve, subset, host solve,
 * tangent, autotune) are appended, up to 65536.  Returns RVE_EINVAL for on
 * not 0 or 1.
 */
int rve_set_kernel_timing(rve_batch* b, int32_t on);

/*
 * Durations (ms, HOST array of at least max doubles) of the fused-kernel
 * launches recorded since timing was last switched, in launch order; waits
 * for those launches to finish.  Returns the number of launches recorded
 * (it may exceed max; only the first max are written), or a negative error
 * code.
 */
int rve_last_kernel_ms(rve_batch* b, int32_t max, double* ms);

/*
 * Orientation tensor of every RVE (Sec. 4 sends it to the macroscale;
 * Sec. 5 measures alignment by P2 = <3 cos^2(theta) - 1>/2):
 *   Omega = <n (x) n>, n = (x_j - x_i)/|x_j - x_i|,
 * averaged over the fibers kept after pruning (active and boundary-to-
 * boundary), at x = F X + h with h the state left by the last solve in
 * `precision` (h = 0 for an RVE not yet solved in it).  P2 along a unit
 * direction a is (3 a.Omega.a - 1)/2.  Unit dyads summed in FP32 per
 * thread, in FP64 across the RVE.
 *   F      device 9*n_rve (the solve's deformation gradients);
 *   omega  device 9*n_rve, symmetric 3x3 row-major, trace 1 (zeros for an
 *          RVE without fibers).
 * Asynchronous on `stream`, ordered after the batch's previous calls.
 */
int rve_orientation(rve_batch* b, const double* F, int32_t precision, double* omega, void* stream);

/* Per-RVE sizes after pruning (HOST arrays of n_rve, any may be NULL). */
int rve_batch_get_sizes(const rve_batch* b, int32_t* free_nodes, int32_t* active_fibers,
                        int32_t* fixed_fibers);

/*
 * Current node positions of RVE r in its reference node order (HOST
 * array of 3 * n_nodes(r) doubles): x = F X + h for free nodes kept,
 * x = F X for boundary and pruned nodes, using F (HOST, 9 doubles) and
 * the fluctuation h left by the last solve in `precision`.  Synchronous.
 */
int rve_get_positions(rve_batch* b, int64_t r, const double* F, int32_t precision,
                      double* x_out);

/*
 * Set the state of RVE r on the given batched precision's path from node
 * positions (HOST, 3 doubles per node in the reference node order, as
 * rve_get_positions returns them) under the deformation gradient F (HOST, 9
 * doubles): the fluctuation of every kept free node becomes x - F X and the
 * state is marked valid, so the next solve with warm_start = 1 starts there
 * (a saved state restored, or a relaxation continued on another path).
 * Boundary and pruned nodes are ignored.  Synchronous.  RVE_EINVAL for an
 * index out of range or the plain precision (which shares the FP64 state:
 * use RVE_PREC_BATCHED_F64).
 */
int rve_set_positions(rve_batch* b, int64_t r, const double* F, int32_t precision, const double* x);

/*
 * Continuous-batching request loop (serving) over a resident pool of RVEs.
 * The paper's RVE batch manager (Sec. 4.3) hands one batched solve per
 * macroscale iteration to the GPU; the server instead takes single requests
 * (rve id, F) as they arrive and batches them at the granularity of DR
 * iterations (Algorithm 2's loop):
 *   - requests queue on the host in arrival order;
 *   - the server has n_slots wave groups (CUDA streams), each with max_wave
 *     request slots; a group runs one wave at a time, and a wave advances
 *     every occupied slot by wave_iters DR iterations (rve_server_set_wave_iters;
 *     0, the default, runs every request to its end within one wave); a solve
 *     that is not done parks on the device (positions, velocities, damping
 *     and iteration count) and resumes in the group's next wave;
 *   - between waves finished requests retire and queued ones take the free
 *     slots; an RVE is in at most one slot at a time, so its warm-start
 *     state advances by one request at a time;
 *   - each request's iterates depend only on its own F, its start state and
 *     wave_iters, so its result is bit-identical alone and in any mix;
 *   - rve_server_step retires finished waves (event query, non-blocking),
 *     admits queued requests and launches the next waves; rve_server_drain
 *     blocks until the queue is empty and no request is on the GPU;
 *   - rve_server_poll returns finished results in completion order with
 *     their latency (seconds from submit to the step that saw them done).
 * The batch's options apply to every solve (precision, tolerance,
 * warm_start: with warm_start = 1 every RVE keeps its converged state on the
 * device between requests).  The plain FP64 path allows n_slots = 1 and
 * wave_iters = 0 only.
 * Pool and admission by device memory (hbm_cap_bytes <= 0: no cap):
 *   - rve_server_create: RVE_EADMIT when the batch, its solver state and the
 *     server's buffers exceed the cap;
 *   - rve_server_add_rves: admits more RVE topologies (arguments as
 *     rve_batch_create, HOST arrays, the batch's options) as a new group of
 *     the pool; their global ids are *first_id .. *first_id + n_rve - 1 (ids
 *     are assigned in admission order and never reused).  RVE_EADMIT, with
 *     nothing admitted, when their device footprint would take the pool over
 *     the cap;
 *   - rve_server_remove_rves: frees the group admitted with first_id (no
 *     request for it may be queued or in flight); the batch given at
 *     creation stays.
 * The batch given at creation must outlive the server; one host thread
 * drives a server; call rve_server_drain before using that batch through the
 * other rve_* calls (which also clears parked solves' state).
 */
typedef struct rve_server rve_server;
typedef struct rve_server_stats {
  int64_t queued;            /* waiting on the host                         */
  int64_t in_flight;         /* in slots on the GPU (running or parked)     */
  int64_t ready;             /* finished, not yet polled                    */
  int64_t completed;         /* finished since creation                     */
  int64_t waves;             /* waves launched since creation               */
  int64_t device_bytes;      /* device memory of the server's own buffers   */
  int64_t pool_rves;         /* RVEs in the pool                            */
  int64_t pool_device_bytes; /* device memory of the pool's batches + state */
  int64_t wave_iters;        /* DR iterations per wave (0: to the end)      */
} rve_server_stats;
int rve_server_create(rve_server** out, rve_batch* b, int32_t n_slots, int32_t max_wave, double hbm_cap_bytes);
/* Iterations per wave (>= 0); only while no request is on the GPU. */
int rve_server_set_wave_iters(rve_server* s, int32_t wave_iters);
int rve_server_add_rves(rve_server* s, int64_t n_rve, const int64_t* node_off, const double* X,
                        const int64_t* fiber_off, const int32_t* conn, const double* L0, const double* EA,
                        const double* B, const uint8_t* is_boundary, const double* V0, int64_t* first_id);
int rve_server_remove_rves(rve_server* s, int64_t first_id);
/* Queue one request for global RVE id rve_id; F is a HOST array of 9 doubles (copied). */
int rve_server_submit(rve_server* s, int64_t rve_id, const double* F, int64_t tag);
int rve_server_step(rve_server* s);
int rve_server_drain(rve_server* s);
/* Copy up to max finished results (HOST arrays: tags[max], sigma[9 max],
 * iters[max], status[max], latency_s[max]; any may be NULL); returns how
 * many were copied, or a negative RVE_E* code. */
int64_t rve_server_poll(rve_server* s, int64_t max, int64_t* tags, double* sigma, int32_t* iters,
                        int32_t* status, double* latency_s);
int rve_server_get_stats(const rve_server* s, rve_server_stats* st);
void rve_server_destroy(rve_server* s);

/* Free everything the batch holds (NULL is ignored). */
void rve_batch_destroy(rve_batch* b);

/* Message of the last failed call on this thread ("" if none). */
const char* rve_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RVE_H */
