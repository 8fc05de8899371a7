/*
 * hsma.h -- C ABI of the GB300 HSMA pair-sum library (libhsma.so).
 *
 * The library evaluates the Harmonic Surface Mapping Algorithm (HSMA) of
 * Liang, Yuan and Xu, "HSMA: An O(N) electrostatics package implemented in
 * LAMMPS", for N point charges in
 *   - a fully periodic box (HSMA3D; the sum of Sec. 2.1, Eq. 3), or
 *   - a slab periodic in x and y between two planar dielectric interfaces
 *     (HSMA2D; the image-charge sum of Sec. 2.1, Eq. 4).
 * One evaluation runs the steps of Sec. 2.2 on one GPU:
 *   near field  -- every particle against the images inside the auxiliary
 *                  sphere B (periodic images; in 2D also reflection images);
 *   check sums  -- the same images onto the monitoring points (and in 2D the
 *                  DtN face grid) that feed the least-squares fit (Eq. 6);
 *   fit + map   -- FP64 coefficients A_n^m of Eq. 5 and the Fibonacci surface
 *                  charges on the sphere (Sec. 2.2, third step);
 *   far field   -- the surface charges onto the particles;
 *   assembly    -- E = 1/2 sum q_i Phi(r_i), F_i = -q_i grad Phi(r_i), and the
 *                  per-atom potential (the outputs of Sec. 3.1).
 *
 * Units are Gaussian with eps_c = 1 (Sec. 2.1, Eq. 2) times the option
 * "coulomb_prefactor" (default 1).
 *
 * Pointers.  Every array argument may be a host pointer or a CUDA device
 * pointer of the current device; the library asks the CUDA runtime which.
 * Arrays are plain C arrays of double: positions x are N*3 row-major
 * (x0 y0 z0 x1 ...), charges q are N, forces are N*3 row-major, potential is N.
 * The caller owns every array it passes.  hsma_eval copies the inputs before
 * returning; hsma_submit copies them before returning, so the caller may
 * reuse its buffers at once.  Results are written when hsma_eval returns
 * HSMA_OK, or when hsma_poll returns HSMA_OK.  On any error the output arrays
 * are left unspecified.
 *
 * Threads.  One handle must not be used by two host threads at once.  Calls
 * on different handles are independent.
 *
 * Errors.  Every int-returning call returns HSMA_OK (0), HSMA_PENDING (1,
 * hsma_poll only) or a negative HSMA_ERR_* code; hsma_last_error gives a
 * one-line message for the last failing call on that handle.
 */
#ifndef HSMA_H
#define HSMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HSMA_OK               0
#define HSMA_PENDING          1
#define HSMA_ERR_ARG        (-1)  /* bad argument: p outside 1..40, M < (p+1)^2 or
                                     M (p+1)^2 > 2^31, |gamma| > 1,
                                     N < 1 or N > 2^28, N times the image shifts
                                     at or above 2^31 (device indices are 32-bit),
                                     dims not 2 or 3, box <= 0, NULL pointer,
                                     unknown option or ticket */
#define HSMA_ERR_NOT_NEUTRAL (-2) /* |sum q| > 1e-10 sum |q| */
#define HSMA_ERR_OUT_OF_SLAB (-3) /* 2D: some z not strictly inside (0, Lz) */
#define HSMA_ERR_NOMEM      (-4)  /* a device or pinned-host allocation failed */
#define HSMA_ERR_BUDGET     (-5)  /* serving: request larger than the HBM budget */
#define HSMA_ERR_TIMEOUT    (-6)  /* a bounded device wait ran out */
#define HSMA_ERR_CUDA       (-7)  /* any other CUDA runtime error */
#define HSMA_ERR_NUMERIC    (-8)  /* the fit lost rank (degenerate geometry), or
                                     the energy is not finite */

typedef struct hsma_ctx* hsma_t;

/*
 * hsma_create -- geometry-only preparation (the paper's "Init", Sec. 3.1).
 *
 * box:   Lx, Ly, Lz > 0.  3D: the periodic cell [0,Lx)x[0,Ly)x[0,Lz).
 *        2D: periodic in x, y; charges must lie in 0 < z < Lz, with the
 *        dielectric interfaces at z = 0 (bottom) and z = Lz (top).
 * dims:  3 (HSMA3D) or 2 (HSMA2D).
 * p:     harmonic order P of Eq. 5, 1..40; (p+1)^2 basis functions.
 * M:     number of Fibonacci surface charges, >= (p+1)^2 and at most
 *        2^31 / (p+1)^2 (the surface map is an M x (p+1)^2 FP64 matrix
 *        built on the host; the same bound holds for n_monitor).
 * gamma_top, gamma_bot: dielectric mismatches of the top and bottom media,
 *        gamma = (eps_c - eps_out)/(eps_c + eps_out) in [-1, 1] (Sec. 2.1,
 *        after Eq. 4).  Ignored when dims == 3.
 * out:   receives the handle.
 * Defaults (changeable with hsma_set_option before the first evaluation):
 * lambda 1.3 (3D) / 1.6 (2D), n_monitor 2(p+1)^2 (Sec. 3.2), dtn_grid 80,
 * precision 1 (FP32 pair arithmetic with compensated FP64 accumulation).
 * The fit matrix is factored once (an SVD pseudo-inverse in FP64) at the
 * first evaluation after a change, and reused by every evaluation.
 * Errors: HSMA_ERR_ARG, HSMA_ERR_NOMEM, HSMA_ERR_CUDA.
 */
int hsma_create(const double box[3], int dims, int p, int M,
                double gamma_top, double gamma_bot, hsma_t* out);

/*
 * hsma_set_option -- change one parameter (Sec. 3.2 lists the paper's set).
 * Keys:
 *   "lambda"            R_s = lambda * R_c, R_c = half the box diagonal; > 1.
 *                       (lambda = 2.6 is the paper's lambda = 1.3 measured
 *                       against the full diagonal.)
 *   "n_monitor"         number of monitoring points N_m, >= (p+1)^2.
 *   "precision"         0 = FP64 pair arithmetic, 1 = FP32 pair arithmetic
 *                       with FP64-compensated accumulation (the paper's
 *                       eps_tol switch of Sec. 3.2 picks FP64 below 1e-6),
 *                       2 = as 1 but with every source-target difference
 *                       formed exactly: coordinates carried as FP32 hi + lo
 *                       pairs, (hi_s - hi_t) + (lo_s - lo_t), so close pairs
 *                       keep FP32 relative accuracy however large the box
 *                       (about 1.4 x the cost of 1).
 *   "dtn_grid"          G, grid points per side on each 2D face (>= 4).
 *   "coulomb_prefactor" multiplies energy, forces and potential.
 *   "timing"            1 = record per-phase CUDA-event times (hsma_get_info).
 *   "chunks"            source chunks per target tile of the near/check
 *                       launch (0 = automatic or autotuned).
 *   "autotune"          1 (default) = on the first evaluation of each N, time
 *                       the near/check launch for a few kernel variants and
 *                       chunk counts and keep the fastest (cached per process
 *                       by N, check-point count and expected image count);
 *                       0 = fixed heuristic.
 *   "targets_per_thread" kernel variant: 1, 2, 4 (scalar FP32), 12, 14
 *                       (packed FP32x2, 2 or 4 targets), 24 (packed, sums in
 *                       shared memory) or 32, 34 (exact differences, 2 or 4
 *                       targets), 44 (exact differences, 4 targets, sums in
 *                       shared memory) for precision 2; turns autotune off.
 *   "graphs"            1 (default) = replay the per-evaluation pipeline as a
 *                       CUDA graph captured on the first evaluation of each N.
 *   "tree_far_order"    1 (default) = above the leaf level, listed cells whose
 *                       centre lies at least sqrt(8) cell widths from the
 *                       target's cell are evaluated to order P - 4 (for
 *                       tree_order >= 8): their truncation bound stays well
 *                       below that of the nearest listed cells at order P.
 *                       0 = every cell to order P.
 *   "tree_count"        1 = the tree evaluation runs its counting instance,
 *                       which also counts the multipole evaluations (M2P)
 *                       and FP32 direct pairs it performs (info keys
 *                       "tree_m2p", "tree_direct_pairs"); slower, for the
 *                       roofline only.  0 (default) = off.
 *   "fused_reduce"      2 = each pair launch sums its per-chunk partials
 *                       itself: the CTA that finishes a target tile's last
 *                       chunk adds that tile's partials in the fixed order
 *                       of the separate reduction (bitwise the same result,
 *                       one launch fewer, partials read back while still in
 *                       L2); 0 = a separate reduction launch; 1 (default) =
 *                       per launch, the fused form where the tile sums are
 *                       short beside the launch's pair work (long launches),
 *                       else the separate one.  Info keys "fused_near" and
 *                       "fused_far" give the choice of the current plan.
 *   "dynamic_schedule"  1 (default) = pair-launch CTAs take (tile, chunk)
 *                       items from a device counter; 0 = a static
 *                       round-robin.  Either way each item writes its own
 *                       partial, so results are the same.
 *   "sphere_mask"       1 (default) = the near set is the images inside the
 *                       sphere B (Sec. 2.2, first step); 0 = every image of
 *                       the enumerated cells (3D: all 27 at lambda <= sqrt 3),
 *                       inside B or not.  The far sources then start 1.5
 *                       cells out and the series converges faster: more
 *                       accurate at equal p, about 4.5 x the near-field cost.
 *   "grad_rows"         1 = append gradient-periodicity rows to the fit: for
 *                       every periodicity row of Eq. 6 three more that ask
 *                       the field (each Cartesian component) to be periodic
 *                       too, weighted by grad_weight * R_c.  Not in the
 *                       paper's fit; 0 (default) = the paper's rows only.
 *   "grad_weight"       weight of those rows in units of R_c (> 0; 0.1).
 *   "surface_rule"      quadrature of the surface charges on the sphere B
 *                       (Sec. 2.2, third step): 0 (default) = M golden-spiral
 *                       points with equal weights; 1 = the Fibonacci lattice
 *                       rule of Sec. 3.2 with F = M and F_w the Fibonacci
 *                       number before it (M must be a Fibonacci number >= 13,
 *                       else HSMA_ERR_ARG), lattice (j + 1/2)/F, (j F_w mod F)/F
 *                       mapped to the sphere through a degree-5 periodising
 *                       map, with the map's Jacobian as the weights; it
 *                       converges as M^-6.
 *   "near_tree"         1 = evaluate the near-field and check-point sums by a
 *                       tree (the paper's O(N) path, which it runs through an
 *                       FMM library): images binned into a uniform octree over
 *                       [-R_s, R_s]^3, multipole expansions of order
 *                       tree_order per cell, FMM interaction lists evaluated
 *                       at each target, direct FP32 pairs with its
 *                       neighbourhood (see tree_leaf_mode).  An
 *                       approximation of the sums: at tree_order 10, force
 *                       RMS about 1e-6 and energy 3e-6 to 5e-6 relative to
 *                       the direct sums.  Needs precision 1
 *                       (an evaluation at precision 0 or 2 returns
 *                       HSMA_ERR_ARG); 0 (default) = direct sums.
 *   "tree_order"        expansion order of the tree: 4, 6, 8, 10 (default),
 *                       12 or 14.
 *   "tree_leaf_level"   leaf level L of the tree (8^L leaves over the root
 *                       cube), 2..6; 0 (default) = about 32 images per
 *                       occupied leaf.
 *   "guard_selftest"    1 = overwrite one byte of the guard band of this
 *                       handle's position buffer (inside its allocation, so
 *                       an in-bounds write), 0 = restore it; lets a test see
 *                       "guard_violations" count it.  Needs an evaluation
 *                       first, else HSMA_ERR_ARG.
 *   "tree_leaf_mode"    the tree's finest level: 1 = summed directly (every
 *                       leaf of the 27 neighbours of the target's cell one
 *                       level up), 2 = leaf multipoles plus direct pairs with
 *                       the 27 neighbouring leaves, 0 (default) = 1 when the
 *                       leaves hold about 48 images or fewer, else 2.
 *   "tree_parts"        1..8 (default 4): each 32-target task of the tree
 *                       evaluation is split into this many work items (every
 *                       tree_parts-th batch of each interaction list), which
 *                       a persistent kernel takes from a queue; the items'
 *                       partial sums are added in a fixed order, so the
 *                       result depends on this value but not on scheduling.
 *   "far_field"         0 (default) = the far field from the M surface charges
 *                       (Eq. 8, the paper's choice); 1 = the fitted series of
 *                       Eq. 5 itself, sum over n >= 1 of A_nm (r/R_c)^n Y_nm,
 *                       and its gradient, per particle (cost N (p+1)^2 instead
 *                       of N M).  The two agree to the surface quadrature's
 *                       error; the series skips that quadrature.
 * On a server handle (hsma_server_create) the keys are
 *   "inject_fail_ticket" fault injection for tests: the request with this
 *                       ticket fails with HSMA_ERR_CUDA when it is admitted,
 *                       without touching the GPU; 0 = off.
 *   "ragged_variant"    pair-kernel code of the ragged launches: 12 (default,
 *                       2 targets per thread, 512-target tiles) or 24 (4
 *                       targets, sums in shared memory, 1024-target tiles)
 *                       at precision 1; 32 (default) or 44 at precision 2.
 *                       Only while the server holds no request.
 *   "ragged_dynamic"    1 (default) = the ragged launches' CTAs take items
 *                       from a device counter; 0 = static round-robin.
 *                       Results are the same either way.
 *   "slot_streams"      1 (default) = each slot's small kernels and copies on
 *                       a stream of its own; 0 = everything on the server's
 *                       stream.  Only while the server holds no request.
 *   "max_batch"         requests per batch at most; 0 (default) = every
 *                       request a free slot admits.  Below the slot count,
 *                       several batches are in flight and a batch's prep
 *                       overlaps the earlier batches' launches.  Results are
 *                       the same either way.
 * Errors: HSMA_ERR_ARG (unknown key or value out of range).
 */
int hsma_set_option(hsma_t h, const char* key, double value);

/*
 * hsma_set_stream -- run this handle's work on the given cudaStream_t
 * (NULL = the library's own stream).  The stream must outlive its use.
 */
int hsma_set_stream(hsma_t h, void* stream);

/*
 * hsma_eval -- one full evaluation (the paper's "Compute", Sec. 3.1 / 2.2).
 * x: N*3 positions, q: N charges (neutral to 1e-10 relative; the residual is
 * removed as q_i -= sum q / N).  3D positions are wrapped into the box; in 2D
 * x and y are wrapped and z must be inside (0, Lz).
 * energy: 1 double (required).  forces: N*3 or NULL.
 * Blocks until the results are written.  Inputs are not scanned: a
 * non-finite position or charge makes the energy non-finite, and the call
 * then returns HSMA_ERR_NUMERIC (hsma_poll does the same for a served
 * request); the handle stays usable.
 * Errors: HSMA_ERR_ARG, HSMA_ERR_NOT_NEUTRAL, HSMA_ERR_OUT_OF_SLAB,
 * HSMA_ERR_NOMEM, HSMA_ERR_NUMERIC, HSMA_ERR_TIMEOUT, HSMA_ERR_CUDA.
 */
int hsma_eval(hsma_t h, const double* x, const double* q, int64_t N,
              double* energy, double* forces);

/*
 * hsma_eval_ex -- hsma_eval that also returns the per-atom potential
 * Phi(r_i) (N doubles, prefactor applied) when potential is not NULL.
 */
int hsma_eval_ex(hsma_t h, const double* x, const double* q, int64_t N,
                 double* energy, double* forces, double* potential);

/*
 * hsma_get_info -- one scalar about the handle or its last evaluation.
 * Keys: "Rc", "Rs", "n_shifts", "n_check", "rank", "Ns" (images in B at the
 * last evaluation), "t_total_ms", "t_prep_ms", "t_near_ms", "t_fit_ms",
 * "t_far_ms", "t_assemble_ms" (with option timing = 1), "chunks",
 * "far_chunks", "far_field", "tree_levels" (leaf level L of the tree, 0 when
 * off), "tree_direct_leaf" (1 when the tree sums its leaf level directly),
 * "kernels_per_eval" (kernel launches of one evaluation), "grid",
 * "slots", "kernel", "tile_targets", "guard_violations" (process-wide: how
 * many device buffers of this library, live or already freed, have had the
 * 256-byte guard band behind their end overwritten; every buffer is
 * allocated with such a band holding a fixed pattern, compared when the
 * buffer is freed and, for live buffers, when this key is read; waits for
 * the device first), "fused_reduce", "dynamic_schedule" (the options),
 * "tree_m2p", "tree_m2p_low", "tree_direct_pairs" (the tree evaluation's
 * work at the last evaluation with option tree_count = 1: multipole
 * evaluations to order P and to the lower far-cell order, direct pairs),
 * "tree_far_order" (the option), "t_tree_eval_ms" (the tree's
 * evaluation kernel alone, with option timing = 1).
 * On a server handle (hsma_server_create) the keys are "batches" (batches
 * enqueued so far), "inflight_at_last_batch" (earlier batches still on the
 * GPU when the last one was enqueued), "queued" (requests waiting for a
 * slot) and "gpu_ms" (the summed device-time spans of the retired batches).
 * Errors: HSMA_ERR_ARG for an unknown key.
 */
int hsma_get_info(hsma_t h, const char* key, double* value);

/*
 * hsma_get_array -- copy an intermediate of the last evaluation to host
 * memory (for checking each step separately).  Names and lengths:
 *   "check_points"  n_check*3  monitoring points, their wraps, 2D face grid
 *   "check_phi"     n_check    Phi_B at the check points
 *   "check_dz"      n_check    dPhi_B/dz at the check points
 *   "coeffs"        (p+1)^2-1  A_n^m for n >= 1 in the basis (r/R_c)^n Y_nm
 *   "surface_points" M*3       Fibonacci points on the sphere B
 *   "surface_q"     M          surface charges Q_m
 *   "grad"          N*3        grad Phi(r_i) (no prefactor)
 * n is the capacity of out in doubles; fails with HSMA_ERR_ARG if too small.
 */
int hsma_get_array(hsma_t h, const char* name, double* out, int64_t n);

/*
 * hsma_geometry_array -- host-only (no GPU needed): build the geometry of a
 * set-up exactly as hsma_create + options would, and copy one array of it:
 *   "T"              M x nv  the composite map from the raw check vector v
 *                    (3D: Phi_B at [monitoring points; wraps]; 2D: [Phi_B;
 *                    dPhi_B/dz] at [monitoring points; wraps; top face;
 *                    bottom face]; with gradient rows followed by
 *                    [dx; dy; dz Phi_B] at [monitoring points; wraps]) to the
 *                    surface charges, row-major.  It is the fit of Sec. 2.2,
 *                    Eq. 6 followed by the surface map.
 *   "check_points"   n_check*3, "surface_points" M*3,
 *   "shifts"         n_shift*5 (sx, sy, zs, zo, factor), identity first,
 *   "sizes"          [n_check, nv, nA, rank, n_shift, Rc, Rs, Rs2].
 * lam <= 0, n_monitor <= 0 or G <= 0 select the defaults; grad_weight > 0
 * adds the gradient-periodicity rows with that weight (option grad_rows),
 * <= 0 leaves them out; surface_rule is the option of that name.  n is the
 * capacity of out in doubles; a too small n is HSMA_ERR_ARG (for "T" it is
 * checked before the matrix is formed).
 * Errors: HSMA_ERR_ARG, HSMA_ERR_NOMEM (host memory), HSMA_ERR_NUMERIC.
 */
int hsma_geometry_array(const double box[3], int dims, int p, int M, double gamma_top,
                        double gamma_bot, double lam, int n_monitor, int G,
                        double grad_weight, int surface_rule, const char* name, double* out,
                        int64_t n);

/*
 * hsma_pair_sum_static -- the direct pair sum (the kernel behind the near
 * field, the check-point sums and the far field) without any device
 * allocation.  The paper has no counterpart.  It exists for callers that
 * cannot call cudaMalloc: engines that hand out all device memory from their
 * own pool and forbid raw cudaMalloc/cudaFree (an allocation behind the pool's
 * back breaks its accounting), plug-ins that run inside such an engine, and
 * real-time loops that must not pay for an allocation or for the
 * synchronisation that freeing implies.
 *
 * targets: n_tgt*3 doubles (x, y, z), device memory of the current device.
 * sources: n_src*4 doubles (x, y, z, q), device memory of the current device.
 * out:     n_tgt*4 doubles, device memory of the current device:
 *          phi(t) = sum_s q_s/|x_s - t| and its gradient with respect to t
 *          (dphi/dx, dphi/dy, dphi/dz), row-major per target.
 *          A source at exactly a target's position divides by zero.
 * precision: 0 = FP64 pairs, 1 = FP32 pairs with compensated accumulation.
 * stream:  cudaStream_t to run on (NULL = the legacy default stream); the call
 *          returns once the work is enqueued, so out is ready when the stream
 *          reaches that point.
 * Scratch: a fixed 64 MiB __device__ array inside the library, one per GPU
 * that loads it, held until the process exits.  Every call shares it and
 * leaves its contents behind; every element a call reads is written by that
 * same call first, so nothing needs clearing.  Calls whose work overlaps on
 * the GPU (other streams, other host threads) race on it: order them.
 * The first call on each device (and the first after that device's context
 * has been replaced, e.g. by cudaDeviceReset) looks up the array's device
 * address with cudaGetSymbolAddress, which may load the module; make that
 * first call before any stream capture.  The call allocates nothing itself.
 * The chunk partial sums are combined by a small fixed-order kernel of its
 * own (8 warps per 32 targets), not by the evaluation's reduction.
 * Limit: (n_tgt + n_src) * (16 bytes in FP32, 32 in FP64) plus 32 * n_tgt
 * bytes of partial sums must fit in 64 MiB; larger inputs are rejected with
 * HSMA_ERR_ARG before any device work.
 * Errors: HSMA_ERR_ARG (NULL pointer, n < 1, precision, size, or a pointer
 * that is not memory of the current device), HSMA_ERR_CUDA.
 */
int hsma_pair_sum_static(const double* targets, int64_t n_tgt, const double* sources,
                         int64_t n_src, double* out, int precision, void* stream);

/* hsma_destroy -- free every resource of the handle (NULL is allowed). */
void hsma_destroy(hsma_t h);

/* hsma_last_error -- message of the last failing call (never NULL). */
const char* hsma_last_error(hsma_t h);

/*
 * Serving: continuous batching of independent HSMA3D requests (MD replicas,
 * Monte Carlo trial states) on one GPU.
 *
 * hsma_server_create -- a request loop with at most `slots` requests on the
 * device at once and `budget_bytes` of device memory for their state.
 * precision as for hsma_set_option (0, 1 or 2).  Requests that arrive while others run
 * are admitted as slots and memory free up; their pair sums share launches.
 * Each request's result is identical to an evaluation of it alone.
 * Each slot runs its request's own small kernels on a stream of its own.
 * Host memory: every request holds pinned copies of its inputs and result
 * from submit to poll; these buffers are pooled by size and kept, for reuse,
 * until hsma_destroy of the server (the pool's size is that of the most
 * requests ever held at once).
 */
int hsma_server_create(int slots, double budget_bytes, int precision, hsma_t* out);

/*
 * hsma_submit -- enqueue one 3D request (cubic or not: box[3]); non-blocking.
 * Copies x and q before returning.  ticket receives the request id.
 * Errors: HSMA_ERR_ARG, HSMA_ERR_NOT_NEUTRAL, HSMA_ERR_BUDGET (the request
 * alone exceeds the budget), HSMA_ERR_NOMEM.
 */
int hsma_submit(hsma_t server, const double* x, const double* q, int64_t N,
                const double box[3], int p, int M, uint64_t* ticket);

/*
 * hsma_poll -- HSMA_PENDING while the request runs; HSMA_OK once energy (1
 * double) and forces (N*3, or NULL) are written, after which the ticket is
 * retired.  A negative code reports that request's failure (and retires the
 * ticket); hsma_last_error(server) then gives that request's own message.
 */
int hsma_poll(hsma_t server, uint64_t ticket, double* energy, double* forces);

/*
 * hsma_server_step -- let the request loop make progress from the calling
 * thread (admit, launch one batch, retire finished requests).  Returns the
 * number of requests still queued or running.  hsma_poll also advances it.
 */
int hsma_server_step(hsma_t server);

/*
 * MD loop: the validation workload of Sec. 4.1 on the device.  A primitive
 * electrolyte of soft spheres (the shifted-truncated LJ repulsion cut at
 * 2^(1/6) sigma, energy 4 eps [(sigma/r)^12 - (sigma/r)^6] + eps) plus the
 * electrostatics of an HSMA3D handle, integrated by velocity Verlet, in the
 * canonical ensemble with a Nose-Hoover thermostat (one thermostat, symmetric
 * Trotter splitting, Q = g kT tdamp^2, g = 3N - 3) or in NVE (tdamp <= 0).
 * Each step runs as one CUDA graph replay on the handle's stream: kick and
 * drift, cell list and LJ forces, the full HSMA evaluation, kick,
 * thermostat, one thermo row.  Nothing returns to the host between steps.
 * The paper runs this loop inside LAMMPS; here it is part of the library.
 */
typedef struct hsma_md* hsma_md_t;

/*
 * hsma_md_create -- start an MD loop around the handle h (its box, p, M,
 * options and coulomb_prefactor, which is l_B kT in reduced units).  With a
 * 2D handle the loop is the confined electrolyte of Sec. 4.3: periodic in x
 * and y, ions kept in 0 < z < Lz by shifted-truncated LJ walls at z = 0 and
 * z = Lz (options wall_sigma 0.5, wall_eps 1.0).
 * x, v: N*3 positions and velocities; q: N charges (host or device).  Copies
 * them, wraps x into the box, computes the forces and takes the first
 * thermostat half step.  h must stay alive and must not be used for another
 * N or have its options changed while the loop exists.
 * Errors: HSMA_ERR_ARG (N < 2, a periodic box side under 3 x 2^(1/6) sigma,
 * bad parameters), HSMA_ERR_NOT_NEUTRAL, HSMA_ERR_OUT_OF_SLAB, HSMA_ERR_NOMEM,
 * HSMA_ERR_CUDA.
 */
int hsma_md_create(hsma_t h, const double* x, const double* v, const double* q, int64_t N,
                   double mass, double dt, double kT, double tdamp, double lj_sigma,
                   double lj_eps, hsma_md_t* out);

/*
 * hsma_md_set_option -- "rdf_every" (accumulate the RDF pair counts every
 * k-th step, 0 = never), "rdf_bins" (200), "rdf_rmax" (5.0, at most L/2)
 * (changing either clears the counts), "cell_capacity" (particles per LJ
 * cell, 8; a run that overflows it fails with HSMA_ERR_ARG); slabs only:
 * "wall_sigma", "wall_eps" (the LJ walls; the forces are recomputed),
 * "zhist_bins" (100: the ion density histogram across the slab, taken with
 * the RDF).
 */
int hsma_md_set_option(hsma_md_t md, const char* key, double value);

/*
 * hsma_md_run -- advance `steps` steps and wait for them.  thermo (NULL or
 * steps*6 doubles, host or device) receives per step: kinetic energy, LJ
 * energy, Coulomb energy, xi, eta, and the conserved extended energy
 * K + U + Q xi^2/2 + g kT eta (K + U in NVE); the LJ column includes the
 * wall energy of a slab.  A slab ion that leaves (0, Lz) fails the run with
 * HSMA_ERR_OUT_OF_SLAB.
 */
int hsma_md_run(hsma_md_t md, int64_t steps, double* thermo);

/*
 * hsma_md_get -- copy state to the host: "x" (N*3, wrapped), "x_unwrapped",
 * "v", "forces" (LJ + Coulomb at the current positions), "rdf" (3*rdf_bins
 * pair counts: cation-anion, cation-cation, anion-anion; in a slab the
 * minimum image is taken in x and y only), "zhist" (2*zhist_bins counts of
 * cations then anions across 0 < z < Lz; slabs), "state" (xi, eta, last K,
 * last U, RDF samples, velocity scale).  n is the capacity of out.
 */
int hsma_md_get(hsma_md_t md, const char* name, double* out, int64_t n);

/* hsma_md_last_error -- message of the last failure on this MD loop. */
const char* hsma_md_last_error(hsma_md_t md);

/* hsma_md_destroy -- free the loop (not the electrostatics handle). */
void hsma_md_destroy(hsma_md_t md);

#ifdef __cplusplus
}
#endif

#endif /* HSMA_H */
