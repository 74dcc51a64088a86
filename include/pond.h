/*
 * pond.h -- C ABI of the GB300 (sm_103a) Particles-on-Demand time step.
 *
 * Method: Kallikounis & Karlin, "Particles on Demand method: theoretical
 * analysis, simplification techniques and model extensions", arXiv:2302.00310.
 * One call of pond_step() advances every cell by the algorithm of Sec. IV.A.3
 * ("Summary of the algorithm"), with the Strang-split quasi-equilibrium
 * relaxation of Sec. IV.B when Pr != 1:
 *   QE half step -> phi_bar^+ at cell centres (Eq. eq:Fbarplus) -> per face:
 *   averaged face frame (Eq. eq::AvgFrame), stencil moved into it by the
 *   moment-invariant frame transformation (Sec. II.B), limited MUSCL half-step
 *   trace (Eq. eq:InterfacePop), interface moments, non-co-moving equilibrium
 *   (Eq. NonComovingEq), face populations (inverse of Eq. eq:FluxTransf) ->
 *   per cell: fluxes moved into the cell frame (Eq. fluxEq), DUGKS update
 *   (Eqs. eq:FinalUpdateDUGKS, eq:FinalUpdateDUGKS_g), new co-moving frame
 *   (Sec. IV.A.1), QE half step.
 *
 * Lattices (Table I): f on D1Q4 (1D) or D2Q16 (2D, 4x4 tensor product), g on
 * D1Q3 / D2Q9.  Population i of a D-dimensional lattice with q nodes per axis
 * has node indices ix = i % q, iy = i / q (x fastest); nodes per axis are in
 * ascending order: D1Q4 (-r2, -r1, r1, r2), r1,2 = sqrt(3 -+ sqrt 6);
 * D1Q3 (-sqrt 3, 0, sqrt 3).
 *
 * Array layouts (all FP64 at the boundary, whatever the internal precision):
 *   fields   [ny][nx]            (x fastest; ny = 1 in 1D)
 *   f        [Qf][ny][nx]        Qf = 4 (1D), 16 (2D) or 25 (D2Q25)
 *   g        [Qg][ny][nx]        Qg = 3 (1D) or 9 (2D); 4 or 16 with g_same_as_f
 * The state is the DUGKS variable phi~ of Eq. eq:variableTransform in each
 * cell's co-moving frame {u, T}; the frame itself is (ux, uy, T).
 *
 * Ownership: host pointers are caller-owned and copied in or out before the
 * call returns.  With on_device = 1 the pointers are caller-owned CUDA device
 * pointers on the context's device; they are read or written in order on the
 * context's stream and the call synchronises that stream before returning.
 * The context owns its device state: either memory it allocated itself, or a
 * caller-provided workspace (e.g. a PyTorch tensor) that must outlive it.
 *
 * Errors: every call returns a pond_status; nothing is thrown across the ABI.
 * Problems detected on the device (nonphysical state, CFL > 1, an iterated
 * face frame that did not converge) set sticky bits read by
 * pond_status_flags(); kernels never trap and never spin.
 *
 * Threading: a context is used by one host thread at a time.
 */
#ifndef POND_H
#define POND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define POND_ABI_VERSION 1

typedef struct pond_ctx pond_ctx;

/* f-lattice of a context (the g-lattice follows: D1Q3 / D2Q9, as in every run of
 * Sec. V, or the f-lattice itself with pond_params.g_same_as_f).  POND_D2Q25: five Gauss-Hermite nodes per axis (the roots of He_5,
 * Table I), frame-invariant moments to fourth order per axis (Sec. II.D.2;
 * the fourth-order runs of the shock-structure problem, Sec. V.B.4); its
 * populations f[25][ny][nx] use node indices ix = i % 5, iy = i / 5, nodes
 * (-r2, -r1, 0, r1, r2), r1,2 = sqrt(5 -+ sqrt 10).  D2Q25 contexts run 8x8
 * tiles: tile 0 or 10 (128 threads, two CTAs per SM) or 2 (160 threads, one
 * CTA); they are not batched (pond_batch_add: POND_E_INVAL). */
typedef enum { POND_D1Q4 = 1, POND_D2Q16 = 2, POND_D2Q25 = 3 } pond_lattice;

typedef enum {
  POND_OK = 0,
  POND_E_INVAL = 1,       /* invalid argument or parameter                  */
  POND_E_NOMEM = 2,       /* device allocation failed / workspace too small */
  POND_E_CUDA = 3,        /* a CUDA runtime call failed                     */
  POND_E_NONPHYSICAL = 4, /* rho <= 0, T <= 0 or NaN appeared               */
  POND_E_NOCONV = 5,      /* iterated face frame did not converge           */
  POND_E_CFL = 6,         /* CFL number above 1 observed                    */
  POND_E_STATE = 7        /* call out of order (e.g. step before init)      */
} pond_status;

/* boundary kinds per side (x-lo, x-hi, y-lo, y-hi), ghost-node method of
 * Sec. IV.D: periodic wrap, zero normal gradient (copy of the boundary cell),
 * a fixed inflow state (its co-moving equilibrium), or a wall half a cell
 * beyond the last cell, with velocity inflow[side][1..2] and temperature
 * inflow[side][3]: the ghost reflects the interior cell (rho_G = rho_B,
 * u_G = 2 u_w - u_B, T_G = 2 T_w - T_B) and carries the Chapman-Enskog
 * non-equilibrium of Sec. IV.D from centred gradients of the last step.
 * Walls go on the y sides in 2D (x sides then periodic or zero-gradient) and
 * on the x sides in 1D, with at least 3 cells across (else POND_E_INVAL). */
enum { POND_BC_PERIODIC = 0, POND_BC_ZERO_GRADIENT = 1, POND_BC_INFLOW = 2, POND_BC_WALL = 3 };
/* arithmetic of the step: all FP64, or the mixed path: FP32 populations,
 * frame (stored as FP32), transformations, reconstruction and collision, with
 * each cell's conserved moments (rho, rho u, rho E) accumulated in FP64, the
 * new frame computed in FP64, and frame transformations whose shifted nodes
 * exceed xi_fp64_threshold built and applied in FP64 */
enum { POND_FP64 = 0, POND_FP32_MIXED = 1 };
/* frame transformation: tensor product of 1D transformations (all Hermite
 * coefficients a, b <= K per axis) or the paper's Grad projection of total
 * order a + b <= K (Sec. V.A) */
enum { POND_TENSOR = 0, POND_GRAD_K = 1 };
/* flux moved into the cell frame as (v^lambda . n) G phi (Eq. fluxEq) or as
 * G (v^lambda_F . n phi) (Appendix C) */
enum { POND_FLUX_MAIN = 0, POND_FLUX_APPC = 1 };
/* slope limiter of the MUSCL reconstruction (Sec. IV.A.2) */
enum { POND_VANLEER = 0, POND_MINMOD = 1 };
/* face frame: average of the adjacent cell frames (Eq. eq::AvgFrame) or the
 * iterated co-moving face frame of the earlier scheme (Sec. IV.A.3): the face
 * frame is replaced by the interface state until they agree to iter_tol
 * (tested in FP64) or iter_max traces were made; a converged face uses the
 * co-moving equilibrium rho W.  An iterate with a nonphysical interface state
 * ends the iteration and the face keeps the previous iterate.  Unconverged
 * faces set POND_FLAG_NOCONV and are counted (pond_status_flags). */
enum { POND_FRAME_AVG = 0, POND_FRAME_ITER = 1 };
/* sticky device flags */
enum { POND_FLAG_NONPHYSICAL = 1u, POND_FLAG_CFL = 2u, POND_FLAG_NOCONV = 4u };

typedef struct {
  double gamma;            /* adiabatic exponent, C_v = 1/(gamma-1) (Sec. III.A) */
  double tau;              /* relaxation time tau_1                              */
  double prandtl;          /* Pr = tau_1/tau_2; 1 disables the QE step          */
  double dx;               /* cell size (square cells in 2D)                     */
  double dt;               /* time step; <= 0: set by pond_init from cfl         */
  double cfl;              /* max|v_i alpha| dt/dx used when dt <= 0 (Sec. V)    */
  int32_t bc[4];           /* POND_BC_* for x-lo, x-hi, y-lo, y-hi               */
  double inflow[4][4];     /* per side: rho, ux, uy, T of the inflow ghost state */
  int32_t precision;       /* POND_FP64 | POND_FP32_MIXED                        */
  int32_t transform;       /* POND_TENSOR | POND_GRAD_K                          */
  int32_t flux_form;       /* POND_FLUX_MAIN | POND_FLUX_APPC                    */
  int32_t limiter;         /* POND_VANLEER | POND_MINMOD                         */
  int32_t flux_frame;      /* POND_FRAME_AVG | POND_FRAME_ITER                   */
  double iter_tol;         /* convergence tolerance of the iterated frame        */
  int32_t iter_max;        /* iteration cap of the iterated frame                */
  double xi_fp64_threshold;/* mixed path: build the frame transformation in FP64
                              when the shift |(u_s-u_F)/sqrt(T_F)| or the scale
                              sqrt(T_s/T_F) exceeds this                          */
  int32_t tile;            /* cells per CTA of the step kernel: 0 automatic
                              (1D: 1; 2D: 10, or on the mixed path 11
                              for grids of at least four waves of three
                              CTAs per SM); 1D: 1 = 252
                              cells; 2D (x by y): 2 = 8x8, 3 = 16x16, 4 = 16x8,
                              5 = 8x8 and 6 = 8x16 with registers capped for two
                              CTAs per SM, 7 = 8x16 and 8 = 8x8 capped for three
                              CTAs per SM, 9 = 8x16 with 192 threads, 10 = 8x14
                              with 128 threads and two CTAs per SM, 11 (mixed
                              path only) = 8x14 with 128 threads capped for
                              three CTAs per SM.  The
                              iterated face frame runs 8x8 (2D) / 252 (1D).
                              Each output depends only on its stencil, so all
                              tiles compute the same step; as separate machine
                              code they may round differently (multiply-add
                              fusion), to the precision of the context.        */
  /* multiscale f-lattice (Sec. II.E lifting and projection, Sec. IV.C
   * switching), when 1: each step every cell takes D1Q4 / D2Q16 where
   *   s_u = max_{d,e} |u_e(x + dx e_d) - u_e(x - dx e_d)| / (2 sqrt T) > ms_theta_u or
   *   s_T = max_d |T(x + dx e_d) - T(x - dx e_d)| / (2 T) > ms_theta_T
   * (the step's start fields, neighbours by the boundary rules), else D1Q3 /
   * D2Q9.  A low cell's state keeps the high lattice's layout, with its
   * coefficients of order 3 along an axis zero in its co-moving frame: the
   * lifting sets the moments the low lattice lacks to their equilibrium
   * values, and the odd central moments of a Gaussian vanish.  A cell that
   * turns low drops them (the projection).  A face takes the higher lattice
   * of its two cells.  The quasi-equilibrium step of a low cell relaxes the
   * third-order content its lattice resolves; a wall ghost takes the lattice
   * of the cell it reflects (a low one drops its Chapman-Enskog content of
   * order 3 along an axis).  Requires D1Q4 / D2Q16, the averaged face frame
   * and tile 0 (or the default: 1 in 1D, 10 in 2D); not batched.  With the
   * main flux form a low cell keeps mass and momentum but not energy exactly
   * (its lattice lacks the third-order moment the energy flux needs in
   * another frame: the mixed path, whose conserved fluxes are otherwise
   * evaluated once per face, adds a low cell's energy flux in the cell's own
   * frame, as the FP64 path does); Appendix C's form keeps all three. */
  int32_t multiscale;
  double ms_theta_u;       /* thresholds on s_u and s_T (the paper states none) */
  double ms_theta_T;
  /* 1: the g-populations on the f-lattice (D1Q4 / D2Q16, invariant to third
   * order) instead of D1Q3 / D2Q9; g needs frame-invariant moments to second
   * order only (Sec. III.C) and every run of the paper uses D2Q9.  g[Qg] then
   * holds 4 (1D) or 16 (2D) populations in the f-lattice's node order.
   * Requires D1Q4 / D2Q16, the averaged face frame, no multiscale and tile 0
   * (or the default: 1 in 1D, 10 in 2D); not batched. */
  int32_t g_same_as_f;
  /* tiles per strip of the step launch: 0 automatic, else 1-8.  A CTA steps a
   * strip of consecutive tiles of one tile row left to right, handing each
   * tile's right-edge x-face records to the next tile instead of computing
   * them twice (a face's record depends only on its stencil, so every strip
   * length gives the same state bit for bit).  Automatic: 2 where that does
   * not lengthen the launch's waves x strip length, else 1; 1 with the
   * iterated face frame.  Batches choose their own (pond_batch_step). */
  int32_t strip;
} pond_params;

/* Fills the defaults: gamma 1.4, tau 1e-4, Pr 1, dx 1, dt 0 (from cfl 0.2),
 * periodic, FP64, tensor, main flux form, van Leer, averaged frame,
 * iter_tol 1e-12, iter_max 10, xi_fp64_threshold 8, tile 0. */
void pond_params_default(pond_params *p);

/* Device bytes a context needs for the given lattice/dims/params (two state
 * buffers plus a small status block).  dims = {nx, ny}; ny is ignored in 1D. */
pond_status pond_workspace_size(pond_lattice lat, const int64_t dims[2], const pond_params *p,
                                size_t *bytes);

/* Creates a context on the current CUDA device.  workspace: caller-owned
 * device memory of at least pond_workspace_size() bytes, 256-byte aligned, or
 * NULL to let the context allocate (and free) its own.  stream: a cudaStream_t
 * (NULL = legacy default stream) on which every kernel of the context runs.
 * Errors: POND_E_INVAL (bad lattice, dims < 2, tau/dx/gamma out of range,
 * unknown option), POND_E_NOMEM, POND_E_CUDA. */
pond_status pond_create(pond_ctx **out, pond_lattice lat, const int64_t dims[2],
                        const pond_params *p, void *workspace, size_t workspace_bytes,
                        void *stream);

/* Sets the state to the co-moving equilibrium of the primitive fields
 * (Eqs. feqPond, geqPond): f = rho W, g = (C_v - D/2) T rho W, frame (u, T).
 * rho, ux, T: [ny][nx]; uy: [ny][nx] in 2D, ignored (may be NULL) in 1D.
 * If params.dt <= 0, dt is set so that max|v_i alpha| dt/dx = params.cfl on
 * this state.  Resets the status flags.  Synchronises the stream. */
pond_status pond_init(pond_ctx *c, const double *rho, const double *ux, const double *uy,
                      const double *T, int on_device);

/* Advances the state by n >= 0 steps (asynchronous on the context stream;
 * consecutive steps are replayed from a captured CUDA graph).  Returns
 * POND_E_STATE before pond_init/pond_set_state, POND_E_INVAL for n < 0. */
pond_status pond_step(pond_ctx *c, int64_t n);

/* rho, u, T of every cell recomputed from the populations (Eqs.
 * eq::ConservationLaws, eq:E).  uy may be NULL in 1D.  Synchronises. */
pond_status pond_moments(pond_ctx *c, double *rho, double *ux, double *uy, double *T,
                         int on_device);

/* Raw state in / out (layouts above).  pond_set_state takes populations that
 * are already in each cell's co-moving frame (ux, uy, T).  Synchronises. */
pond_status pond_get_state(pond_ctx *c, double *f, double *g, double *ux, double *uy,
                           double *T, int on_device);
pond_status pond_set_state(pond_ctx *c, const double *f, const double *g, const double *ux,
                           const double *uy, const double *T, int on_device);

/* Sticky flags (POND_FLAG_*), the largest CFL number max|v_i alpha| dt/dx met
 * since the last reset, and the count of face evaluations whose iterated
 * frame did not converge.  Any pointer may be NULL.  Synchronises.  Returns
 * POND_E_NONPHYSICAL if that flag is set, else POND_OK. */
pond_status pond_status_flags(pond_ctx *c, uint32_t *flags, double *max_cfl,
                              int64_t *noconv_faces);
pond_status pond_reset_flags(pond_ctx *c);

/* Iteration statistics of the iterated face frame (Sec. IV.A.3, the
 * predictor-corrector of the earlier PonD-DUGKS scheme that Sec. V.D compares
 * with), since the last reset: face evaluations (each face once per step),
 * traces made over all of them (the interface state traced in a face frame:
 * one per iterate, plus the retrace at the previous iterate when an iterate
 * turns nonphysical), and the most traces one face evaluation made.  All zero
 * with the averaged frame.  Any pointer may be NULL.  Synchronises. */
pond_status pond_iter_stats(pond_ctx *c, int64_t *face_evals, int64_t *traces, int32_t *max_traces);

/* Multiscale: cell updates made on the high-order f-lattice since the last
 * reset (zero without multiscale).  May be NULL.  Synchronises. */
pond_status pond_ms_stats(pond_ctx *c, int64_t *high_cell_updates);

/* Waits for all work queued on the context stream. */
pond_status pond_sync(pond_ctx *c);

/* Time step in use, steps taken since pond_init/pond_set_state, and the tile
 * code the step kernel runs with. */
pond_status pond_info(pond_ctx *c, double *dt, int64_t *steps, int32_t *tile);

/* Checkpoint and restore.  Not a step of the method: the context's raw state
 * (each cell's Hermite coefficients and frame in the context's arithmetic,
 * exactly as the step kernel keeps them), its step counter, time step and
 * status block, so that a run resumed from a checkpoint continues bit for
 * bit as the uninterrupted run would (pond_get_state/pond_set_state pass
 * populations through an FP64 change of basis, which rounds).
 * pond_checkpoint_size: bytes of a checkpoint of this context.
 * pond_checkpoint: copies it into caller-owned host memory of at least that
 * many bytes; synchronises.  POND_E_STATE before pond_init.
 * pond_restore: loads a checkpoint into a context created with the same
 * lattice, dims, precision and parameters (the time step comes from the
 * checkpoint); POND_E_INVAL if the checkpoint does not match the context.
 * Synchronises. */
pond_status pond_checkpoint_size(pond_ctx *c, size_t *bytes);
pond_status pond_checkpoint(pond_ctx *c, void *host, size_t bytes);
pond_status pond_restore(pond_ctx *c, const void *host, size_t bytes);

/* Releases the context and the device memory it allocated itself. */
void pond_destroy(pond_ctx *c);

/* Static description of a status code. */
const char *pond_strerror(pond_status s);

/* POND_ABI_VERSION of the loaded library. */
int pond_abi_version(void);

/* ---- Batches: many contexts advanced by one persistent kernel -----------------
 * Not a step of the method: a way to run many independent problems (each a
 * context with its own grid, time step, boundaries and parameters) through
 * the same step of Sec. IV.A.3 at once.  Each launch is one time step of
 * every member; a grid of (SMs x resident CTAs) CTAs strides over the tiles
 * of all members, each tile running the same tile step as pond_step().
 * Launches are replayed from a captured CUDA graph (graph_steps launches per
 * chunk); members may join and leave between calls without a new capture.
 *
 * A member's state after a batch step is bit for bit the state pond_step()
 * gives it alone with the same tile shape: both launch the same kernel
 * function, and no result depends on the other members.  Every shape
 * computes the same step (to rounding: each is its own machine code), so the
 * autotuner times candidate shapes on the run's own steps: the first
 * pond_batch_step() call in which every member takes at least graph_steps x
 * (number of shapes) steps runs one chunk with each shape and keeps the
 * fastest, and times them again at the first such call after the stepping
 * members' tiles have grown or shrunk fourfold since.  A fixed tile equal to
 * the contexts' own keeps results bit for bit identical to solo runs.
 *
 * Members must share the batch's dimension, precision and stream, must be
 * initialised, may not use the iterated face frame, and use D1Q4 or D2Q16.  A context belongs
 * to at most one batch; pond_destroy() removes it from its batch.  Batch
 * calls are made from one host thread at a time. */
typedef struct pond_batch pond_batch;
typedef struct {
  int32_t tile;         /* 0: the autotuner picks; else a candidate 2D tile code
                           (mixed: 10, 11, 6; FP64: 10, 9, 6; 1D batches have the
                           one 252-cell tile)                                 */
  int32_t graph_steps;  /* launches per chunk and per captured graph (1-1024) */
  int32_t autotune;     /* 1: time the candidate shapes on the first long call */
} pond_tune;

/* Defaults: tile 0, graph_steps 8, autotune 1. */
void pond_tune_default(pond_tune *t);

/* Creates an empty batch for up to `capacity` members of dimension dim (1 or
 * 2) and precision POND_FP64 / POND_FP32_MIXED, running on `stream` (a
 * cudaStream_t; NULL = legacy default stream, launched without graphs).  It
 * allocates a device descriptor table and two pinned host copies of it.
 * tune may be NULL (defaults). */
pond_status pond_batch_create(pond_batch **out, int32_t dim, int32_t precision, int32_t capacity,
                              const pond_tune *tune, void *stream);

/* Adds / removes a member.  POND_E_INVAL if the context does not fit the
 * batch (dimension, precision, stream, iterated frame, capacity) or is in a
 * batch already; POND_E_STATE if it is not initialised. */
pond_status pond_batch_add(pond_batch *b, pond_ctx *c);
pond_status pond_batch_remove(pond_batch *b, pond_ctx *c);

/* Number of members (in the order they were added; removal keeps the order
 * of the others). */
int32_t pond_batch_size(const pond_batch *b);

/* Advances member i by steps[i] >= 0 time steps (steps NULL: one each), in
 * chunks of graph_steps launches; members with fewer steps drop out of the
 * later launches.  Asynchronous on the batch stream except while the
 * autotuner reads its timings and when the host gets two chunks ahead of
 * the GPU (the descriptor table is double-buffered).  Flags and CFL numbers
 * go to each member's own status (pond_status_flags). */
pond_status pond_batch_step(pond_batch *b, const int64_t *steps);

/* Tile code and grid (CTAs) in use, whether the autotuner has run, and the
 * MLUPS of the chosen shape in its timed chunk (0 if not tuned).  Any
 * pointer may be NULL. */
pond_status pond_batch_info(const pond_batch *b, int32_t *tile, int32_t *grid, int32_t *tuned,
                            double *tuned_mlups);

/* Waits for the batch's work, detaches its members and frees the batch. */
void pond_batch_destroy(pond_batch *b);

/* ---- Step without any device allocation -------------------------------------
 * No counterpart in the paper: this is a calling convention, not a step of
 * the method.  It performs the same FP64 steps as pond_step() for callers that
 * may not call cudaMalloc, for example code that runs while a CUDA graph is
 * being captured in global mode (cudaMalloc is then prohibited), hosts whose
 * device memory belongs to a pool allocator that must not be bypassed, or
 * latency-critical loops that cannot afford cudaMalloc's implicit device
 * synchronisation.
 *
 * The caller passes the state in and gets it back: f, g, ux, uy (2D only; may
 * be NULL in 1D), T are caller-owned FP64 device arrays in the layouts above,
 * holding each cell's populations in its co-moving frame; they are overwritten,
 * in order on `stream`, with the state after n steps.  params: precision must
 * be POND_FP64, flux_frame POND_FRAME_AVG, dt > 0 (no CFL time step); the tile
 * is fixed (8x8 in 2D, 252 cells in 1D).  flags: host pointer or NULL; when
 * given, the call synchronises `stream` and stores the sticky POND_FLAG_* bits
 * of this call.  A synchronisation is not allowed while `stream` is being
 * captured into a CUDA graph (it would invalidate the capture), so flags must
 * be NULL then: a call with flags on a capturing stream returns POND_E_INVAL
 * before any work.  While the call's work runs the arrays hold intermediate
 * values; after a POND_E_CUDA failure their contents are undefined.
 *
 * Its only scratch is one static __device__ array of POND_NOALLOC_SCRATCH_BYTES
 * (a status block plus one state buffer) that every GPU loading this library
 * holds until the process exits; the call allocates and frees nothing.  The
 * first call on a device looks up the array's device address and sets the
 * kernels' shared-memory limits; make that first call before any stream
 * capture.  All calls on a device share the array: calls whose work overlaps
 * on the GPU race.
 *
 * Errors: POND_E_NOMEM when the state does not fit the array (2D FP64:
 * 74,897 cells; 1D: 209,712 cells), POND_E_INVAL for bad arguments (or
 * flags given while `stream` is capturing),
 * POND_E_NONPHYSICAL (only when flags is given), POND_E_CUDA. */
#define POND_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
pond_status pond_step_noalloc(pond_lattice lat, const int64_t dims[2], const pond_params *p,
                              double *f, double *g, double *ux, double *uy, double *T,
                              int64_t n, uint32_t *flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* POND_H */
