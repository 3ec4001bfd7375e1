/*
 * lbm.h -- C ABI of the GB300 (sm_103a) lattice-Boltzmann solver with the
 * moment-conserving wall-link boundary schemes of Li, Chan, Feng & Wang,
 * "Lattice Boltzmann Boundary Conditions for Flow, Convection-Diffusion and
 * MHD Simulations" (arXiv 2506.00907).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Lattice units: dx = dt = 1, c = 1, mu = 1.  Flow on D2Q9 / D3Q19 with
 *   c_s^2 = 1/3; concentration C and the vector magnetic field B on D2Q5 /
 *   D3Q7 with c_h^2 = c_g^2 = 1/4 (weights 1/2, 1/8 in 2D and 1/4, 1/8 in 3D).
 * - Direction numbering (used by lbm_link.dir):
 *     D2Q9 : 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+x+y), 6 (-x+y), 7 (-x-y), 8 (+x-y)
 *     D2Q5 : 0 rest, 1 +x, 2 +y, 3 -x, 4 -y
 *     D3Q19: 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z, 7 (+x+y), 8 (-x-y),
 *            9 (+x-y), 10 (-x+y), 11 (+x+z), 12 (-x-z), 13 (+x-z), 14 (-x+z),
 *            15 (+y+z), 16 (-y-z), 17 (+y-z), 18 (-y+z)
 *     D3Q7 : 0 rest, 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z
 * - Node index n = x + nx*(y + ny*z).  Every axis wraps periodically; a wall is
 *   a layer of solid nodes plus one wall link for every population that would
 *   stream from a solid node into a fluid node.
 * - Body force: Guo forcing with F = rho * accel (the paper, Sec. 2.4, only
 *   says the right-hand side of Eq. 1 "can be modified").  Lorentz force:
 *   magnetic stress 1/2|B|^2 I - BB in the second moment of f^eq (Sec. 2.3).
 * - Host arrays passed in are copied; the caller keeps ownership of every
 *   pointer it passes.  No call throws or aborts; every call returns an
 *   lbm_status and lbm_last_error() gives a message for the last failure.
 * - Device work is issued on the context's stream and is asynchronous unless
 *   the entry point says it synchronises.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* bad argument: sizes, tau <= 1/2, bad or incomplete link list */
    LBM_ENOMEM = 2,     /* device or pinned host allocation failed */
    LBM_ECUDA = 3,      /* a CUDA runtime call failed (message in lbm_last_error) */
    LBM_EUNSTABLE = 4,  /* a non-finite population was found by a check */
    LBM_ETIMEOUT = 5,   /* a bounded device wait gave up */
    LBM_ESTATE = 6      /* call out of order (e.g. stepping a case without walls) */
} lbm_status;

typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1 } lbm_lattice;

/* Storage precision of the populations.  Every precision stores the shifted
 * value p - w_a * phi_ref (phi_ref = rho0, C0 or B0_k of the case), which keeps
 * the small deviations that carry the solution resolvable; FP16S and BF16S
 * store it in 16 bits and compute in FP32, FP32 in FP32, FP64 in FP64.
 * FP16S stores the shifted value times 2^12, so that offsets down to 1.5e-8
 * keep FP16's 11-bit significand (|p - w_a phi_ref| must stay below 16).
 * FP16S and BF16S round the step's results stochastically (the hardware's
 * conversion with random bits; the bits are a hash of the step count, the
 * node and the pair of planes, the same in every launch variant), so that the
 * rounding error has zero mean: rounding to nearest repeats the same error
 * every step at a steady state, which the flow integrates over its diffusion
 * time, and loses every change smaller than half a spacing, which stalls slow
 * transients.  Initialisation and lbm_convert_state round to nearest. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16S = 2, LBM_BF16S = 3 } lbm_prec;

/* physics mask: LBM_FLOW is required */
enum { LBM_FLOW = 1, LBM_CD = 2, LBM_MHD = 4 };

/* One case (one domain).  tau_* > 1/2 (nu = (tau_nu - 1/2)/3, D = (tau_D - 1/2)/4,
 * eta = (tau_eta - 1/2)/4: Eq. 1, 3, 5).  rho0, C0, B0 are the default initial
 * state (rest at equilibrium; the paper initialises with u = 0, Sec. 5.2) and
 * the references of the 16-bit offset storage.  With several concentration
 * species (lbm_config.nspecies > 1), tau_D and C0 are species 0's and
 * tau_Dk[k - 1], C0k[k - 1] those of species k = 1, 2, 3 (ignored otherwise). */
typedef struct {
    int32_t nx, ny, nz;            /* nz = 1 for D2Q9; each >= 1 */
    double tau_nu, tau_D, tau_eta;
    double accel[3];               /* body force per unit mass */
    double rho0, C0, B0[3];
    double tau_Dk[3], C0k[3];      /* concentration species 1..3 */
} lbm_case;

typedef struct {
    lbm_lattice lattice;
    lbm_prec prec;
    uint32_t physics;              /* LBM_FLOW | optional LBM_CD | optional LBM_MHD */
    int32_t ncases;                /* >= 1; all cases are advanced by one launch per step */
    const lbm_case *cases;         /* ncases entries, copied */
    void *stream;                  /* cudaStream_t; NULL = the context creates and owns a non-blocking stream */
    int32_t device;                /* CUDA device ordinal */
    int32_t nspecies;              /* concentration species with LBM_CD: 0 or 1 = one; 2 or 3 = several
                                      (Sec. 4.2.2, text after Eq. 23), then without LBM_MHD */
} lbm_config;

/* Field code of concentration species k in lbm_link.field (k = 0 is the
 * field 1 of a single concentration; the magnetic field keeps 2 + k). */
#define LBM_FIELD_SPECIES(k) ((k) == 0 ? 1 : 4 + (k))
#define LBM_MAX_SPECIES 3

/* Wall-link kinds (Sec. 3-4).  Fields: 0 = f (flow), 1 = h (C, species 0),
 * 2 + k = g_k (B_k), 4 + k = h of concentration species k = 1, 2. */
typedef enum {
    LBM_W_VELOCITY = 0,    /* field f.  Given wall velocity u_wall: Eq. 15 with Eq. 16 for d < 1/2,
                              Eq. 43 for d >= 1/2 (static walls: Bouzidi, Eq. 11/12) */
    LBM_W_GIVEN = 1,       /* h or g_k.  Given C or B_k = phi_wall: Eq. 19/20 (C), Eq. 34/35 (B_k) */
    LBM_W_FLUX = 2,        /* h or g_k.  Flux -lambda dphi/dn = F(phi) = k0 + k1 phi (per link and
                              step, Eq. 23, 48) with the moving-wall correction Eq. 24,
                              imposed by the M scheme, Eq. 25-27 (Robin, Shercliff Eq. 30,
                              zero gradient with k0 = k1 = 0) */
    LBM_W_NEUMANN_BFL = 3, /* h or g_k.  Zero gradient by interpolated bounce-back, Eq. 21/22 */
    /* The two comparison schemes the paper evaluates beside its own (selectable
     * per link; not used by the builders' defaults): */
    LBM_W_VELOCITY_EQ15 = 4,   /* field f.  Eq. 15 with Eq. 16 for every d, Y extrapolated for
                                  d > 1/2; Sec. 5.1 replaces it there by Eq. 43 because it is
                                  unstable (it diverges on walls for every d > 1/2 tried) */
    LBM_W_FLUX_SIMPLIFIED = 5, /* h or g_k.  Flux and move increments as LBM_W_FLUX, added to the
                                  population bounced at X and interpolated as in Eq. 11/12: Eq. 33
                                  at d = 1 (inaccurate at small c_w, Sec. 5.4), Eq. 28 at d = 1/2 */
    /* Open boundaries (Sec. 5.1): a given inlet velocity is LBM_W_VELOCITY with
     * u_wall normal to the boundary (Eq. 41, 43). */
    LBM_W_PRESSURE = 6,        /* field f, flow-only contexts.  Given density rho_w = phi_wall
                                  (pressure rho_w c_s^2): f^eq_a(X) + f^eq_a'(X) - f_rel,a'(Y) with
                                  Y by Eq. 16 for d < 1/2, Eq. 44 for d >= 1/2 (Eq. 42 at d = 1/2);
                                  u(X) extrapolated by Eq. 13 from the fluid velocities at A and E */
    /* (kind 7 is not used by this library) */
    LBM_W_REACTION = 8         /* concentration species i, contexts with several species.  Surface
                                  reaction flux of the case's network (lbm_set_reactions):
                                  increment k0 + k1 R_i(C_1(X), C_2(X), ..) per link and step, with
                                  every species' C(X) by Eq. 13 from its own C at A and E and no
                                  coupled solve (Sec. 4.2.2, text after Eq. 23), imposed with the
                                  moving-wall correction (Eq. 24) by the M scheme (Eq. 25-27); k1 is
                                  the link's share of the wall area (1 for flat walls, Eq. 48) */
} lbm_wall_kind;

/* One wall link: the unknown population of direction dir (pointing from the
 * wall into the fluid) at fluid node A = node, whose neighbour A - e_dir is
 * solid.  d = |AX| / |EA| in (0, 1] is the fraction of the link between A and
 * the wall point X (Eq. 13).  64 bytes. */
typedef struct {
    uint32_t node;
    uint8_t field;                 /* 0 f, 1 h, 2 + k g_k */
    uint8_t dir;
    uint8_t kind;                  /* lbm_wall_kind */
    uint8_t reserved;
    double d;
    double u_wall[3];              /* wall velocity (never extrapolated) */
    double phi_wall;               /* LBM_W_GIVEN: C or B_k on the wall; LBM_W_PRESSURE: density */
    double k0, k1;                 /* LBM_W_FLUX: increment k0 + k1 * phi_X per step;
                                      LBM_W_REACTION: k0 + k1 * R_i(C_X) */
} lbm_link;

/* One surface reaction of a case's network (several species): it runs at
 * rate * prod_m C_m^order[m] per unit wall area and time (order 0, 1 or 2)
 * and produces species i at stoich[i] times that rate (negative: consumed);
 * R_i sums the reactions.  Mass-action kinetics: A + B -> P is order {1, 1, 0},
 * stoich {-1, -1, 1}. */
typedef struct {
    double rate;
    int32_t order[LBM_MAX_SPECIES];
    double stoich[LBM_MAX_SPECIES];
} lbm_reaction;

/* Create a context: validates the configuration, allocates all device memory
 * for every case (two population buffers with guard bands, node flags, the
 * span and tile lists, reduction scratch) and initialises every case at rest
 * (equilibrium of rho0, C0, B0).  Wall-link records and their per-link output
 * are allocated by lbm_set_walls.
 * Errors: LBM_EINVAL (bad config), LBM_ENOMEM, LBM_ECUDA.  *out is NULL on error. */
lbm_status lbm_create(const lbm_config *cfg, lbm_ctx **out);

/* Free all device and host memory of the context.  NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

/* Message of the last failing call on this context ("" if none). */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Geometry and wall links of one case (Sec. 4, 6).
 * solid: host, nx*ny*nz bytes, nonzero = solid.  links: host, nlinks records.
 * The list must hold exactly one link per (fluid node, field, direction) whose
 * upstream neighbour is solid, for every field the physics mask enables.
 * Links whose second fluid node E = A + e_dir is solid are evaluated at
 * d = 1/2 with phi(E) = phi(A) (the paper is silent; this needs no E).
 * Re-initialises the case at rest.  Synchronises.
 * Errors: LBM_EINVAL (range, kind/field mismatch, d outside (0,1], A solid,
 * A - e_dir fluid, duplicate, missing link), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_set_walls(lbm_ctx *ctx, int32_t case_id, const uint8_t *solid,
                         const lbm_link *links, size_t nlinks);

/* Initial state of one case: populations at equilibrium (Eq. 2, 4, 6) of the
 * given host fields, N = nx*ny*nz entries each, u and B as [N][3]; any
 * pointer may be NULL (then rho0, 0, C0, B0).  Resets the step counter of the
 * context's residual history.  Synchronises.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_init_equilibrium(lbm_ctx *ctx, int32_t case_id, const double *rho,
                                const double *u, const double *C, const double *B);

/* Same, from DEVICE fields in FP32 (u and B as [N][3], rho/C may be NULL):
 * the warm-start path.  Asynchronous on the context stream, which reads the
 * fields: work that writes them on another stream must be complete (or
 * ordered before the context stream by the caller). */
lbm_status lbm_init_equilibrium_device(lbm_ctx *ctx, int32_t case_id, const float *rho,
                                       const float *u, const float *C, const float *B);

/* Advance every case by nsteps time steps (Eq. 1, 3, 5 with all wall links).
 * One fused kernel launch per step covers all cases; with graphs enabled
 * (lbm_set_graph) whole blocks of steps replay as one CUDA graph.
 * Asynchronous.  Errors: LBM_EINVAL (nsteps < 0), LBM_ESTATE (walls missing),
 * LBM_ECUDA. */
lbm_status lbm_step(lbm_ctx *ctx, int32_t nsteps);

/* Capture blocks of `steps_per_graph` steps (even, >= 2; 0 disables) as a CUDA
 * graph that lbm_step replays.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_set_graph(lbm_ctx *ctx, int32_t steps_per_graph);

/* Oscillating velocity walls of one case (Stokes' second problem, Sec. 5.2,
 * Eq. 45): from now on every velocity link of field f in the case (kinds
 * LBM_W_VELOCITY and LBM_W_VELOCITY_EQ15) uses u_wall * cos(omega * t + phase)
 * in the step from t to t + 1, the wall velocity taken at t as f^eq(X, t) in
 * Eq. 41/43.  t counts the context's steps since this call for this case
 * (a later call for another case leaves this case's phase alone; a later call
 * for the same case restarts its t at 0).  The motion is part of the state
 * blob (lbm_get_state) and of lbm_convert_state.  The call refolds the wall links of every case
 * (as lbm_set_walls does) and drops existing graphs; from then on a one-block
 * kernel rewrites the velocity coefficient of each oscillating link ahead of
 * every step, also inside captured graphs, so the step kernels themselves
 * carry no term for the motion.  Flux walls of h or g with a nonzero wall velocity would need the
 * same motion in their moving-wall term: a case holding one is refused, here
 * and in later lbm_set_walls calls.  Synchronises.  Errors: LBM_EINVAL (case id,
 * non-finite omega or phase, moving flux wall), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_set_wall_motion(lbm_ctx *ctx, int32_t case_id, double omega, double phase);

/* Macroscopic fields of one case at the current time, FP64, host arrays of N
 * (rho, C) or 3N (u, B) entries; NULL skips.  Solid nodes report 0.  C is
 * concentration species 0.  Synchronises.  Errors: LBM_EINVAL, LBM_ECUDA. */
lbm_status lbm_moments(lbm_ctx *ctx, int32_t case_id, double *rho, double *u,
                       double *C, double *B);

/* Concentration of species k of one case at the current time: host array of
 * N entries (solid nodes 0).  Synchronises.  Errors: LBM_EINVAL (k outside the
 * context's species), LBM_ECUDA. */
lbm_status lbm_species(lbm_ctx *ctx, int32_t case_id, int32_t k, double *C);

/* The surface reaction network of one case (contexts with several species):
 * n <= 4 reactions, copied; used by the case's LBM_W_REACTION links from the
 * next step on (drops captured graphs).  n = 0 clears it (no reaction flux).
 * Errors: LBM_EINVAL (one species, n, order outside 0..2, non-finite),
 * LBM_ECUDA. */
lbm_status lbm_set_reactions(lbm_ctx *ctx, int32_t case_id, int32_t n, const lbm_reaction *reactions);

/* FP64 reductions over the fluid nodes of every case (invariants and the
 * steady-state test; the paper states no convergence criterion):
 * out[8*c + 0..7] = { sum rho, sum C, sum B_x, sum B_y, sum B_z,
 *                     number of non-finite populations,
 *                     sum |phi - phi_prev|^2, sum |phi|^2 }
 * with phi = (u, C, B - B0) (the parts the physics mask enables) and phi_prev
 * the value at the previous call (the first call compares with zero); with
 * several concentration species, slots 2-4 hold sum C_1 .. sum C_3 and
 * phi = (u, C_0, C_1, ..).  The
 * per-node terms are formed in the step's arithmetic precision (FP64 storage:
 * FP64, otherwise FP32, which also keeps phi_prev); every sum over nodes is
 * FP64.  The reduction is deterministic (fixed order).  out: host, 8*ncases
 * doubles.
 * Synchronises.  Returns LBM_EUNSTABLE (after filling out) if any population
 * is not finite, LBM_ETIMEOUT if a bounded device wait of an earlier step
 * gave up.  Errors: LBM_ESTATE (an asynchronous check is in flight), LBM_ECUDA. */
lbm_status lbm_check(lbm_ctx *ctx, double *out);

/* lbm_check in two halves, so that the host need not hold the GPU idle while
 * the result travels back: lbm_check_async enqueues the same reductions and
 * the copy of their record into pinned host memory on the context's stream and
 * returns at once; steps may be enqueued behind it; lbm_check_wait waits for
 * that check only (not for later work) and returns what lbm_check would have
 * returned for it, filling out (host, 8*ncases doubles, may be NULL).  One
 * check may be in flight per context: lbm_check_async and lbm_check refuse a
 * second with LBM_ESTATE, and lbm_check_wait refuses when none is in flight. */
lbm_status lbm_check_async(lbm_ctx *ctx);
lbm_status lbm_check_wait(lbm_ctx *ctx, double *out);

/* Step until every case's relative residual sqrt(sum|phi-phi_prev|^2 / sum|phi|^2)
 * over `interval` steps is below tol, or max_steps are done.  *steps_done and
 * *residual (largest over cases) may be NULL.  Errors: LBM_EUNSTABLE, LBM_ECUDA. */
lbm_status lbm_run_to_steady(lbm_ctx *ctx, int64_t max_steps, int32_t interval, double tol,
                             int64_t *steps_done, double *residual);

/* Freezes (active = 0) or resumes (active != 0) one case.  A frozen case is
 * left out of the step: none of its nodes is read or written, its state is
 * kept identical in both population buffers, and lbm_check reports a zero
 * residual for it while its sums stay those of the frozen state.  The other
 * cases step as they would alone (their arithmetic never reads another
 * case's nodes).  Freezing copies the case's populations once on the device
 * and synchronises the stream; every change rebuilds the step's node and
 * wall-link lists and drops the captured graphs.  A state written into the
 * current buffer from outside the step (initialisation, lbm_set_state,
 * lbm_convert_state, a write through lbm_device_state) is copied to the other
 * buffer of each frozen case before the next step.  Launch variants 1 and 3
 * step every case: freezing is refused while one of them is set, and
 * lbm_set_launch and lbm_autotune refuse them while a case is frozen.
 * Errors: LBM_EINVAL (bad case id, variant 1 or 3 set), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_set_active(lbm_ctx *ctx, int32_t case_id, int32_t active);

/* lbm_run_to_steady case by case: every `interval` steps each active case
 * whose own relative residual is below tol is frozen (lbm_set_active), so
 * that the remaining steps serve only the cases still moving; stops when all
 * are frozen or max_steps are done, then resumes the cases it froze (cases
 * frozen by the caller before the call stay frozen).  *steps_done counts
 * time steps of the whole batch; *residual is the largest of the cases' last
 * measured residuals (INFINITY for a case never measured).  Synchronises.
 * Errors: those of lbm_step, lbm_check and lbm_set_active. */
lbm_status lbm_run_each_to_steady(lbm_ctx *ctx, int64_t max_steps, int32_t interval, double tol,
                                  int64_t *steps_done, double *residual);

/* Checkpoint: size in bytes of the state blob, and copy it out / in (host
 * memory, synchronises).  The blob holds every population of every case, the
 * step count and the wall-motion table of lbm_set_wall_motion (per case
 * omega, phase, on, and the step at which the motion was set); restoring it
 * into a context with the same cases and walls and stepping is bitwise
 * identical to not having stopped, oscillating walls included (a context
 * restored from a blob takes the blob's wall motion).  Errors: LBM_EINVAL
 * (size mismatch, not a blob of this version, a moving flux wall in a case
 * the blob moves), LBM_ECUDA. */
size_t lbm_state_bytes(const lbm_ctx *ctx);
lbm_status lbm_get_state(lbm_ctx *ctx, void *host, size_t bytes);
lbm_status lbm_set_state(lbm_ctx *ctx, const void *host, size_t bytes);

/* Number of steps taken since creation (or the restored state). */
int64_t lbm_steps_done(const lbm_ctx *ctx);

/* Launch shape of the fused step.
 *   variant 0: one thread per node at a time over runs of bulk-fluid
 *              nodes (wall-link nodes are stepped by a second kernel
 *              beside it), in tiles of at most block * nodes_per_thread
 *              nodes (1..8); blocks_per_sm = resident
 *              blocks per SM of a persistent tile loop (0 = one block per
 *              tile, up to 64); min_blocks selects the register budget the
 *              kernel was compiled for, as resident 256-thread blocks per SM:
 *              2D 4, 5 or 6, 3D 2, 3 or 4 (1 = the first).
 *   variant 1: bulk-copy loads and stores (FP32 storage, one
 *              concentration species at most):
 *              persistent blocks of 256 threads copy each plane's source
 *              window of the next tile into shared memory with cp.async.bulk
 *              on mbarriers while computing the current tile, boundary nodes
 *              included, and write each finished tile back with one
 *              cp.async.bulk store per plane (one launch per step).  `block`
 *              is the tile size in nodes and `min_blocks` the register budget,
 *              one of (128, 2), (256, 2), (256, 4), (512, 1), (512, 2);
 *              blocks_per_sm, nodes_per_thread and stages are ignored.
 *   variant 2: as variant 0 (same shapes and register budgets, every
 *              precision), each node reading its pulls unwrapped, at its own
 *              address plus a per-case offset per plane, and only nodes on a
 *              periodic edge reloading the planes whose source wraps; 16-bit
 *              values stay packed two to a register until the collision.
 *   variant 3: shared-memory ring (FP32 storage, one concentration
 *              species at most): persistent
 *              blocks of one producer warp and 8 consumer warps.  The
 *              producer copies each plane's source window of the block's
 *              next tiles into a ring of `stages` (2..8) shared-memory stages
 *              with cp.async.bulk on mbarriers; consumers relax their nodes
 *              from the ring (2D: two x-adjacent nodes per lane with packed
 *              FP32 arithmetic, 3D: one node per lane) and store them to
 *              global memory.  Tiles of 512 (2D) or 256 (3D) nodes;
 *              blocks_per_sm caps the resident blocks per SM (0 = as many as
 *              fit); block, nodes_per_thread and min_blocks are ignored.
 *              Boundary nodes as in variant 0.  Fails with LBM_EINVAL when
 *              the stages do not fit in shared memory.  Not among the
 *              autotuner's candidates.
 * block (variants 0 and 2): 64..256, multiple of 32. */
typedef struct {
    int32_t variant;
    int32_t block;
    int32_t blocks_per_sm;
    int32_t nodes_per_thread;
    int32_t stages;
    int32_t min_blocks;
} lbm_launch;

/* Select the launch shape.  Errors: LBM_EINVAL (out of range, or the
 * pipeline's shared memory does not fit on an SM), LBM_ECUDA. */
lbm_status lbm_set_launch(lbm_ctx *ctx, const lbm_launch *launch);

/* The current launch shape. */
lbm_status lbm_get_launch(const lbm_ctx *ctx, lbm_launch *launch);

/* Autotuner: times the fused step for every candidate launch shape on this
 * context as it runs in production: a CUDA graph of `iters` steps (rounded
 * up to even) is captured and replayed once untimed, then the faster of two
 * timed replays counts (CUDA events).  It keeps the fastest shape, and records it in the text cache file
 * `cache_path` (NULL = no cache) keyed by GPU name, lattice, precision,
 * physics and case sizes; a later call with the same key reads the cache
 * instead of timing.  The context's populations and step count are saved and
 * restored around the timing.  best and best_ms may be NULL.  Candidates:
 * variants 0, 1 and 2 (not 3).  If a candidate's steps fail, the sweep stops,
 * the state and the previous launch shape are restored, every resource of
 * the sweep is released, and the error names the candidate.
 * Errors: LBM_ENOMEM, LBM_ECUDA (or the failing step's status). */
lbm_status lbm_autotune(lbm_ctx *ctx, const char *cache_path, int32_t iters, lbm_launch *best, double *best_ms);

/* Kernel launches issued per time step (for launch accounting): the bulk
 * step over the spans of bulk nodes, plus, when an active case has wall
 * links, the wall-link kernel (one thread per link) and the boundary-node
 * step that uses its values (launch variant 1: one launch in all). */
int32_t lbm_launches_per_step(const lbm_ctx *ctx);

/* Device storage of the current populations (for zero-copy inspection):
 * base pointer, bytes per population, plane stride in elements and element
 * offset of case_id's first plane.  Planes hold the relaxed populations
 * shifted by w_a * phi_ref (FP16S: times 2^12).  Errors: LBM_EINVAL. */
lbm_status lbm_device_state(lbm_ctx *ctx, int32_t case_id, void **base, int32_t *elem_bytes,
                            int64_t *plane_stride, int64_t *case_offset, int32_t *planes);

/* Copies the state of `src` into `dst` at the precision of `dst` (a service
 * of the library; the paper works at one precision).  Both contexts must be on
 * the same device with the same lattice, physics and identical case list; the
 * caller sets the same walls on both (lbm_set_walls copies are per context).
 * Every precision stores p - w_a * phi_ref with the references of the case
 * (rho0, C0, B0), so the stored values are rounded element-wise to the
 * destination type (round to nearest).  The residual snapshot and the step
 * count are copied too, so lbm_check / lbm_run_to_steady on `dst` continue
 * the history of `src`.  Typical use: run a 16-bit storage context towards
 * steady state, then finish in FP32 or FP64.  Synchronises both streams.
 * Errors: LBM_EINVAL (mismatched contexts), LBM_ECUDA. */
lbm_status lbm_convert_state(lbm_ctx *dst, lbm_ctx *src);

/* Allocation-free FP64 reduction of one domain (the paper has no counterpart;
 * this is a service of the library).  It computes, for a population buffer
 * the caller already holds, the same eight numbers lbm_check() reports for a
 * case, but keeps its partial sums in a fixed device array inside the library
 * instead of scratch memory that a context allocated with cudaMalloc.  It is
 * meant for callers that cannot allocate device memory: applications that hand
 * out every byte of the GPU through their own pool or fixed budget, and
 * monitoring hooks that must not change the memory footprint of the job they
 * inspect.
 *   lattice, prec, physics: as in lbm_config.
 *   cs:      host, the case (sizes, accel, rho0, C0, B0).
 *   pops:    device, the case's stored populations (lbm_device_state: base +
 *            case offset), planes of `plane_stride` elements.
 *   flags:   device, nx*ny*nz bytes, nonzero = fluid; NULL counts every node.
 *   snap:    device, 7 * nx*ny*nz doubles holding phi_prev = (u, C, B - B0)
 *            plane by plane, replaced by the current phi (the planes the
 *            lattice and physics can make nonzero; the rest are not touched);
 *            NULL takes phi_prev as zero (sums 6 and 7 then both equal
 *            sum |phi|^2).
 *            Per-node terms are formed as in lbm_check: in FP32 unless the
 *            precision is FP64 (phi_prev is then read rounded to FP32).
 *   out:     host, 8 doubles, the record of lbm_check().
 *   stream:  cudaStream_t (NULL = legacy default stream).  The call
 *            synchronises it (it reads the record back to the host), so it
 *            must not be called while that stream is being captured.
 * Limit: at most LBM_NOALLOC_MAX_NODES nodes (larger domains: LBM_EINVAL, with
 * a message on stderr).  Every call looks up the array's device address on
 * the current device (cudaGetSymbolAddress), so a context torn down and
 * recreated in between is no hazard.  All calls share the one array: calls
 * that overlap on the GPU (other threads or streams) race and must be
 * serialised by the caller.  Every call overwrites what it reads, so nothing
 * needs clearing in between.  FP64 storage is reduced with the FP64 step's
 * rounding policy (no multiply-add contraction), as lbm_check does.
 * Returns LBM_EUNSTABLE (after filling out) if a population is not finite.
 * Errors: LBM_EINVAL, LBM_ECUDA. */
#define LBM_NOALLOC_MAX_NODES (1 << 22)
lbm_status lbm_reduce_noalloc(int32_t lattice, int32_t prec, uint32_t physics, const lbm_case *cs,
                              const void *pops, int64_t plane_stride, const uint8_t *flags, double *snap,
                              double *out, void *stream);

/* ------------------------------------------------------------------------
 * Wall-link builders (host only; no context and no GPU needed).
 * ------------------------------------------------------------------------ */

/* Boundary condition of one field on one wall.  Field f takes LBM_W_VELOCITY;
 * h and g_k take the other kinds.  The flux of LBM_W_FLUX is the physical
 * F(phi) = kappa0 + kappa1 * phi per unit wall area and time (Eq. 17, 30), in
 * lattice units; the builder converts it to the per-link increment
 * k0 + k1 * phi_X (Eq. 23 for flat walls; Eq. 48 with the surface segments for
 * the pipe). */
typedef struct {
    int32_t kind;
    double u_wall[3];
    double phi_wall;
    double kappa0, kappa1;
} lbm_wall_bc;

/* Channel with two flat walls normal to `axis` (0 = x, 1 = y, 2 = z): solid
 * layers at index 0 and n_axis - 1, walls at 1 - d_lo and n_axis - 2 + d_hi
 * (d = |AX| / dx of Eq. 13, the same for axis and diagonal links, Sec. 4.1);
 * the other axes are periodic.  bc[side * 5 + field] for side 0 (low) / 1
 * (high) and field 0 f, 1 h, 2 + k g_k; only fields enabled by `physics` are
 * read.  solid: host output, nx*ny*nz bytes.  links: host output of capacity
 * `cap` records (NULL with cap = 0 to query the count).  *nlinks receives the
 * number of links.  Errors: LBM_EINVAL (sizes, d outside (0, 1], capacity). */
lbm_status lbm_build_channel(int32_t dim, int32_t nx, int32_t ny, int32_t nz, int32_t axis, double d_lo,
                             double d_hi, uint32_t physics, const lbm_wall_bc *bc, uint8_t *solid,
                             lbm_link *links, size_t cap, size_t *nlinks);

/* Circular pipe along x (Sec. 6): fluid where (y - cy)^2 + (z - cz)^2 < R^2
 * with cy = (ny - 1)/2, cz = (nz - 1)/2.  d per node and direction from the
 * intersection of the link with the circle (Fig. 9a).  Flux coefficients are
 * spread over the outer-layer solid points with S_i = (theta_{i+1} -
 * theta_{i-1}) R dx / 2 (azimuth-sorted per axial slice) and split over each
 * point's D3Q7 links by e_a.n / sum e_g.n for e.n > 0 (Eq. 48).  bc[field]
 * for the 5 fields.  Other arguments as lbm_build_channel. */
lbm_status lbm_build_pipe(int32_t nx, int32_t ny, int32_t nz, double R, uint32_t physics, const lbm_wall_bc *bc,
                          uint8_t *solid, lbm_link *links, size_t cap, size_t *nlinks);

/* ------------------------------------------------------------------------
 * Warm-start network (a service of this library, not part of the paper's
 * method): a perceptron with layer widths {4, 64, 64, 64, 2}, tanh hidden
 * layers and a linear output, mapping (x2/R, x3/R, f_Ha, f_cw) of a pipe
 * cross-section to the normalised steady axial velocity and induced field.
 * It is trained on steady fields the solver produced, by this library's own
 * forward, backward and Adam kernels; parameters are FP32 masters with an
 * FP16 copy used by the forward and backward passes (FP32 accumulation).
 * Parameter layout: layer by layer, W (rows = outputs, row-major) then b.
 * ------------------------------------------------------------------------ */
typedef struct lbm_net lbm_net;

/* Number of parameters of the network. */
int64_t lbm_net_num_params(void);

/* dims must be {4, 64, 64, 64, 2} (ndims = 5).  init: host, the initial
 * parameters (the caller draws them).  stream: cudaStream_t (NULL = legacy
 * default).  Errors: LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_net_create(const int32_t *dims, int32_t ndims, const float *init, void *stream, lbm_net **out);
void lbm_net_destroy(lbm_net *net);

/* Copy the FP32 parameters out / in (host; set also resets Adam). */
lbm_status lbm_net_get_params(lbm_net *net, float *host);
lbm_status lbm_net_set_params(lbm_net *net, const float *host);

/* y[n][2] = net(x[n][4]); device arrays; asynchronous on the net's stream. */
lbm_status lbm_net_forward(lbm_net *net, const float *x, float *y, int64_t n);

/* Mean squared error over the n samples (device x[n][4], targets t[n][2])
 * and its gradient, added to the net's gradient accumulator (cleared by
 * lbm_net_adam).  loss (host, may be NULL) receives the loss; grad (host, may
 * be NULL) a copy of the accumulated gradient.  Synchronises when either
 * output is requested. */
lbm_status lbm_net_loss_grad(lbm_net *net, const float *x, const float *t, int64_t n, double *loss, float *grad);

/* One Adam step (bias-corrected) on the accumulated gradient, which is then
 * cleared; refreshes the FP16 copy. */
lbm_status lbm_net_adam(lbm_net *net, float lr, float beta1, float beta2, float eps);

/* Initial fields of a pipe case (axis x, centre ((ny-1)/2, (nz-1)/2), radius
 * R) predicted by the network with features f_ha and f_cw:
 * u = (u_hat * u_scale, 0, 0), B = (b_hat * b_scale, B0, 0) on fluid nodes;
 * device outputs u[N][3], B[N][3] (FP32, N = nx*ny*nz), written on the
 * network's stream, for lbm_init_equilibrium_device. */
lbm_status lbm_net_pipe_fields(lbm_net *net, int32_t nx, int32_t ny, int32_t nz, double R, double f_ha, double f_cw,
                               double u_scale, double b_scale, double B0, float *u, float *B);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
