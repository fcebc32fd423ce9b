/*
 * lbrbc.h -- C ABI of the GB300 (sm_103a) library for the coupled lattice
 * Boltzmann time step with the general local reactive boundary condition of
 * Weinmiller et al., arXiv 2306.10794.
 *
 * One library call advances a flow lattice (D3Q19, or D2Q9 in 2D; BGK or TRT,
 * Sec. 2.1, Eqs. fluid_BGK, fluid_Equilib, fluid_TRT) and a solute
 * advection-diffusion lattice (D3Q7, or D2Q5 / D2Q9 in 2D; BGK or TRT with
 * the rest-fraction weights, Eqs. solute_BGK, solute_equilibrium_function,
 * solute_TRT, RestFraction, RestFractionCs2) by whole time steps.  Every
 * solid-fluid link of the solute lattice carries the reactive boundary
 * condition of Eq. general_RBC with k_i from Eq. k_i_S_New (or Eqs. k_i_S_Ve,
 * k_i_S2, or its anti-bounce-back limit); the reacted mass feeds a per-cell
 * solid fraction (Eq. solidFractionUpdate, adjacent growth, Sec. 2.4) whose
 * thresholds phi <= 0 and phi >= 1 turn cells fluid or solid.
 *
 * Conventions
 *   - Grids are indexed x fastest: cell (x, y, z) is entry x + nx*(y + ny*z)
 *     of every caller array.  2D grids have nz = 1.
 *   - Pointers marked "host" are read (or written) during the call only and
 *     stay owned by the caller.  The library owns all device state of a
 *     simulation; lbrbc_destroy releases it.
 *   - Every entry point returns an lbrbc_status; on failure a message is
 *     available from lbrbc_last_error (per simulation, or for the calling
 *     thread when no simulation exists).  No exception crosses the ABI.
 *   - The library runs its kernels on the CUDA stream given to lbrbc_step
 *     (a cudaStream_t passed as void*).  NULL selects a stream owned by the
 *     simulation and makes the call synchronous.
 *   - There is no CPU fallback: a machine without a usable GPU gets
 *     LBRBC_ERR_CUDA from lbrbc_create.
 *   - The fluid-cell sweep is chosen at creation by the environment variable
 *     LBRBC_FLUID_SWEEP: "dense" (default; one thread per grid cell) or
 *     "list" (compacted fluid cells; not with phase change, where it falls
 *     back to "dense").  Both give bitwise identical results.
 */
#ifndef LBRBC_H
#define LBRBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbrbc_sim lbrbc_sim; /* opaque, owned by the library */

typedef enum {
    LBRBC_OK = 0,
    LBRBC_ERR_ARG = 1,         /* invalid parameter or size                        */
    LBRBC_ERR_CUDA = 2,        /* CUDA runtime error (message has the CUDA text)    */
    LBRBC_ERR_NUMERIC = 3,     /* non-finite or non-positive density/concentration  */
    LBRBC_ERR_TIMEOUT = 4,     /* reserved for bounded device waits                 */
    LBRBC_ERR_STATE = 5,       /* capacity of an internal list exceeded             */
    LBRBC_ERR_UNSUPPORTED = 6  /* lattice / option combination not built            */
} lbrbc_status;

/* Boundary treatment per axis.  OPEN is allowed on x only: x = 0 is a
 * velocity inlet (moving-wall bounce-back for f, anti-bounce-back at
 * c_inlet for g) and x = nx-1 a pressure outlet (anti-bounce-back at
 * rho_outlet for f, anti-bounce-back at the cell's own previous
 * concentration, i.e. zero gradient, for g).  WALL treats positions beyond the
 * axis as inert solid (halfway bounce-back). */
enum { LBRBC_PERIODIC = 0, LBRBC_WALL = 1, LBRBC_OPEN = 2 };

/* k_i of Eq. general_RBC: Eq. k_i_S_New (default), Eq. k_i_S_Ve,
 * Eq. k_i_S2, or k = infinity (anti-bounce-back, C_wall = C_eq). */
enum { LBRBC_SCHEME_NEW = 0, LBRBC_SCHEME_VERHAEGHE = 1, LBRBC_SCHEME_PATEL_JU = 2, LBRBC_SCHEME_ANTI_BB = 3 };

enum { LBRBC_FP32 = 0, LBRBC_FP64 = 1 };

/* Population storage (no counterpart in the paper; results are bitwise the
 * same either way).  DENSE: every cell of the padded grid holds populations.
 * SPARSE: only the stored cells do -- fluid cells, wet boundary cells and the
 * solid cells next to those (the cells one dissolution can turn into
 * boundary cells) -- numbered in row-major order in three ranges, with a
 * neighbour table for streaming; in porous media a warp then moves whole
 * population lines.  When a phase change needs a cell outside the stored set
 * the layout is repacked on the device within that step.  AUTO picks SPARSE
 * when under 85 % of the lanes of the dense grid's 32-cell row segments would
 * hold fluid cells, else DENSE.  Batched domains always use DENSE. */
enum { LBRBC_LAYOUT_AUTO = 0, LBRBC_LAYOUT_DENSE = 1, LBRBC_LAYOUT_SPARSE = 2 };

/* Cell codes of the mask given to lbrbc_create. */
enum { LBRBC_CELL_FLUID = 0, LBRBC_CELL_REACTIVE = 1, LBRBC_CELL_DIRICHLET = 2 };

/* Node classes reported by lbrbc_classes: a solid cell with a fluid
 * neighbour along the solute lattice is a wet boundary node (BOUND). */
enum { LBRBC_CLASS_FLUID = 0, LBRBC_CLASS_BOUND = 1, LBRBC_CLASS_SOLID = 2 };

typedef struct {
    int dim;                 /* 2 or 3                                              */
    int nx, ny, nz;          /* grid size; nz = 1 when dim = 2                      */
    int flow_q;              /* 19 (3D), 9 (2D) or 0 (no flow lattice: u = 0)        */
    int solute_q;            /* 7 (3D), 5 or 9 (2D)                                  */
    int bc[3];               /* LBRBC_PERIODIC / LBRBC_WALL / LBRBC_OPEN (x only)    */
    int scheme;              /* LBRBC_SCHEME_*                                       */
    int phase_change;        /* 1: cells change phase at phi <= 0 / phi >= 1         */
    int precision;           /* LBRBC_FP32 (deviation storage) or LBRBC_FP64         */
    int event_log_capacity;  /* phase-change events kept for lbrbc_events (0: none)  */
    double tau_flow;         /* tau_NS (BGK) or tau_NS^+ (TRT); nu = (tau - 1/2)/3    */
    double magic_flow;       /* Lambda of Eq. fluid_TRT_visc; < 0 selects BGK        */
    double tau_solute;       /* tau_AD (BGK) or tau_AD^+ (TRT): D = cs^2 (tau - 1/2)  */
    double magic_solute;     /* Lambda of Eq. solute_TRT_visc; < 0 selects BGK       */
    double rest_fraction;    /* J0 of Eq. RestFraction (D2Q5/D3Q7); < 0: none        */
    double k_r;              /* reaction rate coefficient (Eq. reactionRateBoundary) */
    double c_eq;             /* equilibrium concentration                           */
    double molar_volume;     /* V_m of Eq. solidFractionUpdate (a_m = dt = 1)        */
    double c_init;           /* initial concentration (unless an init field given)   */
    double rho_init;         /* initial density                                     */
    double c_dirichlet;      /* concentration held by LBRBC_CELL_DIRICHLET cells     */
    double c_inlet;          /* inlet concentration (OPEN x)                        */
    double u_inlet;          /* plug inlet velocity when no inlet profile is given  */
    double rho_outlet;       /* outlet density (OPEN x)                             */
    int layout;              /* LBRBC_LAYOUT_* (0: AUTO)                              */
} lbrbc_params;

/* Optional per-cell inputs; any pointer may be NULL.  All host pointers. */
typedef struct {
    const double *k_field;   /* N: per-voxel k_r replacing k_r on reactive cells    */
    const double *c_init;    /* N: initial concentration                            */
    const double *u_init;    /* 3N (x,y,z interleaved): initial velocity            */
    const double *phi_init;  /* N: initial solid fraction (default 1 reactive, 0 else) */
    const double *inlet_ux;  /* ny*nz: inlet velocity profile u_x(y, z)             */
} lbrbc_init;

/* Create a simulation (Sec. 2; problem statement of Sec. 2.3 / 2.4).
 *   params    host, copied.  tau_* must exceed 1/2; rest_fraction < 1;
 *             k_r, c_eq, molar_volume >= 0; Dirichlet and open boundaries
 *             need a solute lattice.  Violations: LBRBC_ERR_ARG.
 *   mask      host, nx*ny*nz bytes with LBRBC_CELL_* codes, copied.
 *   init      host, optional (may be NULL).
 *   out       receives the simulation handle.
 * The populations start at equilibrium with rho_init, u_init and c_init. */
lbrbc_status lbrbc_create(const lbrbc_params *params, const uint8_t *mask, const lbrbc_init *init,
                          lbrbc_sim **out);

/* Advance n >= 0 time steps (Sec. 2.1-2.4): stream-collide of both lattices,
 * the reactive boundary condition on every solid-fluid link, the reacted-mass
 * ledger, the solid-fraction update and, if enabled, the phase changes with
 * the on-device rebuild of the boundary-link lists.  Kernels are enqueued on
 * `stream` (cudaStream_t; NULL: the simulation's own stream, synchronous). */
lbrbc_status lbrbc_step(lbrbc_sim *sim, int64_t n, void *stream);

/* Moments of the current state (Eqs. fluid_BGK_visc, solute_diffu):
 *   u    3N doubles (x,y,z interleaved), 0 outside fluid cells;
 *   rho  N doubles, 0 outside fluid cells;
 *   c    N doubles, concentration of fluid and boundary cells, 0 in the solid;
 *   phi  N doubles, solid fraction of every cell.
 * Any pointer may be NULL.  device = 1: the pointers are device memory of
 * the simulation's GPU; device = 0: host memory.  Synchronises the stream
 * given to the last lbrbc_step. */
lbrbc_status lbrbc_fields(lbrbc_sim *sim, double *u, double *rho, double *c, double *phi, int device);

/* Node class of every cell (LBRBC_CLASS_*), N bytes, host. */
lbrbc_status lbrbc_classes(lbrbc_sim *sim, uint8_t *out);

/* Mass balance (FP64, deterministic reduction order):
 *   out[0] sum of c over fluid and boundary cells,
 *   out[1] sum of phi / V_m over all cells,
 *   out[2] dissolution charge that had no solid neighbour to pay it,
 *   out[3] cumulative inflow through Dirichlet cells,
 *   out[4] cumulative reacted mass (mass injected by reactive links),
 *   out[5] completed time steps.
 * With walls, periodic axes and Dirichlet cells (no OPEN axis),
 * out[0] + out[1] + out[2] - out[3] is conserved to round-off.
 * `out` is host memory with room for 6 doubles. */
lbrbc_status lbrbc_mass_ledger(lbrbc_sim *sim, double *out);

/* lbrbc_mass_ledger without allocating device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc / cudaFree at this point -- for instance a host program that has
 * handed the GPU's memory to its own pool allocator (a fresh cudaMalloc could
 * fail or fragment it), or a monitoring loop that must not trigger the
 * device-wide synchronisation cudaFree implies.  It returns the same six
 * values as lbrbc_mass_ledger (summation order differs: agreement to
 * round-off).
 *   - Scratch: a file-scope device array of 2 * 4096 + 8 doubles (65.6 KB),
 *     present on every GPU that loads the library until the process exits.
 *     Partial sums are kept per block of 65536 cells, so grids above
 *     4096 * 65536 = 268435456 cells are rejected with LBRBC_ERR_ARG.
 *   - Every call looks up the array's device address with the simulation's
 *     device made current (nothing is cached, so a device reset between
 *     calls is harmless).
 *   - Every call on a device shares the array and leaves its last contents
 *     there; each call overwrites every entry it reads, so nothing needs
 *     clearing.  Calls that overlap on the GPU (two host threads, two
 *     simulations on one device at once) race on it: serialise them.
 *   - Synchronises the stream of the last lbrbc_step.  `out`: host, 6 doubles. */
lbrbc_status lbrbc_mass_ledger_noalloc(lbrbc_sim *sim, double *out);

/* The size rule of lbrbc_mass_ledger_noalloc on its own (host arithmetic,
 * no GPU needed; the paper has no counterpart): a grid of n_cells cells needs
 * ceil(n_cells / cells_per_block) partial pairs and fits if that is at most
 * max_blocks.  lbrbc_mass_ledger_noalloc applies it with max_blocks = 4096
 * and cells_per_block = 65536.  Returns LBRBC_OK, or LBRBC_ERR_ARG with the
 * reason (naming the cell limit) written to msg (host, msg_len bytes,
 * NUL-terminated; may be NULL). */
lbrbc_status lbrbc_noalloc_size_check(int64_t n_cells, int32_t max_blocks, int64_t cells_per_block, char *msg,
                                      int32_t msg_len);

/* Phase-change events logged so far (up to event_log_capacity): on return
 * *count holds the number logged; if step/node/kind are non-NULL the first
 * min(*count, capacity) entries are written (host).  kind: 1 dissolution,
 * 2 precipitation; node is the x-fastest cell index. */
lbrbc_status lbrbc_events(lbrbc_sim *sim, int64_t *count, int64_t capacity, int64_t *step, int64_t *node,
                          int32_t *kind);

/* Discrete adjoint (an extension: the paper computes no gradient): advance
 * n_steps >= 1 steps exactly as lbrbc_step would (the simulation ends
 * n_steps later) and return the reacted mass over those steps,
 *   J = sum over steps and reactive links of m_l  (mass injected into the
 *       fluid; positive for dissolution),
 * with its exact derivatives for this discrete method:
 *   dJ_dk      dJ / d k_r for a uniform change of k_r on every reactive cell,
 *   dJ_dceq    dJ / d c_eq,
 *   dJ_dkfield dJ / d k_r(cell) per cell (N doubles, host, x fastest; may be
 *              NULL; zero outside wet boundary cells).
 * Needs phase_change = 0 (events are not differentiable).  Uses sqrt(n)
 * checkpoints of the full state and recomputes each segment onto a tape, so
 * it needs about 26 sqrt(n) + 10 sqrt(n) population arrays of device memory
 * and costs about two forward passes plus the adjoint sweep.  All pointers
 * host; any may be NULL.  The flow does not depend on k_r or c_eq and is not
 * differentiated. */
lbrbc_status lbrbc_adjoint(lbrbc_sim *sim, int64_t n_steps, double *J, double *dJ_dk, double *dJ_dceq,
                           double *dJ_dkfield);

/* Measurement helper (no counterpart in the paper): advance n (1..4096)
 * steps exactly as lbrbc_step does, but without CUDA graphs and with CUDA
 * events recorded on `stream` around each kernel group; on return
 * ms_out[0..3] hold the mean duration in milliseconds per step of the
 * fluid-cell stream-collide kernel, the wet-boundary kernel (RBC, ledger,
 * solid fraction), the precipitation-share gather and the phase-change
 * group, and *launches (if non-NULL) the kernel launches per step.
 * Synchronises the stream. */
lbrbc_status lbrbc_profile_step(lbrbc_sim *sim, int64_t n, void *stream, double *ms_out, int64_t *launches);

/* out[0] fluid cells, out[1] wet boundary cells at creation, out[2] kernel
 * launches of a time step without phase-change events (host memory, 3
 * entries). */
lbrbc_status lbrbc_info(lbrbc_sim *sim, int64_t *out);

/* Kernel launches of lbrbc_step (host memory, 2 entries): out[0] per time
 * step without phase-change events, out[1] added by a step with events (the
 * phase-change path of Sec. 2.4: events, reclassification, list updates;
 * inside the step graphs it is a conditional node that runs only when the
 * step raised events).  No GPU work, no synchronisation. */
lbrbc_status lbrbc_launch_counts(lbrbc_sim *sim, int64_t *out);

/* Population storage of the simulation (host memory, 4 entries): out[0]
 * LBRBC_LAYOUT_DENSE or LBRBC_LAYOUT_SPARSE, out[1] cells holding
 * populations (SPARSE: stored cells now; DENSE: padded grid slots), out[2]
 * repackings of the SPARSE layout so far, out[3] bytes of population
 * storage.  Synchronises the stream of the last lbrbc_step. */
lbrbc_status lbrbc_layout_info(lbrbc_sim *sim, int64_t *out);

/* ---- Batches of independent domains ------------------------------------
 * Many domains of uneven size and their own parameters (same lattices and
 * precision, 3D, no phase change) advanced together, step pairs replayed
 * from one CUDA graph: either each kernel phase of a step (fluid sweep,
 * wet-boundary list, fluid-end gather) is ONE persistent launch over a
 * schedule of work items from all domains, or (schedule 4) every domain's
 * own kernels run as independent branches of the graph.  Not a construct of
 * the paper: a way to run many of its problems at once. */
typedef struct lbrbc_batch lbrbc_batch; /* opaque, owned by the library */

/* n domains: params[n] (host, copied), masks[n] (host pointers to nx*ny*nz
 * bytes each), inits[n] or NULL.  Errors as lbrbc_create (message from
 * lbrbc_batch_last_error(NULL)); phase_change must be 0. */
lbrbc_status lbrbc_batch_create(int32_t n, const lbrbc_params *params, const uint8_t *const *masks,
                                const lbrbc_init *inits, lbrbc_batch **out);

/* Advance every domain by n steps (stream as in lbrbc_step). */
lbrbc_status lbrbc_batch_step(lbrbc_batch *batch, int64_t n, void *stream);

/* Autotuner: times each candidate schedule (persistent kernels: tile width
 * along x 128/64/32 or fitted to the domain (policies 0-2) or fluid-list
 * chunks (3), domain-major or largest-first interleaved order, 4/8/16
 * blocks per SM; or policy 4, the domains' own kernels as parallel graph
 * branches, 8 x the third entry branch streams: 32/64/128) for `pairs` step
 * pairs plus one warm-up pair -- real steps of every domain -- and keeps the
 * fastest.  choice[3] (host, may be NULL) receives [tile policy, order,
 * blocks per SM]; *ms_per_step (may be NULL) the best time per step in
 * milliseconds. */
lbrbc_status lbrbc_batch_autotune(lbrbc_batch *batch, int32_t pairs, void *stream, int64_t *choice,
                                  double *ms_per_step);

/* Fix the schedule without timing: the three numbers lbrbc_batch_autotune
 * reports (policy 0-4, order 0-1, blocks per SM 1-64; for policy 4 the
 * branch streams are 8 x blocks_per_sm).  LBRBC_ERR_ARG when out of range.
 * Rebuilds the step graphs; call it between steps. */
lbrbc_status lbrbc_batch_schedule(lbrbc_batch *batch, int32_t policy, int32_t order, int32_t blocks_per_sm);

/* out[0] number of domains, out[1] total fluid cells (host, 2 entries). */
lbrbc_status lbrbc_batch_info(lbrbc_batch *batch, int64_t *out);

/* Handle of domain i for lbrbc_fields / lbrbc_mass_ledger / lbrbc_classes /
 * lbrbc_check; owned by the batch (lbrbc_destroy ignores it, lbrbc_step on
 * it fails).  NULL if i is out of range. */
lbrbc_sim *lbrbc_batch_domain(lbrbc_batch *batch, int32_t i);

const char *lbrbc_batch_last_error(lbrbc_batch *batch);
void lbrbc_batch_destroy(lbrbc_batch *batch);

/* Synchronise and report deferred device-side errors (non-finite state,
 * list overflow).  Returns LBRBC_OK, LBRBC_ERR_NUMERIC or LBRBC_ERR_STATE. */
lbrbc_status lbrbc_check(lbrbc_sim *sim);

/* Message of the last failure of `sim`, or of the calling thread's last
 * failed lbrbc_create when sim is NULL.  Never NULL. */
const char *lbrbc_last_error(lbrbc_sim *sim);

/* Release all device and host memory of the simulation.  NULL is a no-op. */
void lbrbc_destroy(lbrbc_sim *sim);

#ifdef __cplusplus
}
#endif

#endif /* LBRBC_H */
