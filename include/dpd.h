/*
 * libdpd -- C ABI of the GB300 (sm_103a) engine for the DPD step loop of
 * arxiv 1804.06205 ("A portable code for dissipative particle dynamics (DPD)
 * simulations with additional specific interactions", CAMUS).
 *
 * The calls follow the paper's statement of the problem:
 *   - eq. 1-2: Newtonian motion, dr/dt = v, m dv/dt = f, all masses 1;
 *   - eq. 3:   f_i = sum_{j != i} (F^C + F^D + F^R + F^S), no exclusions;
 *   - eq. 4:   F^C = a_ij (1 - r) e_ij for r < r_c = 1 (soft repulsion);
 *   - F^D, F^R (named in the paper, forms of Groot and Warren):
 *              F^D = -gamma (1 - r)^2 (e_ij . v~_ij) e_ij,
 *              F^R = sigma (1 - r) theta_ij / sqrt(dt) e_ij,
 *              sigma^2 = 2 gamma kT, theta_ij a unit Gaussian drawn from
 *              Philox4x32-10 with counter (min id, max id, step) so that
 *              theta_ij = theta_ji;
 *   - eqs. 6-8, Fig. 3a: bonded terms F^S (harmonic, modified Morse, and
 *              standard Morse), several records per pair allowed;
 *   - section "Design concept of CAMUS": cells of edge >= r_c rebuilt every
 *              step, no neighbour list;
 *   - Fig. 1:  Groot's modified velocity-Verlet,
 *              r += dt v + dt^2/2 f; v~ = v + lambda dt f; f' = F(r, v~);
 *              v += dt/2 (f + f').
 *
 * Conventions for every call:
 *   - Positions, velocities and forces cross the ABI as host arrays of
 *     n*3 doubles in bead-id order (row i = bead i), caller-allocated.
 *   - All input arrays are caller-owned and copied during the call; the
 *     library owns all device memory and the handle until dpd_destroy.
 *   - Return value 0 (DPD_OK) or a negative DPD_E* code.  Device-side errors
 *     (non-finite state, a device wait that gave up) are sticky on the
 *     handle and reported by the next synchronising call.
 *   - One handle must not be used from two host threads at once.  There is
 *     no global state; handles are independent.
 *   - dpd_step only enqueues work on the handle's stream; the calls marked
 *     "synchronises" wait for it.
 */
#ifndef LIBDPD_DPD_H
#define LIBDPD_DPD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define DPD_OK          0
#define DPD_EINVAL     -1   /* bad argument: L < 3, n <= 0, bad bond, ...     */
#define DPD_ENOMEM     -2   /* device or host allocation failed              */
#define DPD_ECUDA      -3   /* a CUDA runtime call failed                    */
#define DPD_EUNSTABLE  -4   /* a position, velocity or force became NaN/Inf  */
#define DPD_ETIMEOUT   -5   /* a bounded device wait gave up                 */
#define DPD_ENOSTATE   -6   /* dpd_step / dpd_get_state before dpd_set_state */

/* ---- options ----------------------------------------------------------- */
#define DPD_FP32        0   /* FP32 forces, cell-relative FP32 positions     */
#define DPD_FP64        1   /* FP64 everywhere (absolute FP64 positions)     */
#define DPD_NOISE_GAUSS   0 /* theta by Box-Muller (default)                 */
#define DPD_NOISE_UNIFORM 1 /* theta = sqrt(3) (2u - 1)                      */

#define DPD_BOND_HARMONIC    1  /* eq. 6: U = k/2 (r - r0)^2                  */
#define DPD_BOND_MORSE_PAPER 2  /* eq. 7 with Fig. 3a's alpha: |F| =
                                   2 k alpha e (1 - e), e = exp(-alpha|r-r0|),
                                   towards the partner on both sides of r0,
                                   U = k (1 - e)^2                            */
#define DPD_BOND_MORSE       3  /* U = k [(1 - exp(-alpha (r - r0)))^2 - 1]   */

typedef struct dpd_handle dpd_handle;          /* opaque, library-owned */

typedef struct {
    double L[3];          /* periodic box edges; each L >= 3 (cells of edge
                             L/floor(L) >= r_c = 1, at least 3 per side)    */
} dpd_box;

typedef struct {
    int32_t i, j;         /* bead ids, 0 <= i, j < n, i != j                */
    int32_t kind;         /* DPD_BOND_*                                      */
    int32_t pad;          /* ignored                                         */
    double r0;            /* equilibrium distance r_e                        */
    double k;             /* C (harmonic) or K_M / D (Morse kinds)           */
    double alpha;         /* Morse width; ignored for harmonic               */
} dpd_bond;

typedef struct {
    double lambda;        /* velocity-predictor factor of Fig. 1 (0.65)      */
    uint64_t seed;        /* Philox key of the pair noise                    */
    int32_t precision;    /* DPD_FP32 (default) or DPD_FP64                  */
    int32_t noise;        /* DPD_NOISE_GAUSS (default) or DPD_NOISE_UNIFORM  */
    int32_t sample_every; /* accumulate running means every k steps (0=off)  */
    int32_t tile_cells;   /* pair-kernel home cells per block (0 = auto)     */
    int32_t threads;      /* pair-kernel threads per block (0 = auto)        */
    int32_t use_graph;    /* replay steps from captured CUDA graphs (0)      */
    int32_t persistent;   /* 1: each dpd_step / dpd_batch_step call is ONE
                             cooperative launch in which resident blocks run
                             every phase of every step, with bounded grid-wide
                             barriers between phases (0: one launch per kernel
                             per step).  Same bits either way.  Ignored when
                             running means are sampled or graphs are used.   */
    int32_t pad;          /* ignored                                         */
    void *cuda_stream;    /* cudaStream_t to run on; NULL = own stream       */
} dpd_options;

/* Observables of the current state (dpd_observables).
 * kT = sum v^2 / (3n - 3); pressures are (virial)/(3V):
 * p_ideal = sum v^2/(3V), p_cons = sum_{i<j} r_ij.F^C_ij/(3V),
 * p_bond = sum_bonds r_ij.F^S_ij/(3V), p_total = their sum. */
typedef struct {
    int64_t step;         /* evaluation counter of the current force         */
    double momentum[3];   /* sum_i v_i (FP64 accumulation)                   */
    double kT;
    double p_total, p_ideal, p_cons, p_bond;
    double e_pair;        /* sum_{i<j} a_ij (1 - r)^2 / 2                    */
    double e_bond;        /* bond energies                                   */
    double sum_v2;
    double kT_mean, p_mean;   /* running means over sampled steps           */
    int64_t n_samples;
    int32_t status;       /* sticky device status, 0 or a DPD_E* code        */
    int32_t pad;
} dpd_obs;

/* Fill *opt with the defaults (lambda 0.65, seed 0, FP32, Gaussian noise,
 * sample_every 0, automatic tiles, direct launches, not persistent, own
 * stream).  Direct
 * launches use programmatic dependent launch, so each kernel of a step is
 * scheduled while the previous one drains; replaying captured CUDA graphs
 * (use_graph = 1) gives the same bits. */
void dpd_default_options(dpd_options *opt);

/* Create a system (eq. 3-8 parameters).  types[n] in [0, ntypes);
 * a_ij[ntypes*ntypes] symmetric, row-major; gamma >= 0, kT >= 0, dt > 0.
 * bonds[nbonds] and morse[nmorse] are both lists of bonded records (any
 * kind; the split only mirrors 1-2 vs 1-3/1-5 decks, as in Fig. 3b) and may
 * be NULL when their count is 0.  opt may be NULL (defaults).
 * On success *out is a new handle; the state must be set before stepping.
 * Errors: DPD_EINVAL, DPD_ENOMEM, DPD_ECUDA. */
int dpd_create(const dpd_box *box, int64_t n, const int32_t *types, int32_t ntypes,
               const double *a_ij, double gamma, double kT, double dt,
               const dpd_bond *bonds, int64_t nbonds, const dpd_bond *morse, int64_t nmorse,
               const dpd_options *opt, dpd_handle **out);

/* Set positions pos[n*3] and velocities vel[n*3] (bead-id order; positions
 * are wrapped into the box) and the evaluation counter `step`, then
 * evaluate the force f(step) at v~ = v (Fig. 1's starting force).
 * Synchronises.  Errors: DPD_EINVAL (NULL arrays, or a non-finite value,
 * detected on the device; the previous state is then lost), DPD_ECUDA. */
int dpd_set_state(dpd_handle *h, const double *pos, const double *vel, int64_t step);

/* Enqueue nsteps steps of Fig. 1 (nsteps >= 0).  Asynchronous with respect
 * to the host.  Errors: DPD_ENOSTATE, DPD_EINVAL, DPD_ECUDA, or a sticky
 * device error from earlier work. */
int dpd_step(dpd_handle *h, int64_t nsteps);

/* Copy the state to host arrays in bead-id order: pos[n*3] (wrapped into
 * [0, L)), vel[n*3], force[n*3] (total force of the last evaluation) -- any
 * of them may be NULL -- and the evaluation counter to *step (nullable).
 * Synchronises.  Errors: DPD_ENOSTATE, DPD_ECUDA, DPD_EUNSTABLE. */
int dpd_get_state(dpd_handle *h, double *pos, double *vel, double *force, int64_t *step);

/* Observables of the current state (dpd_obs above).  Synchronises. */
int dpd_observables(dpd_handle *h, dpd_obs *out);

/* Unique-pair distance histogram of the current state: counts[nbins] of
 * minimum-image distances in bins of width rmax/nbins, r < rmax.
 * rmax must satisfy 2*ceil(rmax/h)+1 <= n_c in every dimension.
 * Synchronises.  Errors: DPD_EINVAL, DPD_ENOSTATE, DPD_ECUDA. */
int dpd_gr(dpd_handle *h, double rmax, int32_t nbins, uint64_t *counts);

/* The cell division of the current state: key_by_id[n] = cell key
 * (cz*ny + cy)*nx + cx of bead id; order[n] = bead id at each sorted slot
 * (cells ascending, ids ascending inside a cell); cell_start[ncells+1].
 * Any pointer may be NULL.  Synchronises. */
int dpd_get_cells(dpd_handle *h, uint32_t *key_by_id, int64_t *order, int64_t *cell_start);

/* Cells per dimension n_c = floor(L) (cell edge h = L / n_c). */
int dpd_cell_dims(const dpd_handle *h, int64_t nc[3]);

/* Wait for all enqueued work; report sticky device errors. */
int dpd_sync(dpd_handle *h);

/* Number of kernel launches the handle has enqueued so far. */
int64_t dpd_launch_count(const dpd_handle *h);

/* Phase timing with CUDA events on the handle's stream, for benchmarks.
 * dpd_profile_begin(h, max_steps) arms events for the next max_steps steps
 * (max_steps in [1, 100000]); steps beyond that are not timed.
 * dpd_profile_end synchronises and returns, summed over the timed steps,
 * ms[0] = position update + cell division (k_update .. k_gather),
 * ms[1] = pair forces (k_pair), ms[2] = bonds + velocity update + sampled
 * reductions, and *nsteps = the number of steps timed.  Errors: DPD_EINVAL,
 * DPD_ECUDA. */
int dpd_profile_begin(dpd_handle *h, int64_t max_steps);
int dpd_profile_end(dpd_handle *h, double ms[3], int64_t *nsteps);

/* Checkpoint and resume (Fig. 1 carries r, v and the force f(t) from one
 * step to the next, so a faithful restart needs all three).  A checkpoint is
 * an opaque byte string: an 80-byte header (magic "DPDCKPT1", version,
 * precision, n, the evaluation counter, cells per edge, record size, box and
 * seed) followed by one record per bead in bead-id order holding the state in
 * the engine's own representation -- FP32: cell key, cell-relative binary32
 * offset, v and f (40 B); FP64: position, v and f (72 B) -- so that a system
 * restored from it continues bit for bit as if it had never stopped.
 * dpd_checkpoint_bytes: the size of the handle's checkpoint (host only).
 * dpd_get_checkpoint: writes it to buf[bytes] (caller-allocated host memory,
 *   bytes >= the size).  Synchronises.  Errors: DPD_EINVAL (NULL or short
 *   buffer), DPD_ENOSTATE, DPD_ECUDA.
 * dpd_set_checkpoint: replaces the state by the checkpoint's, with no force
 *   evaluation; the handle must have been created with the same parameters
 *   (precision, n, box and seed are checked against the header; types, a_ij,
 *   bonds and the integrator parameters are the caller's responsibility).
 *   Synchronises.  Errors: DPD_EINVAL (mismatched header; or, found on the
 *   device, a cell key out of range or a non-finite value, after which the
 *   previous state is lost), DPD_ECUDA. */
int dpd_checkpoint_bytes(const dpd_handle *h, int64_t *bytes);
int dpd_get_checkpoint(dpd_handle *h, void *buf, int64_t bytes);
int dpd_set_checkpoint(dpd_handle *h, const void *buf, int64_t bytes);

/* Cell division without any allocation.  The paper has no counterpart: it
 * exists for callers that cannot call cudaMalloc -- code whose device memory
 * belongs to a framework allocator or a fixed, pre-budgeted arena, and code
 * that must avoid cudaMalloc's implicit device synchronisation.
 * Computes, for n positions already in device memory, exactly what
 * dpd_set_state + dpd_get_cells give: the periodic wrap into [0, L), the cell
 * key (cz*ny + cy)*nx + cx with n_c = floor(L), and the canonical (cell, id)
 * order.  All buffers are the caller's device memory:
 *   pos_dev[n*3]            input, FP64, bead-id order;
 *   key_dev[n]              output, cell key of each bead id;
 *   order_dev[n]            output, bead id at each sorted slot;
 *   cell_start_dev[ncell+1] output, first slot of each cell (also used as the
 *                           count array, so it is cleared by the call).
 * The work is enqueued on cuda_stream (NULL = the legacy default stream) and
 * the call returns without waiting.  Scratch lives in one fixed array inside
 * the library (16 MiB + 8 KiB per GPU that loads it, held until exit), shared by
 * all calls and keeping the last call's contents: calls that overlap on the
 * GPU race.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make it before any stream capture.
 * Cost: the canonical order inside a cell is found by every bead counting the
 * cell's smaller ids, in parallel, so a cell holding k beads costs k loads per
 * bead.  Physical states hold a few beads per cell; a degenerate input that
 * puts all DPD_NOALLOC_MAX_N beads in one cell (for instance non-finite
 * positions, which the key maps to cell 0) makes the call take seconds.
 * Errors: DPD_EINVAL for NULL pointers, a box edge < 3, n outside
 * [1, DPD_NOALLOC_MAX_N] or more than DPD_NOALLOC_MAX_CELLS cells;
 * DPD_ECUDA if the address lookup or a launch fails. */
#define DPD_NOALLOC_MAX_N     4194304
#define DPD_NOALLOC_MAX_CELLS 4194304
int dpd_cells_noalloc(const double *pos_dev, int64_t n, const dpd_box *box, uint32_t *key_dev,
                      int32_t *order_dev, uint32_t *cell_start_dev, void *cuda_stream);

/* Free the handle and its device memory (NULL is allowed). */
int dpd_destroy(dpd_handle *h);

/* Check of the failure detection on device waits, without a fault.  One block
 * waits on an mbarrier for 16 bytes with the bounded poll loop of the pair
 * kernel's staging wait (each poll is an mbarrier.try_wait).  deliver != 0:
 * a bulk copy delivers the bytes, the wait completes, the call returns DPD_OK.
 * deliver == 0: nothing delivers them, the wait gives up after `tries` polls,
 * the block records the timeout and returns, and the call returns
 * DPD_ETIMEOUT; no copy is in flight, so the CUDA context stays usable.
 * tries in [1, DPD_WAIT_CHECK_MAX_TRIES] (else DPD_EINVAL); cuda_stream: NULL =
 * the legacy default stream.  Allocates nothing; synchronises the stream;
 * DPD_ECUDA if a CUDA call fails. */
#define DPD_WAIT_CHECK_MAX_TRIES (1 << 22)
int dpd_wait_check(int32_t deliver, int32_t tries, void *cuda_stream);

/* Check of the failure detection on the grid-wide barrier of the persistent
 * step kernel (dpd_options.persistent), without a fault.  A cooperative grid of
 * 4 blocks meets at one barrier; complete != 0: the barrier expects the 4 blocks
 * and completes, the call returns DPD_OK; complete == 0: it expects a fifth
 * block that does not exist, so every block waits out `budget_cycles` clock
 * cycles (its clock64() budget), records the timeout and leaves, and the call
 * returns DPD_ETIMEOUT; the CUDA context stays usable.  budget_cycles in
 * [1, DPD_GRID_WAIT_CHECK_MAX_CYCLES] (else DPD_EINVAL); cuda_stream: NULL = the
 * legacy default stream.  Allocates nothing; synchronises the stream;
 * DPD_ECUDA if a CUDA call fails. */
#define DPD_GRID_WAIT_CHECK_MAX_CYCLES 4000000000LL
int dpd_grid_wait_check(int32_t complete, int64_t budget_cycles, void *cuda_stream);

/* Check of the FP64 path's Box-Muller functions of the uniforms u = n 2^-24
 * (n odd): the table-driven ln u (after P. T. P. Tang, ACM TOMS 16, 1990) and
 * cos(2 pi u) with exact quadrant reduction, against the CUDA library's log and
 * cospi over all 2^23 inputs.  *ln_err and *cos_err receive the largest
 * absolute differences.  Allocates and frees its own device memory on the
 * current device; synchronises.  DPD_EINVAL if a pointer is NULL, DPD_ECUDA if
 * a CUDA call fails. */
int dpd_bm_check(double *ln_err, double *cos_err);

/* ---- batches: many independent systems advanced by the same launches ----
 * A batch owns fixed pools sized at creation.  Systems are added (with their
 * state) and removed at any time between steps; dpd_batch_step advances
 * every resident system by the same number of steps, each with its own box,
 * parameters, seed and step counter, in one launch per kernel of Fig. 1's
 * loop for all of them.  A system draws the same noise
 * and follows the same arithmetic alone or in a batch: per-bead sums are in
 * a fixed order and ids, cell keys and Philox counters are its own.
 * Memory admission: dpd_batch_add fails with DPD_ENOMEM when the system's
 * beads, cells (floor(L) per dimension, multiplied), pair-kernel bricks or
 * bond records (two per bond) do not fit next to the resident systems; the
 * caller keeps it queued and retries after a removal. */
typedef struct dpd_batch dpd_batch;

typedef struct {
    int64_t max_beads;     /* bead pool                                      */
    int64_t max_cells;     /* cell pool (also bounds the pair-kernel bricks) */
    int64_t max_bonds;     /* bond pool, in bonds (each uses two records)    */
    int32_t max_systems;   /* resident systems at once                       */
    int32_t pad;
} dpd_batch_capacity;

/* Create an empty batch.  opt: precision, threads, use_graph, cuda_stream
 * (and noise as the default for added systems); NULL = defaults. */
int dpd_batch_create(const dpd_batch_capacity *cap, const dpd_options *opt, dpd_batch **out);

/* Add a system with its parameters (as dpd_create) and its state (as
 * dpd_set_state); *sys receives its index.  lambda, seed and tile_cells (the
 * pair-kernel brick length, 0 = the batch's option or automatic) are per
 * system.  Synchronises.  Errors: DPD_EINVAL, DPD_ENOMEM (does not fit: not
 * admitted), DPD_ECUDA. */
int dpd_batch_add(dpd_batch *b, const dpd_box *box, int64_t n, const int32_t *types,
                  int32_t ntypes, const double *a_ij, double gamma, double kT, double dt,
                  const dpd_bond *bonds, int64_t nbonds, const dpd_bond *morse, int64_t nmorse,
                  double lambda, uint64_t seed, int32_t tile_cells, const double *pos,
                  const double *vel, int64_t step, int32_t *sys);

/* Remove system sys and re-pack the others.  Synchronises. */
int dpd_batch_remove(dpd_batch *b, int32_t sys);

/* Advance every resident system by nsteps (asynchronous). */
int dpd_batch_step(dpd_batch *b, int64_t nsteps);

/* State and observables of one system (as dpd_get_state / dpd_observables). */
int dpd_batch_get_state(dpd_batch *b, int32_t sys, double *pos, double *vel, double *force,
                        int64_t *step);
int dpd_batch_observables(dpd_batch *b, int32_t sys, dpd_obs *out);

/* Pool use: used[4] and cap[4] = beads, cells, bricks, bond records;
 * *nsys = resident systems.  Any pointer may be NULL. */
int dpd_batch_usage(const dpd_batch *b, int64_t used[4], int64_t cap[4], int32_t *nsys);

/* Checkpoints of one resident system, as dpd_checkpoint_bytes /
 * dpd_get_checkpoint / dpd_set_checkpoint.  A checkpoint taken alone restores
 * into a batch and the other way round (same parameters). */
int dpd_batch_checkpoint_bytes(const dpd_batch *b, int32_t sys, int64_t *bytes);
int dpd_batch_get_checkpoint(dpd_batch *b, int32_t sys, void *buf, int64_t bytes);
int dpd_batch_set_checkpoint(dpd_batch *b, int32_t sys, const void *buf, int64_t bytes);

int dpd_batch_sync(dpd_batch *b);
int64_t dpd_batch_launch_count(const dpd_batch *b);

/* Phase timing of the next batch steps, as dpd_profile_begin / _end. */
int dpd_batch_profile_begin(dpd_batch *b, int64_t max_steps);
int dpd_batch_profile_end(dpd_batch *b, double ms[3], int64_t *nsteps);
const char *dpd_batch_last_error(const dpd_batch *b);
int dpd_batch_destroy(dpd_batch *b);

/* Static string for a DPD_E* code. */
const char *dpd_strerror(int code);

/* Detail of the handle's last error (static or handle-owned string);
 * with h == NULL, the detail of this thread's last failed dpd_create. */
const char *dpd_last_error(const dpd_handle *h);

#ifdef __cplusplus
}
#endif
#endif
