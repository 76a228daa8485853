/*
 * lc.h -- C ABI of liblc.so: the link-cell Lennard-Jones force sweep with
 * Newton's third law on one NVIDIA GB300 (sm_103a).
 *
 * The method (Niethammer, Glass, Gracia, "Avoiding Serialization Effects in
 * Data / Dependency aware Task Parallel Algorithms for Spatial
 * Decomposition"):
 *   - Sec. IV: the box is divided into cells whose side is at least the
 *     cutoff r_c, so all partners of a particle lie in its own cell or the 26
 *     neighbouring cells (link-cell method).
 *   - Sec. IV, Fig. 3b: with Newton's third law each pair is computed once;
 *     only the centre cell and 13 of its neighbours (a half-shell) are
 *     visited, and the result is written to both cells.  A cell-cell
 *     interaction (intra- or inter-cell) is the unit of work.
 *   - Sec. IV-V: two cell-cell interactions that share a cell write the same
 *     force accumulators; this write sharing is the race the paper analyses.
 *   - Sec. VI, Strategy 1, Fig. 6: colouring makes the writes of
 *     same-coloured tasks disjoint (LC_SCHED_COLOUR: a cell task keeps its
 *     whole half-shell, so the stride is 3 where the half-shell reaches both
 *     neighbours, x and y, and 2 in z); Strategy 2: tasks run as their
 *     dependences allow (the colour schedule's tasks wait only for their
 *     earlier-coloured neighbours; lc_dag_forces runs the cell-pair task DAG
 *     of a creation order).
 *   - Sec. VIII: commutative updates only need mutual exclusion, not an
 *     order (LC_SCHED_ATOMIC resolves the sharing with atomic adds).
 *   - Sec. VI, Strategy 3: every task writes private buffers, one per
 *     neighbour it serves, and a reduce step sums them afterwards, so no two
 *     tasks write the same memory, at the price of memory (LC_SCHED_BUFFER).
 * Units are reduced Lennard-Jones units, sigma = epsilon = m = 1:
 *   U(r) = 4 (r^-12 - r^-6) for r < r_c (truncated, not shifted),
 *   F_i  = sum_j 24 (2 r^-12 - r^-6) / r^2 (r_i - r_j),
 *   virial W = sum over pairs r_ij . F_ij, kinetic K = 1/2 sum v^2.
 *
 * Conventions for every call:
 *   - Each call returns an lc_status; no call aborts or prints.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *     queued on it; calls that hand results to the host synchronise it.
 *   - Pointers passed in stay owned by the caller; the library reads or
 *     writes them only during the call (host buffers) or, for device
 *     buffers, in stream order before the call's work on `stream` ends.
 *   - Arrays of 3-vectors are [n][3] doubles (x, y, z interleaved), indexed
 *     by particle ID (0 .. n-1) unless stated otherwise.
 *   - A context owns all of its device memory (allocated in lc_create or
 *     lc_batch_create, freed in lc_destroy) and is used from one host thread
 *     at a time.
 */
#ifndef LC_H
#define LC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lc_ctx lc_ctx;

typedef enum {
    LC_OK = 0,
    LC_ERR_INVALID_ARG = 1,   /* NULL pointer, n < 0, rc <= 0, unknown enum   */
    LC_ERR_BOX_TOO_SMALL = 2, /* some L_d / r_c < 3: fewer than 3 cells        */
    LC_ERR_CUDA = 3,          /* a CUDA runtime call failed                    */
    LC_ERR_OOM = 4,           /* device allocation failed                      */
    LC_ERR_NONFINITE = 5,     /* a position or velocity was NaN or infinite    */
    LC_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up            */
    LC_ERR_STATE = 7,         /* call order violated (e.g. no state set)       */
    LC_ERR_RACE = 8,          /* one colour's tasks write a cell twice         */
    LC_ERR_TOO_LARGE = 9      /* size beyond a stated maximum                  */
} lc_status;

/* How the write sharing between cell pairs is resolved (Sec. IV-VI). */
typedef enum {
    LC_SCHED_COLOUR = 0,    /* cell tasks coloured 3-strided in x and y and
                               2-strided in z, run in colour order on a device
                               queue: tasks of one colour write disjoint
                               cells, a task waits (bounded) for its
                               earlier-coloured neighbours; the force
                               additions reach the L2 in the order the waits
                               fix, so forces are bit-reproducible.  A single
                               box's queue tables (about 13 bytes per cell)
                               are built on the first use of the schedule  */
    LC_SCHED_ATOMIC = 1,    /* one pass, both cells updated by atomic adds      */
    LC_SCHED_FULLSHELL = 2, /* all 27 cells, own cell written only, no Newton-3 */
    LC_SCHED_BUFFER = 3,    /* one pass into private per-(cell, offset) buffers,
                               then a fixed-order reduce: no atomics, no phases,
                               forces bit-reproducible from run to run; buffers
                               of 15 x 3 x n floats (FP64: doubles) are
                               allocated on the first use of the schedule    */
    LC_SCHED_LIST = 4       /* not in the paper: Verlet neighbour lists with a
                               skin (lc_set_skin), built from link cells of
                               side >= rc + skin and reused across steps; one
                               thread per particle over its own full list, so
                               no write is shared.  Mixed precision, single
                               box only (2D included)                        */
} lc_schedule;

typedef enum {
    LC_PREC_FP64 = 0,  /* FP64 positions, pair math and accumulation           */
    LC_PREC_MIXED = 1  /* FP32 pair math on cell-local coordinates; FP64 cutoff
                          decision near r_c; Kahan / FP64 cross-cell sums;
                          FP64 positions, velocities, energy and virial        */
} lc_precision;

typedef enum {
    LC_GET_CELL_COUNT = 0, /* int32[ncell]  particles per cell                 */
    LC_GET_CELL_START = 1, /* int32[ncell]  exclusive prefix sum of the counts  */
    LC_GET_PERM = 2,       /* int32[n]      slot -> particle ID (cell-sorted)   */
    LC_GET_COLOUR = 3,     /* int8[ncell]   colour of each cell                 */
    LC_GET_FORCES = 4,     /* double[n][3]  forces of the last evaluation       */
    LC_GET_POS = 5,        /* double[n][3]  positions, wrapped into [0, L)      */
    LC_GET_VEL = 6         /* double[n][3]  velocities                          */
} lc_get_what;

/* Create a context for one periodic orthorhombic box.
 *   box[3]  edge lengths L_x, L_y, L_z (> 0)
 *   rc      cutoff (> 0); cells per dimension nc_d = floor(L_d / rc) (Sec. IV)
 *   n       number of particles (>= 0, < 2^26)
 *   prec    arithmetic of the force sweep
 * Allocates the context's device buffers on the current device (those of
 * particular schedules and options -- LC_SCHED_BUFFER, the colour queue's
 * tables, LC_SCHED_LIST, the staging slots -- on their first use).
 * Errors: LC_ERR_INVALID_ARG, LC_ERR_BOX_TOO_SMALL, LC_ERR_TOO_LARGE,
 * LC_ERR_OOM, LC_ERR_CUDA.  *out is NULL on error. */
lc_status lc_create(const double box[3], double rc, int64_t n, lc_precision prec, lc_ctx **out);

/* Copy the particle state in.  pos, vel: [n][3]; vel may be NULL (zero
 * velocities).  id: reserved, must be NULL (IDs are 0 .. n-1, the row index).
 * on_device != 0: the pointers are device memory, else host memory: page-
 * locked, device-mapped host arrays are read in place by the set-up kernel,
 * other host memory is first copied to the device; either way the call
 * synchronises the stream before returning, so host arrays are the caller's
 * again on return.  Positions may lie outside the box; they are wrapped when
 * binned.  Marks the binning and the forces stale. */
lc_status lc_set_state(lc_ctx *ctx, const double *pos, const double *vel, const int32_t *id,
                       int on_device, void *stream);

/* Host input copied ahead, so that the copy of the next state overlaps the
 * work on the current one.  lc_stage_state queues the copy of pos (and vel,
 * NULL for zero velocities), [n][3] host arrays, into staging slot 0 or 1
 * on copy_stream and returns at once: the host arrays must stay unchanged
 * until the copy is done (copy_stream synchronised, or the slot consumed).
 * A slot is overwritten only after its previous content was consumed.
 * lc_set_state_staged then makes a slot the current state, as
 * lc_set_state would, in stream order on `stream` after the slot's copy.
 * Page-locked host arrays let the copy run concurrently with kernels.
 * The slots (96 bytes per particle) are allocated on first use.  Errors:
 * LC_ERR_INVALID_ARG, LC_ERR_STATE (slot never staged), LC_ERR_OOM,
 * LC_ERR_CUDA. */
lc_status lc_stage_state(lc_ctx *ctx, const double *pos, const double *vel, int32_t slot, void *copy_stream);
lc_status lc_set_state_staged(lc_ctx *ctx, int32_t slot, void *stream);

/* A 2D context (Sec. IV, Fig. 3a: the paper's 2D link-cell case): particles in
 * a periodic box[0] x box[1] rectangle, cells of side >= rc in x and y, the
 * 5-cell half-shell stencil (Newton-3 schedules) or 9 cells (full shell).
 * Positions and velocities keep the [n][3] layout: the z components are
 * ignored on input (every particle lies in one plane, vz = 0) and returned
 * as 0.  Every call below except the batch calls accepts a 2D context; the
 * physics is the 2D Lennard-Jones system (same potential, in-plane
 * distances).  Errors as lc_create; LC_ERR_BOX_TOO_SMALL if box[0] or
 * box[1] holds fewer than 3 cells. */
lc_status lc_create_2d(const double box[2], double rc, int64_t n, lc_precision prec, lc_ctx **out);

/* Counting-sort binning (link-cell construction, Sec. IV): wrap the
 * positions, compute each particle's cell, count, scan and scatter so that
 * every cell's particles are contiguous, ascending by ID inside a cell.  The
 * particle state is stored in that order afterwards.  LC_ERR_NONFINITE if a
 * position is not finite (reported by lc_energy_virial / lc_get, which read
 * the device flag). */
lc_status lc_bin(lc_ctx *ctx, void *stream);

/* One force evaluation with the given schedule (bins first if the positions
 * changed since the last binning).  Also produces the potential energy,
 * the virial and the number of pairs inside r_c.  LC_ERR_OOM if the buffers
 * of LC_SCHED_BUFFER, the tables of LC_SCHED_COLOUR or the lists of
 * LC_SCHED_LIST cannot be allocated (on the schedule's first use: make that
 * first call before any stream capture);
 * LC_ERR_INVALID_ARG for LC_SCHED_LIST on a batch or an FP64 context;
 * LC_ERR_TIMEOUT if a wait of the colour schedule's queue ran out.  LC_SCHED_LIST evaluates
 * from the lists, which it first builds (binning on the list grid) when they
 * are stale -- after lc_set_state, lc_set_skin or any link-cell binning;
 * the first build also sizes them, which synchronises the stream. */
lc_status lc_forces(lc_ctx *ctx, lc_schedule sched, void *stream);

/* nsteps velocity-Verlet steps of size dt (m = 1): v += dt/2 F; x += dt v;
 * bin; F = F(x); v += dt/2 F.  Computes the forces first if they are stale.
 * The step's kernels are captured once into a CUDA graph per (schedule, dt)
 * and replayed: a graph of two steps, and for an odd nsteps a graph of one
 * step at the end.  Potential energy, virial and pair count are accumulated
 * in the last step of the call (lc_energy_virial reports them); the other
 * steps skip that accumulation.  The one-step graph's closing half-kick also
 * forms the kinetic energy of the new velocities, so K after a call with an
 * odd nsteps needs no further pass over them (after an even nsteps,
 * lc_energy_virial forms it: one pass over the velocities).  LC_SCHED_LIST: see the list section below
 * (steps between builds do no binning). */
lc_status lc_verlet_step(lc_ctx *ctx, double dt, int nsteps, lc_schedule sched, void *stream);

/* ---- Verlet neighbour lists (LC_SCHED_LIST) ------------------------------
 * Not part of the paper's method, which sweeps the link cells every step
 * (Sec. IV); an extension that trades memory for fewer candidates per pair.
 * A list build bins the particles on a list grid of cells of side >= rc + skin
 * and records for every particle all partners within rc + skin (both
 * directions).  While no particle has moved by skin / 2 since the build,
 * every pair inside rc is on the lists.  lc_forces(LC_SCHED_LIST) evaluates
 * from the lists (built when stale); lc_verlet_step(LC_SCHED_LIST) reuses them
 * and rebuilds
 * when a particle's displacement since the build exceeds skin / 2, a
 * decision taken on the device inside the step's CUDA graph (a conditional
 * node), so the host never waits.  Positions stay unwrapped between builds
 * (lc_get wraps them).  The link-cell binning is stale after list calls
 * (LC_GET_CELL_COUNT, LC_GET_CELL_START and LC_GET_PERM return LC_ERR_STATE
 * until the next lc_bin).
 *
 * lc_set_skin: skin >= 0 (default 0.4); kmax = entries per particle kept in
 * the list (0: sized from the first build, 1.25 x the longest row + 8).
 * A row longer than kmax is still exact: its partners are swept from the
 * cells.  Waits for the device, then frees the current lists (allocated
 * again on next use: 4 kmax + 36 bytes per particle).  LC_ERR_INVALID_ARG for
 * a negative or non-finite skin or kmax < 0; LC_ERR_BOX_TOO_SMALL if some box
 * edge holds fewer than 3 cells of side rc + skin (checked on first use). */
lc_status lc_set_skin(lc_ctx *ctx, double skin, int32_t kmax);

/* Counters of the lists since the last lc_set_skin: builds, rows longer
 * than kmax over all builds, the longest row seen, steps whose displacement
 * check asked for a rebuild, list entries written over all builds (each
 * pair within rc + skin appears in two rows), and the row capacity kmax.
 * Any output may be NULL.  Synchronises the stream. */
lc_status lc_list_info(lc_ctx *ctx, int64_t *builds, int64_t *long_rows, int64_t *longest_row,
                       int64_t *rebuild_steps, int64_t *entries, int32_t *kmax, void *stream);

/* Energies of the current state, FP64: potential U and virial W of the last
 * force evaluation, kinetic K = 1/2 sum v^2 of the current velocities, and the
 * number of pairs with r < r_c.  Any output pointer may be NULL.  Synchronises
 * the stream; returns LC_ERR_NONFINITE / LC_ERR_TIMEOUT if a device flag
 * was raised. */
lc_status lc_energy_virial(lc_ctx *ctx, double *u_pot, double *k_kin, double *virial,
                           int64_t *npairs, void *stream);

/* The same energies without waiting: queues on `stream` the kinetic-energy
 * reduction (none after lc_verlet_step of an odd nsteps, whose closing
 * kick formed K) and
 * the copy of the 48-byte result block into `out` and returns
 * at once, so the next step can be queued before this one's result is read.
 * out: 48 bytes, 8-byte aligned host memory owned by the caller, valid until
 * the stream has passed the copy; page-locked memory keeps the call
 * asynchronous (pageable memory makes the copy synchronous).  After the
 * stream has passed the copy (an event or a stream synchronisation),
 * lc_result_decode(out, ...) gives U, K, W and the pair count, and the
 * status lc_energy_virial would have returned.  LC_ERR_INVALID_ARG for a
 * batch of boxes (lc_batch_energies), LC_ERR_STATE if no forces were
 * evaluated for the current state. */
lc_status lc_energy_virial_async(lc_ctx *ctx, void *out, void *stream);
lc_status lc_result_decode(const void *out, double *u_pot, double *k_kin, double *virial, int64_t *npairs);

/* Copy one array out (layouts under lc_get_what).  on_device != 0: dst is
 * device memory.  Host copies synchronise the stream. */
lc_status lc_get(lc_ctx *ctx, lc_get_what what, void *dst, int on_device, void *stream);

/* Grid of the context: cells per dimension, number of cell colours (the
 * 2-strided classes of LC_GET_COLOUR), number of colours of LC_SCHED_COLOUR's
 * cell tasks.  Any output may be NULL. */
lc_status lc_grid(const lc_ctx *ctx, int32_t nc[3], int32_t *ncolours, int32_t *nphases);

/* Race and coverage check of a schedule's work decomposition on the device
 * (Sec. IV-VI: the write sharing between cell pairs).  Runs the schedule's
 * own task enumeration without the force arithmetic.  For LC_SCHED_COLOUR
 * (the queue's own tables: the cells at each colour's queue positions) every
 * cell task stamps the cells it may write with its colour and the cells
 * stamped twice within one colour are counted (*conflicts: two tasks of one
 * colour whose writes could meet), as is every queued cell whose entry in
 * the per-cell colour table differs from the colour it is queued under, and
 * every dependence offset that the cell's wait mask includes or omits
 * against that table (the waits must cover exactly the earlier-coloured
 * cells that can share a written cell).  For every schedule each
 * cell pair of the half-shell (the full shell for LC_SCHED_FULLSHELL) must be
 * visited exactly once; *coverage_errors counts the pairs that are not.
 * Its buffers (27 counters per cell) are allocated on the first call
 * (LC_ERR_OOM if they cannot be).  Synchronises the stream. */
lc_status lc_schedule_check(lc_ctx *ctx, lc_schedule sched, int64_t *conflicts,
                            int64_t *coverage_errors, void *stream);

/* ---- Task DAG on the device (Sec. III, Sec. V, Sec. VI Strategy 2) --------
 * The force sweep as the paper's task program: 14 tasks per cell (the
 * intra-cell interaction and the 13 half-shell pairs), each declaring both
 * of its cells inout, so a task depends on the last earlier-created task that
 * touched either cell.  The creation order decides the DAG and with it the
 * critical path (Eq. 1-4, Fig. 5). */
typedef enum {
    LC_ORDER_CELL = 0,   /* outer loop over cells (x fastest), inner loop over
                            the stencil: intra first, then the half-shell
                            offsets in table order (the literature order)   */
    LC_ORDER_LOOPEX = 1  /* loop exchange + 2-strided colouring (Sec. VI,
                            Fig. 6): stencil entries outer (intra first),
                            then colours, then the cells of the colour      */
} lc_order;

/* Builds (once per order; host work O(cells)) the DAG of a single-box
 * context and reports its size: tasks (14 per cell), dependency edges and
 * the critical path counted in tasks.  Any output may be NULL.  Synchronous.
 * LC_ERR_INVALID_ARG for a batch; LC_ERR_TOO_LARGE beyond 2^29 tasks. */
lc_status lc_dag_build(lc_ctx *ctx, lc_order order, int64_t *ntasks, int64_t *nedges,
                       int64_t *critical_path);

/* The same DAG for a grid of nc[0] x nc[1] x nc[2] cells, built on the host
 * only (no context, no GPU): tasks, edges and critical path.  nc[2] == 1
 * means the 2D grid (stencil of 5: the cell and its 4 forward neighbours in
 * the x-y plane, Fig. 3a); otherwise 3D (14).  perm: NULL, or the order of
 * the stencil entries inside a cell for LC_ORDER_CELL, a permutation of
 * 0 .. nperm-1 where entry 0 is the intra-cell task and entry k >= 1 the
 * k-th forward offset in (z, y, x) table order (nperm = 14 in 3D, 5 in 2D).
 * Eq. 1 with equal task times gives the speedup bound tasks / critical_path.
 * LC_ERR_BOX_TOO_SMALL if nc[0] or nc[1] (or, in 3D, nc[2]) < 3,
 * LC_ERR_INVALID_ARG for a bad permutation, LC_ERR_TOO_LARGE beyond 2^29
 * tasks. */
lc_status lc_dag_plan(const int32_t nc[3], lc_order order, const int32_t *perm, int32_t nperm,
                      int64_t *ntasks, int64_t *nedges, int64_t *critical_path);

/* Sets the stencil order inside a cell used by LC_ORDER_CELL on this
 * context (perm as in lc_dag_plan; NULL restores table order); the DAG of
 * that order is rebuilt on its next use.  This is how the orderings of
 * Fig. 5 are run on the device. */
lc_status lc_dag_stencil_order(lc_ctx *ctx, const int32_t *perm, int32_t nperm);

/* One force evaluation by executing the DAG of `order` on the device: a
 * persistent kernel (cooperative launch, every warp resident; a DAG of little
 * parallelism, tasks / critical path of a few, gets eight warps per unit of
 * it and at least four blocks instead of the whole GPU) whose warps
 * claim queue slots, wait for a ready task, run it with plain writes to both
 * cells and release its successors (dependency counting).  Forces, energy,
 * virial and pair count as lc_forces.  wait_seconds (> 0) bounds every wait
 * for a queue slot (default 2 s when <= 0); a wait that runs out makes the
 * call return LC_ERR_TIMEOUT with the forces invalid, the context stays
 * usable.  trace: NULL or device int32[2 * ntasks]; entry 2t / 2t+1 receive
 * the start / end stamp of task t (creation index) on one device-wide
 * counter, so end(p) < start(s) for every edge p -> s.  flags: 0, or
 * LC_DAG_WITHHOLD for a test of the bounded waits (no task is published).
 * Synchronises the stream. */
#define LC_DAG_WITHHOLD 1
lc_status lc_dag_forces(lc_ctx *ctx, lc_order order, double wait_seconds, int flags, int32_t *trace,
                        void *stream);

/* Tile shape of the force kernels: ni = particles of the centre cell held
 * per warp (8 or 16), warps = warps per thread block (1 .. 8), or 16: the
 * atomic schedule of a single 3D box in mixed precision with ni = 16 then
 * runs its row-group kernel (one block of 16 warps per SM; the neighbour
 * cells of up to 21 x-consecutive centre cells copied into shared memory
 * once, by bulk copies, and read from there by the cell tasks; the other
 * schedules and contexts run 8 warps per block).  0 keeps the current value.
 * Used by the autotuner.  Errors: LC_ERR_INVALID_ARG for other values. */
lc_status lc_set_tile(lc_ctx *ctx, int ni, int warps);

/* Number of kernels launched by the last lc_forces / lc_verlet_step call
 * per force evaluation and per step (for accounting; per step: the
 * two-step graph's kernels halved, rounded down). */
lc_status lc_launch_counts(const lc_ctx *ctx, int32_t *per_force, int32_t *per_step);

/* Kernels in the step graphs that lc_verlet_step launched last: the
 * one-step graph (which ends an odd step count) and the two-step graph; 0
 * for one not launched yet.  A call of n steps with the same schedule
 * launches two_steps * (n / 2) + one_step * (n % 2) kernels.  Any output
 * may be NULL. */
lc_status lc_launch_counts_graphs(const lc_ctx *ctx, int32_t *one_step, int32_t *two_steps);

/* ---- batches of independent boxes --------------------------------------
 * A batch context holds nbox independent periodic boxes (each with its own
 * edges, cutoff and particle count) and runs every stage over all boxes in
 * one launch: binning, the force sweep, integration.  With LC_SCHED_COLOUR
 * the force sweep is one persistent launch fed by a device work queue whose
 * items are single cell tasks (box, colour, cell).  The (box, colour) groups
 * are ordered by the colour's position k / colours(box) in its box's chain,
 * so the boxes interleave and every box's chain advances at the same pace;
 * within a box the order is colour-major.  A cell task waits only for the
 * earlier-coloured tasks of its own box that could write a common cell
 * (bounded waits, LC_ERR_TIMEOUT), and the per-box energies are summed in a
 * fixed order.
 * Particles are numbered box after box: box b owns IDs
 * [n_0 + ... + n_{b-1}, ... + n_b).  lc_set_state, lc_forces,
 * lc_verlet_step, lc_get (all but LC_GET_COLOUR) and lc_destroy take a batch
 * context; lc_energy_virial returns sums over the boxes. */

/* box: [nbox][3] edges, rc: [nbox] cutoffs, n: [nbox] particle counts
 * (host arrays).  nbox <= 65535, total particles < 2^26.  Errors as
 * lc_create. */
lc_status lc_batch_create(int32_t nbox, const double *box, const double *rc, const int64_t *n,
                          lc_precision prec, lc_ctx **out);

/* Per-box energies of the current state into host arrays of nbox entries
 * (any may be NULL): potential U and virial W of the last force evaluation,
 * kinetic K, pairs inside r_c.  Synchronises the stream.  The per-box U and W
 * are summed with FP64 atomics for the atomic, full-shell and buffer
 * schedules (order not fixed: the last bits may differ between runs) and in
 * a fixed order for the colour schedule. */
lc_status lc_batch_energies(lc_ctx *ctx, double *u_pot, double *k_kin, double *virial, int64_t *npairs,
                            void *stream);

/* nsteps velocity-Verlet steps of every box of a batch (as lc_verlet_step)
 * with the colour schedule on the device work queue: Sec. VI, Strategy 1
 * (colouring) for the disjoint writes of concurrent tasks, Strategy 2 (tasks
 * run as their dependences allow) for the order, over all boxes at once.
 * Steps are captured in CUDA graphs (two steps, one step) and replayed.
 * LC_ERR_INVALID_ARG for a single-box context; LC_ERR_TIMEOUT if a wait of
 * the queue ran out (see lc_set_queue_wait). */
lc_status lc_batch_step(lc_ctx *ctx, double dt, int32_t nsteps, void *stream);

/* Limit of one wait of the colour schedule's device queue (seconds, default
 * 2) and flags: LC_QUEUE_WITHHOLD makes no task publish its completion, so
 * every wait for an earlier-coloured task runs out and the evaluation ends
 * with LC_ERR_TIMEOUT (a test of the bounded waits; the context stays
 * usable).  Waits for the device and drops the captured step graphs.
 * LC_ERR_INVALID_ARG for seconds outside (0, 1e6] or unknown flags. */
#define LC_QUEUE_WITHHOLD 1
lc_status lc_set_queue_wait(lc_ctx *ctx, double seconds, int32_t flags);

/* Number of boxes (0 for a single-box context), total particles, total cells. */
lc_status lc_batch_info(const lc_ctx *ctx, int32_t *nbox, int64_t *total_particles, int64_t *total_cells);

/* Binning without any device allocation, for callers that cannot allocate
 * device memory (work issued while another component captures a CUDA graph,
 * code confined to a memory pool it was handed, embedded users that only
 * pass pointers).  The paper has no counterpart: it is an interface
 * convenience around the counting sort of lc_bin.
 *   pos         device, [n][3] doubles by particle ID (any values; wrapped)
 *   box, rc     host; cells nc_d = floor(L_d / rc), each >= 3
 *   cell_count  device, int32[ncell], written: particles per cell
 *   cell_start  device, int32[ncell], written: exclusive prefix sum
 *   perm        device, int32[n], written: slot -> particle ID, cell-sorted,
 *               ascending ID inside a cell (the same arrays as lc_get's
 *               CELL_COUNT / CELL_START / PERM after lc_bin)
 * Work is queued on `stream`; the call does not synchronise.  Its scratch is
 * one fixed array of device memory inside the library (about 25 MB, held by
 * every GPU that loads the library until the process exits), so
 * n <= 1,048,576 and ncell <= 1,048,576 (LC_ERR_TOO_LARGE otherwise).  The
 * array's device address is looked up on the first call on each device
 * and again on the first call in every new CUDA context of that device
 * (after cudaDeviceReset, for example), with that device current: make
 * those first calls before any stream capture.  All calls share the array:
 * calls that overlap on the GPU race, so order them on one stream.
 * Non-finite positions are binned into cell 0 (no flag is reported).  If a
 * CUDA error is already pending on entry (from the caller's earlier work)
 * the call returns LC_ERR_CUDA, queues nothing and leaves that error
 * pending; only errors raised by this call's own launches are cleared.
 * Errors: LC_ERR_INVALID_ARG, LC_ERR_BOX_TOO_SMALL, LC_ERR_TOO_LARGE,
 * LC_ERR_CUDA. */
lc_status lc_bin_noalloc(const double *pos, int64_t n, const double box[3], double rc, int32_t *cell_count,
                         int32_t *cell_start, int32_t *perm, void *stream);

/* ---- measurement ---------------------------------------------------------
 * FP32 fused multiply-add throughput of the current device, the denominator
 * of the force sweep's roofline: every thread of 8 blocks of 256 per SM runs
 * eight independent chains of `iters` packed f32x2 FMAs (four flops each),
 * after a short warm-up launch.  flops: the flops of the timed launch;
 * seconds: its duration between two CUDA events on `stream`.  Synchronises
 * the stream; allocates nothing on the device.  The paper has no
 * counterpart (it states no hardware rate).  Errors: LC_ERR_INVALID_ARG
 * (iters <= 0, null outputs), LC_ERR_CUDA. */
lc_status lc_probe_fp32(int32_t iters, double *flops, double *seconds, void *stream);

void lc_destroy(lc_ctx *ctx);

/* Static string naming a status code. */
const char *lc_status_str(lc_status s);

#ifdef __cplusplus
}
#endif

#endif /* LC_H */
