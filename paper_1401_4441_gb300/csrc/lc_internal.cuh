// Internal declarations shared by the translation units of liblc.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lc.h"

namespace lc {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
// Slots are packed with a 5-bit neighbour index into one int32 (see lc_force.cu).
constexpr int64_t kMaxParticles = int64_t(1) << 26;
// Relative half-width of the band around r_c^2 inside which the FP32 r^2 of
// the mixed path is not trusted to decide the cutoff (its error bound is
// below 1e-6 relative for cell-local coordinates; see lc_force.cu).
constexpr float kCutBand = 4.0e-6f;

constexpr int kNumSched = 4;     // colour, atomic, full shell, buffer
constexpr int kNumGraphs = 4 * kNumSched;   // captured steps: (two, one) x schedule x buffer parity
constexpr int kNumFbuf = 15;     // buffer schedule: intra j side, 13 offsets, i side

// Rounding residuals of the FP32 cell-local offsets are stored as
// q = rint(r * kLoScale), |q| <= 511, i.e. in units of 2^-23 / 511.
constexpr float kLoScale = (float)(511.0 * 8388608.0);
constexpr float kLoUnit = (float)(1.0 / (511.0 * 8388608.0));

__device__ __forceinline__ float lo_residual(unsigned w, int d) {
    return (float)((int)((w >> (10 * d)) & 1023u) - 512) * kLoUnit;
}

// Error flags raised on the device (bit mask in Ctx::d_err).
enum : int { kErrNonfinite = 1, kErrTimeout = 2 };

// Geometry of one periodic box with its cell grid.
struct Grid {
    double L[3];      // box edges
    double h[3];      // cell sides L / nc
    double inv[3];    // nc / L (one FP64 division each)
    int nc[3];        // cells per dimension (>= 3)
    int ncell;
    double rc, rc2;   // cutoff and its square (FP64, rc * rc)
    float hf[3];      // FP32 cell sides
    float hl[3];      // h - hf rounded to FP32 (double-float cell side)
    float invf[3];    // nc / L in FP32
    float Lf_lo[3];   // FP32 value below L: hi < Lf_lo implies x < L
    float cmargin[3]; // distance from a cell face below which binning is exact FP64
    float rc2f_lo, rc2f_hi;  // FP32 band around rc^2 for the mixed path
    int dims;         // 3, or 2: one cell layer in z, positions in the x-y plane
    int ncolours;
    int class_count[3][3];   // cells of colour class a along dimension d
    int colour_of_raw[27];   // raw colour cx + 3 cy + 9 cz -> colour rank (-1 absent)
    int raw_of_colour[27];   // inverse
    // colour schedule (LC_SCHED_COLOUR): a cell's class along dimension d is
    // c mod cs_p[d] for the cells of the full periods and a class of its own
    // for each cell past the last full period; cs_p = 3 where the half-shell
    // reaches both neighbours (x, y; x in 2D), 2 where it reaches one (z; y
    // in 2D), so two cells of one class triple never write the same cell.
    // Colour = rank of the triple's code a0 + 5 a1 + 25 a2 among those present.
    int cs_p[3];
    int cs_ncls[3];               // classes per dimension (at most cs_p + 2)
    int cs_ncolours;
    int cs_colour_of_raw[125];    // -1: absent
    int cs_raw_of_colour[125];
    int cs_first[126];            // queue position of the first cell of each colour
    // ceil(2^64 / nc_x) and ceil(2^64 / (nc_x nc_y)): the high word of
    // c * div is the exact quotient for every 32-bit cell index c
    unsigned long long divx, divxy;
};

// Cell coordinates of a cell index, the quotients by multiply-high with the
// grid's precomputed ceil(2^64 / d) (exact for every 32-bit index).
__device__ __forceinline__ void cell_coords(const Grid &g, int c, int out[3]) {
    const int q1 = (int)__umul64hi((unsigned long long)(unsigned)c, g.divx);    // c / nc_x
    const int q2 = (int)__umul64hi((unsigned long long)(unsigned)c, g.divxy);   // c / (nc_x nc_y)
    out[0] = c - q1 * g.nc[0];
    out[1] = q1 - q2 * g.nc[1];
    out[2] = q2;
}

// Offsets of the 27-cell stencil and the phase groups, in constant memory.
// 3D: 13 forward offsets of 26; 2D (offsets in the x-y plane): 4 of 8.
struct Stencil {
    int nh, nf;         // half-shell offsets (13 / 4), full-shell cells (27 / 9)
    int hs[13][3];      // forward half-shell, (z, y, x) lexicographic
    int group_of[13];   // phase group (0..3) of each half-shell offset
    int group_first[5]; // offsets of group g are group_list[group_first[g] .. group_first[g+1])
    int group_list[13];
    int full[27][3];    // all offsets, centre first
    // offsets between two cells whose half-shell tasks (centre + forward
    // offsets) can write a common cell: differences of two stencil entries
    int ndep;           // 62 (3D) / 12 (2D)
    int dep[62][3];
};

void make_stencil(Stencil *s, int dims = 3);
void make_grid(Grid *g, const double box[3], double rc, int dims = 3);

// One box of a batch: its grid, the FP32 shift tables of its 27 offsets,
// and where its cells and particles sit in the batch's global numbering
// (boxes are concatenated: box b owns cells [cell_off, cell_off + ncell)
// and slots [part_off, part_off + n)).
struct BoxDev {
    Grid g;
    float sh[27][3];   // o * h rounded to FP32, offset index (ox+1) + 3 (oy+1) + 9 (oz+1)
    float sl[27][3];   // o * h - sh, rounded to FP32
    int cell_off, part_off, n, pad;
};
void make_box(BoxDev *b, const double box[3], double rc, int cell_off, int part_off, int n);

// Double-buffered particle state in cell-sorted order.
struct State {
    double *x, *y, *z;     // wrapped positions
    double *vx, *vy, *vz;  // velocities
    int *id;               // particle ID of each slot
};

// Task DAG of one task-creation order (Sec. III, Sec. V, Sec. VI Strategy 2):
// tasks are cell-cell interactions (cell A, k) with k = 0 intra-cell and
// k = 1..13 half-shell offset k - 1; a task depends on the last earlier task
// that touched either of its cells (both are inout).
struct DagDev {
    int ntasks, nroots;
    int64_t nedges, critical_path;
    int *task;          // [T] creation order: A << 4 | k
    int *succ_start;    // [T + 1] CSR of the successors
    int *succ;          // [E]
    int *pred_count;    // [T] predecessors of each task
    int *cnt;           // [T] unfinished predecessors (reset per evaluation)
    int *queue;         // [T] ready tasks in publication order, -1 = not yet
    int *queue_init;    // [T] the roots in creation order, then -1
    int *ctrl;          // [4] next slot to claim, next slot to publish, trace clock, spare
    int *ctrl_init;     // [4] 0, nroots, 0, 0
};

struct Ctx {
    Grid g;
    int64_t n;
    lc_precision prec;
    int ni, warps;         // tile shape of the force kernels
    int num_sms;
    State cur, nxt;
    // binning
    int *d_cell;           // cell of each particle (previous order)
    int *d_rank;           // arrival rank inside its cell (atomic, unstable)
    int *d_count;          // [ncell]
    int *d_start;          // [ncell + 1]
    int *d_src;            // slot -> index in the previous order
    int *d_cellt;          // slot -> its cell (written with d_src)
    int *d_key;            // slot -> particle ID (before the final ranking)
    int *d_blocksums;      // scan partials
    int8_t *d_colour;      // [ncell]
    int *d_cs_cell;        // colour queue of a single box: position -> cell
    int8_t *d_cs_rank;     // colour of every cell (per box)
    unsigned long long *d_cs_dep;   // per cell: dependence offsets with an earlier colour (bit e)
    float4 *d_p4;          // FP32 cell-centre offsets (sorted) + packed residuals
    // forces
    double *fx, *fy, *fz;  // FP64 forces in sorted order
    float2 *kx, *ky, *kz;  // Kahan (sum, compensation) accumulators, colour + mixed
    double *d_warp_acc;    // per-warp partials: [nwarp_max][4] (s6, s12, K, spare)
    long long *d_warp_pairs;
    double *d_kin_part;    // per-block partial sums of v^2 (kinetic_blocks of them)
    bool kin_valid;        // d_kin_part holds the partials of the current velocities
    bool kin_final;        // d_result[3] holds their K (implies kin_valid)
    unsigned *d_kin_ticket;   // k_kick's count of finished blocks (block + 48; zero between launches)
    // one 64-byte device block, read back in one copy: U, W, pairs (as
    // double), K, then the pair count and the error flags
    double *d_result;      // [4] U, W, npairs (as double), K  (block + 0)
    long long *d_npairs;   // block + 32
    int *d_err;            // block + 40
    void *h_out;           // page-locked host copy of the block
    int nwarp_max;
    int nwarp_used;        // warps of the last force evaluation (their partials are reduced)
    // colour schedule: per-cell completion flags, the queue counter and the
    // per-cell energy partials (s6, s12, spare, spare) and pair counts
    int *d_cs_done;        // [ncell]
    int *d_cs_ctrl;        // [2]: next queue item, spare
    double *d_cell_acc;    // [ncell][4]
    long long *d_cell_pairs;   // [ncell]
    double cs_wait_s;      // limit of one wait of the colour queue (seconds)
    int cs_withhold;       // test: no task publishes its completion
    // batch: colour-queue items (box, colour, first cell of the colour, cells),
    // ordered by colour, then box
    int4 *d_cs_items;
    int cs_nitems;
    // check buffers
    int *d_stamp;
    unsigned long long *d_visit;
    unsigned long long *d_counters;
    // status
    bool have_state, binned, forces_valid;
    int launches_force, launches_step;
    int launches_one, launches_two;   // kernels of the one-step and two-step graphs last launched
    // batch of independent boxes (nbox > 0); single box: nbox == 0
    int nbox;
    BoxDev *h_boxes;          // host copy
    BoxDev *d_boxes;
    unsigned short *d_cell_box;   // box of each global cell
    unsigned short *d_slot_box;   // box of each slot
    double *d_box_acc;        // [nbox][2] sums of r^-6 and r^-12 (pairs once)
    unsigned long long *d_box_pairs;
    double *d_box_out;        // [nbox][4] U, W, pairs, K
    int stats_full;           // last statistics came from the full shell
    // two staging slots for host input copied ahead (lc_stage_state): raw
    // [n][3] positions and velocities, allocated on first use, with events
    // for "copy done" and "consumed"
    double *d_stage[2];
    cudaEvent_t ev_staged[2], ev_consumed[2];
    bool stage_has_vel[2];
    DagDev *dag[2];        // per task-creation order, built on first use
    int dag_perm[14];      // stencil order inside a cell for the cell order
    int dag_perm_n;        // 0: table order
    // buffer schedule: per-(cell, offset) private force buffers [15][3][n]
    // (float for the mixed path, double for FP64), allocated on first use
    void *d_fbuf;
    // graphs of Verlet steps: two steps at 2 * schedule + state-buffer
    // parity, one step at 2 * kNumSched + the same
    cudaGraphExec_t graph[kNumGraphs];
    double graph_dt[kNumGraphs];
    int graph_launches[kNumGraphs];   // kernels in each
    double *state_a;       // cur.x of buffer set A (parity reference)
    // Verlet neighbour lists (LC_SCHED_LIST): a coarser list grid with
    // cells of side >= rc + skin, fixed-point offsets from the build cells'
    // centres and one list row per particle, allocated on first use
    double skin;
    int list_kmax_req;     // row capacity requested (0: sized from the first build)
    int list_kmax;         // row capacity of d_nbr
    int list_shift;        // offsets are stored in units of 2^-list_shift
    Grid gl;               // list grid; its cutoff fields are those of g
    unsigned *d_nbr;       // [kmax][n]: slot << 6 | (o_x + 1) | (o_y + 1) << 2 | (o_z + 1) << 4
    int *d_nn;             // [n] row lengths (a row longer than kmax is swept from the cells)
    int4 *d_q4;            // [2n]: offsets now, then at the build; w = build cell
    unsigned long long *d_list_stats;   // builds, long rows, longest row, rebuild steps, entries; + 2 control words
    bool list_valid;       // the lists match the current slot order and state
    cudaGraphExec_t list_graph[4];      // (one / two steps) x (state-buffer parity)
    double list_graph_dt[4];
    int list_graph_launches[4];         // kernels in each
};

// ---- kernels / launchers (stream-ordered, return cudaError_t) -------------
// Binning; kicks = 1 / 2 fuses the start of a Verlet step (kick + drift of
// step dt) / also the previous step's closing kick into the cell pass.
cudaError_t launch_bin(Ctx *c, cudaStream_t s, int *launches, int kicks = 0, double dt = 0.0);
cudaError_t launch_forces(Ctx *c, lc_schedule sched, cudaStream_t s, int *launches, bool stats = true,
                          bool *pot_deferred = nullptr);
cudaError_t launch_kick(Ctx *c, double dt, cudaStream_t s, bool kin = false, bool pot = false);
cudaError_t launch_kinetic(Ctx *c, cudaStream_t s);
cudaError_t launch_energy_reduce(Ctx *c, cudaStream_t s, int full);
// the same reduction over n partials given as [n][4] doubles and [n] pair counts
cudaError_t launch_energy_reduce_parts(Ctx *c, cudaStream_t s, int full, const double *acc, const long long *pairs,
                                       int n);
cudaError_t launch_box_energy(Ctx *c, cudaStream_t s, int full);
// per-box U, W and pairs from per-cell partials (colour schedule), fixed order
cudaError_t launch_box_energy_cells(Ctx *c, cudaStream_t s);
// Forces by executing a task DAG on the device (dependency counting, bounded
// waits); trace: optional [2T] start / end stamps.
// withhold != 0 publishes no ready task (a test of the bounded waits).
cudaError_t launch_forces_dag(Ctx *c, const DagDev *d, long long wait_ns, int withhold, int32_t *trace,
                              cudaStream_t s, int *launches);
cudaError_t build_dag(const Ctx *c, const Stencil &st, int order, DagDev **out);
void free_dag(DagDev *d);
// Host-only DAG of a grid of nc cells (no device work): returns the critical path.
int64_t dag_plan_host(const int nc[3], int order, const int *perm, int nperm, int64_t *ntasks, int64_t *nedges);
cudaError_t launch_box_kinetic(Ctx *c, cudaStream_t s);
cudaError_t launch_colour(Ctx *c, cudaStream_t s);
cudaError_t upload_stencil(const Stencil &st3, const Stencil &st2);
int kinetic_blocks(const Ctx *c);
cudaError_t launch_schedule_check(Ctx *c, lc_schedule sched, cudaStream_t s);
cudaError_t launch_unsort_vec(Ctx *c, const double *a, const double *b, const double *cc,
                              double *dst, cudaStream_t s, int wrap);
cudaError_t launch_set_state(Ctx *c, const double *pos, const double *vel, cudaStream_t s);
// Verlet neighbour lists (lc_list.cu)
bool make_list_grid(Ctx *c);   // false: fewer than 3 list cells in some dimension
cudaError_t launch_list_build(Ctx *c, cudaStream_t s, bool write);
cudaError_t launch_list_rebuild(Ctx *c, cudaStream_t s, bool copy_back, int *launches);
cudaError_t launch_list_forces(Ctx *c, cudaStream_t s, bool stats, int *launches);
cudaError_t capture_list_steps(Ctx *c, double dt, int nsteps, cudaGraphExec_t *out, int *launches);
cudaError_t init_force_kernels();

// cell-start scan of the binning (lc_bin.cu), also launched by lc_noalloc.cu:
// tiles of kScanTile counts, one block of kScanThreads each; partial[] holds
// one int per tile, ticket one zero-initialised counter (reset by the
// kernel); start[] needs ncell + 1 ints; id == nullptr: identity IDs
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
__global__ void k_scan_tiles_ticket(int ncell, const int *__restrict__ count, int *__restrict__ local, int *partial,
                                    unsigned *ticket);
// cellt (optional): the cell of each provisional slot, read by k_rank_gather
// instead of a dependent gather of cell[src[t]]
__global__ void k_scatter_starts(int n, int ncell, const int *__restrict__ cell, const int *__restrict__ rank,
                                 const int *__restrict__ local, const int *__restrict__ partial,
                                 const int *__restrict__ id, int *__restrict__ src, int *__restrict__ key,
                                 int *__restrict__ start, int *__restrict__ cellt = nullptr);

// ---- small device helpers ----------------------------------------------------
// A particle's v^2 added to a thread's partial as three fused multiply-adds
// (the FP64 pipe is the scarce one: three operations instead of five
// products and sums plus the addition), and the block sum of 256 thread
// partials in a fixed order (butterfly inside each warp, then the eight warp
// sums in warp order): every kernel that forms kinetic-energy partials gets
// the same bits for the same state.
constexpr int kKinThreads = 256;
__device__ __forceinline__ double kin_add(double acc, double vx, double vy, double vz) {
    return fma(vz, vz, fma(vy, vy, fma(vx, vx, acc)));
}
__device__ __forceinline__ double block_sum_kin(double acc, double *red) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, m));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    double t = red[0];
#pragma unroll
    for (int w = 1; w < kKinThreads / 32; ++w) t = __dadd_rn(t, red[w]);
    __syncthreads();   // red is free again when the caller reuses it
    return t;
}

// Periodic wrap into [0, L), each operation rounded once (no contraction):
// x - L floor(x / L), then one correction for the rounding edge cases.
// For x in (0, L) that formula returns x itself (x / L rounds below
// 1, so floor gives 0), which the fast path returns without the FP64
// division.
__device__ __forceinline__ double wrap_coord(double x, double L) {
    if (x > 0.0 && x < L) return x;
    double q = floor(__ddiv_rn(x, L));
    double p = __dmul_rn(q, L);
    double y = __dsub_rn(x, p);
    if (y >= L) y = __dsub_rn(y, L);
    if (y < 0.0) y = __dadd_rn(y, L);
    if (y >= L) y = 0.0;
    return y;
}

// Cell coordinate of a wrapped coordinate: (int)(x * (nc / L)), clamped.
__device__ __forceinline__ int cell_coord(double xw, double inv, int nc) {
    int c = (int)__dmul_rn(xw, inv);
    c = c > nc - 1 ? nc - 1 : c;
    return c < 0 ? 0 : c;
}

// Exact FP32 -> FP64 conversion by rearranging the IEEE-754 bit fields
// (binary32: 1/8/23 bits, binary64: 1/11/52): integer operations only, so it
// does not occupy the FP64 pipe.  Zeros and subnormals map to signed zero,
// infinities and NaNs keep their class.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned a = b & 0x7fffffffu;                          // |f|: exponent and mantissa adjacent
    unsigned hi = (a >> 3) + (896u << 20);                       // normal: exponent 127 -> 1023 bias
    hi = a >= 0x7f800000u ? ((a >> 3) | 0x7ff00000u) : hi;       // inf / nan: exponent all ones
    hi = a < 0x00800000u ? 0u : hi;                              // zero and subnormals: zero
    const unsigned lo = a < 0x00800000u ? 0u : (b << 29);        // low three mantissa bits
    return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)lo);
}

// FP32 view of an FP64 value without the FP64 pipe: the binary64 sign,
// exponent and top 23 mantissa bits rearranged as binary32 (truncation, so
// |hi| <= |x| and |x - hi| < 2^-23 |x|), and the remaining 29 mantissa bits as a
// second FP32 value lo (rounded to 24 bits: |x - hi - lo| <= 2^-47 |x|).
// Valid for 2^-100 <= |x| < 2^100 (callers treat other magnitudes, zero
// included, on an exact FP64 path).
struct Split {
    float hi, lo;
};
__device__ __forceinline__ bool split_f64(double x, Split &s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ffu) - 1023;
    if (e < -100 || e >= 100) return false;
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const unsigned man_hi = (unsigned)((b >> 29) & 0x7fffffu);
    s.hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | man_hi);
    const unsigned low = (unsigned)(b & 0x1fffffffull);          // 29 bits
    const float scale = __uint_as_float((unsigned)(e - 52 + 127) << 23);   // 2^(e-52)
    const float l = __uint2float_rn(low) * scale;
    s.lo = sign ? -l : l;
    return true;
}

// Cell coordinate of a coordinate without FP64 arithmetic when that is safe:
// returns false (caller takes the exact FP64 path: wrap, multiply, truncate)
// unless x lies strictly inside (0, L) and x * nc / L is at least 1e-4 away
// from an integer, in which case the FP32 estimate has the same floor.
// The FP32 estimate of x * nc / L has relative error below 4e-7, i.e. below
// 4e-7 nc absolute; `margin` (2e-6 nc + 1e-6) keeps a factor 5 of headroom.
__device__ __forceinline__ bool cell_coord_fast(const Split &s, float Lf_lo, float invf, int nc, float margin,
                                                int &c) {
    if (!(s.hi > 0.0f && s.hi < Lf_lo)) return false;
    const float t = (s.hi + s.lo) * invf - 0.5f;
    const float r = (t + 8388608.0f) - 8388608.0f;          // nearest integer to t
    if (fabsf(t - r) > 0.5f - margin) return false;         // too close to a cell face
    c = (int)r;
    c = c > nc - 1 ? nc - 1 : c;
    return true;
}

__host__ __device__ __forceinline__ int colour_class(int c, int nc) {
    return ((nc & 1) && c == nc - 1) ? 2 : (c & 1);
}

// Colour schedule: class of cell coordinate c along a dimension of nc cells
// with class stride p, the number of cells of class a, and the coordinate of
// the t-th cell of class a.
__host__ __device__ __forceinline__ int cs_class(int c, int nc, int p) {
    const int full = p * (nc / p);
    return c < full ? c % p : p + (c - full);
}
__host__ __device__ __forceinline__ int cs_count(int a, int nc, int p) { return a < p ? nc / p : 1; }
__host__ __device__ __forceinline__ int cs_coord(int a, int t, int nc, int p) {
    return a < p ? a + p * t : p * (nc / p) + (a - p);
}

// Offset x - (c + 1/2) h of one coordinate from the centre of its cell c,
// as an unevaluated FP32 sum hi + lo, formed in double-float arithmetic
// (TwoProduct / TwoSum) from the hi + lo split of the FP64 coordinate.
__device__ __forceinline__ void cell_offset_df(const Grid &g, const Split &sp, int c, int d, float &hi, float &lo) {
    const float cf = (float)c + 0.5f;
    const float ph = cf * g.hf[d];
    const float pl = fmaf(cf, g.hf[d], -ph) + cf * g.hl[d];
    const float sum = sp.hi - ph;                    // TwoSum(hi, -ph)
    const float bb = sum - sp.hi;
    const float e2 = (sp.hi - (sum - bb)) + (-ph - bb);
    const float rest = (sp.lo - pl) + e2;
    hi = sum + rest;
    lo = rest - (hi - sum);
}

// FP32 offset of a particle from the centre (c + 1/2) h of cell cc; the
// rounding residual of each offset (|r| <= 2^-23 for |offset| < 4) is kept
// as a 10-bit signed fraction of 2^-23 in the spare fourth word (offset +
// residual equals x - (c + 1/2) h to ~2e-10).
__device__ __forceinline__ float4 cell_offset_p4(const Grid &g, const Split (&sp)[3], const int (&cc)[3]) {
    float hi[3];
    unsigned w = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float res;
        cell_offset_df(g, sp[d], cc[d], d, hi[d], res);
        int q = __float2int_rn(res * kLoScale);
        q = q > 511 ? 511 : (q < -511 ? -511 : q);
        w |= (unsigned)(q + 512) << (10 * d);
    }
    return make_float4(hi[0], hi[1], hi[2], __uint_as_float(w));
}

}  // namespace lc
