// Link-cell Lennard-Jones force sweep: the three schedules of the cell-pair
// work (colour phases, atomic accumulation, full shell) in FP64 and mixed
// precision.
//
// Work decomposition (paper Sec. IV): a task is a centre cell A together
// with a list of neighbour cells B = A + o.  For the Newton-3 schedules the
// offsets come from the 13-offset half-shell (Fig. 3b) and the intra-cell
// interaction (i < j) is part of the task; both A and every B are written
// (the write sharing of Sec. IV-V).  The full-shell schedule visits all 27
// cells, counts every pair from both sides and writes A only.
//
// One warp runs one task.  The neighbour particles of the task are listed in
// shared memory (slot + neighbour index) and processed 32 at a time, one per
// lane ("lanes = j").  The centre cell's particles are held NI at a time in
// shared memory and the loop over them is unrolled, so each lane keeps a
// private partial force for every i in registers (acc[NI][3]) and its own
// j's force in three more registers: both sides of Newton's third law
// accumulate without any communication in the inner loop.  At the end of a
// task the per-lane partials of the i's are summed across the warp by a
// butterfly reduce-scatter (NI*3 values, about one shuffle per value).
//
// Mixed precision: positions are FP32 offsets from the cell centre (|x| <
// 0.65 h), the neighbour's offset o*h is added in FP32, and the pair force is
// FP32 with a Newton-refined hardware reciprocal.  The error of the FP32 r^2
// stays below 1e-6 * r_c^2; candidates within kCutBand of r_c^2 are decided
// again from the FP64 positions with the exact arithmetic of the definition
// ((x_i - x_j) - s L, products and sums rounded once), so the set of pairs
// inside r_c is the FP64 set.  Per-task partials enter the per-particle
// accumulators as FP64 (atomic schedule) or Kahan-compensated FP32 pairs
// (colour schedule, owner writes); energies are Kahan-summed per lane and
// reduced in FP64.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#include "lc_internal.cuh"
#include "lc_pair.cuh"

namespace lc {

__constant__ Stencil c_st;    // 3D stencil tables
__constant__ Stencil c_st2;   // 2D (x-y plane) stencil tables

__device__ __forceinline__ const Stencil &stencil(int dims) { return dims == 2 ? c_st2 : c_st; }

// kColourQ: cell tasks in colour order on a device queue (LC_SCHED_COLOUR)
enum Mode : int { kAtomic = 1, kFullShell = 2, kBuffer = 3, kDag = 4, kColourQ = 5 };

constexpr int kJCap = 512;      // neighbour slots listed per batch (per warp)
constexpr int kMaxNb = 27;      // neighbour cells per task
constexpr int kJdCap = 256;     // pruned neighbours whose data is kept in shared memory
constexpr int kPruneRounds = 4; // neighbour rounds of 32 whose loads the prune issues together

struct ForceArgs {
    Grid g;
    const float4 *p4;           // FP32 cell-centre offsets + packed rounding residuals
    const double *x, *y, *z;
    const int *start, *count;
    double *fx, *fy, *fz;
    float2 *kx, *ky, *kz;
    float *bf;                  // buffer schedule, mixed: [15][3][n] private partial forces
    double *bd;                 // buffer schedule, FP64: [15][3][n]
    size_t n;                   // particles (buffer stride)
    double *warp_acc;           // [W][4] (single-launch sweeps: one slot per block)
    long long *warp_pairs;      // [W]
    int group, colour;          // colour phase
    int ntasks;
    // colour queue: per-cell completion flags, the queue counter, the limit
    // of one wait for a cell, per-cell energy partials
    int *cs_done;
    int *cs_ctrl;
    int *err;
    long long wait_ns;
    double *cell_acc;
    long long *cell_pairs;
    const int4 *cs_items;       // batch: (box, colour, global cell, 1) per queue item
    const int *cs_cell;         // single box: queue position -> cell (colour-major, cells ascending)
    const int8_t *cs_rank;      // colour (rank) of every cell, per box
    const unsigned long long *cs_dep;   // per cell: bit e = dependence offset e has an earlier colour
    int withhold;               // test of the bounded waits: no task publishes its completion
    int stats;                  // accumulate energy, virial and pair count
    int pairx;                  // 2D atomic: a task is two x-adjacent cells (see single_task)
    float sh[27][3];            // o * h rounded to FP32, offset index (ox+1) + 3 (oy+1) + 9 (oz+1)
    float sl[27][3];            // o * h - sh, rounded to FP32
    // batch of boxes (BATCHED kernels): per-box grids, box of every global
    // cell, per-box statistics accumulators
    const BoxDev *boxes;
    const unsigned short *cell_box;
    double *box_acc;
    unsigned long long *box_pairs;
};

// ---------------------------------------------------------------- tasks ----
struct TaskCells {
    int A;            // centre cell (global index)
    int cA[3];        // its coordinates in its box
    int nnb;          // neighbour cells listed (self first when present)
    bool self;        // intra-cell interaction included
    int nself;        // leading entries whose pairs are taken once by slot order (0, 1, or 2)
    int pairx;        // 1: the task is cells A and A + x (2D atomic), see single_task
    int group;        // colour: the phase's offset group; DAG: the offset index
    int dims;         // 3, or 2 (stencil in the x-y plane)
    const Grid *g;    // the box's grid
    const float (*sh)[3], (*sl)[3];   // the box's shift tables
    int cell_off;     // first global cell of the box
    int box;
};

__device__ __forceinline__ void cell_xyz(const Grid &g, int c, int out[3]) { cell_coords(g, c, out); }

// Neighbour k of the task (k < nnb): offset and periodic image.
// Entries of a two-cell task (cells A and A + x of the 2D atomic schedule),
// as offsets from A: the two cells themselves (both ordered by slot), the
// cell after them, and the four cells of the next row from A - x to A + 2x.
// The pairs each cell needs are among them; the others (A with the two
// outer cells, A + x with A - x + y) lie at least a cell side, >= r_c, apart
// and never pass the cutoff, so every pair inside r_c is taken once.
__constant__ int c_pair_off[7][2] = {{0, 0}, {1, 0}, {2, 0}, {-1, 1}, {0, 1}, {1, 1}, {2, 1}};

template <int MODE>
__device__ __forceinline__ void task_offset(int group, int k, bool self, int dims, int o[3], int pairx = 0) {
    if (MODE == kAtomic && pairx) {
        o[0] = c_pair_off[k][0]; o[1] = c_pair_off[k][1]; o[2] = 0;
        return;
    }
    if (self) {
        if (k == 0) { o[0] = o[1] = o[2] = 0; return; }
        --k;
    }
    const Stencil &S = stencil(dims);
    if (MODE == kFullShell) {            // all offsets, centre first
        o[0] = S.full[k + 1][0]; o[1] = S.full[k + 1][1]; o[2] = S.full[k + 1][2];
    } else if (MODE == kAtomic || MODE == kBuffer || MODE == kColourQ) {
        o[0] = S.hs[k][0]; o[1] = S.hs[k][1]; o[2] = S.hs[k][2];
    } else {                             // kDag: one neighbour, half-shell offset `group`
        o[0] = S.hs[group][0]; o[1] = S.hs[group][1]; o[2] = S.hs[group][2];
    }
}

// Single-box task t: the cell and its neighbour count (2D atomic: a pair of
// x-adjacent cells); used by the force and check kernels.
template <int MODE>
__device__ __forceinline__ void single_task(const Grid &g, int group, int colour, int t, TaskCells &tc,
                                            int pairx = 0) {
    tc.group = group;
    tc.dims = g.dims;
    tc.pairx = 0;
    const Stencil &S = stencil(g.dims);
    if (MODE == kAtomic && pairx) {
        // 2D atomic: task t = cells (2 tx, ty) and (2 tx + 1, ty); an odd
        // row's last cell is a task of its own (the one-cell half-shell)
        const int nhx = (g.nc[0] + 1) >> 1;
        const int ty = t / nhx, tx = t - ty * nhx;
        tc.cA[0] = 2 * tx; tc.cA[1] = ty; tc.cA[2] = 0;
        tc.A = tc.cA[0] + g.nc[0] * ty;
        tc.self = true;
        tc.pairx = (tc.cA[0] + 1 < g.nc[0]) ? 1 : 0;
        tc.nself = tc.pairx ? 2 : 1;
        tc.nnb = tc.pairx ? 7 : S.nh + 1;
    } else {
        tc.A = t;
        cell_xyz(g, t, tc.cA);
        tc.self = true;
        tc.nself = 1;
        tc.nnb = (MODE == kFullShell) ? S.nf : S.nh + 1;
    }
}

// sh / sl: the single box's shift tables (a shared-memory copy of a.sh / a.sl)
template <int MODE, bool BATCHED, bool PX = false>
__device__ __forceinline__ TaskCells make_task(const ForceArgs &a, int t, const float (*sh)[3], const float (*sl)[3]) {
    TaskCells tc;
    if constexpr (BATCHED) {
        // task t = global cell t of the batch (atomic and full-shell schedules)
        const int box = a.cell_box[t];
        const BoxDev &bd = a.boxes[box];
        tc.g = &bd.g; tc.sh = bd.sh; tc.sl = bd.sl; tc.cell_off = bd.cell_off; tc.box = box;
        tc.A = t;
        cell_xyz(bd.g, t - bd.cell_off, tc.cA);
        tc.group = 0;
        tc.dims = 3;
        tc.self = true;
        tc.nself = 1;
        tc.pairx = 0;
        tc.nnb = (MODE == kFullShell) ? 27 : 14;
    } else {
        tc.g = &a.g; tc.sh = sh; tc.sl = sl; tc.cell_off = 0; tc.box = 0;
        single_task<MODE>(a.g, a.group, a.colour, t, tc, PX ? 1 : 0);
    }
    return tc;
}

// ----------------------------------------------------- per-warp scratch ----
template <typename T>
struct alignas(16) WarpSmem {
    float4 ipa[16];             // mixed: particles 2m, 2m+1 as (x, x', y, y')
    float4 ipb[16];             // mixed: (z, z', rz, rz') with r the rounding residual
    float4 ipc[16];             // mixed: (rx, rx', ry, ry')
    int2 islot2[16];            // mixed: (slot, slot')
    float corr[32][3];          // mixed: i-side forces of the band pairs around r_c
    double corr64[16][3];       // mixed: i-side forces of the close pairs (FP64)
    T ix[32], iy[32], iz[32];   // FP64: centre-cell particles
    int islot[32];
    int jl[kJCap];              // slot | (neighbour index << 26)
    int jk[kJCap];              // mixed: the entries of jl within r_c of the i chunk's box
    float4 jd[kJdCap];          // mixed: their FP32 offsets + residuals (the first kJdCap)
    int nb_start[kMaxNb], nb_count[kMaxNb];
    int nb_img[kMaxNb];         // periodic image s_d in {-1,0,1} as (s+1) in 2-bit fields
    float4 nb_sh[kMaxNb];       // o * h rounded to FP32 (mixed), w unused
    float4 nb_sl[kMaxNb];       // o * h - nb_sh, rounded to FP32
};

// The FP64 value of a partial force (exact).  The hardware conversion here:
// on the neighbour-side and centre-side additions it measured faster than
// the integer rearrangement of the bits (atomic 0.344 -> 0.341 ms, colour
// 0.605 -> 0.597 ms on the 1M liquid).
template <typename T>
__device__ __forceinline__ double to_f64(T v) {
    if constexpr (std::is_same<T, float>::value) return (double)v;
    else return v;
}

// One task's partial force on one particle enters its accumulator: the FP32
// partial v and, for the mixed path, the FP64 sum c of its close pairs.
// (The close-pair sum is nonzero only for the rare close pairs: it is added
// on a separate path, so the common one does no FP64 arithmetic, which runs
// at a small fraction of the FP32 rate on this GPU.)
template <int MODE, bool MIXED, typename T>
__device__ __forceinline__ void write_force(const ForceArgs &a, int slot, T vx, T vy, T vz, double cx = 0.0,
                                            double cy = 0.0, double cz = 0.0) {
    const bool close = MIXED && nonzero3(cx, cy, cz);
    // kColourQ: the tasks that touch a cell never run at the same time and
    // run in the order the queue's dependences fix, so these adds neither
    // conflict nor change order from run to run; the L2's reduction units
    // perform them (RED), so the warp does not wait for the read
    if constexpr (MODE == kAtomic || MODE == kColourQ) {
        atomicAdd(a.fx + slot, to_f64(vx));
        atomicAdd(a.fy + slot, to_f64(vy));
        atomicAdd(a.fz + slot, to_f64(vz));
        if (close) {
            atomicAdd(a.fx + slot, cx);
            atomicAdd(a.fy + slot, cy);
            atomicAdd(a.fz + slot, cz);
        }
    } else if constexpr (MODE == kFullShell) {
        if (close) {
            a.fx[slot] = to_f64(vx) + cx; a.fy[slot] = to_f64(vy) + cy; a.fz[slot] = to_f64(vz) + cz;
        } else {
            a.fx[slot] = to_f64(vx); a.fy[slot] = to_f64(vy); a.fz[slot] = to_f64(vz);
        }
    } else if constexpr (MIXED) {
        float2 kx = a.kx[slot], ky = a.ky[slot], kz = a.kz[slot];
        kahan_add(kx, (float)vx); kahan_add(ky, (float)vy); kahan_add(kz, (float)vz);
        if (close) { kahan_add64(kx, cx); kahan_add64(ky, cy); kahan_add64(kz, cz); }
        a.kx[slot] = kx; a.ky[slot] = ky; a.kz[slot] = kz;
    } else {
        a.fx[slot] += vx; a.fy[slot] += vy; a.fz[slot] += vz;
    }
}

// Buffer schedule (Sec. VI, Strategy 3): a task's partial force on a particle
// goes to the buffer of the role it plays there -- buffer 0: the j side of
// an intra-cell pair, 1..13: the j side of half-shell offset 1..13, 14: the
// i side -- and every (buffer, particle) entry has exactly one writing task,
// so plain stores suffice.  `add`: a later centre-cell chunk of the same
// task adds to its own earlier store (same lane, program order).
constexpr int kIBuf = kNumFbuf - 1;

template <typename T>
__device__ __forceinline__ T *fbuf(const ForceArgs &a) {
    if constexpr (std::is_same<T, float>::value) return a.bf;
    else return a.bd;
}

template <typename T>
__device__ __forceinline__ void buffer_store(const ForceArgs &a, int buf, int slot, bool add, T vx, T vy, T vz) {
    T *p = fbuf<T>(a) + (size_t)buf * 3 * a.n + slot;
    if (add) { vx += p[0]; vy += p[a.n]; vz += p[2 * a.n]; }
    p[0] = vx; p[a.n] = vy; p[2 * a.n] = vz;
}

// Fixed-order reduce of the buffer schedule: F = sum over the 15 buffers in
// buffer order (deterministic).  FP32 partials are summed as an unevaluated
// pair hi + lo with Knuth's TwoSum (every rounding error kept, no FP64 pipe:
// GB300 runs FP64 at a small fraction of the FP32 rate); FP64 partials of
// the FP64 path are added in FP64.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += e;
}

template <typename T>
__global__ void k_buffer_reduce(size_t n, const T *buf, double *fx, double *fy, double *fz) {
    for (size_t s = blockIdx.x * (size_t)blockDim.x + threadIdx.x; s < n; s += (size_t)gridDim.x * blockDim.x) {
        double f[3];
        if constexpr (std::is_same<T, float>::value) {
            float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int b = 0; b < kNumFbuf; ++b)
#pragma unroll
                for (int d = 0; d < 3; ++d) two_sum_add(hi[d], lo[d], buf[((size_t)b * 3 + d) * n + s]);
#pragma unroll
            for (int d = 0; d < 3; ++d) f[d] = f32_to_f64_bits(hi[d]) + f32_to_f64_bits(lo[d]);
        } else {
            f[0] = f[1] = f[2] = 0.0;
#pragma unroll
            for (int b = 0; b < kNumFbuf; ++b)
#pragma unroll
                for (int d = 0; d < 3; ++d) f[d] += buf[((size_t)b * 3 + d) * n + s];
        }
        fx[s] = f[0]; fy[s] = f[1]; fz[s] = f[2];
    }
}

// Exact FP64 cutoff decision, the definition's arithmetic (each op rounded once).
__device__ __forceinline__ bool exact_inside(const ForceArgs &a, double rc2, int si, int sj, const double sL[3]) {
    double dx = __dsub_rn(__dsub_rn(a.x[si], a.x[sj]), sL[0]);
    double dy = __dsub_rn(__dsub_rn(a.y[si], a.y[sj]), sL[1]);
    double dz = __dsub_rn(__dsub_rn(a.z[si], a.z[sj]), sL[2]);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rc2;
}

// --------------------------------------------------------- the kernel -----
// Lane accumulators of one warp across its tasks.
struct LaneEnergy {
    float2 s6, s12;   // Kahan pairs (mixed)
    double d6, d12;   // FP64 sums (FP64 path)
    long long pairs;
};

// A neighbour slot as loaded for one lane (prefetched one chunk ahead).
struct JLoad {
    int w;            // slot | neighbour index << 26, or -1 past the list
    float4 p;         // mixed: FP32 offsets + packed residuals
    double x, y, z;   // FP64 path
};

template <bool MIXED>
__device__ __forceinline__ JLoad load_j(const ForceArgs &a, const int *jl, int e, int nj) {
    JLoad r;
    r.w = -1;
    if (e < nj) {
        r.w = jl[e];
        const int sj = r.w & ((1 << 26) - 1);
        if constexpr (MIXED) {
            r.p = a.p4[sj];
        } else {
            r.x = a.x[sj]; r.y = a.y[sj]; r.z = a.z[sj];
        }
    }
    return r;
}

// Mixed: entry e of a pruned list, its data from shared memory when the
// prune staged it (jdata != nullptr), else from global memory.
__device__ __forceinline__ JLoad load_j_staged(const ForceArgs &a, const int *jl, const float4 *jdata, int e, int nj) {
    JLoad r;
    r.w = -1;
    if (e < nj) {
        r.w = jl[e];
        r.p = jdata ? jdata[e] : a.p4[r.w & ((1 << 26) - 1)];
    }
    return r;
}

// Neighbour cells of a task: start, count, FP32 shift and periodic image per
// entry, filled by lanes 0 .. nnb-1.
template <bool MIXED, int MODE>
__device__ __forceinline__ void setup_neighbours(const ForceArgs &a, WarpSmem<typename std::conditional<MIXED, float, double>::type> &sm,
                                                 const TaskCells &tc, int lane) {
    const Grid &g = *tc.g;
    // neighbour table: lane k fills entry k (no FP64: shifts come from the
    // per-offset tables, the periodic image is kept as a code)
    if (lane < tc.nnb) {
        int o[3];
        task_offset<MODE>(tc.group, lane, tc.self, tc.dims, o);
        int c[3];
        int img = 0;
        for (int d = 0; d < 3; ++d) {
            c[d] = tc.cA[d] + o[d];
            int sgn = 0;
            if (c[d] >= g.nc[d]) { c[d] -= g.nc[d]; sgn = 1; }
            else if (c[d] < 0) { c[d] += g.nc[d]; sgn = -1; }
            img |= (sgn + 1) << (2 * d);
        }
        const int oi = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);
        sm.nb_sh[lane] = make_float4(tc.sh[oi][0], tc.sh[oi][1], tc.sh[oi][2], 0.f);
        sm.nb_sl[lane] = make_float4(tc.sl[oi][0], tc.sl[oi][1], tc.sl[oi][2], 0.f);
        sm.nb_img[lane] = img;
        const int B = tc.cell_off + c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
        sm.nb_start[lane] = a.start[B];
        sm.nb_count[lane] = a.count[B];
    }
    __syncwarp();
}

// Neighbour metadata of a task held in registers (lane b: entry b), so a
// warp can issue the loads of its next task before computing the current one.
struct NbPre {
    int start, count;   // of neighbour entry `lane`
    int img, oi;        // its periodic image code and offset index
    int dbl;            // two-cell task: the entry lies two cells along x (shift 2 h_x)
    int a0, na;         // the centre's first slot and count (both cells of a two-cell task)
    int nA;             // particles of cell A (the rest belong to A + x)
};

template <int MODE, bool PX = false>
__device__ __forceinline__ NbPre load_neighbours(const ForceArgs &a, const TaskCells &tc, int lane) {
    NbPre p;
    p.start = 0; p.count = 0; p.img = 0; p.oi = 13; p.dbl = 0;
    if (lane < tc.nnb) {
        const Grid &g = *tc.g;
        int o[3];
        task_offset<MODE>(tc.group, lane, tc.self, tc.dims, o, PX ? tc.pairx : 0);
        int c[3];
        int img = 0;
        for (int d = 0; d < 3; ++d) {
            c[d] = tc.cA[d] + o[d];
            int sgn = 0;
            if (c[d] >= g.nc[d]) { c[d] -= g.nc[d]; sgn = 1; }
            else if (c[d] < 0) { c[d] += g.nc[d]; sgn = -1; }
            img |= (sgn + 1) << (2 * d);
        }
        p.dbl = PX && o[0] == 2;   // o * h = 2 * (h rounded to FP32): the table's entry doubled, exactly
        p.oi = (o[0] - p.dbl + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);
        p.img = img;
        const int B = tc.cell_off + c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
        p.start = a.start[B];
        p.count = a.count[B];
    }
    p.a0 = a.start[tc.A];
    p.nA = a.count[tc.A];
    p.na = p.nA + ((PX && tc.pairx) ? a.count[tc.A + 1] : 0);
    return p;
}

template <typename S, bool PX = false>
__device__ __forceinline__ void commit_neighbours(S &sm, const TaskCells &tc, const NbPre &p, int lane) {
    if (lane < tc.nnb) {
        float4 sh4 = make_float4(tc.sh[p.oi][0], tc.sh[p.oi][1], tc.sh[p.oi][2], 0.f);
        float4 sl4 = make_float4(tc.sl[p.oi][0], tc.sl[p.oi][1], tc.sl[p.oi][2], 0.f);
        if (PX && p.dbl) { sh4.x *= 2.0f; sl4.x *= 2.0f; }
        sm.nb_sh[lane] = sh4;
        sm.nb_sl[lane] = sl4;
        sm.nb_img[lane] = p.img;
        sm.nb_start[lane] = p.start;
        sm.nb_count[lane] = p.count;
    }
    __syncwarp();
}

// Next batch of neighbour slots (slot | entry << 26) into sm.jl; returns
// how many were listed.  (b, kin) is the walk position over the entries.
template <typename S>
__device__ __forceinline__ int fill_batch(S &sm, int nnb, int &b, int &kin, int lane) {
    int nj = 0;
    while (b < nnb && nj < kJCap) {
        const int cnt = sm.nb_count[b] - kin;
        const int take = min(cnt, kJCap - nj);
        const int st = sm.nb_start[b] + kin;
        for (int k = lane; k < take; k += kWarp) sm.jl[nj + k] = (st + k) | (b << 26);
        nj += take;
        kin += take;
        if (kin >= sm.nb_count[b]) { ++b; kin = 0; }
    }
    __syncwarp();
    return nj;
}

// The task's whole neighbour list in one pass: lane b (< nnb) writes the
// entries of neighbour b at its exclusive prefix of the counts.  Returns the
// total; the list is written only if it fits (total <= kJCap), otherwise
// the caller walks it in batches with fill_batch.
template <typename S>
__device__ __forceinline__ int list_all(S &sm, const NbPre &pre, int nnb, int lane) {
    const int cnt = lane < nnb ? pre.count : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(kFull, incl, kWarp - 1);
    if (total <= kJCap) {
        const int base = incl - cnt;
        for (int k = 0; k < cnt; ++k) sm.jl[base + k] = (pre.start + k) | (lane << 26);
    }
    __syncwarp();
    return total;
}

// Keeps the entries of sm.jl[0 .. total) whose particle lies within r_c of
// the box [bmin, bmax] spanned by the staged centre particles (FP32, with a
// relative margin of 1e-4 on r_c^2, so no pair inside r_c is dropped) and
// compacts them, in list order, into sm.jk.  Returns how many were kept.
// Buffer schedule: a dropped neighbour's entry for this task is zero and is
// written as such by the first centre chunk.
template <int MODE>
__device__ __forceinline__ void prune_test(const ForceArgs &a, const WarpSmem<float> &sm, int e, int total,
                                           float3 bmin, float3 bmax, float keep2, bool first_chunk, int &w,
                                           float4 &p, bool &keep) {
    keep = false;
    if (e < total) {
        const int sj = w & ((1 << 26) - 1);
        const float4 sh = sm.nb_sh[w >> 26];
        const float px = p.x + sh.x, py = p.y + sh.y, pz = p.z + sh.z;
        const float dx = fmaxf(fmaxf(bmin.x - px, px - bmax.x), 0.f);
        const float dy = fmaxf(fmaxf(bmin.y - py, py - bmax.y), 0.f);
        const float dz = fmaxf(fmaxf(bmin.z - pz, pz - bmax.z), 0.f);
        keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < keep2;
        if constexpr (MODE == kBuffer) {
            if (!keep && first_chunk) buffer_store<float>(a, w >> 26, sj, false, 0.f, 0.f, 0.f);
        }
    }
}

// Keeps the entries of sm.jl[0 .. total) whose particle lies within r_c of
// the box [bmin, bmax] spanned by the staged centre particles (FP32, with a
// relative margin of 1e-4 on r_c^2, so no pair inside r_c is dropped) and
// compacts them, in list order, into sm.jk, their data into sm.jd (the
// first kJdCap).  Returns how many were kept.  Buffer schedule: a dropped
// neighbour's entry for this task is zero and is written as such by the
// first centre chunk.
template <int MODE>
__device__ __forceinline__ int prune_list(const ForceArgs &a, WarpSmem<float> &sm, int total, float3 bmin,
                                          float3 bmax, float keep2, bool first_chunk, int lane) {
    int nk = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int e0 = 0; e0 < total; e0 += kPruneRounds * kWarp) {
        // kPruneRounds rounds per step: all their loads in flight before any test
        int w[kPruneRounds];
        float4 p[kPruneRounds];
        const int rounds = min(kPruneRounds, (total - e0 + kWarp - 1) / kWarp);   // warp-uniform
#pragma unroll
        for (int r = 0; r < kPruneRounds; ++r) {
            const int e = e0 + r * kWarp + lane;
            w[r] = 0;
            p[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e < total) { w[r] = sm.jl[e]; p[r] = a.p4[w[r] & ((1 << 26) - 1)]; }
        }
#pragma unroll
        for (int r = 0; r < kPruneRounds; ++r) {
            if (r >= rounds) break;   // rounds past the list's end
            const int e = e0 + r * kWarp + lane;
            bool k;
            prune_test<MODE>(a, sm, e, total, bmin, bmax, keep2, first_chunk, w[r], p[r], k);
            const unsigned m = __ballot_sync(kFull, k);
            if (k) {
                const int pos = nk + __popc(m & below);
                sm.jk[pos] = w[r];
                if (pos < kJdCap) sm.jd[pos] = p[r];
            }
            nk += __popc(m);
        }
    }
    __syncwarp();
    return nk;
}

// Sum the i chunk's per-lane partials over the lanes and let the owner
// lanes write them (plus the near-r_c corrections of the mixed path).
// Mixed: column sums through the pruned-data scratch (free once the chunk
// loop has run; the next i chunk prunes again): a chunk of 16 as packed
// pairs (column_sum_pairs, the owner of element e on lane pair_element), a
// chunk of 8 one element per lane (lane l < 8 owning element l).  FP64: a
// shuffle reduce-scatter.
template <bool MIXED, int NI, int MODE, typename T, typename S>
__device__ __forceinline__ void write_i_chunk(const ForceArgs &a, S &sm, T (&ax)[NI], T (&ay)[NI], T (&az)[NI],
                                              int a0, int i0, int na, int lane) {
    if constexpr (MIXED) {
        float sx, sy, sz;
        int e = lane;
        bool owner = lane < NI;
        if constexpr (NI == 16) {
            float2 *scratch = reinterpret_cast<float2 *>(sm.jd);
            static_assert(sizeof(sm.jd) >= sizeof(float2) * 32 * kPairStride, "column-sum scratch");
            float2 px[8], py[8], pz[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                px[k] = make_float2(ax[2 * k], ax[2 * k + 1]);
                py[k] = make_float2(ay[2 * k], ay[2 * k + 1]);
                pz[k] = make_float2(az[2 * k], az[2 * k + 1]);
            }
            sx = column_sum_pairs(px, scratch, lane);
            sy = column_sum_pairs(py, scratch, lane);
            sz = column_sum_pairs(pz, scratch, lane);
            e = pair_element(lane);
            owner = pair_owner(lane);
        } else {
            float *scratch = reinterpret_cast<float *>(sm.jd);
            static_assert(sizeof(sm.jd) >= sizeof(float) * 32 * kColStride, "column-sum scratch");
            sx = column_sum<NI>(ax, scratch, lane);
            sy = column_sum<NI>(ay, scratch, lane);
            sz = column_sum<NI>(az, scratch, lane);
        }
        __syncwarp();   // order the j-side writes to A before the i-side ones; the scratch is free again
        if (owner) {
            const int ii = i0 + e;
            if (ii < na) {
                const float vx = sx + sm.corr[e][0], vy = sy + sm.corr[e][1], vz = sz + sm.corr[e][2];
                const double c[3] = {sm.corr64[e][0], sm.corr64[e][1], sm.corr64[e][2]};
                if constexpr (MODE == kBuffer) {
                    float wx = vx, wy = vy, wz = vz;
                    if (nonzero3(c[0], c[1], c[2])) {
                        wx += (float)c[0]; wy += (float)c[1]; wz += (float)c[2];
                    }
                    buffer_store<float>(a, kIBuf, a0 + ii, false, wx, wy, wz);
                } else {
                    write_force<MODE, true, float>(a, a0 + ii, vx, vy, vz, c[0], c[1], c[2]);
                }
            }
        }
        __syncwarp();
        return;
    }
    reduce_scatter<T, NI>(ax, lane);
    reduce_scatter<T, NI>(ay, lane);
    reduce_scatter<T, NI>(az, lane);
    __syncwarp();   // order the j-side writes to A before the i-side ones
    const int elem = scattered_element<NI>(lane);
    if ((lane & ((32 / NI) - 1)) == 0) {
        const int ii = i0 + elem;
        if (ii < na) {
            if constexpr (MODE == kBuffer) {
                buffer_store<T>(a, kIBuf, a0 + ii, false, ax[0], ay[0], az[0]);
            } else {
                write_force<MODE, MIXED, T>(a, a0 + ii, ax[0], ay[0], az[0]);
            }
        }
    }
    __syncwarp();
}

// Per-box statistics of one i chunk (batched kernels): warp sums, one set
// of FP64 / integer atomics per chunk into the box's accumulators.
__device__ __forceinline__ void box_stats(const ForceArgs &a, int box, double s6, double s12, long long np) {
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        s6 += __shfl_xor_sync(kFull, s6, m);
        s12 += __shfl_xor_sync(kFull, s12, m);
        np += __shfl_xor_sync(kFull, np, m);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(a.box_acc + 2 * box + 0, s6);
        atomicAdd(a.box_acc + 2 * box + 1, s12);
        atomicAdd(a.box_pairs + box, (unsigned long long)np);
    }
}

template <int NI, int MODE, bool STATS, bool BATCHED, bool PX = false>
__device__ void run_task_mixed(const ForceArgs &a, WarpSmem<float> &sm, const TaskCells &tc, const NbPre &pre,
                               int lane, LaneEnergy &le) {
    constexpr bool N3 = (MODE != kFullShell);
    const Grid &g = *tc.g;
    const int a0 = pre.a0;
    const int na = pre.na;
    const float rc2lo = g.rc2f_lo, rc2hi = g.rc2f_hi;
    const int total = list_all(sm, pre, tc.nnb, lane);   // reused by every i chunk

    for (int i0 = 0; i0 < na; i0 += NI) {
        // bounding box of the chunk's particles (FP32 offsets), from the staging loads
        float3 bmin = make_float3(1.0e30f, 1.0e30f, 1.0e30f), bmax = make_float3(-1.0e30f, -1.0e30f, -1.0e30f);
        if (lane < NI) {   // stage the i chunk (far-away sentinels past the end)
            const int ii = i0 + lane;
            float4 p = make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
            unsigned q = 0x20080200u;   // all three residuals zero
            if (ii < na) {
                p = a.p4[a0 + ii];
                q = __float_as_uint(p.w);
            }
            float rx = lo_residual(q, 0);
            if (ii < na) {
                if (PX && tc.pairx && ii >= pre.nA) {
                    // cell A + x of a two-cell task: into A's frame by its
                    // shift h_x, added as the neighbours' shifts are
                    // (Fast2Sum, the error joining the residual)
                    const float sh = tc.sh[14][0], sl = tc.sl[14][0];   // offset (1, 0, 0)
                    const float sum = sh + p.x;
                    rx = ((p.x - (sum - sh)) + rx) + sl;
                    p.x = sum;
                }
                bmin = make_float3(p.x, p.y, p.z);
                bmax = bmin;
            }
            float *A = reinterpret_cast<float *>(sm.ipa);
            float *B = reinterpret_cast<float *>(sm.ipb);
            float *C = reinterpret_cast<float *>(sm.ipc);
            int *S = reinterpret_cast<int *>(sm.islot2);
            const int m = lane >> 1, h = lane & 1;
            A[4 * m + h] = p.x;
            A[4 * m + 2 + h] = p.y;
            B[4 * m + h] = p.z;
            B[4 * m + 2 + h] = lo_residual(q, 2);
            C[4 * m + h] = rx;
            C[4 * m + 2 + h] = lo_residual(q, 1);
            S[2 * m + h] = ii < na ? a0 + ii : 0x7fffffff;
            sm.corr[lane][0] = sm.corr[lane][1] = sm.corr[lane][2] = 0.f;
            sm.corr64[lane][0] = sm.corr64[lane][1] = sm.corr64[lane][2] = 0.0;
        }
        // the box is only used by the prune (lists longer than one chunk)
        if (total > kWarp) {
#pragma unroll
            for (int m = 16; m >= 1; m >>= 1) {
                bmin.x = fminf(bmin.x, __shfl_xor_sync(kFull, bmin.x, m));
                bmin.y = fminf(bmin.y, __shfl_xor_sync(kFull, bmin.y, m));
                bmin.z = fminf(bmin.z, __shfl_xor_sync(kFull, bmin.z, m));
                bmax.x = fmaxf(bmax.x, __shfl_xor_sync(kFull, bmax.x, m));
                bmax.y = fmaxf(bmax.y, __shfl_xor_sync(kFull, bmax.y, m));
                bmax.z = fmaxf(bmax.z, __shfl_xor_sync(kFull, bmax.z, m));
            }
        }
        float2 ax2[NI / 2], ay2[NI / 2], az2[NI / 2];
#pragma unroll
        for (int k = 0; k < NI / 2; ++k) ax2[k] = ay2[k] = az2[k] = make_float2(0.f, 0.f);
        float2 e6 = make_float2(0.f, 0.f), e12 = make_float2(0.f, 0.f);
        int npair = 0;
        __syncwarp();

        // centre pairs of this chunk that hold a particle (the tile's tail is sentinels)
        const int kpairs = (min(NI, na - i0) + 1) >> 1;
        int b = 0, kin = 0;
        while (b < tc.nnb) {
            int nj = total;
            const int *list = sm.jk;
            if (total <= kWarp) {                            // one chunk whatever the prune keeps
                b = tc.nnb;
                list = sm.jl;
            } else if (total <= kJCap) {                     // listed once above: prune it
                b = tc.nnb;
                nj = prune_list<MODE>(a, sm, total, bmin, bmax, g.rc2f_hi * 1.0001f, i0 == 0, lane);
            } else {                                         // long lists: in batches, unpruned
                nj = fill_batch(sm, tc.nnb, b, kin, lane);
                list = sm.jl;
            }
            const float4 *jdata = (list == sm.jk && nj <= kJdCap) ? sm.jd : nullptr;   // staged by the prune
            JLoad nxt = load_j_staged(a, list, jdata, lane, nj);
            for (int jc = 0; jc < nj; jc += kWarp) {
                const JLoad cur = nxt;
                nxt = load_j_staged(a, list, jdata, jc + kWarp + lane, nj);   // prefetch
                const bool valid = cur.w >= 0;
                const int sj = valid ? (cur.w & ((1 << 26) - 1)) : 0x7fffffff;
                const int nb = valid ? (cur.w >> 26) : 0;
                const bool is_self = PX ? (valid && nb < tc.nself) : (valid && tc.self && nb == 0);
                const int jlim = (N3 && is_self) ? sj : 0x7fffffff;   // Newton-3 intra: slot_i < slot_j
                const int jexcl = (!N3 && is_self) ? sj : -1;         // full shell: skip i == j
                // the j position in the centre cell's frame as hi + lo: the
                // shift o*h added by Fast2Sum (|o*h| >= |x_j| when o != 0)
                // plus the stored rounding residual
                float pj[3] = {-1.0e15f, -1.0e15f, -1.0e15f}, lj[3] = {0.f, 0.f, 0.f};
                if (valid) {
                    const float4 Sh4 = sm.nb_sh[nb], Sl4 = sm.nb_sl[nb];
                    const float pin[3] = {cur.p.x, cur.p.y, cur.p.z};
                    const unsigned q = __float_as_uint(cur.p.w);
                    const float res[3] = {lo_residual(q, 0), lo_residual(q, 1), lo_residual(q, 2)};
                    const float Sh[3] = {Sh4.x, Sh4.y, Sh4.z}, Sl[3] = {Sl4.x, Sl4.y, Sl4.z};
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float sum = Sh[d] + pin[d];
                        const float err = pin[d] - (sum - Sh[d]);
                        pj[d] = sum;
                        lj[d] = (err + res[d]) + Sl[d];
                    }
                }
                float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;   // sum of f d over the i's (j gets -g)
                bool amb = false;
                if (__any_sync(kFull, is_self))
                    pair_loop<NI, N3, true, STATS>(sm, pj, lj, jlim, jexcl, rc2lo, rc2hi, ax2, ay2, az2, gx, gy, gz,
                                                   e6, e12, npair, amb, kpairs);
                else
                    pair_loop<NI, N3, false, STATS>(sm, pj, lj, jlim, jexcl, rc2lo, rc2hi, ax2, ay2, az2, gx, gy, gz,
                                                    e6, e12, npair, amb, kpairs);
                float fjx = -(gx.x + gx.y), fjy = -(gy.x + gy.y), fjz = -(gz.x + gz.y);
                double cj[3] = {0.0, 0.0, 0.0};   // the j side of its close pairs (FP64)
                if (__any_sync(kFull, amb)) {
                    // rare: candidates within the band around r_c^2 are decided
                    // with the FP64 definition and the ones inside added in
                    // FP32; pairs closer than kClose are computed and summed in
                    // FP64 (i side through the warp's shared correction slots)
                    double sL[3];
                    for (int d = 0; d < 3; ++d) sL[d] = image_shift(g, sm.nb_img[nb], d);
#pragma unroll 1
                    for (int k = 0; k < NI; ++k) {
                        const int si = reinterpret_cast<const int *>(sm.islot2)[k];
                        const bool ok = N3 ? (si < jlim) : (si != jexcl);
                        const float dx = (staged(sm.ipa, k, 0) + -pj[0]) + (staged(sm.ipc, k, 0) + -lj[0]);
                        const float dy = (staged(sm.ipa, k, 1) + -pj[1]) + (staged(sm.ipc, k, 1) + -lj[1]);
                        const float dz = (staged(sm.ipb, k, 0) + -pj[2]) + (staged(sm.ipb, k, 1) + -lj[2]);
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (!(valid && ok && r2 < rc2hi) || loop_hit(r2, rc2lo)) continue;
                        if (loop_close(r2, rc2lo)) {
                            double F[3];
                            const double s6d = pair_force_f64(a.x, a.y, a.z, si, sj, sL, F);
                            atomicAdd(&sm.corr64[k][0], F[0]);
                            atomicAdd(&sm.corr64[k][1], F[1]);
                            atomicAdd(&sm.corr64[k][2], F[2]);
                            cj[0] -= F[0]; cj[1] -= F[1]; cj[2] -= F[2];
                            if (STATS) {
                                const float s6 = (float)s6d;
                                e6.x += s6;
                                e12.x = fmaf(s6, s6, e12.x);
                                npair += 1;
                            }
                        } else if (exact_inside(a, g.rc2, si, sj, sL)) {   // the band around r_c^2
                            const float inv = rcp_nr(r2);
                            const float s6 = inv * inv * inv;
                            const float f = (s6 * inv) * fmaf(48.0f, s6, -24.0f);
                            atomicAdd(&sm.corr[k][0], f * dx);
                            atomicAdd(&sm.corr[k][1], f * dy);
                            atomicAdd(&sm.corr[k][2], f * dz);
                            fjx = fmaf(-f, dx, fjx); fjy = fmaf(-f, dy, fjy); fjz = fmaf(-f, dz, fjz);
                            if (STATS) {
                                e6.x += s6;
                                e12.x = fmaf(s6, s6, e12.x);
                                npair += 1;
                            }
                        }
                    }
                }
                if (N3 && valid) {
                    if constexpr (MODE == kBuffer) {
                        if (nonzero3(cj[0], cj[1], cj[2])) {
                            fjx += (float)cj[0]; fjy += (float)cj[1]; fjz += (float)cj[2];
                        }
                        buffer_store<float>(a, nb, sj, i0 > 0, fjx, fjy, fjz);
                    } else {
                        write_force<MODE, true, float>(a, sj, fjx, fjy, fjz, cj[0], cj[1], cj[2]);
                    }
                }
            }
            __syncwarp();
        }
        float ax[NI], ay[NI], az[NI];
#pragma unroll
        for (int k = 0; k < NI / 2; ++k) {
            ax[2 * k] = ax2[k].x; ax[2 * k + 1] = ax2[k].y;
            ay[2 * k] = ay2[k].x; ay[2 * k + 1] = ay2[k].y;
            az[2 * k] = az2[k].x; az[2 * k + 1] = az2[k].y;
        }
        write_i_chunk<true, NI, MODE>(a, sm, ax, ay, az, a0, i0, na, lane);
        if (STATS) {
            if constexpr (BATCHED) {
                box_stats(a, tc.box, f32_to_f64_bits(e6.x) + f32_to_f64_bits(e6.y),
                          f32_to_f64_bits(e12.x) + f32_to_f64_bits(e12.y), npair);
            } else {
                kahan_add(le.s6, e6.x + e6.y);
                kahan_add(le.s12, e12.x + e12.y);
                le.pairs += npair;
            }
        }
    }
}

// FP64: the definition's arithmetic in double precision throughout.
template <int NI, int MODE, bool BATCHED>
__device__ void run_task_fp64(const ForceArgs &a, WarpSmem<double> &sm, const TaskCells &tc, int lane, LaneEnergy &le) {
    constexpr bool N3 = (MODE != kFullShell);
    const Grid &g = *tc.g;
    setup_neighbours<false, MODE>(a, sm, tc, lane);
    const int a0 = a.start[tc.A];
    const int na = a.count[tc.A];
    const double rc2 = g.rc2;
    for (int i0 = 0; i0 < na; i0 += NI) {
        if (lane < NI) {
            const int ii = i0 + lane;
            const bool in = ii < na;
            const int s = in ? a0 + ii : 0x7fffffff;
            sm.ix[lane] = in ? a.x[s] : 1.0e15;
            sm.iy[lane] = in ? a.y[s] : 1.0e15;
            sm.iz[lane] = in ? a.z[s] : 1.0e15;
            sm.islot[lane] = s;
        }
        double ax[NI], ay[NI], az[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) ax[k] = ay[k] = az[k] = 0.0;
        double e6 = 0.0, e12 = 0.0;
        int npair = 0;
        __syncwarp();
        int b = 0, kin = 0;
        while (b < tc.nnb) {
            const int nj = fill_batch(sm, tc.nnb, b, kin, lane);
            JLoad nxt = load_j<false>(a, sm.jl, lane, nj);
            for (int jc = 0; jc < nj; jc += kWarp) {
                const JLoad cur = nxt;
                nxt = load_j<false>(a, sm.jl, jc + kWarp + lane, nj);
                const bool valid = cur.w >= 0;
                const int sj = valid ? (cur.w & ((1 << 26) - 1)) : 0x7fffffff;
                const int nb = valid ? (cur.w >> 26) : 0;
                const bool is_self = valid && tc.self && nb == 0;
                const int jlim = (N3 && is_self) ? sj : 0x7fffffff;
                const int jexcl = (!N3 && is_self) ? sj : -1;
                const double pjx = valid ? cur.x : -1.0e15, pjy = valid ? cur.y : -1.0e15,
                             pjz = valid ? cur.z : -1.0e15;
                const int img = sm.nb_img[nb];
                const double sLx = image_shift(g, img, 0), sLy = image_shift(g, img, 1), sLz = image_shift(g, img, 2);
                double fjx = 0.0, fjy = 0.0, fjz = 0.0;
#pragma unroll
                for (int k = 0; k < NI; ++k) {
                    const int si = sm.islot[k];
                    const bool ok = N3 ? (si < jlim) : (si != jexcl);
                    const double dx = __dsub_rn(__dsub_rn(sm.ix[k], pjx), sLx);
                    const double dy = __dsub_rn(__dsub_rn(sm.iy[k], pjy), sLy);
                    const double dz = __dsub_rn(__dsub_rn(sm.iz[k], pjz), sLz);
                    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    const bool hit = ok && (r2 < rc2);
                    const double inv = hit ? 1.0 / r2 : 0.0;
                    const double s6 = inv * inv * inv;
                    const double f = (s6 * inv) * (48.0 * s6 - 24.0);
                    ax[k] += f * dx; ay[k] += f * dy; az[k] += f * dz;
                    if (N3) { fjx -= f * dx; fjy -= f * dy; fjz -= f * dz; }
                    e6 += s6;
                    e12 += s6 * s6;
                    npair += hit ? 1 : 0;
                }
                if (N3 && valid) {
                    if constexpr (MODE == kBuffer) buffer_store<double>(a, nb, sj, i0 > 0, fjx, fjy, fjz);
                    else write_force<MODE, false, double>(a, sj, fjx, fjy, fjz);
                }
            }
            __syncwarp();
        }
        write_i_chunk<false, NI, MODE>(a, sm, ax, ay, az, a0, i0, na, lane);
        if constexpr (BATCHED) {
            box_stats(a, tc.box, e6, e12, npair);
        } else {
            le.d6 += e6;
            le.d12 += e12;
            le.pairs += npair;
        }
    }
}

// Colour schedule: task t of colour k of one box (grid g, shift tables sh /
// sl, first global cell cell_off).  Waits until the earlier-coloured tasks
// whose written cells can meet this task's have published their completion
// (the cells at the stencil's dependency offsets), runs the cell task with
// plain writes and stores the task's energy partials (summed in a fixed
// order afterwards); the caller publishes its completion.  Returns false if
// a wait ran out (error flag set).
template <bool MIXED, int NI, bool STATS>
__device__ bool colour_task(const ForceArgs &a, WarpSmem<typename std::conditional<MIXED, float, double>::type> &sm,
                            const Grid &g, const float (*sh)[3], const float (*sl)[3], int cell_off, int k, int A,
                            int lane) {
    const Stencil &S = stencil(g.dims);
    int cA[3];
    cell_coords(g, A - cell_off, cA);
    const unsigned long long waits = a.cs_dep[A];   // the dependence offsets with an earlier colour
    bool timed_out = false;
    for (int e = lane; e < S.ndep; e += kWarp) {
        if (!((waits >> e) & 1ull)) continue;
        int cn[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            cn[d] = cA[d] + S.dep[e][d];
            cn[d] = cn[d] < 0 ? cn[d] + g.nc[d] : (cn[d] >= g.nc[d] ? cn[d] - g.nc[d] : cn[d]);
        }
        const int N = cell_off + cn[0] + g.nc[0] * (cn[1] + g.nc[1] * cn[2]);
        if (ld_acquire(a.cs_done + N) != 0) continue;
        const unsigned long long t0 = global_ns();
        unsigned sleep = 64;
        timed_out = true;
        for (unsigned it = 0; it < (1u << 22); ++it) {
            __nanosleep(sleep);
            if (sleep < 2048) sleep <<= 1;   // back off: few loads on the flag
            if (ld_acquire(a.cs_done + N) != 0) { timed_out = false; break; }
            if ((it & 7) == 7) {
                if (ld_relaxed(a.err) & kErrTimeout) break;
                if ((long long)(global_ns() - t0) > a.wait_ns) break;
            }
        }
        if (timed_out) break;
    }
    if (__any_sync(kFull, timed_out)) {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        return false;
    }
    // every flag a lane saw set was published with a release store and read
    // with an acquire load, so that task's writes happen before the lane's
    // later accesses; the warp barrier carries the order to the other lanes
    // (an acquire fence here instead cost 0.05 ms per evaluation at 1M)
    __syncwarp();
    TaskCells tc;
    tc.g = &g; tc.sh = sh; tc.sl = sl; tc.cell_off = cell_off; tc.box = 0;
    tc.A = A; tc.cA[0] = cA[0]; tc.cA[1] = cA[1]; tc.cA[2] = cA[2];
    tc.group = 0; tc.dims = g.dims; tc.self = true; tc.nself = 1; tc.pairx = 0; tc.nnb = S.nh + 1;
    LaneEnergy lt;
    lt.s6 = make_float2(0.f, 0.f);
    lt.s12 = make_float2(0.f, 0.f);
    lt.d6 = lt.d12 = 0.0;
    lt.pairs = 0;
    if constexpr (MIXED) {
        const NbPre pre = load_neighbours<kColourQ>(a, tc, lane);
        commit_neighbours<WarpSmem<float>>(sm, tc, pre, lane);
        run_task_mixed<NI, kColourQ, STATS, false>(a, sm, tc, pre, lane, lt);
    } else {
        run_task_fp64<NI, kColourQ, false>(a, sm, tc, lane, lt);
    }
    if (STATS) {
        double s6 = MIXED ? (f32_to_f64_bits(lt.s6.x) - f32_to_f64_bits(lt.s6.y)) : lt.d6;
        double s12 = MIXED ? (f32_to_f64_bits(lt.s12.x) - f32_to_f64_bits(lt.s12.y)) : lt.d12;
        long long np = lt.pairs;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            s6 += __shfl_xor_sync(kFull, s6, m);
            s12 += __shfl_xor_sync(kFull, s12, m);
            np += __shfl_xor_sync(kFull, np, m);
        }
        if (lane == 0) {
            a.cell_acc[4 * (size_t)A + 0] = s6;
            a.cell_acc[4 * (size_t)A + 1] = s12;
            a.cell_pairs[A] = np;
        }
    }
    __syncwarp();   // every lane's writes ordered before lane 0's later release (cumulative)
    return true;
}

// The statistics of a single-launch sweep (atomic, full shell, buffer)
// summed per block: the block's warps' partials in warp order into slot
// blockIdx.x (written, not added: no clearing before the launch), so the
// final reduction reads one slot per block instead of one per warp.  A
// shared-memory sum behind a block barrier; no fence, which would make the
// compiler return a value from every force reduction of the sweep.
__device__ __forceinline__ void block_stats(const ForceArgs &a, double s6, double s12, long long np, int wib,
                                            int lane) {
    __shared__ double f6[8], f12[8];   // k_force blocks hold at most 8 warps
    __shared__ long long fp[8];
    if (lane == 0) { f6[wib] = s6; f12[wib] = s12; fp[wib] = np; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t6 = f6[0], t12 = f12[0];
        long long tp = fp[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { t6 += f6[w]; t12 += f12[w]; tp += fp[w]; }
        a.warp_acc[4 * blockIdx.x + 0] = t6;
        a.warp_acc[4 * blockIdx.x + 1] = t12;
        a.warp_pairs[blockIdx.x] = tp;
    }
}

template <bool MIXED, int NI, int MODE, bool STATS, bool BATCHED, bool PX = false>
__global__ void __launch_bounds__(256, MIXED ? 2 : 1) k_force(ForceArgs a) {
    using T = typename std::conditional<MIXED, float, double>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WarpSmem<T> &sm = reinterpret_cast<WarpSmem<T> *>(smem_raw)[wib];
    const int W = gridDim.x * (blockDim.x >> 5);
    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    LaneEnergy le;
    le.s6 = make_float2(0.f, 0.f);
    le.s12 = make_float2(0.f, 0.f);
    le.d6 = le.d12 = 0.0;
    le.pairs = 0;
    // the single box's shift tables in shared memory: the lanes of a task
    // read them with 14 different indices, which parameter space serialises
    __shared__ float s_sh[27][3], s_sl[27][3];
    for (int k = threadIdx.x; k < 81; k += blockDim.x) {
        (&s_sh[0][0])[k] = (&a.sh[0][0])[k];
        (&s_sl[0][0])[k] = (&a.sl[0][0])[k];
    }
    __syncthreads();
    if constexpr (MODE == kColourQ) {
        // Colour schedule: the queue holds cell tasks in colour order
        // (colour-major; a batch: (box, colour) groups by the colour's
        // position in its box's chain, one cell per item).  Cells of one
        // colour write disjoint cells; a task first
        // waits (bounded) until the earlier-coloured tasks of its box that
        // could share a written cell have published -- they were claimed
        // earlier, so running warps hold them -- then runs with plain writes.
        // A finished task is published right after its warp's next claim
        // is issued, so that its reductions drain while the claim's atomic
        // is in flight; the warp waits for nothing in between, which keeps
        // the argument above.
        int pend = -1;   // finished task not yet published
        for (;;) {
            int q = 0;
            if (lane == 0) q = atomicAdd(a.cs_ctrl, 1);
            if (lane == 0 && pend >= 0 && !a.withhold) st_release(a.cs_done + pend, 1);
            pend = -1;
            q = __shfl_sync(kFull, q, 0);
            if (q >= a.ntasks) break;
            bool ok = true;
            int A;
            if constexpr (BATCHED) {
                const int4 it = a.cs_items[q];   // (box, colour, global cell)
                const BoxDev &bd = a.boxes[it.x];
                A = it.z;
                ok = colour_task<MIXED, NI, STATS>(a, sm, bd.g, bd.sh, bd.sl, bd.cell_off, it.y, it.z, lane);
            } else {
                A = a.cs_cell[q];
                ok = colour_task<MIXED, NI, STATS>(a, sm, a.g, s_sh, s_sl, 0, (int)a.cs_rank[A], A, lane);
            }
            if (!ok) break;
            pend = A;
        }
    } else if constexpr (MIXED) {
        for (int t = w; t < a.ntasks; t += W) {
            const TaskCells tc = make_task<MODE, BATCHED, PX>(a, t, s_sh, s_sl);
            const NbPre pre = load_neighbours<MODE, PX>(a, tc, lane);
            commit_neighbours<WarpSmem<float>, PX>(sm, tc, pre, lane);
            run_task_mixed<NI, MODE, STATS, BATCHED, PX>(a, sm, tc, pre, lane, le);
        }
    } else {
        for (int t = w; t < a.ntasks; t += W) {
            TaskCells tc = make_task<MODE, BATCHED>(a, t, s_sh, s_sl);
            run_task_fp64<NI, MODE, BATCHED>(a, sm, tc, lane, le);
        }
    }
    // warp reduction of the energy partials in FP64, fixed order
    double s6 = MIXED ? (f32_to_f64_bits(le.s6.x) - f32_to_f64_bits(le.s6.y)) : le.d6;
    double s12 = MIXED ? (f32_to_f64_bits(le.s12.x) - f32_to_f64_bits(le.s12.y)) : le.d12;
    long long np = le.pairs;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        s6 += __shfl_xor_sync(kFull, s6, m);
        s12 += __shfl_xor_sync(kFull, s12, m);
        np += __shfl_xor_sync(kFull, np, m);
    }
    if constexpr (STATS && !BATCHED && MODE != kColourQ) {
        block_stats(a, s6, s12, np, wib, lane);
    } else if (STATS && !BATCHED && lane == 0) {
        a.warp_acc[4 * w + 0] += s6;
        a.warp_acc[4 * w + 1] += s12;
        a.warp_pairs[w] += np;
    }
}

// ------------------------------------- row groups (atomic schedule, 3D) ----
// The atomic schedule's single-box 3D sweep with the neighbour data of a
// group of consecutive centre cells staged once per block.  A group is a run
// of up to kRowGMax x-consecutive centre cells of one (y, z) row; the
// forward half-shells of its cells lie in five rows of cells, (y, z),
// (y + 1, z), (y - 1, z + 1), (y, z + 1), (y + 1, z + 1), over x0 - 1 ..
// x0 + G, each row one to three contiguous runs of slots (cell order is x
// fastest; a run breaks where the row wraps around the periodic boundary).
// One warp copies them into a shared-memory slot by bulk copies (TMA,
// cp.async.bulk, one per run) and the block's warps take the group's cells as
// tasks, reading every neighbour from shared memory: each particle is read
// from L2 once per group instead of once per task, and no warp waits on a
// gather latency in its prune.  Two slots per block: the warp that finishes
// a group's last task refills its slot with the block's next group while the
// others work on the group in the other slot.  Runs that do not fit a slot
// are read from global memory instead.  The task itself is the atomic
// schedule's (the same pair loop, pruning, rare path and writes).
#ifndef ROW_G
#define ROW_G 21
#define ROW_CAP 4096
#define ROW_SLOTS 2
#endif
constexpr int kRowWarps = 16;
constexpr int kRowGMax = ROW_G;                     // centre cells per group
constexpr int kRowRows = 5;
constexpr int kRowCells = kRowRows * (kRowGMax + 2);
constexpr int kRowCap = ROW_CAP;                    // staged particles per slot
constexpr int kRowSlots = ROW_SLOTS;                // groups staged ahead per block
constexpr int kRowJl = 512;                         // listed neighbour entries per batch
constexpr int kRowUnstaged = 1 << 25;               // list entry flag: data in global memory

struct RowSlot {
    float4 data[kRowCap];
    int boff[kRowCells];      // buffer offset of each table cell (-1: not staged)
    int gstart[kRowCells];    // its first slot
    int count[kRowCells];
    int img[kRowCells];       // its periodic image code seen from the group's centre row
    int tag;                  // local group index whose data is in place
    int group;                // its global group index (-1: past the last group)
    int y, z, x0, ntask;
    int done;                 // tasks of the group finished
    int phase;                // parity of the mbarrier's next phase
    unsigned long long bar;   // mbarrier of the bulk copies
};

struct alignas(16) RowWarp {
    float4 ipa[8], ipb[8], ipc[8];   // the centre chunk in pairs, as in WarpSmem
    int2 islot2[8];
    float corr[16][3];
    double corr64[16][3];
    float4 nb_sh[14], nb_sl[14];
    int nb_base[14];                 // slot = nb_base + entry index (staged or not)
    int nb_boff[14], nb_count[14], nb_img[14];
    union {
        int jl[kRowJl];              // entry index | unstaged flag | neighbour << 26
        float4 jd[(32 * kPairStride * 2 + 3) / 4];   // the column sums' scratch (write_i_chunk)
    };
};

struct RowArgs {
    int G, nseg, ngroups;            // centre cells per group, groups per row, groups
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned:
// float4 entries) from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Row of the group's table for a half-shell offset (oy, oz).
__device__ __forceinline__ int row_of(int oy, int oz) { return oz == 0 ? oy : 3 + oy; }
__device__ __forceinline__ int row_oy(int r) { return r == 0 ? 0 : (r == 1 ? 1 : r - 3); }
__device__ __forceinline__ int row_oz(int r) { return r < 2 ? 0 : 1; }

// One warp stages local group li of the block into slot S: the block's
// groups are blockIdx.x + li * gridDim.x (increasing in li, so once one is
// past the last group all later ones are), fills the cell table, copies the
// runs that fit, waits for the copies (bounded) and publishes the tag.
// Returns false on a timeout.
__device__ bool row_stage(const ForceArgs &a, const RowArgs &r, RowSlot &S, int li, int *s_end, int lane) {
    const Grid &g = a.g;
    const int gid = blockIdx.x + li * gridDim.x;
    if (gid >= r.ngroups) {
        if (lane == 0) {
            S.group = -1;
            atomicMin(s_end, li);
            __threadfence_block();
            *(volatile int *)&S.tag = li;
        }
        __syncwarp();
        return true;
    }
    const int seg = gid % r.nseg, row = gid / r.nseg;
    const int y = row % g.nc[1], z = row / g.nc[1];
    const int x0 = seg * r.G;
    const int ntask = min(r.G, g.nc[0] - x0);
    const int nk = ntask + 2;   // table cells per row: x0 - 1 .. x0 + ntask
    // the runs: per row, the cell before x0 when it wraps, the cells inside
    // the box, the cell after the last when it wraps (lane p: row p / 3)
    int p_first = 0, p_cells = 0, p_k0 = 0;   // first global cell, cells, first table column
    int p_bytes = 0, p_gs = 0;
    if (lane < 3 * kRowRows) {
        const int rr = lane / 3, kind = lane % 3;
        int yy = y + row_oy(rr), zz = z + row_oz(rr);
        yy = yy < 0 ? yy + g.nc[1] : (yy >= g.nc[1] ? yy - g.nc[1] : yy);
        zz = zz >= g.nc[2] ? zz - g.nc[2] : zz;
        const int rbase = g.nc[0] * (yy + g.nc[1] * zz);
        const int xlo = x0 - 1, xhi = x0 + ntask;
        int xa = 0, xb = -1, k0 = 0;
        if (kind == 0) {
            if (xlo < 0) { xa = xb = g.nc[0] - 1; k0 = 0; }
        } else if (kind == 1) {
            xa = max(xlo, 0); xb = min(xhi, g.nc[0] - 1); k0 = xa - xlo;
        } else {
            if (xhi >= g.nc[0]) { xa = xb = 0; k0 = nk - 1; }
        }
        if (xb >= xa) {
            p_first = rbase + xa;
            p_cells = xb - xa + 1;
            p_k0 = rr * (r.G + 2) + k0;
            p_gs = a.start[p_first];
            p_bytes = 16 * (a.start[p_first + p_cells - 1] + a.count[p_first + p_cells - 1] - p_gs);
        }
    }
    // buffer offsets: inclusive scan of the run sizes in lane order
    int incl = p_bytes;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const int v = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += v;
    }
    const bool fits = p_cells > 0 && incl <= 16 * kRowCap;
    const int p_off = (incl - p_bytes) >> 4;   // entries
    const unsigned total = __reduce_add_sync(kFull, fits ? (unsigned)p_bytes : 0u);
    // the cell table: lane-parallel over the runs' cells
    for (int p = 0; p < 3 * kRowRows; ++p) {
        const int cells = __shfl_sync(kFull, p_cells, p);
        if (cells == 0) continue;
        const int first = __shfl_sync(kFull, p_first, p), k0 = __shfl_sync(kFull, p_k0, p);
        const int gs = __shfl_sync(kFull, p_gs, p), off = __shfl_sync(kFull, p_off, p);
        const bool st = __shfl_sync(kFull, fits, p);
        for (int c = lane; c < cells; c += kWarp) {
            const int ci = k0 + c, gc = first + c;
            const int s0 = a.start[gc];
            S.gstart[ci] = s0;
            S.count[ci] = a.count[gc];
            S.boff[ci] = st ? off + (s0 - gs) : -1;
            // periodic image of the cell as the group's centres see it
            const int rr = ci / (r.G + 2), k = ci - rr * (r.G + 2);
            const int xi = x0 - 1 + k, yi = y + row_oy(rr), zi = z + row_oz(rr);
            const int sx = xi < 0 ? -1 : (xi >= g.nc[0] ? 1 : 0);
            const int sy = yi < 0 ? -1 : (yi >= g.nc[1] ? 1 : 0);
            const int sz = zi >= g.nc[2] ? 1 : 0;
            S.img[ci] = (sx + 1) | ((sy + 1) << 2) | ((sz + 1) << 4);
        }
    }
    if (lane == 0) {
        S.group = gid; S.y = y; S.z = z; S.x0 = x0; S.ntask = ntask; S.done = 0;
    }
    // the slot's previous readers finished before its last task was counted
    // (release there, acquire by the counting atomic): order their generic
    // reads before the asynchronous copies' writes
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_expect_tx(&S.bar, total);
    __syncwarp();
    if (fits && p_bytes > 0) bulk_g2s(&S.data[p_off], a.p4 + p_gs, (unsigned)p_bytes, &S.bar);
    // wait for the copies (bounded: a second limit if the first runs out,
    // so that no copy is in flight when the warp leaves)
    bool ok = true;
    if (lane == 0) {
        const unsigned par = (unsigned)S.phase;
        const unsigned long long t0 = global_ns();
        unsigned it = 0;
        while (!mbar_try_wait(&S.bar, par)) {
            if ((++it & 255) == 0 && (long long)(global_ns() - t0) > a.wait_ns) { ok = false; break; }
        }
        if (!ok) {
            atomicOr(a.err, kErrTimeout);
            const unsigned long long t1 = global_ns();
            while (!mbar_try_wait(&S.bar, par) && (long long)(global_ns() - t1) < 4 * a.wait_ns) {}
        }
        S.phase = (int)(par ^ 1u);
        __threadfence_block();
        *(volatile int *)&S.tag = li;
    }
    ok = __shfl_sync(kFull, ok, 0);
    __syncwarp();
    return ok;
}

// Waits (bounded) until slot S holds local group li.  Returns 1 when it
// does, 0 past the block's last group, -1 on a timeout (error flag set).
__device__ int row_wait(const ForceArgs &a, const RowSlot &S, int li, const int *s_end) {
    int res = 1;
    if ((threadIdx.x & 31) == 0) {
        const unsigned long long t0 = global_ns();
        unsigned sleep = 32, it = 0;
        for (;;) {
            if (*(volatile const int *)&S.tag == li) {
                if (*(volatile const int *)&S.group < 0) res = 0;   // past the last group
                break;
            }
            if (*(volatile const int *)s_end <= li) { res = 0; break; }
            if ((++it & 15) == 0) {
                if (*(volatile const int *)a.err & kErrTimeout) { res = -1; break; }
                if ((long long)(global_ns() - t0) > a.wait_ns) { atomicOr(a.err, kErrTimeout); res = -1; break; }
            }
            __nanosleep(sleep);
            if (sleep < 1024) sleep <<= 1;
        }
        __threadfence_block();
    }
    res = __shfl_sync(kFull, res, 0);
    __syncwarp();
    return res;
}

// Neighbour entry e of a listed batch: data from the slot or, flagged, from
// global memory; its slot.
__device__ __forceinline__ float4 row_data(const ForceArgs &a, const RowSlot &S, const RowWarp &W, int w) {
    const int idx = w & (kRowUnstaged - 1);
    return (w & kRowUnstaged) ? a.p4[W.nb_base[w >> 26] + idx] : S.data[idx];
}

// List neighbour entries from (b, kin) until kRowJl are listed; returns how many.
__device__ __forceinline__ int row_list(RowWarp &W, int &b, int &kin, int lane) {
    int nj = 0;
    while (b < 14 && nj < kRowJl) {
        const int cnt = W.nb_count[b] - kin;
        const int take = min(cnt, kRowJl - nj);
        const int boff = W.nb_boff[b];
        const int tagb = (b << 26) | (boff < 0 ? kRowUnstaged : 0);
        const int base = (boff < 0 ? 0 : boff) + kin;
        for (int k = lane; k < take; k += kWarp) W.jl[nj + k] = (base + k) | tagb;
        nj += take;
        kin += take;
        if (kin >= W.nb_count[b]) { ++b; kin = 0; }
    }
    __syncwarp();
    return nj;
}

// One task: centre cell x0 + t of the slot's group, its 13 forward
// neighbours and itself (the atomic schedule's task).
template <bool STATS>
__device__ __forceinline__ void row_task(const ForceArgs &a, const RowArgs &r, const RowSlot &S, RowWarp &W, int t, int lane,
                         const float (*sh)[3], const float (*sl)[3], LaneEnergy &le) {
    const Grid &g = a.g;
    // neighbour table, in the stencil's order: self, then the forward offsets
    if (lane < 14) {
        int o[3] = {0, 0, 0};
        if (lane > 0) {
            const int k = lane - 1;   // forward offsets, z then y then x ascending
            if (k == 0) { o[0] = 1; }
            else if (k < 4) { o[0] = k - 2; o[1] = 1; }
            else { o[0] = (k - 4) % 3 - 1; o[1] = (k - 4) / 3 - 1; o[2] = 1; }
        }
        const int ci = row_of(o[1], o[2]) * (r.G + 2) + t + 1 + o[0];
        const int boff = S.boff[ci], gs = S.gstart[ci];
        const int oi = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);
        W.nb_sh[lane] = make_float4(sh[oi][0], sh[oi][1], sh[oi][2], 0.f);
        W.nb_sl[lane] = make_float4(sl[oi][0], sl[oi][1], sl[oi][2], 0.f);
        W.nb_base[lane] = boff >= 0 ? gs - boff : gs;
        W.nb_boff[lane] = boff;
        W.nb_count[lane] = S.count[ci];
        W.nb_img[lane] = S.img[ci];
    }
    __syncwarp();
    const int na = W.nb_count[0];
    const int a0 = W.nb_base[0] + (W.nb_boff[0] < 0 ? 0 : W.nb_boff[0]);   // first slot of the centre cell
    const int c0 = W.nb_boff[0];                                              // its buffer offset (-1: global)
    const float rc2lo = g.rc2f_lo, rc2hi = g.rc2f_hi;
    constexpr int NI = 16;
    for (int i0 = 0; i0 < na; i0 += NI) {
        float3 bmin = make_float3(1.0e30f, 1.0e30f, 1.0e30f), bmax = make_float3(-1.0e30f, -1.0e30f, -1.0e30f);
        if (lane < NI) {
            const int ii = i0 + lane;
            float4 p = make_float4(1.0e15f, 1.0e15f, 1.0e15f, 0.f);
            unsigned q = 0x20080200u;   // all three residuals zero
            if (ii < na) {
                p = c0 >= 0 ? S.data[c0 + ii] : a.p4[a0 + ii];
                q = __float_as_uint(p.w);
                bmin = make_float3(p.x, p.y, p.z);
                bmax = bmin;
            }
            float *A = reinterpret_cast<float *>(W.ipa);
            float *B = reinterpret_cast<float *>(W.ipb);
            float *C = reinterpret_cast<float *>(W.ipc);
            int *Sl = reinterpret_cast<int *>(W.islot2);
            const int m = lane >> 1, h = lane & 1;
            A[4 * m + h] = p.x;
            A[4 * m + 2 + h] = p.y;
            B[4 * m + h] = p.z;
            B[4 * m + 2 + h] = lo_residual(q, 2);
            C[4 * m + h] = lo_residual(q, 0);
            C[4 * m + 2 + h] = lo_residual(q, 1);
            Sl[2 * m + h] = ii < na ? a0 + ii : 0x7fffffff;
            W.corr[lane][0] = W.corr[lane][1] = W.corr[lane][2] = 0.f;
            W.corr64[lane][0] = W.corr64[lane][1] = W.corr64[lane][2] = 0.0;
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            bmin.x = fminf(bmin.x, __shfl_xor_sync(kFull, bmin.x, m));
            bmin.y = fminf(bmin.y, __shfl_xor_sync(kFull, bmin.y, m));
            bmin.z = fminf(bmin.z, __shfl_xor_sync(kFull, bmin.z, m));
            bmax.x = fmaxf(bmax.x, __shfl_xor_sync(kFull, bmax.x, m));
            bmax.y = fmaxf(bmax.y, __shfl_xor_sync(kFull, bmax.y, m));
            bmax.z = fmaxf(bmax.z, __shfl_xor_sync(kFull, bmax.z, m));
        }
        float2 ax2[NI / 2], ay2[NI / 2], az2[NI / 2];
#pragma unroll
        for (int k = 0; k < NI / 2; ++k) ax2[k] = ay2[k] = az2[k] = make_float2(0.f, 0.f);
        float2 e6 = make_float2(0.f, 0.f), e12 = make_float2(0.f, 0.f);
        int npair = 0;
        __syncwarp();
        const int kpairs = (min(NI, na - i0) + 1) >> 1;
        const float keep2 = g.rc2f_hi * 1.0001f;
        const unsigned below = (1u << lane) - 1u;
        int b = 0, kin = 0;
        while (b < 14) {
            int nj = row_list(W, b, kin, lane);
            if (nj > kWarp) {
                // prune in place: keep the entries within r_c of the chunk's box
                int nk = 0;
                for (int e0 = 0; e0 < nj; e0 += kWarp) {
                    const int e = e0 + lane;
                    bool keep = false;
                    int w = 0;
                    if (e < nj) {
                        w = W.jl[e];
                        const float4 p = row_data(a, S, W, w);
                        const float4 s4 = W.nb_sh[w >> 26];
                        const float px = p.x + s4.x, py = p.y + s4.y, pz = p.z + s4.z;
                        const float dx = fmaxf(fmaxf(bmin.x - px, px - bmax.x), 0.f);
                        const float dy = fmaxf(fmaxf(bmin.y - py, py - bmax.y), 0.f);
                        const float dz = fmaxf(fmaxf(bmin.z - pz, pz - bmax.z), 0.f);
                        keep = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < keep2;
                    }
                    const unsigned mk = __ballot_sync(kFull, keep);
                    if (keep) W.jl[nk + __popc(mk & below)] = w;   // nk + rank <= e: read before written
                    nk += __popc(mk);
                }
                __syncwarp();
                nj = nk;
            }
            int wn = lane < nj ? W.jl[lane] : -1;
            float4 pn = wn >= 0 ? row_data(a, S, W, wn) : make_float4(0.f, 0.f, 0.f, 0.f);
            for (int jc = 0; jc < nj; jc += kWarp) {
                const int w = wn;
                const float4 pc = pn;
                const int en = jc + kWarp + lane;   // prefetch the next chunk's entry
                wn = en < nj ? W.jl[en] : -1;
                pn = wn >= 0 ? row_data(a, S, W, wn) : make_float4(0.f, 0.f, 0.f, 0.f);
                const bool valid = w >= 0;
                const int nb = valid ? (w >> 26) : 0;
                const int sj = valid ? W.nb_base[nb] + (w & (kRowUnstaged - 1)) : 0x7fffffff;
                const bool is_self = valid && nb == 0;
                const int jlim = is_self ? sj : 0x7fffffff;   // Newton-3 intra: slot_i < slot_j
                float pj[3] = {-1.0e15f, -1.0e15f, -1.0e15f}, lj[3] = {0.f, 0.f, 0.f};
                if (valid) {
                    const float4 Sh4 = W.nb_sh[nb], Sl4 = W.nb_sl[nb];
                    const float pin[3] = {pc.x, pc.y, pc.z};
                    const unsigned q = __float_as_uint(pc.w);
                    const float res[3] = {lo_residual(q, 0), lo_residual(q, 1), lo_residual(q, 2)};
                    const float Shv[3] = {Sh4.x, Sh4.y, Sh4.z}, Slv[3] = {Sl4.x, Sl4.y, Sl4.z};
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const float sum = Shv[d] + pin[d];
                        const float err = pin[d] - (sum - Shv[d]);
                        pj[d] = sum;
                        lj[d] = (err + res[d]) + Slv[d];
                    }
                }
                float2 gx = make_float2(0.f, 0.f), gy = gx, gz = gx;
                bool amb = false;
                if (__any_sync(kFull, is_self))
                    pair_loop<NI, true, true, STATS>(W, pj, lj, jlim, -1, rc2lo, rc2hi, ax2, ay2, az2, gx, gy, gz, e6,
                                                     e12, npair, amb, kpairs);
                else
                    pair_loop<NI, true, false, STATS>(W, pj, lj, jlim, -1, rc2lo, rc2hi, ax2, ay2, az2, gx, gy, gz, e6,
                                                      e12, npair, amb, kpairs);
                float fjx = -(gx.x + gx.y), fjy = -(gy.x + gy.y), fjz = -(gz.x + gz.y);
                double cj[3] = {0.0, 0.0, 0.0};
                if (__any_sync(kFull, amb)) {
                    // rare: the band around r_c^2 decided in FP64 and added in
                    // FP32; pairs closer than kClose computed and summed in FP64
                    double sL[3];
                    for (int d = 0; d < 3; ++d) sL[d] = image_shift(g, W.nb_img[nb], d);
#pragma unroll 1
                    for (int k = 0; k < NI; ++k) {
                        const int si = reinterpret_cast<const int *>(W.islot2)[k];
                        const bool ok = si < jlim;
                        const float dx = (staged(W.ipa, k, 0) + -pj[0]) + (staged(W.ipc, k, 0) + -lj[0]);
                        const float dy = (staged(W.ipa, k, 1) + -pj[1]) + (staged(W.ipc, k, 1) + -lj[1]);
                        const float dz = (staged(W.ipb, k, 0) + -pj[2]) + (staged(W.ipb, k, 1) + -lj[2]);
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (!(valid && ok && r2 < rc2hi) || loop_hit(r2, rc2lo)) continue;
                        if (loop_close(r2, rc2lo)) {
                            double F[3];
                            const double s6d = pair_force_f64(a.x, a.y, a.z, si, sj, sL, F);
                            atomicAdd(&W.corr64[k][0], F[0]);
                            atomicAdd(&W.corr64[k][1], F[1]);
                            atomicAdd(&W.corr64[k][2], F[2]);
                            cj[0] -= F[0]; cj[1] -= F[1]; cj[2] -= F[2];
                            if (STATS) {
                                const float s6 = (float)s6d;
                                e6.x += s6;
                                e12.x = fmaf(s6, s6, e12.x);
                                npair += 1;
                            }
                        } else if (exact_inside(a, g.rc2, si, sj, sL)) {
                            const float inv = rcp_nr(r2);
                            const float s6 = inv * inv * inv;
                            const float f = (s6 * inv) * fmaf(48.0f, s6, -24.0f);
                            atomicAdd(&W.corr[k][0], f * dx);
                            atomicAdd(&W.corr[k][1], f * dy);
                            atomicAdd(&W.corr[k][2], f * dz);
                            fjx = fmaf(-f, dx, fjx); fjy = fmaf(-f, dy, fjy); fjz = fmaf(-f, dz, fjz);
                            if (STATS) {
                                e6.x += s6;
                                e12.x = fmaf(s6, s6, e12.x);
                                npair += 1;
                            }
                        }
                    }
                }
                if (valid) write_force<kAtomic, true, float>(a, sj, fjx, fjy, fjz, cj[0], cj[1], cj[2]);
            }
            __syncwarp();
        }
        float ax[NI], ay[NI], az[NI];
#pragma unroll
        for (int k = 0; k < NI / 2; ++k) {
            ax[2 * k] = ax2[k].x; ax[2 * k + 1] = ax2[k].y;
            ay[2 * k] = ay2[k].x; ay[2 * k + 1] = ay2[k].y;
            az[2 * k] = az2[k].x; az[2 * k + 1] = az2[k].y;
        }
        // the listing is rebuilt for the next centre chunk: its space holds
        // the column sums
        write_i_chunk<true, NI, kAtomic>(a, W, ax, ay, az, a0, i0, na, lane);
        if (STATS) {
            kahan_add(le.s6, e6.x + e6.y);
            kahan_add(le.s12, e12.x + e12.y);
            le.pairs += npair;
        }
    }
}

template <bool STATS>
__global__ void __launch_bounds__(kRowWarps * 32, 1) k_force_rows(ForceArgs a, RowArgs r) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowSlot *slot = reinterpret_cast<RowSlot *>(smem_raw);
    RowWarp *wsm = reinterpret_cast<RowWarp *>(smem_raw + kRowSlots * sizeof(RowSlot));
    __shared__ int s_next, s_end;
    __shared__ float s_sh[27][3], s_sl[27][3];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int w = blockIdx.x * kRowWarps + wib;
    for (int k = threadIdx.x; k < 81; k += blockDim.x) {
        (&s_sh[0][0])[k] = (&a.sh[0][0])[k];
        (&s_sl[0][0])[k] = (&a.sl[0][0])[k];
    }
    if (threadIdx.x == 0) {
        s_next = 0;
        s_end = 0x7fffffff;
        for (int k = 0; k < kRowSlots; ++k) {
            slot[k].tag = -1;
            slot[k].group = -1;
            slot[k].done = 0;
            slot[k].phase = 0;
            mbar_init(&slot[k].bar, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    LaneEnergy le;
    le.s6 = make_float2(0.f, 0.f);
    le.s12 = make_float2(0.f, 0.f);
    le.d6 = le.d12 = 0.0;
    le.pairs = 0;
    bool ok = true;
    if (wib < kRowSlots) ok = row_stage(a, r, slot[wib], wib, &s_end, lane);
    while (ok) {
        int tl = 0;
        if (lane == 0) tl = atomicAdd(&s_next, 1);
        tl = __shfl_sync(kFull, tl, 0);
        const int li = tl / r.G, t = tl - li * r.G;
        RowSlot &S = slot[li % kRowSlots];
        const int st = row_wait(a, S, li, &s_end);
        if (st <= 0) break;
        if (t < S.ntask) row_task<STATS>(a, r, S, wsm[wib], t, lane, s_sh, s_sl, le);
        // count the task; the warp that counts the group's last one refills
        // the slot with the block's group li + kRowSlots
        __syncwarp();
        int d = 0;
        if (lane == 0) {
            __threadfence_block();
            d = atomicAdd(&S.done, 1) + 1;
            __threadfence_block();
        }
        d = __shfl_sync(kFull, d, 0);
        if (d == r.G) ok = row_stage(a, r, S, li + kRowSlots, &s_end, lane);
    }
    double s6 = f32_to_f64_bits(le.s6.x) - f32_to_f64_bits(le.s6.y);
    double s12 = f32_to_f64_bits(le.s12.x) - f32_to_f64_bits(le.s12.y);
    long long np = le.pairs;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        s6 += __shfl_xor_sync(kFull, s6, m);
        s12 += __shfl_xor_sync(kFull, s12, m);
        np += __shfl_xor_sync(kFull, np, m);
    }
    if (STATS && lane == 0) {
        a.warp_acc[4 * w + 0] += s6;
        a.warp_acc[4 * w + 1] += s12;
        a.warp_pairs[w] += np;
    }
}

// ------------------------------------------------ device task DAG ----
// Sec. VI, Strategy 2 and Sec. III / V: the tasks of one creation order run
// as a dependency-counted DAG.  A persistent warp claims the next queue slot,
// waits (bounded) until a ready task is published there, runs it -- one
// cell-cell interaction, exclusive plain writes to both cells, which the DAG
// orders -- and then decrements its successors' counters; the warp that
// drops a counter to zero publishes that task.
struct DagArgs {
    const int *task, *succ_start, *succ;
    int *cnt, *queue, *ctrl, *err;
    int32_t *trace;              // optional [2T]: start and end stamps of each task
    int ntasks;
    long long wait_ns;           // limit of one wait for a queue slot
};

constexpr unsigned kDagMaxSpins = 1u << 24;   // second bound on one wait

// Task (A, k): k = 0 the intra-cell interaction of A, k = 1..13 the pair
// (A, A + half-shell offset k - 1).
__device__ __forceinline__ TaskCells dag_task(const ForceArgs &a, int A, int k) {
    TaskCells tc;
    tc.g = &a.g; tc.sh = a.sh; tc.sl = a.sl; tc.cell_off = 0; tc.box = 0;
    tc.A = A;
    cell_xyz(a.g, A, tc.cA);
    tc.self = (k == 0);
    tc.nself = tc.self ? 1 : 0;
    tc.pairx = 0;
    tc.group = k > 0 ? k - 1 : 0;
    tc.dims = a.g.dims;
    tc.nnb = 1;
    return tc;
}

template <bool MIXED, int NI>
__global__ void __launch_bounds__(256, MIXED ? 2 : 1) k_force_dag(ForceArgs a, DagArgs d) {
    using T = typename std::conditional<MIXED, float, double>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    WarpSmem<T> &sm = reinterpret_cast<WarpSmem<T> *>(smem_raw)[wib];
    const int w = blockIdx.x * (blockDim.x >> 5) + wib;
    LaneEnergy le;
    le.s6 = make_float2(0.f, 0.f);
    le.s12 = make_float2(0.f, 0.f);
    le.d6 = le.d12 = 0.0;
    le.pairs = 0;
    int next = -1;   // a successor this warp made ready and runs itself (continuation)
    for (;;) {
        int tid = next;
        next = -1;
        if (tid < 0) {
            int pos = 0;
            if (lane == 0) pos = atomicAdd(d.ctrl + 0, 1);
            pos = __shfl_sync(kFull, pos, 0);
            if (pos >= d.ntasks) break;
            if (lane == 0) {
                // wait for a task to be published at this slot, or for every
                // task to be done (tasks run as continuations are never
                // published, so the last slots stay empty)
                const unsigned long long t0 = global_ns();
                bool gave_up = true;
                for (unsigned it = 0; it < kDagMaxSpins; ++it) {
                    tid = ld_acquire(d.queue + pos);
                    if (tid >= 0) { gave_up = false; break; }
                    if (ld_acquire(d.ctrl + 3) >= d.ntasks) { gave_up = false; break; }   // all done
                    if ((it & 15) == 15) {
                        if (ld_acquire(d.err) & kErrTimeout) break;              // another warp gave up
                        if ((long long)(global_ns() - t0) > d.wait_ns) break;
                    }
                    __nanosleep(200);
                }
                if (gave_up) { atomicOr(d.err, kErrTimeout); tid = -1; }
            }
            tid = __shfl_sync(kFull, tid, 0);
            __syncwarp();               // order the lanes' reads after lane 0's acquire
            if (tid < 0) break;
        }
        if (d.trace && lane == 0) d.trace[2 * tid] = atomicAdd(d.ctrl + 2, 1);
        const int code = d.task[tid];
        const TaskCells tc = dag_task(a, code >> 4, code & 15);
        if constexpr (MIXED) {
            const NbPre pre = load_neighbours<kDag>(a, tc, lane);
            commit_neighbours(sm, tc, pre, lane);
            run_task_mixed<NI, kDag, true, false>(a, sm, tc, pre, lane, le);
        } else {
            run_task_fp64<NI, kDag, false>(a, sm, tc, lane, le);
        }
        // the lanes' force writes are ordered before every lane's release
        // below by the warp barrier (release is cumulative)
        __syncwarp();
        if (d.trace && lane == 0) d.trace[2 * tid + 1] = atomicAdd(d.ctrl + 2, 1);
        const int e1 = d.succ_start[tid + 1];
        for (int e = d.succ_start[tid] + lane; e < e1; e += kWarp) {
            const int sc = d.succ[e];
            // acquire-release decrement: it releases this task's writes, and
            // the decrement that reaches zero acquires those of every
            // predecessor (they released theirs on the same counter)
            const bool ready = atom_add_acq_rel(d.cnt + sc, -1) == 1;
            // the first ready successor (lowest lane, first round) becomes
            // this warp's next task; the others are published
            const unsigned m = __ballot_sync(__activemask(), ready);
            const bool keep = ready && next < 0 && lane == __ffs(m) - 1;
            if (ready && !keep) {
                const int p = atomicAdd(d.ctrl + 1, 1);
                st_release(d.queue + p, sc);
            }
            const int kept = __shfl_sync(__activemask(), keep ? sc : -1, m ? __ffs(m) - 1 : 0);
            if (next < 0 && m) next = kept;
        }
        next = __shfl_sync(kFull, next, 0);
        if (lane == 0) atomicAdd(d.ctrl + 3, 1);   // tasks done
        if (next >= 0) {
            // the lane whose decrement reached zero acquired the
            // predecessors' writes; the warp barrier carries that order to
            // the other lanes
            __syncwarp();
        }
    }
    double s6 = MIXED ? (f32_to_f64_bits(le.s6.x) - f32_to_f64_bits(le.s6.y)) : le.d6;
    double s12 = MIXED ? (f32_to_f64_bits(le.s12.x) - f32_to_f64_bits(le.s12.y)) : le.d12;
    long long np = le.pairs;
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        s6 += __shfl_xor_sync(kFull, s6, m);
        s12 += __shfl_xor_sync(kFull, s12, m);
        np += __shfl_xor_sync(kFull, np, m);
    }
    if (lane == 0) {
        a.warp_acc[4 * w + 0] += s6;
        a.warp_acc[4 * w + 1] += s12;
        a.warp_pairs[w] += np;
    }
}

// Colour + mixed: Kahan accumulators -> FP64 forces.
__global__ void k_kahan_finalize(int n, const float2 *kx, const float2 *ky, const float2 *kz,
                                 double *fx, double *fy, double *fz) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        float2 a = kx[s], b = ky[s], c = kz[s];
        fx[s] = (double)a.x - (double)a.y;
        fy[s] = (double)b.x - (double)b.y;
        fz[s] = (double)c.x - (double)c.y;
    }
}

// ------------------------------------------------------ schedule check ----
// Replays a schedule's task enumeration: each task stamps the cells it
// writes (colour schedule: with its phase; a second stamp in the same phase
// is a conflict) and counts its visits of every (cell, offset) pair.
template <int MODE>
__global__ void k_check(Grid g, int group, int colour, int ntasks, int phase, int *stamp,
                        unsigned long long *visit, unsigned long long *counters) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntasks; t += gridDim.x * blockDim.x) {
        TaskCells tc;
        single_task<MODE>(g, group, colour, t, tc);
        for (int k = 0; k < tc.nnb; ++k) {
            int o[3];
            task_offset<MODE>(group, k, tc.self, tc.dims, o);
            int c[3];
            for (int d = 0; d < 3; ++d) {
                c[d] = tc.cA[d] + o[d];
                if (c[d] >= g.nc[d]) c[d] -= g.nc[d];
                else if (c[d] < 0) c[d] += g.nc[d];
            }
            int B = c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
            int oi = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);   // 0..26
            atomicAdd(visit + (size_t)tc.A * 27 + oi, 1ull);
            (void)B;
        }
    }
}

// Replays the colour schedule's colour k: every cell A of colour k stamps the
// cells its task writes (A and A + o for the forward offsets, all distinct)
// with k; a cell stamped twice within one colour is written by two tasks of
// that colour (a conflict).  Each task counts its visits of (A, o).
__global__ void k_check_cs(Grid g, int k, const int *cs_cell, const int8_t *cs_rank,
                           const unsigned long long *cs_dep, int *stamp, unsigned long long *visit,
                           unsigned long long *counters) {
    // the queue's own tables: the cells at colour k's queue positions, each
    // of which must carry colour k in the per-cell table the waits read
    const int first = g.cs_first[k], ntask = g.cs_first[k + 1] - first;
    const Stencil &S = stencil(g.dims);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntask; t += gridDim.x * blockDim.x) {
        const int Ai = cs_cell[first + t];
        if ((int)cs_rank[Ai] != k) atomicAdd(counters + 0, 1ull);
        int cA[3];
        cell_coords(g, Ai, cA);
        const size_t A = (size_t)Ai;
        // the waits' mask: exactly the dependence cells of an earlier colour
        for (int e = 0; e < S.ndep; ++e) {
            int n[3];
            for (int d = 0; d < 3; ++d) n[d] = (cA[d] + S.dep[e][d] + g.nc[d]) % g.nc[d];
            const bool earlier = (int)cs_rank[n[0] + g.nc[0] * (n[1] + g.nc[1] * n[2])] < k;
            if (earlier != (((cs_dep[Ai] >> e) & 1ull) != 0)) atomicAdd(counters + 0, 1ull);
        }
        for (int h = -1; h < S.nh; ++h) {
            int o[3] = {0, 0, 0};
            if (h >= 0) { o[0] = S.hs[h][0]; o[1] = S.hs[h][1]; o[2] = S.hs[h][2]; }
            int c[3];
            for (int d = 0; d < 3; ++d) c[d] = (cA[d] + o[d] + g.nc[d]) % g.nc[d];
            if (atomicExch(stamp + c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]), k) == k) atomicAdd(counters + 0, 1ull);
            atomicAdd(visit + A * 27 + (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1), 1ull);
        }
    }
}

// Expected visits: 1 for the centre and the half-shell offsets (Newton-3
// schedules) or all 27 offsets (full shell), 0 otherwise.
__global__ void k_check_cover(Grid g, int full, const unsigned long long *visit, unsigned long long *counters) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.ncell * 27; t += gridDim.x * blockDim.x) {
        int oi = t % 27;
        int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, oi / 9 - 1};
        bool fwd = (o[2] > 0) || (o[2] == 0 && o[1] > 0) || (o[2] == 0 && o[1] == 0 && o[0] > 0);
        bool centre = (o[0] == 0 && o[1] == 0 && o[2] == 0);
        const bool in_plane = g.dims != 2 || o[2] == 0;     // 2D: offsets in the x-y plane only
        unsigned long long want = (in_plane && (full || fwd || centre)) ? 1ull : 0ull;
        if (visit[t] != want) atomicAdd(counters + 1, 1ull);
    }
}

// ------------------------------------------------------------ launchers --
template <bool MIXED, int NI>
static size_t smem_bytes(int warps) {
    using T = typename std::conditional<MIXED, float, double>::type;
    return sizeof(WarpSmem<T>) * (size_t)warps;
}

// Warps per block of the per-warp-task kernels (a setting of 16 selects the
// row-group kernel for the atomic schedule; the others run 8).
static int task_warps(const Ctx *c) { return c->warps > 8 ? 8 : c->warps; }

// One resident wave: SMs x the blocks that fit on an SM (cached per shape).
template <bool MIXED, int NI, int MODE, bool STATS, bool BATCHED, bool PX = false>
static int force_blocks(Ctx *c) {
    static int cache[17] = {0};
    const int warps = task_warps(c);
    if (!cache[warps]) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force<MIXED, NI, MODE, STATS, BATCHED, PX>, warps * 32,
                                                      smem_bytes<MIXED, NI>(warps));
        if (per_sm < 1) per_sm = 1;
        cache[warps] = per_sm;
    }
    int blocks = c->num_sms * cache[warps];
    const int maxb = c->nwarp_max / warps;
    return blocks < maxb ? blocks : maxb;
}

template <bool MIXED, int NI, int MODE, bool STATS, bool BATCHED, bool PX = false>
static cudaError_t launch_one(Ctx *c, ForceArgs &a, cudaStream_t s) {
    const int warps = task_warps(c);
    const size_t sm = smem_bytes<MIXED, NI>(warps);
    const int blocks = force_blocks<MIXED, NI, MODE, STATS, BATCHED, PX>(c);
    if (STATS && !BATCHED && MODE != kColourQ) c->nwarp_used = blocks;   // one statistics slot per block
    else if (blocks * warps > c->nwarp_used) c->nwarp_used = blocks * warps;
    k_force<MIXED, NI, MODE, STATS, BATCHED, PX><<<blocks, warps * 32, sm, s>>>(a);
    return cudaGetLastError();
}

template <bool MIXED, int NI, int MODE>
static cudaError_t launch_mode(Ctx *c, ForceArgs &a, cudaStream_t s, bool stats) {
    // the FP64 comparator always accumulates its statistics; batches run
    // the centre-cell tile of 16 (atomic and full-shell schedules)
    if constexpr (MODE == kColourQ && NI == 16) {
        if (c->nbox > 0) {   // the colour queue over the boxes' cells
            if (!MIXED || stats) return launch_one<MIXED, NI, MODE, true, true>(c, a, s);
            return launch_one<MIXED, NI, MODE, (MIXED ? false : true), true>(c, a, s);
        }
    }
    if constexpr (MODE != kColourQ && NI == 16) {
        if (c->nbox > 0) {
            if (!MIXED || stats) return launch_one<MIXED, NI, MODE, true, true>(c, a, s);
            return launch_one<MIXED, NI, MODE, (MIXED ? false : true), true>(c, a, s);
        }
    }
    if constexpr (MIXED && MODE == kAtomic) {
        if (a.pairx) {   // two-cell tasks (2D)
            if (stats) return launch_one<true, NI, kAtomic, true, false, true>(c, a, s);
            return launch_one<true, NI, kAtomic, false, false, true>(c, a, s);
        }
    }
    if (!MIXED || stats) return launch_one<MIXED, NI, MODE, true, false>(c, a, s);
    return launch_one<MIXED, NI, MODE, (MIXED ? false : true), false>(c, a, s);
}

// Row-group kernel of the atomic schedule: the group geometry (runs of up
// to kRowGMax centre cells per row, equal lengths) and one block of 16 warps
// per SM.
static size_t rows_smem() { return kRowSlots * sizeof(RowSlot) + kRowWarps * sizeof(RowWarp); }

static RowArgs row_args(const Ctx *c) {
    RowArgs r;
    r.nseg = (c->g.nc[0] + kRowGMax - 1) / kRowGMax;
    r.G = (c->g.nc[0] + r.nseg - 1) / r.nseg;
    r.ngroups = r.nseg * c->g.nc[1] * c->g.nc[2];
    return r;
}

// The row-group kernel serves single 3D boxes in mixed precision with the
// centre tile of 16 when the tile setting asks for it (warps = 16).
static bool use_rows(const Ctx *c) {
    return c->warps == 16 && c->ni == 16 && c->nbox == 0 && c->g.dims == 3 && c->prec == LC_PREC_MIXED;
}

static cudaError_t launch_rows(Ctx *c, ForceArgs &a, cudaStream_t s, bool stats) {
    RowArgs r = row_args(c);
    a.err = c->d_err;
    a.wait_ns = (long long)(c->cs_wait_s * 1.0e9);
    const int blocks = c->num_sms;
    if (blocks * kRowWarps > c->nwarp_used) c->nwarp_used = blocks * kRowWarps;
    if (stats) k_force_rows<true><<<blocks, kRowWarps * 32, rows_smem(), s>>>(a, r);
    else k_force_rows<false><<<blocks, kRowWarps * 32, rows_smem(), s>>>(a, r);
    return cudaGetLastError();
}

// FP32 shift tables o * h = sh + sl for the 27 offsets.
static void fill_shift_tables(const Ctx *c, ForceArgs &a) {
    for (int oi = 0; oi < 27; ++oi) {
        const int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, oi / 9 - 1};
        for (int d = 0; d < 3; ++d) {
            const double S = (double)o[d] * c->g.h[d];
            const float Sh = (float)S;
            a.sh[oi][d] = Sh;
            a.sl[oi][d] = (float)(S - (double)Sh);
        }
    }
}

template <bool MIXED, int NI>
static cudaError_t launch_sched(Ctx *c, lc_schedule sched, cudaStream_t s, int *launches, bool stats) {
    ForceArgs a;
    a.g = c->g;
    a.p4 = c->d_p4;
    a.x = c->cur.x; a.y = c->cur.y; a.z = c->cur.z;
    a.start = c->d_start; a.count = c->d_count;
    a.fx = c->fx; a.fy = c->fy; a.fz = c->fz;
    a.kx = c->kx; a.ky = c->ky; a.kz = c->kz;
    a.warp_acc = c->d_warp_acc; a.warp_pairs = c->d_warp_pairs;
    a.group = 0; a.colour = 0;
    a.pairx = 0;
    a.stats = stats ? 1 : 0;
    a.boxes = c->d_boxes;
    a.cell_box = c->d_cell_box;
    a.box_acc = c->d_box_acc;
    a.box_pairs = c->d_box_pairs;
    a.bf = static_cast<float *>(c->d_fbuf);
    a.bd = static_cast<double *>(c->d_fbuf);
    a.n = (size_t)c->n;
    fill_shift_tables(c, a);
    cudaError_t e = cudaSuccess;
    const size_t nbytes = sizeof(double) * (size_t)c->n;
    if (sched == LC_SCHED_COLOUR) {
        // cell tasks in colour order on the device queue
        e = cudaMemsetAsync(c->fx, 0, 3 * nbytes, s);
        if (e) return e;
        a.ntasks = c->nbox > 0 ? c->cs_nitems : c->g.ncell;   // batch: one item per cell
        if ((e = cudaMemsetAsync(c->d_cs_done, 0, sizeof(int) * (size_t)c->g.ncell, s))) return e;
        if ((e = cudaMemsetAsync(c->d_cs_ctrl, 0, sizeof(int) * 2, s))) return e;
        a.cs_done = c->d_cs_done;
        a.cs_ctrl = c->d_cs_ctrl;
        a.err = c->d_err;
        a.wait_ns = (long long)(c->cs_wait_s * 1.0e9);
        a.withhold = c->cs_withhold;
        a.cell_acc = c->d_cell_acc;
        a.cell_pairs = c->d_cell_pairs;
        a.cs_items = c->d_cs_items;
        a.cs_cell = c->d_cs_cell;
        a.cs_rank = c->d_cs_rank;
        a.cs_dep = c->d_cs_dep;
        e = launch_mode<MIXED, NI, kColourQ>(c, a, s, stats);
        if (e) return e;
        ++*launches;
    } else if (sched == LC_SCHED_ATOMIC) {
        e = cudaMemsetAsync(c->fx, 0, 3 * nbytes, s);
        if (e) return e;
        a.ntasks = c->g.ncell;   // a batch: the total cell count of all boxes
        if (MIXED && c->nbox == 0 && c->g.dims == 2) {
            // sparse 2D cells: two x-adjacent cells per task (half the tasks)
            a.pairx = 1;
            a.ntasks = ((c->g.nc[0] + 1) / 2) * c->g.nc[1];
        }
        if (MIXED && NI == 16 && use_rows(c)) e = launch_rows(c, a, s, stats);
        else e = launch_mode<MIXED, NI, kAtomic>(c, a, s, stats);
        ++*launches;
    } else if (sched == LC_SCHED_BUFFER) {
        // every buffer entry is written by its one task: no clearing
        using T = typename std::conditional<MIXED, float, double>::type;
        a.ntasks = c->g.ncell;
        e = launch_mode<MIXED, NI, kBuffer>(c, a, s, stats);
        ++*launches;
        if (e) return e;
        k_buffer_reduce<T><<<c->num_sms * 8, 256, 0, s>>>((size_t)c->n, static_cast<const T *>(c->d_fbuf),
                                                         c->fx, c->fy, c->fz);
        ++*launches;
        e = cudaGetLastError();
    } else {
        a.ntasks = c->g.ncell;
        e = launch_mode<MIXED, NI, kFullShell>(c, a, s, stats);
        ++*launches;
    }
    return e;
}

template <bool MIXED>
static cudaError_t launch_dag(Ctx *c, const DagDev *dd, long long wait_ns, int32_t *trace, cudaStream_t s) {
    ForceArgs a;
    memset(&a, 0, sizeof(a));
    a.g = c->g;
    a.p4 = c->d_p4;
    a.x = c->cur.x; a.y = c->cur.y; a.z = c->cur.z;
    a.start = c->d_start; a.count = c->d_count;
    a.fx = c->fx; a.fy = c->fy; a.fz = c->fz;
    a.kx = c->kx; a.ky = c->ky; a.kz = c->kz;
    a.warp_acc = c->d_warp_acc; a.warp_pairs = c->d_warp_pairs;
    a.stats = 1;
    fill_shift_tables(c, a);
    DagArgs d;
    d.task = dd->task; d.succ_start = dd->succ_start; d.succ = dd->succ;
    d.cnt = dd->cnt; d.queue = dd->queue; d.ctrl = dd->ctrl; d.err = c->d_err;
    d.trace = trace;
    d.ntasks = dd->ntasks;
    d.wait_ns = wait_ns;
    const int warps = task_warps(c);
    const size_t smem = smem_bytes<MIXED, 16>(warps);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_force_dag<MIXED, 16>, warps * 32, smem);
    if (e) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int blocks = c->num_sms * per_sm;
    if (blocks > c->nwarp_max / warps) blocks = c->nwarp_max / warps;
    // a DAG with little parallelism (tasks / critical path of a few, as in
    // the cell-major creation orders) gets eight warps per unit of it, at
    // least four blocks: fewer warps polling the queue shortens every hand-off
    const double width = (double)dd->ntasks / (double)(dd->critical_path > 0 ? dd->critical_path : 1);
    const double want = ceil(8.0 * width / warps);
    if (want < (double)blocks) blocks = want < 4.0 ? (blocks < 4 ? blocks : 4) : (int)want;
    c->nwarp_used = blocks * warps;
    // every warp may wait for another one: all of them must be resident
    void *args[] = {&a, &d};
    return cudaLaunchCooperativeKernel((const void *)k_force_dag<MIXED, 16>, dim3(blocks), dim3(warps * 32), args,
                                      smem, s);
}

cudaError_t launch_forces_dag(Ctx *c, const DagDev *d, long long wait_ns, int withhold, int32_t *trace,
                              cudaStream_t s, int *launches) {
    cudaError_t e;
    const bool mixed = (c->prec == LC_PREC_MIXED);
    if ((e = cudaMemsetAsync(c->d_warp_acc, 0, sizeof(double) * 4 * (size_t)c->nwarp_max, s))) return e;
    if ((e = cudaMemsetAsync(c->d_warp_pairs, 0, sizeof(long long) * (size_t)c->nwarp_max, s))) return e;
    if (mixed) e = cudaMemsetAsync(c->kx, 0, 3 * sizeof(float2) * (size_t)c->n, s);
    else e = cudaMemsetAsync(c->fx, 0, 3 * sizeof(double) * (size_t)c->n, s);
    if (e) return e;
    if ((e = cudaMemcpyAsync(d->cnt, d->pred_count, sizeof(int) * (size_t)d->ntasks, cudaMemcpyDeviceToDevice, s)))
        return e;
    if ((e = cudaMemcpyAsync(d->queue, d->queue_init, sizeof(int) * (size_t)d->ntasks, cudaMemcpyDeviceToDevice, s)))
        return e;
    if ((e = cudaMemcpyAsync(d->ctrl, d->ctrl_init, sizeof(int) * 4, cudaMemcpyDeviceToDevice, s))) return e;
    if (withhold) {   // nothing published: every wait for a queue slot runs out
        if ((e = cudaMemsetAsync(d->queue, 0xff, sizeof(int) * (size_t)d->ntasks, s))) return e;
        if ((e = cudaMemsetAsync(d->ctrl + 1, 0, sizeof(int), s))) return e;
    }
    e = mixed ? launch_dag<true>(c, d, wait_ns, trace, s) : launch_dag<false>(c, d, wait_ns, trace, s);
    if (e) return e;
    ++*launches;
    if (mixed) {
        k_kahan_finalize<<<c->num_sms * 8, 256, 0, s>>>((int)c->n, c->kx, c->ky, c->kz, c->fx, c->fy, c->fz);
        ++*launches;
        if ((e = cudaGetLastError())) return e;
    }
    c->stats_full = 0;
    e = launch_energy_reduce(c, s, 0);
    ++*launches;
    return e;
}

// The sweeps whose statistics come as one slot per block (block_stats),
// written by the launch itself: one launch of k_force over a single box,
// the colour queue excepted (its per-cell partials are summed in cell order
// afterwards).  Their slots need no clearing.
static bool block_slots(const Ctx *c, lc_schedule sched) {
    if (c->nbox > 0) return false;
    if (sched == LC_SCHED_ATOMIC) return !(c->ni == 16 && use_rows(c));
    return sched == LC_SCHED_FULLSHELL || sched == LC_SCHED_BUFFER;
}

// pot_deferred (non-null): the final sum of a single box's statistics slots
// is left to the caller's next kernel (the closing kick) and *pot_deferred
// says whether it was.
cudaError_t launch_forces(Ctx *c, lc_schedule sched, cudaStream_t s, int *launches, bool stats,
                          bool *pot_deferred) {
    if (pot_deferred) *pot_deferred = false;
    cudaError_t e;
    const bool mixed = (c->prec == LC_PREC_MIXED);
    if (!mixed) stats = true;
    if (stats && !block_slots(c, sched)) {
        if (c->nbox > 0) {
            if ((e = cudaMemsetAsync(c->d_box_acc, 0, sizeof(double) * 2 * (size_t)c->nbox, s))) return e;
            if ((e = cudaMemsetAsync(c->d_box_pairs, 0, sizeof(unsigned long long) * (size_t)c->nbox, s))) return e;
        } else {
            if ((e = cudaMemsetAsync(c->d_warp_acc, 0, sizeof(double) * 4 * (size_t)c->nwarp_max, s))) return e;
            if ((e = cudaMemsetAsync(c->d_warp_pairs, 0, sizeof(long long) * (size_t)c->nwarp_max, s))) return e;
        }
    }
    c->nwarp_used = 0;
    if (c->ni == 8 && c->nbox == 0)
        e = mixed ? launch_sched<true, 8>(c, sched, s, launches, stats) : launch_sched<false, 8>(c, sched, s, launches, stats);
    else
        e = mixed ? launch_sched<true, 16>(c, sched, s, launches, stats) : launch_sched<false, 16>(c, sched, s, launches, stats);
    if (e) return e;
    if (stats) {
        c->stats_full = (sched == LC_SCHED_FULLSHELL);
        if (c->nbox > 0 && sched == LC_SCHED_COLOUR) e = launch_box_energy_cells(c, s);
        else if (c->nbox > 0) e = launch_box_energy(c, s, sched == LC_SCHED_FULLSHELL);
        else if (sched == LC_SCHED_COLOUR) {   // per-cell partials, reduced in cell order (two kernels)
            e = launch_energy_reduce_parts(c, s, 0, c->d_cell_acc, c->d_cell_pairs, c->g.ncell);
            ++*launches;
        } else if (pot_deferred) {
            *pot_deferred = true;
            return e;
        } else {
            e = launch_energy_reduce(c, s, sched == LC_SCHED_FULLSHELL);
        }
        ++*launches;
    }
    return e;
}

cudaError_t launch_schedule_check(Ctx *c, lc_schedule sched, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(c->d_stamp, 0xff, sizeof(int) * (size_t)c->g.ncell, s);
    if (e) return e;
    e = cudaMemsetAsync(c->d_visit, 0, sizeof(unsigned long long) * 27 * (size_t)c->g.ncell, s);
    if (e) return e;
    e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * 4, s);
    if (e) return e;
    const int blocks = c->num_sms * 4;
    if (sched == LC_SCHED_COLOUR) {
        for (int k = 0; k < c->g.cs_ncolours; ++k)
            k_check_cs<<<blocks, 256, 0, s>>>(c->g, k, c->d_cs_cell, c->d_cs_rank, c->d_cs_dep, c->d_stamp,
                                              c->d_visit, c->d_counters);
    } else if (sched == LC_SCHED_ATOMIC || sched == LC_SCHED_BUFFER) {
        k_check<kAtomic><<<blocks, 256, 0, s>>>(c->g, 0, 0, c->g.ncell, 0, c->d_stamp, c->d_visit, c->d_counters);
    } else {
        k_check<kFullShell><<<blocks, 256, 0, s>>>(c->g, 0, 0, c->g.ncell, 0, c->d_stamp, c->d_visit, c->d_counters);
    }
    k_check_cover<<<blocks, 256, 0, s>>>(c->g, sched == LC_SCHED_FULLSHELL, c->d_visit, c->d_counters);
    return cudaGetLastError();
}

template <bool MIXED, int NI, bool STATS>
static cudaError_t attrs_for() {
    cudaError_t e;
    const int bytes = (int)smem_bytes<MIXED, NI>(8);
    if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kColourQ, STATS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kAtomic, STATS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if constexpr (MIXED)
        if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kAtomic, STATS, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kFullShell, STATS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kBuffer, STATS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if constexpr (NI == 16) {
        if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kColourQ, STATS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
        if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kAtomic, STATS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
        if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kFullShell, STATS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
        if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kBuffer, STATS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    }
    return cudaSuccess;
}

// Opt the force kernels into the shared memory of the largest tile shape
// (called once per context, before any stream capture).
cudaError_t init_force_kernels() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_force_dag<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<true, 16>(8))) ||
        (e = cudaFuncSetAttribute(k_force_dag<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_bytes<false, 16>(8))))
        return e;
    if ((e = cudaFuncSetAttribute(k_force_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem())) ||
        (e = cudaFuncSetAttribute(k_force_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem())))
        return e;
    if ((e = attrs_for<true, 8, true>()) || (e = attrs_for<true, 16, true>()) || (e = attrs_for<true, 8, false>()) ||
        (e = attrs_for<true, 16, false>()) || (e = attrs_for<false, 8, true>()) || (e = attrs_for<false, 16, true>()))
        return e;
    return cudaSuccess;
}

cudaError_t upload_stencil(const Stencil &st3, const Stencil &st2) {
    cudaError_t e = cudaMemcpyToSymbol(c_st, &st3, sizeof(Stencil));
    if (!e) e = cudaMemcpyToSymbol(c_st2, &st2, sizeof(Stencil));
    return e;
}

}  // namespace lc
