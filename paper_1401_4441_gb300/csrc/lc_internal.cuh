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

// Rounding residuals of the FP32 cell-local coordinates are stored as
// q = rint(r * kLoScale), |q| <= 511, i.e. in units of 2^-23 / 511.
constexpr double kLoScale = 511.0 * 8388608.0;
constexpr float kLoUnit = (float)(1.0 / (511.0 * 8388608.0));

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
    float rc2f_lo, rc2f_hi;  // FP32 band around rc^2 for the mixed path
    int ncolours;
    int class_count[3][3];   // cells of colour class a along dimension d
    int colour_of_raw[27];   // raw colour cx + 3 cy + 9 cz -> colour rank (-1 absent)
    int raw_of_colour[27];   // inverse
};

// Offsets of the 27-cell stencil and the phase groups, in constant memory.
struct Stencil {
    int hs[13][3];      // forward half-shell, (z, y, x) lexicographic
    int group_of[13];   // phase group (0..3) of each half-shell offset
    int group_first[5]; // offsets of group g are group_list[group_first[g] .. group_first[g+1])
    int group_list[13];
    int full[27][3];    // all 27 offsets, centre first
};

void make_stencil(Stencil *s);
void make_grid(Grid *g, const double box[3], double rc);

// Double-buffered particle state in cell-sorted order.
struct State {
    double *x, *y, *z;     // wrapped positions
    double *vx, *vy, *vz;  // velocities
    int *id;               // particle ID of each slot
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
    int *d_blocksums;      // scan partials
    int8_t *d_colour;      // [ncell]
    float4 *d_p4;          // FP32 cell-centre-local coordinates, sorted
    // forces
    double *fx, *fy, *fz;  // FP64 forces in sorted order
    float2 *kx, *ky, *kz;  // Kahan (sum, compensation) accumulators, colour + mixed
    double *d_warp_acc;    // per-warp partials: [nwarp_max][4] (s6, s12, K, spare)
    long long *d_warp_pairs;
    double *d_kin_part;    // per-block partial sums of v^2
    double *d_result;      // [4] U, W, npairs (as double), K
    long long *d_npairs;
    int *d_err;
    int nwarp_max;
    // check buffers
    int *d_stamp;
    unsigned long long *d_visit;
    unsigned long long *d_counters;
    // status
    bool have_state, binned, forces_valid;
    int launches_force, launches_step;
    // graphs of two Verlet steps: one per (schedule, state-buffer parity)
    cudaGraphExec_t graph[6];
    double graph_dt[6];
    double *state_a;       // cur.x of buffer set A (parity reference)
};

// ---- kernels / launchers (stream-ordered, return cudaError_t) -------------
cudaError_t launch_bin(Ctx *c, cudaStream_t s, int *launches);
cudaError_t launch_forces(Ctx *c, lc_schedule sched, cudaStream_t s, int *launches);
cudaError_t launch_kick_drift(Ctx *c, double dt, cudaStream_t s);
cudaError_t launch_kick(Ctx *c, double dt, cudaStream_t s);
cudaError_t launch_kinetic(Ctx *c, cudaStream_t s);
cudaError_t launch_energy_reduce(Ctx *c, cudaStream_t s, int full);
cudaError_t launch_colour(Ctx *c, cudaStream_t s);
cudaError_t upload_stencil(const Stencil &st);
int kinetic_blocks(const Ctx *c);
cudaError_t launch_schedule_check(Ctx *c, lc_schedule sched, cudaStream_t s);
cudaError_t launch_unsort_vec(Ctx *c, const double *a, const double *b, const double *cc,
                              double *dst, cudaStream_t s, int wrap);
cudaError_t launch_set_state(Ctx *c, const double *pos, const double *vel, cudaStream_t s);
int force_grid_warps(const Ctx *c);
cudaError_t init_force_kernels();

// ---- small device helpers ----------------------------------------------------
// Periodic wrap into [0, L), each operation rounded once (no contraction):
// x - L floor(x / L), then one correction for the rounding edge cases.
__device__ __forceinline__ double wrap_coord(double x, double L) {
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

__host__ __device__ __forceinline__ int colour_class(int c, int nc) {
    return ((nc & 1) && c == nc - 1) ? 2 : (c & 1);
}

}  // namespace lc
