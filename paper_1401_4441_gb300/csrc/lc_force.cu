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

#include <type_traits>

#include "lc_internal.cuh"

namespace lc {

__constant__ Stencil c_st;

enum Mode : int { kColour = 0, kAtomic = 1, kFullShell = 2 };

constexpr int kJCap = 512;      // neighbour slots listed per batch (per warp)
constexpr int kMaxNb = 27;      // neighbour cells per task

struct ForceArgs {
    Grid g;
    const float4 *p4;
    const double *x, *y, *z;
    const int *start, *count;
    double *fx, *fy, *fz;
    float2 *kx, *ky, *kz;
    double *warp_acc;           // [W][4]
    long long *warp_pairs;      // [W]
    int group, colour;          // colour phase
    int ntasks;
};

// ---------------------------------------------------------------- tasks ----
struct TaskCells {
    int A;            // centre cell
    int cA[3];        // its coordinates
    int nnb;          // neighbour cells listed (self first when present)
    bool self;        // intra-cell interaction included
};

__device__ __forceinline__ void cell_xyz(const Grid &g, int c, int out[3]) {
    out[0] = c % g.nc[0];
    int r = c / g.nc[0];
    out[1] = r % g.nc[1];
    out[2] = r / g.nc[1];
}

// Task t of a colour phase: the t-th cell (x fastest) of colour `colour`.
__device__ __forceinline__ int colour_task_cell(const Grid &g, int colour, int t, int cA[3]) {
    int raw = g.raw_of_colour[colour];
    int a[3] = {raw % 3, (raw / 3) % 3, raw / 9};
    int n0 = g.class_count[0][a[0]], n1 = g.class_count[1][a[1]];
    int t3[3] = {t % n0, (t / n0) % n1, t / (n0 * n1)};
    for (int d = 0; d < 3; ++d) cA[d] = (a[d] == 2) ? g.nc[d] - 1 : 2 * t3[d] + a[d];
    return cA[0] + g.nc[0] * (cA[1] + g.nc[1] * cA[2]);
}

__device__ __forceinline__ int colour_ntasks(const Grid &g, int colour) {
    int raw = g.raw_of_colour[colour];
    int a[3] = {raw % 3, (raw / 3) % 3, raw / 9};
    return g.class_count[0][a[0]] * g.class_count[1][a[1]] * g.class_count[2][a[2]];
}

// Neighbour k of the task (k < nnb): offset and periodic image.
template <int MODE>
__device__ __forceinline__ void task_offset(int group, int k, bool self, int o[3]) {
    if (self) {
        if (k == 0) { o[0] = o[1] = o[2] = 0; return; }
        --k;
    }
    if (MODE == kFullShell) {            // all 27 offsets, centre first
        o[0] = c_st.full[k + 1][0]; o[1] = c_st.full[k + 1][1]; o[2] = c_st.full[k + 1][2];
    } else if (MODE == kAtomic) {
        o[0] = c_st.hs[k][0]; o[1] = c_st.hs[k][1]; o[2] = c_st.hs[k][2];
    } else {
        int kk = c_st.group_list[c_st.group_first[group] + k];
        o[0] = c_st.hs[kk][0]; o[1] = c_st.hs[kk][1]; o[2] = c_st.hs[kk][2];
    }
}

template <int MODE>
__device__ __forceinline__ TaskCells make_task(const Grid &g, int group, int colour, int t) {
    TaskCells tc;
    if (MODE == kColour) {
        tc.A = colour_task_cell(g, colour, t, tc.cA);
        tc.self = (group == 0);
        tc.nnb = (c_st.group_first[group + 1] - c_st.group_first[group]) + (tc.self ? 1 : 0);
    } else {
        tc.A = t;
        cell_xyz(g, t, tc.cA);
        tc.self = true;
        tc.nnb = (MODE == kFullShell) ? 27 : 14;
    }
    return tc;
}

// ----------------------------------------------------- per-warp scratch ----
template <typename T>
struct alignas(16) WarpSmem {
    T ix[32], iy[32], iz[32];   // centre-cell particles of the current i chunk
    int islot[32];
    int jl[kJCap];              // slot | (neighbour index << 26)
    int nb_start[kMaxNb], nb_count[kMaxNb], nb_cell[kMaxNb];
    float nb_sh[kMaxNb][3];     // o * h rounded to FP32 (mixed)
    float nb_sl[kMaxNb][3];     // o * h - nb_sh, rounded to FP32
    double nb_sL[kMaxNb][3];    // periodic image s * L in FP64
};

// Reciprocal: hardware approximation refined by one Newton-Raphson step
// y <- y (2 - r y), written as two FMAs.
__device__ __forceinline__ float rcp_nr(float r) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r));
    float e = fmaf(-r, y, 1.0f);
    return fmaf(y, e, y);
}

// Butterfly reduce-scatter of v[NI] over the 32 lanes of a warp.  On return
// lane l holds in v[0] the warp-wide sum of element (l / (32 / NI)) % NI.
template <typename T, int NI>
__device__ __forceinline__ void reduce_scatter(T (&v)[NI], int lane) {
#pragma unroll
    for (int half = NI / 2, m = 16; half >= 1; half >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            T send = up ? v[k] : v[k + half];
            T keep = up ? v[k + half] : v[k];
            v[k] = keep + __shfl_xor_sync(kFull, send, m);
        }
    }
    // remaining lanes above the NI split hold partial sums of the same element
#pragma unroll
    for (int m = 16 / NI; m >= 1; m >>= 1) v[0] += __shfl_xor_sync(kFull, v[0], m);
}

// Kahan-compensated accumulation of v into (s, c): true sum ~ s - c.
__device__ __forceinline__ void kahan_add(float2 &acc, float v) {
    float y = v - acc.y;
    float t = acc.x + y;
    acc.y = (t - acc.x) - y;
    acc.x = t;
}

template <int MODE, bool MIXED>
__device__ __forceinline__ void write_force(const ForceArgs &a, int slot, double vx, double vy, double vz) {
    if (MODE == kAtomic) {
        atomicAdd(a.fx + slot, vx);
        atomicAdd(a.fy + slot, vy);
        atomicAdd(a.fz + slot, vz);
    } else if (MODE == kFullShell) {
        a.fx[slot] = vx; a.fy[slot] = vy; a.fz[slot] = vz;
    } else if (MIXED) {
        float2 kx = a.kx[slot], ky = a.ky[slot], kz = a.kz[slot];
        kahan_add(kx, (float)vx); kahan_add(ky, (float)vy); kahan_add(kz, (float)vz);
        a.kx[slot] = kx; a.ky[slot] = ky; a.kz[slot] = kz;
    } else {
        a.fx[slot] += vx; a.fy[slot] += vy; a.fz[slot] += vz;
    }
}

// Exact FP64 cutoff decision, the definition's arithmetic (each op rounded once).
__device__ __forceinline__ bool exact_inside(const ForceArgs &a, int si, int sj, const double sL[3]) {
    double dx = __dsub_rn(__dsub_rn(a.x[si], a.x[sj]), sL[0]);
    double dy = __dsub_rn(__dsub_rn(a.y[si], a.y[sj]), sL[1]);
    double dz = __dsub_rn(__dsub_rn(a.z[si], a.z[sj]), sL[2]);
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < a.g.rc2;
}

// --------------------------------------------------------- the kernel -----
// Lane accumulators of one warp across its tasks.
struct LaneEnergy {
    float2 s6, s12;   // Kahan pairs (mixed)
    double d6, d12;   // FP64 sums (FP64 path)
    long long pairs;
};

template <bool MIXED, int NI, int MODE>
__device__ void run_task(const ForceArgs &a, WarpSmem<typename std::conditional<MIXED, float, double>::type> &sm,
                         const TaskCells &tc, int lane, LaneEnergy &le) {
    using T = typename std::conditional<MIXED, float, double>::type;
    constexpr bool N3 = (MODE != kFullShell);
    const Grid &g = a.g;

    // neighbour table: lane k fills entry k
    if (lane < tc.nnb) {
        int o[3];
        task_offset<MODE>(a.group, lane, tc.self, o);
        int c[3];
        double sL[3];
        for (int d = 0; d < 3; ++d) {
            c[d] = tc.cA[d] + o[d];
            sL[d] = 0.0;
            if (c[d] >= g.nc[d]) { c[d] -= g.nc[d]; sL[d] = g.L[d]; }
            else if (c[d] < 0) { c[d] += g.nc[d]; sL[d] = -g.L[d]; }
            const double S = (double)o[d] * g.h[d];
            const float Sh = (float)S;
            sm.nb_sh[lane][d] = Sh;
            sm.nb_sl[lane][d] = (float)(S - (double)Sh);
            sm.nb_sL[lane][d] = sL[d];
        }
        int B = c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
        sm.nb_cell[lane] = B;
        sm.nb_start[lane] = a.start[B];
        sm.nb_count[lane] = a.count[B];
    }
    __syncwarp();
    const int a0 = a.start[tc.A];
    const int na = a.count[tc.A];
    const T far_i = (T)1.0e15, far_j = (T)-1.0e15;
    const float rc2lo = g.rc2f_lo, rc2hi = g.rc2f_hi;
    const float rc2mid = 0.5f * (rc2lo + rc2hi), band = 0.5f * (rc2hi - rc2lo);
    const T rc2 = MIXED ? (T)0 : (T)g.rc2;

    for (int i0 = 0; i0 < na; i0 += NI) {
        // stage the i chunk
        if (lane < NI) {
            int ii = i0 + lane;
            if (ii < na) {
                int s = a0 + ii;
                if (MIXED) {
                    float4 p = a.p4[s];
                    sm.ix[lane] = (T)p.x; sm.iy[lane] = (T)p.y; sm.iz[lane] = (T)p.z;
                } else {
                    sm.ix[lane] = (T)a.x[s]; sm.iy[lane] = (T)a.y[s]; sm.iz[lane] = (T)a.z[s];
                }
                sm.islot[lane] = s;
            } else {
                sm.ix[lane] = far_i; sm.iy[lane] = far_i; sm.iz[lane] = far_i;
                sm.islot[lane] = 0x7fffffff;
            }
        }
        T ax[NI], ay[NI], az[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) { ax[k] = ay[k] = az[k] = (T)0; }
        T e6 = 0, e12 = 0;
        int npair = 0;
        __syncwarp();

        // walk the neighbour cells in batches of at most kJCap slots
        int b = 0, kin = 0;
        while (b < tc.nnb) {
            int nj = 0;
            while (b < tc.nnb && nj < kJCap) {
                int cnt = sm.nb_count[b] - kin;
                int take = min(cnt, kJCap - nj);
                int st = sm.nb_start[b] + kin;
                for (int k = lane; k < take; k += kWarp) sm.jl[nj + k] = (st + k) | (b << 26);
                nj += take;
                kin += take;
                if (kin >= sm.nb_count[b]) { ++b; kin = 0; }
            }
            __syncwarp();
            for (int jc = 0; jc < nj; jc += kWarp) {
                const int e = jc + lane;
                const bool valid = e < nj;
                int sj = 0x7fffffff, nb = 0;
                T pjx = far_j, pjy = far_j, pjz = far_j;
                // mixed: the j position in the centre cell's frame as an
                // unevaluated sum hi + lo (the shift o*h added by Fast2Sum,
                // |o*h| >= |x_j| whenever o != 0, plus the stored residual)
                float ljx = 0.f, ljy = 0.f, ljz = 0.f;
                if (valid) {
                    int w = sm.jl[e];
                    sj = w & ((1 << 26) - 1);
                    nb = w >> 26;
                    if (MIXED) {
                        const float4 p = a.p4[sj];
                        const unsigned q = __float_as_uint(p.w);
                        const float pin[3] = {p.x, p.y, p.z};
                        float hi[3], lo[3];
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            const float Sh = sm.nb_sh[nb][d];
                            const float s = Sh + pin[d];
                            const float err = pin[d] - (s - Sh);
                            const float res = (float)((int)((q >> (10 * d)) & 1023u) - 512) * kLoUnit;
                            hi[d] = s;
                            lo[d] = (err + res) + sm.nb_sl[nb][d];
                        }
                        pjx = hi[0]; pjy = hi[1]; pjz = hi[2];
                        ljx = lo[0]; ljy = lo[1]; ljz = lo[2];
                    } else {
                        pjx = (T)a.x[sj]; pjy = (T)a.y[sj]; pjz = (T)a.z[sj];
                    }
                }
                const bool is_self = valid && tc.self && nb == 0;
                // Newton-3 intra pairs need slot_i < slot_j; full shell skips i == j
                const int jlim = (N3 && is_self) ? sj : 0x7fffffff;
                const int jexcl = (!N3 && is_self) ? sj : -1;
                T sLx = 0, sLy = 0, sLz = 0;
                if (!MIXED) { sLx = (T)sm.nb_sL[nb][0]; sLy = (T)sm.nb_sL[nb][1]; sLz = (T)sm.nb_sL[nb][2]; }
                T fjx = 0, fjy = 0, fjz = 0;
                bool amb = false;
#pragma unroll
                for (int k = 0; k < NI; ++k) {
                    const int si = sm.islot[k];
                    const bool ok = N3 ? (si < jlim) : (si != jexcl);
                    T dx, dy, dz, r2;
                    if (MIXED) {
                        dx = (sm.ix[k] - pjx) - (T)ljx;
                        dy = (sm.iy[k] - pjy) - (T)ljy;
                        dz = (sm.iz[k] - pjz) - (T)ljz;
                        r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    } else {
                        dx = __dsub_rn(__dsub_rn(sm.ix[k], pjx), sLx);
                        dy = __dsub_rn(__dsub_rn(sm.iy[k], pjy), sLy);
                        dz = __dsub_rn(__dsub_rn(sm.iz[k], pjz), sLz);
                        r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    }
                    bool hit;
                    T inv;
                    if (MIXED) {
                        hit = ok && ((float)r2 < rc2lo);
                        amb |= ok && (fabsf((float)r2 - rc2mid) < band);
                        inv = (T)rcp_nr((float)r2);
                        inv = hit ? inv : (T)0;   // masks r2 = 0 (i == j) as well
                    } else {
                        hit = ok && (r2 < rc2);
                        inv = hit ? (T)1.0 / r2 : (T)0;
                    }
                    const T s6 = inv * inv * inv;
                    const T f = (s6 * inv) * ((T)48 * s6 - (T)24);
                    ax[k] += f * dx; ay[k] += f * dy; az[k] += f * dz;
                    if (N3) { fjx -= f * dx; fjy -= f * dy; fjz -= f * dz; }
                    e6 += s6;
                    e12 += s6 * s6;
                    npair += hit ? 1 : 0;
                }
                if (MIXED && __any_sync(kFull, amb)) {
                    // candidates near r_c: decide with the FP64 definition
                    double sL[3] = {sm.nb_sL[nb][0], sm.nb_sL[nb][1], sm.nb_sL[nb][2]};
#pragma unroll
                    for (int k = 0; k < NI; ++k) {
                        const int si = sm.islot[k];
                        const bool ok = N3 ? (si < jlim) : (si != jexcl);
                        float dx = ((float)sm.ix[k] - (float)pjx) - ljx;
                        float dy = ((float)sm.iy[k] - (float)pjy) - ljy;
                        float dz = ((float)sm.iz[k] - (float)pjz) - ljz;
                        float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (valid && ok && fabsf(r2 - rc2mid) < band && exact_inside(a, si, sj, sL)) {
                            float inv = rcp_nr(r2);
                            float s6 = inv * inv * inv;
                            float f = (s6 * inv) * (48.0f * s6 - 24.0f);
                            ax[k] += (T)(f * dx); ay[k] += (T)(f * dy); az[k] += (T)(f * dz);
                            if (N3) { fjx -= (T)(f * dx); fjy -= (T)(f * dy); fjz -= (T)(f * dz); }
                            e6 += (T)s6;
                            e12 += (T)(s6 * s6);
                            npair += 1;
                        }
                    }
                }
                if (N3 && valid) write_force<MODE, MIXED>(a, sj, (double)fjx, (double)fjy, (double)fjz);
            }
            __syncwarp();
        }
        // the i chunk's forces: reduce-scatter over lanes, owners write
        reduce_scatter<T, NI>(ax, lane);
        reduce_scatter<T, NI>(ay, lane);
        reduce_scatter<T, NI>(az, lane);
        __syncwarp();   // order the j-side writes to A before the i-side ones
        // element held by this lane after the butterfly: bit (4 - k) of the
        // lane selects bit (log2 NI - 1 - k) of the element index
        int bits = 0;
        for (int n = NI; n > 1; n >>= 1) ++bits;
        int elem = 0;
        for (int k = 0; k < bits; ++k) elem |= ((lane >> (4 - k)) & 1) << (bits - 1 - k);
        const int lowmask = (32 / NI) - 1;
        if ((lane & lowmask) == 0) {
            const int ii = i0 + elem;
            if (ii < na) write_force<MODE, MIXED>(a, a0 + ii, (double)ax[0], (double)ay[0], (double)az[0]);
        }
        // energies of this chunk
        if (MIXED) {
            kahan_add(le.s6, (float)e6);
            kahan_add(le.s12, (float)e12);
        } else {
            le.d6 += (double)e6;
            le.d12 += (double)e12;
        }
        le.pairs += npair;
        __syncwarp();
    }
}

template <bool MIXED, int NI, int MODE>
__global__ void __launch_bounds__(256) k_force(ForceArgs a) {
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
    for (int t = w; t < a.ntasks; t += W) {
        TaskCells tc = make_task<MODE>(a.g, a.group, a.colour, t);
        run_task<MIXED, NI, MODE>(a, sm, tc, lane, le);
    }
    // warp reduction of the energy partials in FP64, fixed order
    double s6 = MIXED ? ((double)le.s6.x - (double)le.s6.y) : le.d6;
    double s12 = MIXED ? ((double)le.s12.x - (double)le.s12.y) : le.d12;
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
        TaskCells tc = make_task<MODE>(g, group, colour, t);
        for (int k = 0; k < tc.nnb; ++k) {
            int o[3];
            task_offset<MODE>(group, k, tc.self, o);
            int c[3];
            for (int d = 0; d < 3; ++d) {
                c[d] = tc.cA[d] + o[d];
                if (c[d] >= g.nc[d]) c[d] -= g.nc[d];
                else if (c[d] < 0) c[d] += g.nc[d];
            }
            int B = c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
            int oi = (o[0] + 1) + 3 * (o[1] + 1) + 9 * (o[2] + 1);   // 0..26
            atomicAdd(visit + (size_t)tc.A * 27 + oi, 1ull);
            if (MODE == kColour && B != tc.A) {
                int old = atomicExch(stamp + B, phase);
                if (old == phase) atomicAdd(counters + 0, 1ull);
            }
        }
        if (MODE == kColour) {
            int old = atomicExch(stamp + tc.A, phase);
            if (old == phase) atomicAdd(counters + 0, 1ull);
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
        unsigned long long want = (full || fwd || centre) ? 1ull : 0ull;
        if (visit[t] != want) atomicAdd(counters + 1, 1ull);
    }
}

// ------------------------------------------------------------ launchers --
template <bool MIXED, int NI>
static size_t smem_bytes(int warps) {
    using T = typename std::conditional<MIXED, float, double>::type;
    return sizeof(WarpSmem<T>) * (size_t)warps;
}

template <bool MIXED, int NI, int MODE>
static cudaError_t launch_one(Ctx *c, ForceArgs &a, cudaStream_t s) {
    const int warps = c->warps;
    const size_t sm = smem_bytes<MIXED, NI>(warps);
    int blocks = force_grid_warps(c) / warps;
    k_force<MIXED, NI, MODE><<<blocks, warps * 32, sm, s>>>(a);
    return cudaGetLastError();
}

template <bool MIXED, int NI>
static cudaError_t launch_sched(Ctx *c, lc_schedule sched, cudaStream_t s, int *launches) {
    ForceArgs a;
    a.g = c->g;
    a.p4 = c->d_p4;
    a.x = c->cur.x; a.y = c->cur.y; a.z = c->cur.z;
    a.start = c->d_start; a.count = c->d_count;
    a.fx = c->fx; a.fy = c->fy; a.fz = c->fz;
    a.kx = c->kx; a.ky = c->ky; a.kz = c->kz;
    a.warp_acc = c->d_warp_acc; a.warp_pairs = c->d_warp_pairs;
    a.group = 0; a.colour = 0;
    cudaError_t e = cudaSuccess;
    const size_t nbytes = sizeof(double) * (size_t)c->n;
    if (sched == LC_SCHED_COLOUR) {
        if (MIXED) {
            e = cudaMemsetAsync(c->kx, 0, 3 * sizeof(float2) * (size_t)c->n, s);
        } else {
            e = cudaMemsetAsync(c->fx, 0, 3 * nbytes, s);
        }
        if (e) return e;
        for (int g = 0; g < 4; ++g)
            for (int k = 0; k < c->g.ncolours; ++k) {
                a.group = g; a.colour = k;
                int raw = c->g.raw_of_colour[k];
                a.ntasks = c->g.class_count[0][raw % 3] * c->g.class_count[1][(raw / 3) % 3] *
                           c->g.class_count[2][raw / 9];
                e = launch_one<MIXED, NI, kColour>(c, a, s);
                if (e) return e;
                ++*launches;
            }
        if (MIXED) {
            k_kahan_finalize<<<c->num_sms * 8, 256, 0, s>>>((int)c->n, c->kx, c->ky, c->kz, c->fx, c->fy, c->fz);
            ++*launches;
            e = cudaGetLastError();
        }
    } else if (sched == LC_SCHED_ATOMIC) {
        e = cudaMemsetAsync(c->fx, 0, 3 * nbytes, s);
        if (e) return e;
        a.ntasks = c->g.ncell;
        e = launch_one<MIXED, NI, kAtomic>(c, a, s);
        ++*launches;
    } else {
        a.ntasks = c->g.ncell;
        e = launch_one<MIXED, NI, kFullShell>(c, a, s);
        ++*launches;
    }
    return e;
}

int force_grid_warps(const Ctx *c) {
    // persistent-style grid: 16 resident warps per SM
    int per_sm = 16;
    int w = c->num_sms * per_sm;
    w = (w / c->warps) * c->warps;
    return w > 0 ? w : c->warps;
}

cudaError_t launch_forces(Ctx *c, lc_schedule sched, cudaStream_t s, int *launches) {
    cudaError_t e = cudaMemsetAsync(c->d_warp_acc, 0, sizeof(double) * 4 * (size_t)c->nwarp_max, s);
    if (e) return e;
    e = cudaMemsetAsync(c->d_warp_pairs, 0, sizeof(long long) * (size_t)c->nwarp_max, s);
    if (e) return e;
    const bool mixed = (c->prec == LC_PREC_MIXED);
    switch (c->ni) {
        case 8: e = mixed ? launch_sched<true, 8>(c, sched, s, launches) : launch_sched<false, 8>(c, sched, s, launches); break;
        case 32: e = mixed ? launch_sched<true, 32>(c, sched, s, launches) : launch_sched<false, 32>(c, sched, s, launches); break;
        default: e = mixed ? launch_sched<true, 16>(c, sched, s, launches) : launch_sched<false, 16>(c, sched, s, launches); break;
    }
    if (e) return e;
    e = launch_energy_reduce(c, s, sched == LC_SCHED_FULLSHELL);
    ++*launches;
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
        int phase = 0;
        for (int g = 0; g < 4; ++g)
            for (int k = 0; k < c->g.ncolours; ++k, ++phase) {
                int raw = c->g.raw_of_colour[k];
                int nt = c->g.class_count[0][raw % 3] * c->g.class_count[1][(raw / 3) % 3] *
                         c->g.class_count[2][raw / 9];
                k_check<kColour><<<blocks, 256, 0, s>>>(c->g, g, k, nt, phase, c->d_stamp, c->d_visit, c->d_counters);
            }
    } else if (sched == LC_SCHED_ATOMIC) {
        k_check<kAtomic><<<blocks, 256, 0, s>>>(c->g, 0, 0, c->g.ncell, 0, c->d_stamp, c->d_visit, c->d_counters);
    } else {
        k_check<kFullShell><<<blocks, 256, 0, s>>>(c->g, 0, 0, c->g.ncell, 0, c->d_stamp, c->d_visit, c->d_counters);
    }
    k_check_cover<<<blocks, 256, 0, s>>>(c->g, sched == LC_SCHED_FULLSHELL, c->d_visit, c->d_counters);
    return cudaGetLastError();
}

template <bool MIXED, int NI>
static cudaError_t attrs_for() {
    cudaError_t e;
    const int bytes = (int)smem_bytes<MIXED, NI>(16);
    if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kColour>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(k_force<MIXED, NI, kAtomic>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    return cudaFuncSetAttribute(k_force<MIXED, NI, kFullShell>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Opt the force kernels into the shared memory of the largest tile shape
// (called once per context, before any stream capture).
cudaError_t init_force_kernels() {
    cudaError_t e;
    if ((e = attrs_for<true, 8>()) || (e = attrs_for<true, 16>()) || (e = attrs_for<true, 32>()) ||
        (e = attrs_for<false, 8>()) || (e = attrs_for<false, 16>()) || (e = attrs_for<false, 32>()))
        return e;
    return cudaSuccess;
}

cudaError_t upload_stencil(const Stencil &st) {
    return cudaMemcpyToSymbol(c_st, &st, sizeof(Stencil));
}

}  // namespace lc
