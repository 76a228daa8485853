// Verlet neighbour lists with a skin on top of the link cells: an extension
// of the paper's method (the paper sweeps the link cells every step,
// Sec. IV), kept beside it as LC_SCHED_LIST.
//
// A list build bins the particles on a coarser "list grid" whose cells have
// side >= rc + skin, so every partner within rc + skin lies in the 27
// surrounding cells, and records for each particle all such partners (both
// directions: a full list).  Until some particle has moved by skin / 2 since
// the build, every pair inside rc is on the lists, and a force evaluation is
// one thread per particle over its own row -- each thread writes only its
// own force, so there is no write sharing to resolve at all.
//
//   k_list_build  one warp per list cell: the cell's particles against the
//                 candidates of its 27 neighbours (FP32 test with margin),
//                 appended to the rows in candidate order; also the
//                 fixed-point offsets of the force kernel
//   k_list_force  one thread per particle: its row, exact fixed-point
//                 displacements, FP32 pair terms, FP64 cutoff decision in
//                 the band around rc
//   k_list_drift  kick + drift of a velocity-Verlet step (same FMAs as the
//                 link-cell step), new offsets, displacement check; its
//                 last block sets the CUDA-graph condition that runs the
//                 rebuild
//
// Positions are not wrapped between builds (the offsets stay continuous);
// the rebuild's binning wraps them.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lc_internal.cuh"

namespace lc {

constexpr int kLBWarps = 4;     // warps per block of the build
constexpr int kLBCap = 1024;    // candidates listed per batch (per warp)
constexpr int kListThreads = 256;
constexpr int kPF = 4;          // list entries in flight per thread (force kernel)

struct ListArgs {
    Grid g;                     // list grid (rc fields: the force cutoff)
    int n, kmax;
    const float4 *p4;           // offsets from the binning (build)
    int4 *q4;                   // fixed-point offsets now; w = build cell
    int4 *qb;                   // the same at the build (displacement check)
    double *x, *y, *z;          // FP64 positions
    const int *start, *count;   // list cells at the build
    unsigned *nbr;              // [kmax][n]
    int *nn;                    // [n]
    float rl2;                  // (rc + skin)^2 with a relative margin (build test)
    float scale, inv_scale;     // 2^k, 2^-k: offsets are in units of 2^-k
    float scale2;               // 2^2k
    int hq[3];                  // cell sides in units of 2^-k
    float rc2s_lo, rc2s_hi;     // FP32 band around rc^2, in units of 2^-2k
    double *fx, *fy, *fz;
    double *warp_acc;
    long long *warp_pairs;
    unsigned long long *stats;  // builds, long rows, longest row, rebuild steps, entries
    unsigned *ctl;              // rebuild flag, block ticket
    int *err;
};

// round(x * 2^k) for x = hi + lo (|x| 2^k < 2^30): hi * 2^k is exact, its
// integer part exact, the fractional part exact (|hi 2^k| < 2^23) or zero.
__device__ __forceinline__ int quantize(float hi, float lo, float scale) {
    const float S = hi * scale;
    const int i1 = __float2int_rn(S);
    const float r1 = S - __int2float_rn(i1);
    return i1 + __float2int_rn(fmaf(lo, scale, r1));
}

// Periodic image of neighbour offset o of cell coordinate c: -1, 0, +1.
__device__ __forceinline__ int image_of(int c, int o, int nc) {
    const int t = c + o;
    return t >= nc ? 1 : (t < 0 ? -1 : 0);
}

// ------------------------------------------------------------- build -----
// One warp per list cell and chunk of up to 32 of its particles, in two
// phases per batch of candidates (the particles of the 27 surrounding cells,
// in table order):
//   test  lane = candidate: FP32 distance to every chunk particle, two per
//         packed f32x2 operation; the ballot of each (round, particle) goes
//         to shared memory
//   emit  lane = chunk particle: walks its bits in candidate order and
//         appends the entries; the t-th append of every lane writes row t,
//         so the stores of a warp are contiguous
struct alignas(16) BuildSmem {
    unsigned mask[kLBCap / 32][32];    // [round][chunk particle]: candidates within rc + skin
    float ipx[32], ipy[32], ipz[32];   // chunk particles (FP32 offsets); far past the chunk
    unsigned jl[kLBCap];               // candidate entries: slot << 6 | cell-shift code
    int nb_start[27], nb_count[27], nb_code[27];
};

__device__ __forceinline__ float2 lds2(const float *p) { return *reinterpret_cast<const float2 *>(p); }

template <bool WRITE>
__global__ void __launch_bounds__(kLBWarps * 32) k_list_build(ListArgs a) {
    __shared__ BuildSmem smem[kLBWarps];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    BuildSmem &sm = smem[wib];
    const int W = gridDim.x * kLBWarps;
    const Grid &g = a.g;
    const int nf = g.dims == 2 ? 9 : 27;
    int my_max = 0, my_long = 0;
    long long my_entries = 0;
    for (int A = blockIdx.x * kLBWarps + wib; A < g.ncell; A += W) {
        const int a0 = a.start[A], na = a.count[A];
        if (na == 0) continue;
        int cA[3];
        cell_coords(g, A, cA);
        if (lane < nf) {   // neighbour table: entry lane = offset index (z, y, x) lexicographic
            const int oi = g.dims == 2 ? 9 + lane : lane;
            const int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, oi / 9 - 1};
            int c[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                c[d] = cA[d] + o[d];
                c[d] = c[d] >= g.nc[d] ? c[d] - g.nc[d] : (c[d] < 0 ? c[d] + g.nc[d] : c[d]);
            }
            const int B = c[0] + g.nc[0] * (c[1] + g.nc[1] * c[2]);
            sm.nb_start[lane] = a.start[B];
            sm.nb_count[lane] = a.count[B];
            sm.nb_code[lane] = (o[0] + 1) | ((o[1] + 1) << 2) | ((o[2] + 1) << 4);
        }
        __syncwarp();
        for (int i0 = 0; i0 < na; i0 += 32) {
            const int ni = min(32, na - i0);
            const int si = a0 + i0 + lane;
            float4 pi = make_float4(1.0e30f, 1.0e30f, 1.0e30f, 0.f);
            if (lane < ni) pi = a.p4[si];
            sm.ipx[lane] = pi.x; sm.ipy[lane] = pi.y; sm.ipz[lane] = pi.z;
            const int nii = (ni + 1) & ~1;   // chunk particles tested, in pairs
            int cnt = 0;                     // this lane's row length
            __syncwarp();
            int b = 0, kin = 0;
            while (b < nf) {
                int nj = 0;   // next batch of candidates, in table order
                while (b < nf && nj < kLBCap) {
                    const int take = min(sm.nb_count[b] - kin, kLBCap - nj);
                    const unsigned st = (unsigned)(sm.nb_start[b] + kin), code = (unsigned)sm.nb_code[b];
                    for (int k = lane; k < take; k += 32) sm.jl[nj + k] = ((st + k) << 6) | code;
                    nj += take;
                    kin += take;
                    if (kin >= sm.nb_count[b]) { ++b; kin = 0; }
                }
                __syncwarp();
                const int nr = (nj + 31) >> 5;
                for (int r = 0; r < nr; ++r) {   // test
                    const int e = r * 32 + lane;
                    const bool valid = e < nj;
                    int sj = -1;
                    float2 px = make_float2(1.0e30f, 1.0e30f), py = px, pz = px;
                    if (valid) {
                        const unsigned w = sm.jl[e];
                        sj = (int)(w >> 6);
                        const float4 q = a.p4[sj];
                        const float x = q.x + (float)((int)(w & 3u) - 1) * g.hf[0];
                        const float y = q.y + (float)((int)((w >> 2) & 3u) - 1) * g.hf[1];
                        const float z = q.z + (float)((int)((w >> 4) & 3u) - 1) * g.hf[2];
                        px = make_float2(-x, -x); py = make_float2(-y, -y); pz = make_float2(-z, -z);
                    }
                    const int self = sj - (a0 + i0);   // chunk index of the candidate itself, if it is one
                    for (int ii = 0; ii < nii; ii += 2) {
                        const float2 dx = __fadd2_rn(lds2(&sm.ipx[ii]), px);
                        const float2 dy = __fadd2_rn(lds2(&sm.ipy[ii]), py);
                        const float2 dz = __fadd2_rn(lds2(&sm.ipz[ii]), pz);
                        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                        const unsigned m0 = __ballot_sync(kFull, r2.x < a.rl2 && self != ii);
                        const unsigned m1 = __ballot_sync(kFull, r2.y < a.rl2 && self != ii + 1);
                        if (lane == 0) *reinterpret_cast<uint2 *>(&sm.mask[r][ii]) = make_uint2(m0, m1);
                    }
                }
                __syncwarp();
                if (lane < ni) {   // emit: this lane's bits, round by round
                    int r = 0;
                    unsigned m = sm.mask[0][lane];
                    for (;;) {
                        while (m == 0u && ++r < nr) m = sm.mask[r][lane];
                        if (m == 0u) break;
                        const int bit = __ffs(m) - 1;
                        m &= m - 1u;
                        if (WRITE && cnt < a.kmax) a.nbr[(size_t)cnt * (size_t)a.n + (size_t)si] = sm.jl[r * 32 + bit];
                        ++cnt;
                    }
                }
                __syncwarp();
            }
            if (lane < ni) {
                a.nn[si] = cnt;
                if (WRITE) {
                    const float4 p = pi;
                    const unsigned wr = __float_as_uint(p.w);
                    int4 q;
                    q.x = quantize(p.x, lo_residual(wr, 0), a.scale);
                    q.y = quantize(p.y, lo_residual(wr, 1), a.scale);
                    q.z = quantize(p.z, lo_residual(wr, 2), a.scale);
                    q.w = A;
                    a.q4[si] = q;
                    a.qb[si] = q;
                }
                my_max = max(my_max, cnt);
                my_long += cnt > a.kmax ? 1 : 0;
                my_entries += cnt;
            }
            __syncwarp();
        }
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        my_max = max(my_max, __shfl_xor_sync(kFull, my_max, m));
        my_long += __shfl_xor_sync(kFull, my_long, m);
        my_entries += __shfl_xor_sync(kFull, my_entries, m);
    }
    if (lane == 0) {
        atomicMax(a.stats + 2, (unsigned long long)my_max);
        if (WRITE && my_long) atomicAdd(a.stats + 1, (unsigned long long)my_long);
        if (WRITE && my_entries) atomicAdd(a.stats + 4, (unsigned long long)my_entries);
    }
    if (WRITE && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(a.stats + 0, 1ull);
}

// ------------------------------------------------------------- forces ----
// Exact FP64 cutoff decision (each operation rounded once), the image of
// the pair from the build cell of i and the entry's offset.
__device__ __forceinline__ bool exact_inside_list(const ListArgs &a, int i, int sj, int celli, unsigned w) {
    int cA[3];
    cell_coords(a.g, celli, cA);
    double sL[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int im = image_of(cA[d], (int)((w >> (2 * d)) & 3u) - 1, a.g.nc[d]);
        sL[d] = im == 0 ? 0.0 : (im > 0 ? a.g.L[d] : -a.g.L[d]);
    }
    const double dx = __dsub_rn(__dsub_rn(a.x[i], a.x[sj]), sL[0]);
    const double dy = __dsub_rn(__dsub_rn(a.y[i], a.y[sj]), sL[1]);
    const double dz = __dsub_rn(__dsub_rn(a.z[i], a.z[sj]), sL[2]);
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < a.g.rc2;
}

// Two list entries of particle i, one per half of the packed f32x2
// operations: displacement in exact integer arithmetic (offsets in units of
// 2^-k, the entry's cell shift from the block's table; modular, the result
// fits), one rounding to FP32, then the pair terms, masked rather than
// branched on (the FP64 decision in the band around rc is the only branch,
// and it is rare).  live = false: a padding slot, no contribution.
template <bool STATS>
__device__ __forceinline__ void list_pair2(const ListArgs &a, const int4 *shift, int i, const int4 &qi, unsigned w0,
                                           const int4 &q0, bool live0, unsigned w1, const int4 &q1, bool live1,
                                           float2 &fx, float2 &fy, float2 &fz, float2 &e6, float2 &e12, int &np) {
    const int4 s0 = shift[w0 & 63u], s1 = shift[w1 & 63u];
    const float2 dx = make_float2((float)(int)((unsigned)qi.x - (unsigned)q0.x - (unsigned)s0.x),
                                  (float)(int)((unsigned)qi.x - (unsigned)q1.x - (unsigned)s1.x));
    const float2 dy = make_float2((float)(int)((unsigned)qi.y - (unsigned)q0.y - (unsigned)s0.y),
                                  (float)(int)((unsigned)qi.y - (unsigned)q1.y - (unsigned)s1.y));
    const float2 dz = make_float2((float)(int)((unsigned)qi.z - (unsigned)q0.z - (unsigned)s0.z),
                                  (float)(int)((unsigned)qi.z - (unsigned)q1.z - (unsigned)s1.z));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));   // units of 2^-2k
    bool t0 = live0 && r2.x < a.rc2s_lo, t1 = live1 && r2.y < a.rc2s_lo;
    if (live0 && r2.x < a.rc2s_hi && !t0) t0 = exact_inside_list(a, i, (int)(w0 >> 6), qi.w, w0);
    if (live1 && r2.y < a.rc2s_hi && !t1) t1 = exact_inside_list(a, i, (int)(w1 >> 6), qi.w, w1);
    float2 y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.x) : "f"(r2.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.y) : "f"(r2.y));
    const float2 e = __ffma2_rn(make_float2(-r2.x, -r2.y), y, make_float2(1.0f, 1.0f));   // Newton step
    y = __ffma2_rn(y, e, y);
    float2 inv = __fmul2_rn(y, make_float2(a.scale2, a.scale2));   // r^-2
    inv.x = t0 ? inv.x : 0.0f;
    inv.y = t1 ? inv.y : 0.0f;
    const float2 s6 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
    const float2 g = __ffma2_rn(s6, make_float2(48.0f, 48.0f), make_float2(-24.0f, -24.0f));
    const float2 f = __fmul2_rn(__fmul2_rn(s6, inv), __fmul2_rn(g, make_float2(a.inv_scale, a.inv_scale)));
    fx = __ffma2_rn(f, dx, fx);
    fy = __ffma2_rn(f, dy, fy);
    fz = __ffma2_rn(f, dz, fz);
    if (STATS) {
        e6 = __fadd2_rn(e6, s6);
        e12 = __ffma2_rn(s6, s6, e12);
        np += (t0 ? 1 : 0) + (t1 ? 1 : 0);
    }
}

template <bool STATS>
__global__ void __launch_bounds__(kListThreads) k_list_force(ListArgs a) {
    // cell shift of every entry code (o_d + 1 in two bits per axis), in
    // units of 2^-k
    __shared__ int4 shift[64];
    if (threadIdx.x < 64) {
        const int c = threadIdx.x;
        shift[c] = make_int4(((c & 3) - 1) * a.hq[0], (((c >> 2) & 3) - 1) * a.hq[1], (((c >> 4) & 3) - 1) * a.hq[2], 0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float2 e6 = make_float2(0.f, 0.f), e12 = make_float2(0.f, 0.f);
    int np = 0;
    const size_t n = (size_t)a.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
        const int4 qi = a.q4[i];
        const int cnt = a.nn[i];
        float2 fx = make_float2(0.f, 0.f), fy = fx, fz = fx;
        if (cnt <= a.kmax) {
            // software pipeline: the next kPF entries load while the
            // current ones' partner offsets load and are used
            const unsigned *row = a.nbr + i;
            unsigned w[kPF];
#pragma unroll
            for (int j = 0; j < kPF; ++j) w[j] = j < cnt ? __ldcs(row + (size_t)j * n) : 0u;
            for (int k = 0; k < cnt; k += kPF) {
                int4 q[kPF];
#pragma unroll
                for (int j = 0; j < kPF; ++j) q[j] = k + j < cnt ? a.q4[w[j] >> 6] : qi;
                unsigned wn[kPF];
#pragma unroll
                for (int j = 0; j < kPF; ++j)
                    wn[j] = k + kPF + j < cnt ? __ldcs(row + (size_t)(k + kPF + j) * n) : 0u;
#pragma unroll
                for (int j = 0; j < kPF; j += 2)
                    list_pair2<STATS>(a, shift, i, qi, w[j], q[j], k + j < cnt, w[j + 1], q[j + 1], k + j + 1 < cnt,
                                      fx, fy, fz, e6, e12, np);
#pragma unroll
                for (int j = 0; j < kPF; ++j) w[j] = wn[j];
            }
        } else {
            // a row longer than the list's capacity: the partners are swept
            // from the 27 list cells around the build cell (cells of side
            // >= rc + skin hold every partner within rc while no particle
            // has moved by skin / 2)
            int cA[3];
            cell_coords(a.g, qi.w, cA);
            const int nf = a.g.dims == 2 ? 9 : 27;
            for (int e = 0; e < nf; ++e) {
                const int oi = a.g.dims == 2 ? 9 + e : e;
                const int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, oi / 9 - 1};
                int c[3];
                for (int d = 0; d < 3; ++d) {
                    c[d] = cA[d] + o[d];
                    c[d] = c[d] >= a.g.nc[d] ? c[d] - a.g.nc[d] : (c[d] < 0 ? c[d] + a.g.nc[d] : c[d]);
                }
                const int B = c[0] + a.g.nc[0] * (c[1] + a.g.nc[1] * c[2]);
                const unsigned code = (unsigned)((o[0] + 1) | ((o[1] + 1) << 2) | ((o[2] + 1) << 4));
                const int b0 = a.start[B], b1 = b0 + a.count[B];
                for (int j = b0; j < b1; ++j) {
                    const unsigned wj = ((unsigned)j << 6) | code;
                    list_pair2<STATS>(a, shift, i, qi, wj, a.q4[j], j != i, wj, qi, false, fx, fy, fz, e6, e12, np);
                }
            }
        }
        a.fx[i] = f32_to_f64_bits(fx.x + fx.y);
        a.fy[i] = f32_to_f64_bits(fy.x + fy.y);
        a.fz[i] = f32_to_f64_bits(fz.x + fz.y);
    }
    if (STATS) {   // block partials in FP64, fixed order: one slot per block
        __shared__ double r6[kListThreads / 32], r12[kListThreads / 32];
        __shared__ long long rp[kListThreads / 32];
        double s6 = f32_to_f64_bits(e6.x) + f32_to_f64_bits(e6.y);
        double s12 = f32_to_f64_bits(e12.x) + f32_to_f64_bits(e12.y);
        long long p = np;
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            s6 += __shfl_xor_sync(kFull, s6, m);
            s12 += __shfl_xor_sync(kFull, s12, m);
            p += __shfl_xor_sync(kFull, p, m);
        }
        const int wib = threadIdx.x >> 5;
        if (lane == 0) { r6[wib] = s6; r12[wib] = s12; rp[wib] = p; }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < kListThreads / 32; ++k) { s6 += r6[k]; s12 += r12[k]; p += rp[k]; }
            a.warp_acc[4 * blockIdx.x + 0] = s6;
            a.warp_acc[4 * blockIdx.x + 1] = s12;
            a.warp_pairs[blockIdx.x] = p;
        }
    }
}

// -------------------------------------------------------------- drift ----
// Velocity-Verlet opening of a step between builds: KICKS = 1: v += h F,
// x += dt v; KICKS = 2: the previous step's closing v += h F first (the
// same FMAs as the link-cell step).  Then the fixed-point offsets from the
// build cell's centre and the displacement since the build; a block that
// sees a displacement above the threshold raises the rebuild flag, and the
// last block to finish turns the flag into the graph condition.
struct ListDrift {
    double half, dt;
    double *vx, *vy, *vz;
    const double *fx, *fy, *fz;
    float thr2;                 // rebuild when |displacement|^2 > thr2
    int use_cond;
    cudaGraphConditionalHandle cond;
};

template <int KICKS>
__global__ void __launch_bounds__(kListThreads) k_list_drift(ListArgs a, ListDrift dr) {
    bool exceed = false;
    const Grid &g = a.g;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < a.n; s += gridDim.x * blockDim.x) {
        double X[3] = {a.x[s], a.y[s], a.z[s]};
        double v[3] = {dr.vx[s], dr.vy[s], dr.vz[s]};
        const double f[3] = {dr.fx[s], dr.fy[s], dr.fz[s]};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (KICKS == 2) v[d] = fma(dr.half, f[d], v[d]);
            v[d] = fma(dr.half, f[d], v[d]);
            X[d] = fma(dr.dt, v[d], X[d]);
        }
        dr.vx[s] = v[0]; dr.vy[s] = v[1]; dr.vz[s] = v[2];
        a.x[s] = X[0]; a.y[s] = X[1]; a.z[s] = X[2];
        const int4 b = a.qb[s];
        int cc[3];
        cell_coords(g, b.w, cc);
        const int bq[3] = {b.x, b.y, b.z};
        int q[3];
        float d2 = 0.f;
        bool bad = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            Split sp;
            if (!split_f64(X[d], sp)) {   // |x| < 2^-100 (taken as 0), huge or not finite
                bad = bad || !(fabs(X[d]) < 1.0);
                sp.hi = sp.lo = 0.0f;
            }
            float hi, lo;
            cell_offset_df(g, sp, cc[d], d, hi, lo);
            const float dd = hi - __int2float_rn(bq[d]) * a.inv_scale;
            d2 = fmaf(dd, dd, d2);
            // far from the build cell: no offset (the rebuild recomputes it)
            const bool far = !(fabsf(hi) * a.scale < 1.0e9f);
            bad = bad || far;
            q[d] = far ? 0 : quantize(hi, lo, a.scale);
        }
        if (bad && !(isfinite(X[0]) && isfinite(X[1]) && isfinite(X[2]))) atomicOr(a.err, kErrNonfinite);
        exceed = exceed || bad || !(d2 <= dr.thr2);
        a.q4[s] = make_int4(q[0], q[1], q[2], b.w);
    }
    const int any = __syncthreads_or(exceed ? 1 : 0);
    if (threadIdx.x == 0) {
        if (any) atomicOr(a.ctl + 0, 1u);
        __threadfence();
        const unsigned t = atomicAdd(a.ctl + 1, 1u);
        if (t == gridDim.x - 1) {   // the last block: every flag is in
            __threadfence();
            const unsigned flag = atomicExch(a.ctl + 0, 0u);
            atomicExch(a.ctl + 1, 0u);
            if (dr.use_cond) cudaGraphSetConditional(dr.cond, flag ? 1u : 0u);
            if (flag) atomicAdd(a.stats + 3, 1ull);
        }
    }
}

__global__ void k_copy_state(int n, State src, State dst) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        dst.x[s] = src.x[s]; dst.y[s] = src.y[s]; dst.z[s] = src.z[s];
        dst.vx[s] = src.vx[s]; dst.vy[s] = src.vy[s]; dst.vz[s] = src.vz[s];
        dst.id[s] = src.id[s];
    }
}

// -------------------------------------------------------------- host -----
bool make_list_grid(Ctx *c) {
    const double rl = c->g.rc + c->skin;
    for (int d = 0; d < c->g.dims; ++d)
        if (floor(c->g.L[d] / rl) < 3.0) return false;
    make_grid(&c->gl, c->g.L, rl, c->g.dims);
    c->gl.rc = c->g.rc;
    c->gl.rc2 = c->g.rc2;
    c->gl.rc2f_lo = c->g.rc2f_lo;
    c->gl.rc2f_hi = c->g.rc2f_hi;
    // unit 2^-k: per-axis displacements of any two particles of
    // neighbouring list cells (< 2 h + skin) stay below 2^30 units
    double hmax = 0.0;
    for (int d = 0; d < 3; ++d) hmax = c->gl.h[d] > hmax ? c->gl.h[d] : hmax;
    const double B = 2.0 * hmax + c->skin + 1.0;
    c->list_shift = (int)floor(log2((double)(1 << 30) / B));
    if (c->list_shift > 40) c->list_shift = 40;
    return true;
}

static ListArgs list_args(const Ctx *c) {
    ListArgs a;
    a.g = c->gl;
    a.n = (int)c->n;
    a.kmax = c->list_kmax;
    a.p4 = c->d_p4;
    a.q4 = c->d_q4;
    a.qb = c->d_q4 + c->n;
    a.x = c->cur.x; a.y = c->cur.y; a.z = c->cur.z;
    a.start = c->d_start;
    a.count = c->d_count;
    a.nbr = c->d_nbr;
    a.nn = c->d_nn;
    const double rl = c->g.rc + c->skin;
    a.rl2 = (float)(rl * rl * (1.0 + 2.0e-5));
    const int k = c->list_shift;
    a.scale = ldexpf(1.0f, k);
    a.inv_scale = ldexpf(1.0f, -k);
    a.scale2 = ldexpf(1.0f, 2 * k);
    for (int d = 0; d < 3; ++d) a.hq[d] = (int)llrint(ldexp(c->gl.h[d], k));
    a.rc2s_lo = c->g.rc2f_lo * a.scale2;
    a.rc2s_hi = c->g.rc2f_hi * a.scale2;
    a.fx = c->fx; a.fy = c->fy; a.fz = c->fz;
    a.warp_acc = c->d_warp_acc;
    a.warp_pairs = c->d_warp_pairs;
    a.stats = c->d_list_stats;
    a.ctl = reinterpret_cast<unsigned *>(c->d_list_stats + 5);
    a.err = c->d_err;
    return a;
}

// One thread per particle (grid-stride beyond nwarp_max blocks, whose
// statistics slots bound the grid).
static int list_blocks(const Ctx *c) {
    const int want = (int)((c->n + kListThreads - 1) / kListThreads);
    const int cap = c->nwarp_max;
    return want < 1 ? 1 : (want < cap ? want : cap);
}

cudaError_t launch_list_build(Ctx *c, cudaStream_t s, bool write) {
    if (c->n == 0) return cudaSuccess;
    ListArgs a = list_args(c);
    int blocks = (c->gl.ncell + kLBWarps - 1) / kLBWarps;
    if (blocks > c->num_sms * 6) blocks = c->num_sms * 6;   // six resident per SM (shared memory)
    if (write) k_list_build<true><<<blocks, kLBWarps * 32, 0, s>>>(a);
    else k_list_build<false><<<blocks, kLBWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

// Bin on the list grid and build the lists.  copy_back: return the binned
// state to the buffers it came from (a captured step must leave the state
// where the next replay expects it).
cudaError_t launch_list_rebuild(Ctx *c, cudaStream_t s, bool copy_back, int *launches) {
    const Grid saved = c->g;
    c->g = c->gl;
    cudaError_t e = launch_bin(c, s, launches, 0, 0.0);
    c->g = saved;
    if (e) return e;
    if (copy_back && c->n > 0) {
        k_copy_state<<<c->num_sms * 8, 256, 0, s>>>((int)c->n, c->cur, c->nxt);
        if ((e = cudaGetLastError())) return e;
        ++*launches;
        const State t = c->cur; c->cur = c->nxt; c->nxt = t;
    }
    if (c->n > 0) ++*launches;
    return launch_list_build(c, s, true);
}

cudaError_t launch_list_forces(Ctx *c, cudaStream_t s, bool stats, int *launches) {
    if (c->n > 0) {
        ++*launches;
        ListArgs a = list_args(c);
        const int blocks = list_blocks(c);
        if (stats) k_list_force<true><<<blocks, kListThreads, 0, s>>>(a);
        else k_list_force<false><<<blocks, kListThreads, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
        c->nwarp_used = blocks;   // one statistics slot per block
    }
    if (!stats) return cudaSuccess;
    if (c->n == 0) {   // no warps: zero statistics
        c->nwarp_used = 1;
        cudaError_t e = cudaMemsetAsync(c->d_warp_acc, 0, sizeof(double) * 4, s);
        if (!e) e = cudaMemsetAsync(c->d_warp_pairs, 0, sizeof(long long), s);
        if (e) return e;
    }
    c->stats_full = 1;
    ++*launches;
    return launch_energy_reduce(c, s, 1);   // every pair appears in two rows
}

static cudaError_t launch_list_drift(Ctx *c, double dt, int kicks, const cudaGraphConditionalHandle *cond,
                                     cudaStream_t s) {
    ListArgs a = list_args(c);
    ListDrift dr;
    dr.half = 0.5 * dt;
    dr.dt = dt;
    dr.vx = c->cur.vx; dr.vy = c->cur.vy; dr.vz = c->cur.vz;
    dr.fx = c->fx; dr.fy = c->fy; dr.fz = c->fz;
    const double t = 0.5 * c->skin - 1.0e-6;
    dr.thr2 = t > 0.0 ? (float)(t * t) : 0.0f;
    dr.use_cond = cond != nullptr;
    dr.cond = cond ? *cond : 0;
    const int blocks = list_blocks(c);
    if (kicks == 2) k_list_drift<2><<<blocks, kListThreads, 0, s>>>(a, dr);
    else k_list_drift<1><<<blocks, kListThreads, 0, s>>>(a, dr);
    return cudaGetLastError();
}

// nsteps (1 or 2) list steps as one CUDA graph: per step the drift kernel,
// a conditional node whose body (bin on the list grid, copy back, build) runs
// only when the drift kernel saw a displacement above skin / 2, and the
// force kernel; then the closing kick.  Statistics in the last step.
cudaError_t capture_list_steps(Ctx *c, double dt, int nsteps, cudaGraphExec_t *out, int *launches) {
    *out = nullptr;
    cudaStream_t cap = nullptr, body_s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&body_s, cudaStreamNonBlocking);
    if (e) {
        if (cap) cudaStreamDestroy(cap);
        return e;
    }
    const State saved_cur = c->cur, saved_nxt = c->nxt;
    cudaGraph_t graph = nullptr;
    int per = 0;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    bool capturing = !e;
    for (int k = 0; k < nsteps && !e; ++k) {
        cudaStreamCaptureStatus st;
        cudaGraph_t g_cap = nullptr;
        e = cudaStreamGetCaptureInfo(cap, &st, nullptr, &g_cap, nullptr, nullptr, nullptr);
        cudaGraphConditionalHandle h = 0;
        if (!e) e = cudaGraphConditionalHandleCreate(&h, g_cap, 0, cudaGraphCondAssignDefault);
        if (!e) e = launch_list_drift(c, dt, k == 0 ? 1 : 2, &h, cap);
        ++per;   // the rebuild's launches (in the conditional body) are not counted
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        if (!e) e = cudaStreamGetCaptureInfo(cap, &st, nullptr, &g_cap, &deps, nullptr, &ndeps);
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeIf;
        p.conditional.size = 1;
        cudaGraphNode_t cn = nullptr;
        if (!e) e = cudaGraphAddNode(&cn, g_cap, deps, nullptr, ndeps, &p);
        if (!e) e = cudaStreamUpdateCaptureDependencies(cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (!e) {
            cudaGraph_t body = p.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(body_s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (!e) {
                int body_launches = 0;
                cudaError_t eb = launch_list_rebuild(c, body_s, true, &body_launches);
                cudaGraph_t got = nullptr;
                cudaError_t ee = cudaStreamEndCapture(body_s, &got);
                e = eb ? eb : ee;
            }
        }
        if (!e) e = launch_list_forces(c, cap, k == nsteps - 1, &per);
    }
    if (!e) e = launch_kick(c, dt, cap);
    ++per;
    if (capturing) {
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (!e) e = e2;
    }
    c->cur = saved_cur;   // the copy-back keeps the buffers in place
    c->nxt = saved_nxt;
    if (!e) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(body_s);
    cudaStreamDestroy(cap);
    if (e) {
        cudaGetLastError();
        *out = nullptr;
    }
    if (launches) *launches = per;
    return e;
}

}  // namespace lc
