// Pair arithmetic and warp helpers shared by the link-cell force kernels
// (lc_force.cu: the per-cell-task sweep; lc_blk.cu: the block-staged sweep).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "lc_internal.cuh"

namespace lc {

// Pairs closer than kClose (r^2 < kClose2) have their force recomputed in
// FP64: the FP32 r^2 carries about one ulp of rounding, which the r^-14 of
// the force amplifies about sevenfold, and the largest pair forces (the
// closest pairs) set the largest per-particle errors.
constexpr float kClose2 = 0.9025f;   // (0.95 sigma)^2

__device__ __forceinline__ double image_shift(const Grid &g, int img, int d) {
    const int s = ((img >> (2 * d)) & 3) - 1;
    return s == 0 ? 0.0 : (s > 0 ? g.L[d] : -g.L[d]);
}

// Shared-memory vector load kept inside the loop (volatile): the centre-cell
// particles are re-read per candidate instead of being pinned in registers,
// which keeps the kernel at two resident blocks per SM.
__device__ __forceinline__ float4 lds4(const float4 *p) {
    float4 v;
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// Reciprocal: hardware approximation refined by one Newton-Raphson step
// y <- y (2 - r y), written as two FMAs.
__device__ __forceinline__ float rcp_nr(float r) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r));
    float e = fmaf(-r, y, 1.0f);
    return fmaf(y, e, y);
}

// Butterfly reduce-scatter of v[NI] over the 32 lanes of a warp.  On return
// lane l holds in v[0] the warp-wide sum of element e(l), where fold k (lane
// bit 4 - k) picks bit log2(NI) - 1 - k of e; lanes that differ only in the
// low log2(32 / NI) bits hold the same element.
template <typename T, int NI>
__device__ __forceinline__ void reduce_scatter(T (&v)[NI], int lane) {
#pragma unroll
    for (int half = NI / 2, m = 16; half >= 1; half >>= 1, m >>= 1) {
        const bool up = (lane & m) != 0;
        if constexpr (std::is_same<T, float>::value) {
            if (half >= 2) {   // pairs of adjacent elements: one f32x2 add per pair
#pragma unroll
                for (int k = 0; k < half; k += 2) {
                    const float2 keep = make_float2(up ? v[k + half] : v[k], up ? v[k + half + 1] : v[k + 1]);
                    const float2 recv = make_float2(__shfl_xor_sync(kFull, up ? v[k] : v[k + half], m),
                                                    __shfl_xor_sync(kFull, up ? v[k + 1] : v[k + half + 1], m));
                    const float2 sum = __fadd2_rn(keep, recv);
                    v[k] = sum.x;
                    v[k + 1] = sum.y;
                }
                continue;
            }
        }
#pragma unroll
        for (int k = 0; k < half; ++k) {
            T send = up ? v[k] : v[k + half];
            T keep = up ? v[k + half] : v[k];
            v[k] = keep + __shfl_xor_sync(kFull, send, m);
        }
    }
#pragma unroll
    for (int m = 16 / NI; m >= 1; m >>= 1) v[0] += __shfl_xor_sync(kFull, v[0], m);
}

// Sum over the 32 lanes of every lane's NI partials through per-warp shared
// scratch s (32 * 17 floats; the odd row stride makes both the row writes
// and the column reads free of bank conflicts): lane (i, g) = (lane mod NI,
// lane / NI) adds rows g NI .. g NI + NI - 1 of column i, then the 32 / NI
// group sums are added by a butterfly over g.  Lanes l < NI return the sum
// of element l.  A fixed order: the same bits on every run.  Unlike the
// shuffle butterfly the loads and adds of one column are independent, so
// they overlap.
constexpr int kColStride = 17;
template <int NI>
__device__ __forceinline__ float column_sum(const float (&v)[NI], float *s, int lane) {
    __syncwarp();   // the scratch's previous readers are done
#pragma unroll
    for (int i = 0; i < NI; ++i) s[lane * kColStride + i] = v[i];
    __syncwarp();
    const float *col = s + (lane / NI) * NI * kColStride + (lane & (NI - 1));
    float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < NI; ++r) t[r & 3] += col[r * kColStride];
    float sum = (t[0] + t[1]) + (t[2] + t[3]);
#pragma unroll
    for (int m = NI; m < 32; m <<= 1) sum += __shfl_xor_sync(kFull, sum, m);
    return sum;
}

// The same sums for a chunk of 16 held as 8 packed pairs per lane (pair k
// = elements 2k, 2k + 1): every lane stores its pairs as one row of 8-byte
// words (row stride kPairStride pairs, odd, so that neither the row stores
// nor the column reads conflict); lane (p = l & 7, h = l >> 3) adds pair p
// over rows 8h .. 8h + 7 with packed adds; two shuffle levels finish the sum
// and split the pair on the way: lanes with h = 0 (l < 8) end with element
// 2p, lanes with h = 2 (16 <= l < 24) with element 2p + 1 (pair_element).
// A fixed order, so the bits are reproducible.  Returns the lane's sum,
// valid on those 16 lanes.
constexpr int kPairStride = 9;
__device__ __forceinline__ int pair_element(int lane) { return 2 * (lane & 7) + ((lane >> 4) & 1); }
__device__ __forceinline__ bool pair_owner(int lane) { return (lane & 8) == 0; }
__device__ __forceinline__ float column_sum_pairs(const float2 (&v)[8], float2 *s, int lane) {
    __syncwarp();   // the scratch's previous readers are done
#pragma unroll
    for (int k = 0; k < 8; ++k) s[lane * kPairStride + k] = v[k];
    __syncwarp();
    const float2 *col = s + 8 * (lane >> 3) * kPairStride + (lane & 7);
    float2 t0 = col[0], t1 = col[kPairStride];
#pragma unroll
    for (int r = 2; r < 8; r += 2) {
        t0 = __fadd2_rn(t0, col[r * kPairStride]);
        t1 = __fadd2_rn(t1, col[(r + 1) * kPairStride]);
    }
    const float2 t = __fadd2_rn(t0, t1);
    const bool keep_x = lane < 16;   // h < 2 keeps element 2p, h >= 2 element 2p + 1
    const float mine = keep_x ? t.x : t.y;
    float r = mine + __shfl_xor_sync(kFull, keep_x ? t.y : t.x, 16);
    r += __shfl_xor_sync(kFull, r, 8);
    return r;
}

template <int NI>
__device__ __forceinline__ int scattered_element(int lane) {
    int bits = 0;
    for (int n = NI; n > 1; n >>= 1) ++bits;
    int e = 0;
    for (int k = 0; k < bits; ++k) e |= ((lane >> (4 - k)) & 1) << (bits - 1 - k);
    return e;
}

// Kahan-compensated accumulation of v into (s, c): true sum ~ s - c.
__device__ __forceinline__ void kahan_add(float2 &acc, float v) {
    float y = v - acc.y;
    float t = acc.x + y;
    acc.y = (t - acc.x) - y;
    acc.x = t;
}

// Mixed-precision candidate loop (SM: per-warp scratch holding the staged
// centre pairs ipa / ipb / ipc and their slots islot2) of one 32-slot neighbour chunk against the
// NI staged centre-cell particles, two of them per packed f32x2 operation.
// SELF: the chunk holds intra-cell entries (slot order decides the pair);
// The candidate loop's own classification of an r^2 in FP32, with its
// arithmetic: computed in the loop (kClose2 <= r^2 < rc2lo), close (below
// that range: FP64 in the rare path), or neither (the band around r_c^2,
// decided exactly).
__device__ __forceinline__ bool loop_hit(float r2, float rc2lo) {
    const float mid = 0.5f * (rc2lo + kClose2), half = 0.5f * (rc2lo - kClose2);
    return fabsf(r2 + -mid) < half;
}
__device__ __forceinline__ bool loop_close(float r2, float rc2lo) {
    return !loop_hit(r2, rc2lo) && r2 < 0.5f * (rc2lo + kClose2);
}

// STATS: accumulate energy partials and the pair count.
template <int NI, bool N3, bool SELF, bool STATS, typename SM>
__device__ __forceinline__ void pair_loop(const SM &sm, const float (&pj)[3], const float (&lj)[3],
                                          int jlim, int jexcl, float rc2lo, float rc2hi,
                                          float2 (&ax2)[NI / 2], float2 (&ay2)[NI / 2], float2 (&az2)[NI / 2],
                                          float2 &gx, float2 &gy, float2 &gz, float2 &e6, float2 &e12,
                                          int &npair, bool &amb, int kpairs) {
    const float2 one2 = make_float2(1.0f, 1.0f);
    const float mid = 0.5f * (rc2lo + kClose2), half = 0.5f * (rc2lo - kClose2);
    const float2 nmid2 = make_float2(-mid, -mid);
    const float2 c48 = make_float2(48.0f, 48.0f), cm24 = make_float2(-24.0f, -24.0f);
    const float2 npx = make_float2(-pj[0], -pj[0]), npy = make_float2(-pj[1], -pj[1]), npz = make_float2(-pj[2], -pj[2]);
    const float2 nlx = make_float2(-lj[0], -lj[0]), nly = make_float2(-lj[1], -lj[1]), nlz = make_float2(-lj[2], -lj[2]);
#pragma unroll
    for (int m = 0; m < NI / 2; ++m) {
        if (m >= kpairs) break;   // the rest of the tile holds only sentinels (warp-uniform)
        const float4 A = lds4(&sm.ipa[m]);
        const float4 B = lds4(&sm.ipb[m]);
        const float4 C = lds4(&sm.ipc[m]);
        bool oka = true, okb = true;
        if (SELF) {
            const int2 sl = sm.islot2[m];
            oka = N3 ? (sl.x < jlim) : (sl.x != jexcl);
            okb = N3 ? (sl.y < jlim) : (sl.y != jexcl);
        }
        // d = (x_i - x_j,hi) + (r_i - x_j,lo): both residuals carried
        const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(A.x, A.y), npx), __fadd2_rn(make_float2(C.x, C.y), nlx));
        const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(A.z, A.w), npy), __fadd2_rn(make_float2(C.z, C.w), nly));
        const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(B.x, B.y), npz), __fadd2_rn(make_float2(B.z, B.w), nlz));
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
        const bool neara = oka && (r2.x < rc2hi), nearb = okb && (r2.y < rc2hi);
        // FP32 here: kClose2 <= r^2 < rc2lo, as |r^2 - mid| < half (one
        // packed add); the band around r_c^2 and the close pairs go to the
        // rare path, which classifies them by the same arithmetic
        const float2 t = __fadd2_rn(r2, nmid2);
        const bool hita = neara && (fabsf(t.x) < half), hitb = nearb && (fabsf(t.y) < half);
        amb |= (neara && !hita) || (nearb && !hitb);
        float2 y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.x) : "f"(r2.x));
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y.y) : "f"(r2.y));
        const float2 e = __ffma2_rn(make_float2(-r2.x, -r2.y), y, one2);   // Newton step
        y = __ffma2_rn(y, e, y);
        y.x = hita ? y.x : 0.0f;   // masks misses and r2 = 0 (i == j)
        y.y = hitb ? y.y : 0.0f;
        const float2 s6 = __fmul2_rn(__fmul2_rn(y, y), y);
        const float2 f = __fmul2_rn(__fmul2_rn(s6, y), __ffma2_rn(s6, c48, cm24));
        ax2[m] = __ffma2_rn(f, dx, ax2[m]);
        ay2[m] = __ffma2_rn(f, dy, ay2[m]);
        az2[m] = __ffma2_rn(f, dz, az2[m]);
        if (N3) {
            gx = __ffma2_rn(f, dx, gx);
            gy = __ffma2_rn(f, dy, gy);
            gz = __ffma2_rn(f, dz, gz);
        }
        if (STATS) {
            e6 = __fadd2_rn(e6, s6);
            e12 = __ffma2_rn(s6, s6, e12);
            npair += (hita ? 1 : 0) + (hitb ? 1 : 0);
        }
    }
}

__device__ __forceinline__ float staged(const float4 *arr, int k, int comp) {
    // component comp (0: x or z, 1: y or slot) of staged particle k
    const float *f = reinterpret_cast<const float *>(arr);
    return f[4 * (k >> 1) + 2 * comp + (k & 1)];
}

// Device clock, acquire loads and release stores of the device queues.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int atom_add_acq_rel(int *p, int v) {
    int old;
    asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// FP64 force on particle si from sj (slots of the FP64 positions, image
// shift sL of sj), the definition's arithmetic: for the close pairs, whose
// FP32 force would carry the FP32 rounding of r^2 amplified by r^-14.
// Returns s6 = r^-6 for the energy.
__device__ __forceinline__ double pair_force_f64(const double *x, const double *y, const double *z, int si, int sj,
                                                 const double sL[3], double F[3]) {
    const double Dx = __dsub_rn(__dsub_rn(x[si], x[sj]), sL[0]);
    const double Dy = __dsub_rn(__dsub_rn(y[si], y[sj]), sL[1]);
    const double Dz = __dsub_rn(__dsub_rn(z[si], z[sj]), sL[2]);
    const double inv = 1.0 / (Dx * Dx + Dy * Dy + Dz * Dz);
    const double s6 = inv * inv * inv;
    const double fd = s6 * inv * (48.0 * s6 - 24.0);
    F[0] = fd * Dx; F[1] = fd * Dy; F[2] = fd * Dz;
    return s6;
}

// Whether any of three FP64 values is nonzero, by integer operations on
// their bits (a zero of either sign has no bit set below the sign): FP64
// compares would run on the FP64 pipe, a small fraction of the FP32 rate.
__device__ __forceinline__ bool nonzero3(double a, double b, double c) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(a) |
                                    (unsigned long long)__double_as_longlong(b) |
                                    (unsigned long long)__double_as_longlong(c);
    return (bits << 1) != 0ull;
}

// Adds an FP64 value to an FP32 Kahan pair (sum, compensation): as its
// rounded FP32 value and the FP32 rounding of the rest.
__device__ __forceinline__ void kahan_add64(float2 &acc, double v) {
    const float hi = (float)v;
    kahan_add(acc, hi);
    kahan_add(acc, (float)(v - (double)hi));
}

}  // namespace lc
