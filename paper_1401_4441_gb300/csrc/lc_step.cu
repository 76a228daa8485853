// Velocity-Verlet integration (m = 1) and the FP64 reductions of energy,
// virial and kinetic energy.  All state lives in cell-sorted order, so the
// integrator streams contiguous FP64 arrays:
//   v <- v + (dt/2) F,  x <- x + dt v   (wrap happens in the next binning),
// each update one FP64 fused multiply-add (one rounding).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lc_internal.cuh"

namespace lc {

// K = 1/2 sum of the block partials of v^2, in a fixed order: thread t adds
// partials t, t + kKinThreads, ... ascending (four loads in flight; the
// zeros past the end leave the non-negative sum unchanged), then the
// block's tree.
__device__ __forceinline__ double final_kin(int nb, const double *part, double *red) {
    double a = 0.0;
    for (int b0 = 0; b0 < nb; b0 += 4 * kKinThreads) {
        double v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int b = b0 + r * kKinThreads + (int)threadIdx.x;
            v[r] = b < nb ? __ldcg(part + b) : 0.0;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) a = __dadd_rn(a, v[r]);
    }
    return 0.5 * block_sum_kin(a, red);
}

// U, W and the pair count from nw statistics slots (s6, s12 at [4 w],
// [4 w + 1], the pair count in pairs[w]), summed by one block of kKinThreads
// threads in a fixed order: thread t takes slots t, t + kKinThreads, ...,
// then a butterfly inside each warp, then the warps in order.  The full
// shell sees every pair twice.  out[0] = U, out[1] = W, out[2] = pairs.
struct PotArgs {
    int nw;                      // slots (0: nothing to sum)
    int full;
    const double *acc;
    const long long *pairs;
    double *out;
    long long *npairs;
};
__device__ __forceinline__ void pot_sum(const PotArgs &p) {
    __shared__ double r6[kKinThreads / 32], r12[kKinThreads / 32];
    __shared__ long long rp[kKinThreads / 32];
    double a6 = 0.0, a12 = 0.0;
    long long ap = 0;
    for (int w = threadIdx.x; w < p.nw; w += kKinThreads) {
        a6 += p.acc[4 * w + 0];
        a12 += p.acc[4 * w + 1];
        ap += p.pairs[w];
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) {
        a6 += __shfl_xor_sync(0xffffffffu, a6, m);
        a12 += __shfl_xor_sync(0xffffffffu, a12, m);
        ap += __shfl_xor_sync(0xffffffffu, ap, m);
    }
    if ((threadIdx.x & 31) == 0) { r6[threadIdx.x >> 5] = a6; r12[threadIdx.x >> 5] = a12; rp[threadIdx.x >> 5] = ap; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s6 = r6[0], s12 = r12[0];
        long long sp = rp[0];
        for (int w = 1; w < kKinThreads / 32; ++w) { s6 += r6[w]; s12 += r12[w]; sp += rp[w]; }
        const double scale = p.full ? 0.5 : 1.0;
        p.out[0] = scale * 4.0 * (s12 - s6);          // U = 4 sum (r^-12 - r^-6)
        p.out[1] = scale * 24.0 * (2.0 * s12 - s6);   // W = sum r.F = 24 sum (2 r^-12 - r^-6)
        const long long np = p.full ? sp / 2 : sp;
        p.out[2] = (double)np;
        *p.npairs = np;
    }
}

__global__ void __launch_bounds__(kKinThreads) k_final_pot(PotArgs p) { pot_sum(p); }

// Closing half-kick v <- v + (dt/2) F.  KIN: fused with the kinetic energy
// of the new velocities -- each block forms the partial sum of v^2 that
// k_kinetic would (same grid, same particles per thread, same order), and
// the block that finishes last (ticket) adds the partials with final_kin
// into the result block, so K needs no further pass.  pot.nw > 0: block 0
// first sums the force sweep's statistics slots (pot_sum), in place of a
// launch of k_final_pot between the sweep and the kick.
template <bool KIN>
__global__ void __launch_bounds__(kKinThreads) k_kick(int n, double half, State st, const double *__restrict__ fx,
                                                      const double *__restrict__ fy, const double *__restrict__ fz,
                                                      double *__restrict__ part, unsigned *ticket,
                                                      double *__restrict__ out, PotArgs pot) {
    if (pot.nw > 0 && blockIdx.x == 0) pot_sum(pot);
    double acc = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const double vx = fma(half, fx[s], st.vx[s]);
        const double vy = fma(half, fy[s], st.vy[s]);
        const double vz = fma(half, fz[s], st.vz[s]);
        st.vx[s] = vx;
        st.vy[s] = vy;
        st.vz[s] = vz;
        if (KIN) acc = kin_add(acc, vx, vy, vz);
    }
    if constexpr (!KIN) return;
    __shared__ double red[kKinThreads];
    __shared__ bool last;
    const double t = block_sum_kin(acc, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = t;
        __threadfence();   // the partial is visible before the ticket counts it
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const double k = final_kin(gridDim.x, part, red);
    if (threadIdx.x == 0) {
        out[3] = k;
        *ticket = 0u;   // ready for the next launch
    }
}

// Block partial sums of v^2 (grid-stride, fixed assignment: deterministic;
// the same arithmetic as the partials the state set-up forms).
__global__ void __launch_bounds__(kKinThreads) k_kinetic(int n, State st, double *__restrict__ part) {
    __shared__ double red[kKinThreads];
    double acc = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        acc = kin_add(acc, st.vx[s], st.vy[s], st.vz[s]);
    const double t = block_sum_kin(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kKinThreads) k_final_kin(int nb, const double *__restrict__ part,
                                                           double *__restrict__ out) {
    __shared__ double red[kKinThreads];
    const double k = final_kin(nb, part, red);
    if (threadIdx.x == 0) out[3] = k;
}

// Per-box statistics of a batch: U, W and pair count from the box
// accumulators of the force kernel (full shell: each pair seen twice).
__global__ void k_box_energy(int nbox, int full, const double *__restrict__ acc,
                             const unsigned long long *__restrict__ pairs, double *__restrict__ out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbox; b += gridDim.x * blockDim.x) {
        const double scale = full ? 0.5 : 1.0;
        const double s6 = acc[2 * b], s12 = acc[2 * b + 1];
        out[4 * b + 0] = scale * 4.0 * (s12 - s6);
        out[4 * b + 1] = scale * 24.0 * (2.0 * s12 - s6);
        out[4 * b + 2] = (double)(full ? pairs[b] / 2 : pairs[b]);
    }
}

// Kinetic energy per box: one block per box over its slot range, fixed order.
__global__ void __launch_bounds__(256) k_box_kinetic(const BoxDev *__restrict__ boxes, State st, double *__restrict__ out) {
    __shared__ double red[256];
    const BoxDev &bd = boxes[blockIdx.x];
    double acc = 0.0;
    for (int s = bd.part_off + threadIdx.x; s < bd.part_off + bd.n; s += blockDim.x) {
        const double vx = st.vx[s], vy = st.vy[s], vz = st.vz[s];
        acc += vx * vx + vy * vy + vz * vz;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int m = 128; m > 0; m >>= 1) {
        if (threadIdx.x < m) red[threadIdx.x] += red[threadIdx.x + m];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[4 * blockIdx.x + 3] = 0.5 * red[0];
}

// Per-box statistics from per-cell partials: one block per box, its cells in
// order, a fixed reduction tree (the same bits on every run).
__global__ void __launch_bounds__(256) k_box_energy_cells(const BoxDev *__restrict__ boxes,
                                                          const double *__restrict__ acc,
                                                          const long long *__restrict__ pairs,
                                                          double *__restrict__ out) {
    __shared__ double r6[256], r12[256];
    __shared__ long long rp[256];
    const BoxDev &bd = boxes[blockIdx.x];
    double a6 = 0.0, a12 = 0.0;
    long long ap = 0;
    for (int c = bd.cell_off + threadIdx.x; c < bd.cell_off + bd.g.ncell; c += blockDim.x) {
        a6 += acc[4 * (size_t)c];
        a12 += acc[4 * (size_t)c + 1];
        ap += pairs[c];
    }
    r6[threadIdx.x] = a6; r12[threadIdx.x] = a12; rp[threadIdx.x] = ap;
    __syncthreads();
    for (int m = 128; m > 0; m >>= 1) {
        if (threadIdx.x < m) {
            r6[threadIdx.x] += r6[threadIdx.x + m];
            r12[threadIdx.x] += r12[threadIdx.x + m];
            rp[threadIdx.x] += rp[threadIdx.x + m];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[4 * blockIdx.x + 0] = 4.0 * (r12[0] - r6[0]);
        out[4 * blockIdx.x + 1] = 24.0 * (2.0 * r12[0] - r6[0]);
        out[4 * blockIdx.x + 2] = (double)rp[0];
    }
}

cudaError_t launch_box_energy_cells(Ctx *c, cudaStream_t s) {
    k_box_energy_cells<<<c->nbox, 256, 0, s>>>(c->d_boxes, c->d_cell_acc, c->d_cell_pairs, c->d_box_out);
    return cudaGetLastError();
}

cudaError_t launch_box_energy(Ctx *c, cudaStream_t s, int full) {
    k_box_energy<<<(c->nbox + 255) / 256, 256, 0, s>>>(c->nbox, full, c->d_box_acc, c->d_box_pairs, c->d_box_out);
    return cudaGetLastError();
}

cudaError_t launch_box_kinetic(Ctx *c, cudaStream_t s) {
    k_box_kinetic<<<c->nbox, 256, 0, s>>>(c->d_boxes, c->cur, c->d_box_out);
    return cudaGetLastError();
}

static PotArgs pot_args(const Ctx *c, int full) {
    PotArgs p;
    p.nw = c->nwarp_used > 0 ? c->nwarp_used : c->nwarp_max;   // the rest are zero
    p.full = full;
    p.acc = c->d_warp_acc;
    p.pairs = c->d_warp_pairs;
    p.out = c->d_result;
    p.npairs = c->d_npairs;
    return p;
}

cudaError_t launch_kick(Ctx *c, double dt, cudaStream_t s, bool kin, bool pot) {
    if (c->n == 0) return pot ? launch_energy_reduce(c, s, c->stats_full) : cudaSuccess;
    PotArgs p = pot_args(c, c->stats_full);
    if (!pot) p.nw = 0;
    if (kin)
        k_kick<true><<<kinetic_blocks(c), kKinThreads, 0, s>>>((int)c->n, 0.5 * dt, c->cur, c->fx, c->fy, c->fz,
                                                               c->d_kin_part, c->d_kin_ticket, c->d_result, p);
    else
        k_kick<false><<<kinetic_blocks(c), kKinThreads, 0, s>>>((int)c->n, 0.5 * dt, c->cur, c->fx, c->fy, c->fz,
                                                                nullptr, nullptr, nullptr, p);
    return cudaGetLastError();
}

int kinetic_blocks(const Ctx *c) { return c->num_sms * 8; }

// K into the result block.  Nothing to do when a closing kick with the
// kinetic energy (k_kick<true>) or an earlier call already put the current
// velocities' K there; the pass over the velocities is skipped while the
// partials still describe them (the state set-up and the kick form them).
cudaError_t launch_kinetic(Ctx *c, cudaStream_t s) {
    if (c->kin_final) return cudaSuccess;
    const int nb = kinetic_blocks(c);
    double *part = c->d_kin_part;
    if (!c->kin_valid) k_kinetic<<<nb, kKinThreads, 0, s>>>((int)c->n, c->cur, part);
    k_final_kin<<<1, kKinThreads, 0, s>>>(nb, part, c->d_result);
    cudaError_t e = cudaGetLastError();
    if (!e) c->kin_valid = c->kin_final = true;
    return e;
}

// First level of the per-cell partials' sum: block b takes the cells of
// one contiguous range, its threads a fixed stride within it, then a fixed
// tree: partials in the per-warp slots' layout for k_final_pot.
__global__ void __launch_bounds__(256) k_cell_parts(int n, int per_block, const double *__restrict__ acc,
                                                    const long long *__restrict__ pairs,
                                                    double *__restrict__ part, long long *__restrict__ part_pairs) {
    __shared__ double r6[256], r12[256];
    __shared__ long long rp[256];
    const int c0 = blockIdx.x * per_block, c1 = min(n, c0 + per_block);
    double a6 = 0.0, a12 = 0.0;
    long long ap = 0;
    for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
        a6 += acc[4 * (size_t)c];
        a12 += acc[4 * (size_t)c + 1];
        ap += pairs[c];
    }
    r6[threadIdx.x] = a6; r12[threadIdx.x] = a12; rp[threadIdx.x] = ap;
    __syncthreads();
    for (int m = 128; m > 0; m >>= 1) {
        if (threadIdx.x < m) {
            r6[threadIdx.x] += r6[threadIdx.x + m];
            r12[threadIdx.x] += r12[threadIdx.x + m];
            rp[threadIdx.x] += rp[threadIdx.x + m];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[4 * blockIdx.x + 0] = r6[0];
        part[4 * blockIdx.x + 1] = r12[0];
        part_pairs[blockIdx.x] = rp[0];
    }
}

// U, W and the pair count from n per-cell partials (acc[4 c], acc[4 c + 1]:
// sums of r^-6 and r^-12; pairs[c]) in two fixed-order levels: many blocks
// over contiguous cell ranges into the per-warp slots, then k_final_pot.
cudaError_t launch_energy_reduce_parts(Ctx *c, cudaStream_t s, int full, const double *acc, const long long *pairs,
                                       int n) {
    int nb = std::min(c->nwarp_max, 2 * c->num_sms);
    const int per_block = std::max(256, (n + nb - 1) / nb);
    nb = std::max(1, (n + per_block - 1) / per_block);
    k_cell_parts<<<nb, 256, 0, s>>>(n, per_block, acc, pairs, c->d_warp_acc, c->d_warp_pairs);
    PotArgs p = pot_args(c, full);
    p.nw = nb;
    k_final_pot<<<1, kKinThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_energy_reduce(Ctx *c, cudaStream_t s, int full) {
    k_final_pot<<<1, kKinThreads, 0, s>>>(pot_args(c, full));
    return cudaGetLastError();
}

}  // namespace lc
