// Counting-sort binning of the link-cell method (paper Sec. IV: cells of
// side >= r_c, partners only in the 27 surrounding cells).
//
//   k_cellid      wrap, cell index, count per cell (warp-aggregated atomics;
//                 the atomic's return value gives a provisional rank)
//   k_scan_tiles_ticket  exclusive prefix sum of the counts per tile; the
//                 last block scans the tile totals
//   k_scatter_starts  provisional slot start[cell] + rank: source index and
//                 ID; the final cell starts
//   k_rank_gather one thread per slot: final rank = number of the cell's
//                 particles with a smaller ID (so the result does not depend
//                 on the order in which the atomics were served); gather the
//                 FP64 state into that slot and write the FP32
//                 cell-centre-local coordinates of the mixed-precision sweep.
// Cell indices and wraps avoid the FP64 pipe except near a cell face or for
// a coordinate outside (0, L), where the exact FP64 formula decides.
// The final permutation is stable by particle ID inside each cell, so the
// whole binning is bit-exact and reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lc_internal.cuh"

namespace lc {

// BATCHED: slot s belongs to box slot_box[s] (boxes keep their slot ranges),
// whose grid gives the local cell; the global cell adds the box's offset.
// KICKS: velocity-Verlet updates fused in front of the cell index (the
// integrator's pass over the state and the binning's first pass become
// one): 0 none; 1 v += h F, x += dt v (the start of a step); 2 the previous
// step's closing v += h F first (same forces, same FMAs as two launches).
struct Drift {
    double half, dt;
    double *vx, *vy, *vz;
    const double *fx, *fy, *fz;
};

template <bool BATCHED, int KICKS>
__global__ void k_cellid(Grid g1, const BoxDev *__restrict__ boxes, const unsigned short *__restrict__ slot_box, int n,
                         double *__restrict__ x, double *__restrict__ y, double *__restrict__ z, Drift dr,
                         int *__restrict__ cell, int *__restrict__ rank, int *__restrict__ count, int *__restrict__ err) {
    const int lane = threadIdx.x & 31;
    for (int s0 = blockIdx.x * blockDim.x; s0 < n; s0 += gridDim.x * blockDim.x) {
        const int s = s0 + threadIdx.x;
        const bool act = s < n;
        int c = 0;
        if (act) {
            const BoxDev *bd = BATCHED ? &boxes[slot_box[s]] : nullptr;
            const Grid &g = BATCHED ? bd->g : g1;
            double X[3] = {x[s], y[s], z[s]};
            if constexpr (KICKS > 0) {
                double v[3] = {dr.vx[s], dr.vy[s], dr.vz[s]};
                const double f[3] = {dr.fx[s], dr.fy[s], dr.fz[s]};
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    if (KICKS == 2) v[d] = fma(dr.half, f[d], v[d]);
                    v[d] = fma(dr.half, f[d], v[d]);
                    X[d] = fma(dr.dt, v[d], X[d]);
                }
                dr.vx[s] = v[0]; dr.vy[s] = v[1]; dr.vz[s] = v[2];
                x[s] = X[0]; y[s] = X[1]; z[s] = X[2];
            }
            int cc[3];
            bool fast = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Split sp;
                fast = fast && split_f64(X[d], sp) &&
                       cell_coord_fast(sp, g.Lf_lo[d], g.invf[d], g.nc[d], g.cmargin[d], cc[d]);
            }
            if (fast) {
                c = cc[0] + g.nc[0] * (cc[1] + g.nc[1] * cc[2]);
            } else if (isfinite(X[0]) && isfinite(X[1]) && isfinite(X[2])) {
                // exact FP64 path: outside (0, L) or within the margin of a cell face
                for (int d = 0; d < 3; ++d) cc[d] = cell_coord(wrap_coord(X[d], g.L[d]), g.inv[d], g.nc[d]);
                c = cc[0] + g.nc[0] * (cc[1] + g.nc[1] * cc[2]);
            } else {
                atomicOr(err, kErrNonfinite);
            }
            if (BATCHED) c += bd->cell_off;
        }
        // lanes of a warp mostly share cells (the previous order is cell
        // sorted): one atomic per distinct cell, ranks by lane order
        const unsigned mask = __ballot_sync(kFull, act);
        if (act) {
            const unsigned peers = __match_any_sync(mask, c);
            const int leader = __ffs(peers) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(count + c, __popc(peers));
            base = __shfl_sync(peers, base, leader);
            cell[s] = c;
            rank[s] = base + __popc(peers & ((1u << lane) - 1u));
        }
    }
}

// Block-level exclusive scan of the kScanTile counts of tile `tile` into
// out[]; returns the tile's total (valid in every thread).
__device__ __forceinline__ int scan_tile(int tile, int ncell, const int *__restrict__ count, int *__restrict__ out) {
    __shared__ int warp_tot[kScanThreads / 32];
    __shared__ int tile_tot;
    const int base = tile * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < ncell) ? count[base + k] : 0;
        sum += v[k];
    }
    // warp inclusive scan of the thread sums
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = sum;
#pragma unroll
    for (int m = 1; m < 32; m <<= 1) {
        int t = __shfl_up_sync(kFull, inc, m);
        if (lane >= m) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int t = warp_tot[lane];
        int ti = t;
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            int u = __shfl_up_sync(kFull, ti, m);
            if (lane >= m) ti += u;
        }
        warp_tot[lane] = ti - t;   // exclusive
        if (lane == 31) tile_tot = ti;
    }
    __syncthreads();
    int run = warp_tot[wid] + inc - sum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < ncell) out[base + k] = run;
        run += v[k];
    }
    return tile_tot;
}

// In-place exclusive scan of partial[0, ntiles) by one block (loops if there
// are more tiles than threads).
__device__ __forceinline__ void scan_partials(int ntiles, int *partial) {
    __shared__ int warp_tot[kScanThreads / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b0 = 0; b0 < ntiles; b0 += kScanThreads) {
        int i = b0 + threadIdx.x;
        int v = i < ntiles ? __ldcg(&partial[i]) : 0;
        int inc = v;
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            int t = __shfl_up_sync(kFull, inc, m);
            if (lane >= m) inc += t;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int t = warp_tot[lane];
            int ti = t;
#pragma unroll
            for (int m = 1; m < 32; m <<= 1) {
                int u = __shfl_up_sync(kFull, ti, m);
                if (lane >= m) ti += u;
            }
            warp_tot[lane] = ti - t;
        }
        __syncthreads();
        int c0 = carry;
        if (i < ntiles) partial[i] = c0 + warp_tot[wid] + inc - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = c0 + warp_tot[wid] + inc;
        __syncthreads();
    }
}

// Tile scans into local[] and the tile totals to partial[]; the block that
// finishes last (a ticket counter, no waiting) scans the totals in place, so
// partial[k] becomes the start of tile k, and resets the ticket for the next
// launch.  Cell c then starts at local[c] + partial[c / kScanTile], which
// k_scatter_starts writes out.
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles_ticket(int ncell, const int *__restrict__ count,
                                                                   int *__restrict__ local, int *partial,
                                                                   unsigned *ticket) {
    __shared__ bool last;
    const int tot = scan_tile(blockIdx.x, ncell, count, local);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = tot;
        __threadfence();   // the total is visible before the ticket is taken
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();       // every other block's total is visible
    scan_partials(gridDim.x, partial);
    if (threadIdx.x == 0) *ticket = 0u;
}

// Provisional slot of every particle (cell start + the rank its count
// atomic returned): its source index and ID (identity when id is null).
// The cell start is the tile-local start plus the tile's start; the same
// threads then write every cell's final start (and start[ncell] = n).
__global__ void k_scatter_starts(int n, int ncell, const int *__restrict__ cell, const int *__restrict__ rank,
                                 const int *__restrict__ local, const int *__restrict__ partial,
                                 const int *__restrict__ id, int *__restrict__ src, int *__restrict__ key,
                                 int *__restrict__ start, int *__restrict__ cellt) {
    const int stride = gridDim.x * blockDim.x;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += stride) {
        const int c = cell[s];
        const int t = local[c] + partial[c / kScanTile] + rank[s];
        src[t] = s;
        key[t] = id ? id[s] : s;
        if (cellt) cellt[t] = c;
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += stride)
        start[c] = local[c] + partial[c / kScanTile];
    if (blockIdx.x == 0 && threadIdx.x == 0) start[ncell] = n;
}

// One thread per slot t of the new order (its cell from the scatter).  Rank = number of the cell's
// particles with a smaller ID (IDs are unique), so slot = start + rank is
// stable by ID whatever order the atomics were served in.
template <bool BATCHED>
__global__ void k_rank_gather(Grid g1, const BoxDev *__restrict__ boxes, const unsigned short *__restrict__ slot_box,
                              int n, int write_p4, const int *__restrict__ start,
                              const int *__restrict__ count, const int *__restrict__ cellt,
                              const int *__restrict__ src, const int *__restrict__ key, State in, State out,
                              float4 *__restrict__ p4) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int s = src[t];
        const int my_id = key[t];
        const int c = cellt[t];   // written by the scatter: no dependent gather through src
        // the particle's state is loaded before the rank loop so that its
        // latency overlaps the key loads
        double X[3] = {in.x[s], in.y[s], in.z[s]};
        const double V[3] = {in.vx[s], in.vy[s], in.vz[s]};
        const int base = start[c], cnt = count[c];
        // four independent loads in flight per step (the keys are L1 hits
        // shared with the cell's other slots; the loop is latency-bound)
        int r = 0, k = 0;
        for (; k + 4 <= cnt; k += 4) {
            const int k0 = key[base + k], k1 = key[base + k + 1], k2 = key[base + k + 2], k3 = key[base + k + 3];
            r += (k0 < my_id ? 1 : 0) + (k1 < my_id ? 1 : 0) + (k2 < my_id ? 1 : 0) + (k3 < my_id ? 1 : 0);
        }
        for (; k < cnt; ++k) r += (key[base + k] < my_id) ? 1 : 0;
        const int dst = base + r;
        const BoxDev *bd = BATCHED ? &boxes[slot_box[t]] : nullptr;
        const Grid &g = BATCHED ? bd->g : g1;
        const int cl = BATCHED ? c - bd->cell_off : c;
        int cc[3];
        cell_coords(g, cl, cc);
        Split sp[3];
        bool fast = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) fast = fast && split_f64(X[d], sp[d]) && sp[d].hi > 0.0f && sp[d].hi < g.Lf_lo[d];
        if (!fast) {
            // exact wrap (rare: the particle left the box or sits at 0)
            for (int d = 0; d < 3; ++d) {
                X[d] = wrap_coord(X[d], g.L[d]);
                if (!split_f64(X[d], sp[d])) sp[d].hi = sp[d].lo = 0.0f;
            }
        }
        out.x[dst] = X[0]; out.y[dst] = X[1]; out.z[dst] = X[2];
        out.vx[dst] = V[0]; out.vy[dst] = V[1]; out.vz[dst] = V[2];
        out.id[dst] = my_id;
        if (write_p4) p4[dst] = cell_offset_p4(g, sp, cc);
    }
}

__global__ void k_colour(Grid g, int8_t *colour) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < g.ncell; c += gridDim.x * blockDim.x) {
        int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
        int raw = colour_class(cx, g.nc[0]) + 3 * colour_class(cy, g.nc[1]) + 9 * colour_class(cz, g.nc[2]);
        colour[c] = (int8_t)g.colour_of_raw[raw];
    }
}

cudaError_t launch_colour(Ctx *c, cudaStream_t s) {
    k_colour<<<c->num_sms * 4, 256, 0, s>>>(c->g, c->d_colour);
    return cudaGetLastError();
}

// One resident wave of 256-thread blocks of `kernel` (its register count
// decides how many fit on an SM): the grid-stride loops then run without a
// partial second wave.
template <typename K>
static int one_wave(const Ctx *c, K kernel, int *cache) {
    if (!*cache) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1) {
            cudaGetLastError();
            per_sm = 4;
        }
        *cache = per_sm;
    }
    return c->num_sms * *cache;
}

template <bool BATCHED, int KICKS>
static void cellid_launch(Ctx *c, int, const Drift &dr, cudaStream_t s) {
    static int per_sm = 0;
    const int grid_n = one_wave(c, k_cellid<BATCHED, KICKS>, &per_sm);
    k_cellid<BATCHED, KICKS><<<grid_n, 256, 0, s>>>(c->g, BATCHED ? c->d_boxes : nullptr,
                                                    BATCHED ? c->d_slot_box : nullptr, (int)c->n, c->cur.x, c->cur.y,
                                                    c->cur.z, dr, c->d_cell, c->d_rank, c->d_count, c->d_err);
}

cudaError_t launch_bin(Ctx *c, cudaStream_t s, int *launches, int kicks, double dt) {
    const int n = (int)c->n;
    const int ncell = c->g.ncell;
    const int ntiles = (ncell + kScanTile - 1) / kScanTile;
    const int grid_n = c->num_sms * 8;
    cudaError_t e = cudaMemsetAsync(c->d_count, 0, sizeof(int) * (size_t)ncell, s);
    if (e) return e;
    if (n > 0) {
        Drift dr;
        dr.half = 0.5 * dt; dr.dt = dt;
        dr.vx = c->cur.vx; dr.vy = c->cur.vy; dr.vz = c->cur.vz;
        dr.fx = c->fx; dr.fy = c->fy; dr.fz = c->fz;
        const bool b = c->nbox > 0;
        if (kicks == 0) b ? cellid_launch<true, 0>(c, grid_n, dr, s) : cellid_launch<false, 0>(c, grid_n, dr, s);
        else if (kicks == 1) b ? cellid_launch<true, 1>(c, grid_n, dr, s) : cellid_launch<false, 1>(c, grid_n, dr, s);
        else b ? cellid_launch<true, 2>(c, grid_n, dr, s) : cellid_launch<false, 2>(c, grid_n, dr, s);
        ++*launches;
    }
    // two-pass scan: tile scans (the last tile block scans the tile totals),
    // then the starts completed inside k_scatter_starts
    int *local = c->d_start + (ncell + 1);
    unsigned *ticket = reinterpret_cast<unsigned *>(c->d_blocksums + ntiles);
    k_scan_tiles_ticket<<<ntiles, kScanThreads, 0, s>>>(ncell, c->d_count, local, c->d_blocksums, ticket);
    k_scatter_starts<<<grid_n, 256, 0, s>>>(n, ncell, c->d_cell, c->d_rank, local, c->d_blocksums, c->cur.id,
                                            c->d_src, c->d_key, c->d_start, c->d_cellt);
    *launches += 2;
    if (n > 0) {
        static int per_sm_b = 0, per_sm_s = 0;
        if (c->nbox > 0)
            k_rank_gather<true><<<one_wave(c, k_rank_gather<true>, &per_sm_b), 256, 0, s>>>(
                c->g, c->d_boxes, c->d_slot_box, n, c->prec == LC_PREC_MIXED, c->d_start, c->d_count, c->d_cellt,
                c->d_src, c->d_key, c->cur, c->nxt, c->d_p4);
        else
            k_rank_gather<false><<<one_wave(c, k_rank_gather<false>, &per_sm_s), 256, 0, s>>>(
                c->g, nullptr, nullptr, n, c->prec == LC_PREC_MIXED, c->d_start, c->d_count, c->d_cellt, c->d_src,
                c->d_key, c->cur, c->nxt, c->d_p4);
        *launches += 1;
    }
    e = cudaGetLastError();
    if (e) return e;
    State t = c->cur; c->cur = c->nxt; c->nxt = t;
    c->list_valid = false;   // the slot order changed
    return cudaSuccess;
}

// ---------------------------------------------------------- state I/O ---
// New state from [n][3] arrays in one pass: positions, velocities (zero
// when vel is null), identity IDs, and the block partials of v^2.  2D
// contexts: the particles sit at z = zval inside the single cell layer (a
// value away from the layer's faces) with vz = 0; the z the caller gave is
// ignored.
__global__ void __launch_bounds__(kKinThreads) k_set_state(int n, const double *__restrict__ pos,
                                                           const double *__restrict__ vel, int plane, double zval,
                                                           State st, double *__restrict__ kin_part) {
    __shared__ double red[kKinThreads];
    double acc = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const double x = pos[3 * (size_t)s], y = pos[3 * (size_t)s + 1];
        const double z = plane ? zval : pos[3 * (size_t)s + 2];
        double vx = 0.0, vy = 0.0, vz = 0.0;
        if (vel) {
            vx = vel[3 * (size_t)s]; vy = vel[3 * (size_t)s + 1];
            vz = plane ? 0.0 : vel[3 * (size_t)s + 2];
        }
        st.x[s] = x; st.y[s] = y; st.z[s] = z;
        st.vx[s] = vx; st.vy[s] = vy; st.vz[s] = vz;
        st.id[s] = s;
        acc = kin_add(acc, vx, vy, vz);
    }
    const double t = block_sum_kin(acc, red);
    if (threadIdx.x == 0) kin_part[blockIdx.x] = t;
}

// dst[id[s]] = (a[s], b[s], c[s]); wrap != 0 wraps positions into [0, L);
// 2D contexts report z components as 0.
__global__ void k_unsort_vec(int n, Grid g1, const BoxDev *__restrict__ boxes, const unsigned short *__restrict__ slot_box,
                             int wrap, const int *__restrict__ id, const double *__restrict__ a,
                             const double *__restrict__ b, const double *__restrict__ cc, double *__restrict__ dst) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        double va = a[s], vb = b[s], vc = cc[s];
        const Grid &g = boxes ? boxes[slot_box[s]].g : g1;
        if (wrap) {
            va = wrap_coord(va, g.L[0]); vb = wrap_coord(vb, g.L[1]); vc = wrap_coord(vc, g.L[2]);
        }
        if (g.dims == 2) vc = 0.0;
        int i = id[s];
        dst[3 * i + 0] = va; dst[3 * i + 1] = vb; dst[3 * i + 2] = vc;
    }
}

cudaError_t launch_set_state(Ctx *c, const double *pos, const double *vel, cudaStream_t s) {
    const int n = (int)c->n;
    c->kin_valid = c->kin_final = false;
    if (n == 0) return cudaSuccess;
    k_set_state<<<kinetic_blocks(c), kKinThreads, 0, s>>>(n, pos, vel, c->g.dims == 2, 0.25 * c->g.L[2], c->cur,
                                                          c->d_kin_part);
    cudaError_t e = cudaGetLastError();
    if (!e) c->kin_valid = true;
    return e;
}

cudaError_t launch_unsort_vec(Ctx *c, const double *a, const double *b, const double *cc, double *dst,
                              cudaStream_t s, int wrap) {
    const int n = (int)c->n;
    if (n == 0) return cudaSuccess;
    k_unsort_vec<<<c->num_sms * 8, 256, 0, s>>>(n, c->g, c->nbox > 0 ? c->d_boxes : nullptr, c->d_slot_box, wrap,
                                                 c->cur.id, a, b, cc, dst);
    return cudaGetLastError();
}

}  // namespace lc
