// Allocation-free binning: lc_bin_noalloc (declared in include/lc.h).
//
// Some callers cannot allocate device memory: code that runs while a CUDA
// graph is being captured by someone else, callers that own a fixed memory
// budget (a pool handed to them by a framework or a real-time loop that must
// not touch the allocator), and embedded users that only hand over
// pointers.  For them this file offers one entry point that performs the
// counting-sort binning of the link-cell method on caller-owned device
// buffers and allocates nothing: its scratch (cell index, provisional rank,
// slot source, key per particle, cell starts, scan partials) lives in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// Limits: at most kNoAllocMaxParticles particles and kNoAllocMaxCells cells
// per call (about 25 MB of device memory in total).  All calls share the one
// array and it keeps the contents of the last call: calls that overlap on the
// GPU (different streams without ordering, or several host threads) race.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "lc_internal.cuh"

namespace lc {

constexpr int64_t kNoAllocMaxParticles = int64_t(1) << 20;
constexpr int64_t kNoAllocMaxCells = int64_t(1) << 20;
constexpr int kNoAllocTiles = (int)((kNoAllocMaxCells + kScanTile - 1) / kScanTile) + 1;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
    int cell[kNoAllocMaxParticles];
    int rank[kNoAllocMaxParticles];
    int src[kNoAllocMaxParticles];
    int key[kNoAllocMaxParticles];
    int start[kNoAllocMaxCells + 1];
    int local[kNoAllocMaxCells + 1];
    int partial[kNoAllocTiles];
    unsigned ticket;   // zero at load; the scan resets it after each use
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Cell of every particle of an [n][3] position array (variant of k_cellid:
// interleaved input, identity IDs).  Counts go to the caller's array.
__global__ void k_na_cellid(Grid g, int n, const double *__restrict__ pos, int *__restrict__ cell,
                            int *__restrict__ rank, int *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    for (int s0 = blockIdx.x * blockDim.x; s0 < n; s0 += gridDim.x * blockDim.x) {
        const int s = s0 + threadIdx.x;
        const bool act = s < n;
        int c = 0;
        if (act) {
            const double X[3] = {pos[3 * s + 0], pos[3 * s + 1], pos[3 * s + 2]};
            int cc[3];
            bool fast = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Split sp;
                fast = fast && split_f64(X[d], sp) &&
                       cell_coord_fast(sp, g.Lf_lo[d], g.invf[d], g.nc[d], g.cmargin[d], cc[d]);
            }
            if (!fast && isfinite(X[0]) && isfinite(X[1]) && isfinite(X[2])) {
                for (int d = 0; d < 3; ++d) cc[d] = cell_coord(wrap_coord(X[d], g.L[d]), g.inv[d], g.nc[d]);
                fast = true;
            }
            // non-finite positions are binned into cell 0
            if (fast) c = cc[0] + g.nc[0] * (cc[1] + g.nc[1] * cc[2]);
        }
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

// Final slot = cell start + number of the cell's particles with a smaller ID.
__global__ void k_na_rank(int n, const int *__restrict__ start, const int *__restrict__ count,
                          const int *__restrict__ cell, const int *__restrict__ src, const int *__restrict__ key,
                          int *__restrict__ perm) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int my_id = key[t];
        const int c = cell[src[t]];
        const int base = start[c], cnt = count[c];
        int r = 0;
        for (int k = 0; k < cnt; ++k) r += (key[base + k] < my_id) ? 1 : 0;
        perm[base + r] = my_id;
    }
}

// Device address of the scratch array, looked up with the device current
// and cached per device together with the ID of the CUDA context it was
// looked up in: after cudaDeviceReset (or with another context current) the
// context ID differs and the address is looked up again, so a kernel never
// gets an address from a context that no longer exists.  The context ID
// comes from the driver's cuCtxGetCurrent / cuCtxGetId, reached through the
// runtime's driver entry points (no link against the driver library).
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

static cudaError_t current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return cudaErrorContextIsDestroyed;
    return get_id(ctx, id) == 0 ? cudaSuccess : cudaErrorContextIsDestroyed;
}

static cudaError_t scratch_address(NoAllocScratch **out) {
    static std::mutex mu;
    static NoAllocScratch *addr[kMaxDevices] = {nullptr};
    static unsigned long long ctx_of[kMaxDevices] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    unsigned long long ctx = 0;
    if (addr[dev]) {
        e = current_context_id(&ctx);
        if (e != cudaSuccess) return e;
    }
    if (!addr[dev] || ctx != ctx_of[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // also creates the context if needed
        if (e != cudaSuccess) return e;
        if ((e = current_context_id(&ctx)) != cudaSuccess) return e;
        addr[dev] = static_cast<NoAllocScratch *>(p);
        ctx_of[dev] = ctx;
    }
    *out = addr[dev];
    return cudaSuccess;
}

}  // namespace lc

using namespace lc;

extern "C" lc_status lc_bin_noalloc(const double *pos, int64_t n, const double box[3], double rc,
                                    int32_t *cell_count, int32_t *cell_start, int32_t *perm, void *stream) {
    if (!box || !(rc > 0.0) || n < 0 || !cell_count || !cell_start || (n > 0 && (!pos || !perm)))
        return LC_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(box[d] > 0.0) || !isfinite(box[d])) return LC_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (floor(box[d] / rc) < 3.0) return LC_ERR_BOX_TOO_SMALL;
    if (n > kNoAllocMaxParticles) return LC_ERR_TOO_LARGE;
    if (floor(box[0] / rc) * floor(box[1] / rc) * floor(box[2] / rc) > (double)kNoAllocMaxCells)
        return LC_ERR_TOO_LARGE;

    // an error left pending by the caller's earlier work is not ours to
    // clear: report it and leave it pending
    if (cudaPeekAtLastError() != cudaSuccess) return LC_ERR_CUDA;
    NoAllocScratch *sc = nullptr;
    cudaError_t e = scratch_address(&sc);
    if (e != cudaSuccess) { cudaGetLastError(); return LC_ERR_CUDA; }
    Grid g;
    make_grid(&g, box, rc);
    const int ncell = g.ncell;
    const int nn = (int)n;
    const int ntiles = (ncell + kScanTile - 1) / kScanTile;
    cudaStream_t s = (cudaStream_t)stream;
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid_n = (nsm > 0 ? nsm : 1) * 8;
    if ((e = cudaMemsetAsync(cell_count, 0, sizeof(int32_t) * (size_t)ncell, s)) != cudaSuccess) {
        cudaGetLastError();
        return LC_ERR_CUDA;
    }
    if (nn > 0) k_na_cellid<<<grid_n, 256, 0, s>>>(g, nn, pos, sc->cell, sc->rank, cell_count);
    k_scan_tiles_ticket<<<ntiles, kScanThreads, 0, s>>>(ncell, cell_count, sc->local, sc->partial, &sc->ticket);
    k_scatter_starts<<<grid_n, 256, 0, s>>>(nn, ncell, sc->cell, sc->rank, sc->local, sc->partial, nullptr, sc->src,
                                            sc->key, sc->start);
    if (nn > 0) {
        k_na_rank<<<grid_n, 256, 0, s>>>(nn, sc->start, cell_count, sc->cell, sc->src, sc->key, perm);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cell_start, sc->start, sizeof(int32_t) * (size_t)ncell, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) { cudaGetLastError(); return LC_ERR_CUDA; }
    return LC_OK;
}
