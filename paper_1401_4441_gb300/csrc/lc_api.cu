// Host side of the C ABI declared in include/lc.h: context set-up, buffer
// ownership, call-order checks, CUDA-graph capture of the Verlet step.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <vector>
#include <algorithm>
#include <utility>
#include "lc_internal.cuh"

namespace lc {

void make_stencil(Stencil *s, int dims) {
    memset(s, 0, sizeof(*s));
    const int zlo = dims == 2 ? 0 : -1, zhi = dims == 2 ? 0 : 1;
    int k = 0;
    for (int oz = zlo; oz <= zhi; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                bool fwd = oz > 0 || (oz == 0 && oy > 0) || (oz == 0 && oy == 0 && ox > 0);
                if (!fwd) continue;
                s->hs[k][0] = ox; s->hs[k][1] = oy; s->hs[k][2] = oz;
                ++k;
            }
    s->nh = k;
    // Offsets with pairwise different parity patterns (|ox|,|oy|,|oz|) may
    // share a colour phase: two same-colour cells differ by an even number of
    // cells per dimension, so A + o == A' + o' forces o == o' (mod 2).
    // Each offset goes to the first group that lacks its pattern.
    bool used[4][8] = {};
    int cnt[4] = {0, 0, 0, 0};
    int members[4][13];
    for (int i = 0; i < s->nh; ++i) {
        int pat = (s->hs[i][0] != 0) + 2 * (s->hs[i][1] != 0) + 4 * (s->hs[i][2] != 0);
        int g = 0;
        while (used[g][pat]) ++g;
        used[g][pat] = true;
        s->group_of[i] = g;
        members[g][cnt[g]++] = i;
    }
    int pos = 0;
    for (int g = 0; g < 4; ++g) {
        s->group_first[g] = pos;
        for (int i = 0; i < cnt[g]; ++i) s->group_list[pos++] = members[g][i];
    }
    s->group_first[4] = pos;
    // full shell: centre first, then the others in (z, y, x) order
    s->full[0][0] = s->full[0][1] = s->full[0][2] = 0;
    int f = 1;
    for (int oz = zlo; oz <= zhi; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                if (!ox && !oy && !oz) continue;
                s->full[f][0] = ox; s->full[f][1] = oy; s->full[f][2] = oz;
                ++f;
            }
    s->nf = f;
    // differences of two entries of the centre + forward stencil: the
    // offsets between cells whose tasks can write a common cell
    int ent[14][3] = {{0, 0, 0}};
    for (int k = 0; k < s->nh; ++k)
        for (int d = 0; d < 3; ++d) ent[k + 1][d] = s->hs[k][d];
    s->ndep = 0;
    for (int a = 0; a <= s->nh; ++a)
        for (int b = 0; b <= s->nh; ++b) {
            const int o[3] = {ent[a][0] - ent[b][0], ent[a][1] - ent[b][1], ent[a][2] - ent[b][2]};
            if (!o[0] && !o[1] && !o[2]) continue;
            bool seen = false;
            for (int k = 0; k < s->ndep && !seen; ++k)
                seen = s->dep[k][0] == o[0] && s->dep[k][1] == o[1] && s->dep[k][2] == o[2];
            if (!seen) {
                for (int d = 0; d < 3; ++d) s->dep[s->ndep][d] = o[d];
                ++s->ndep;
            }
        }
}

void make_grid(Grid *g, const double box[3], double rc, int dims) {
    memset(g, 0, sizeof(*g));
    g->dims = dims;
    g->rc = rc;
    g->rc2 = rc * rc;
    g->ncell = 1;
    for (int d = 0; d < 3; ++d) {
        g->L[d] = box[d];
        g->nc[d] = (dims == 2 && d == 2) ? 1 : (int)floor(box[d] / rc);   // 2D: one layer of side L_z
        g->h[d] = box[d] / (double)g->nc[d];
        g->inv[d] = (double)g->nc[d] / box[d];
        g->hf[d] = (float)g->h[d];
        g->hl[d] = (float)(g->h[d] - (double)g->hf[d]);
        g->invf[d] = (float)g->inv[d];
        g->Lf_lo[d] = (float)(box[d] * (1.0 - 1.0e-6));
        g->cmargin[d] = (float)(2.0e-6 * g->nc[d] + 1.0e-6);
        g->ncell *= g->nc[d];
    }
    float rc2f = (float)g->rc2;
    g->rc2f_lo = rc2f * (1.0f - kCutBand);
    g->rc2f_hi = rc2f * (1.0f + kCutBand);
    for (int d = 0; d < 3; ++d) {
        for (int a = 0; a < 3; ++a) g->class_count[d][a] = 0;
        for (int c = 0; c < g->nc[d]; ++c) g->class_count[d][colour_class(c, g->nc[d])]++;
    }
    int r = 0;
    for (int raw = 0; raw < 27; ++raw) {
        int a[3] = {raw % 3, (raw / 3) % 3, raw / 9};
        bool present = g->class_count[0][a[0]] && g->class_count[1][a[1]] && g->class_count[2][a[2]];
        g->colour_of_raw[raw] = present ? r : -1;
        g->raw_of_colour[raw] = -1;
        if (present) { g->raw_of_colour[r] = raw; ++r; }
    }
    g->ncolours = r;
    // colour schedule: class strides, classes and the colour queue order
    for (int d = 0; d < 3; ++d) {
        const bool two_sided = dims == 3 ? d < 2 : d == 0;
        g->cs_p[d] = (dims == 2 && d == 2) ? 1 : (two_sided ? 3 : 2);
        g->cs_ncls[d] = g->cs_p[d] + (g->nc[d] - g->cs_p[d] * (g->nc[d] / g->cs_p[d]));
    }
    r = 0;
    g->cs_first[0] = 0;
    for (int raw = 0; raw < 125; ++raw) {
        const int a[3] = {raw % 5, (raw / 5) % 5, raw / 25};
        g->cs_colour_of_raw[raw] = -1;
        g->cs_raw_of_colour[raw] = -1;
        if (a[0] >= g->cs_ncls[0] || a[1] >= g->cs_ncls[1] || a[2] >= g->cs_ncls[2]) continue;
        g->cs_colour_of_raw[raw] = r;
        g->cs_raw_of_colour[r] = raw;
        g->cs_first[r + 1] = g->cs_first[r] + cs_count(a[0], g->nc[0], g->cs_p[0]) *
                                                  cs_count(a[1], g->nc[1], g->cs_p[1]) *
                                                  cs_count(a[2], g->nc[2], g->cs_p[2]);
        ++r;
    }
    g->cs_ncolours = r;
    // exact division by multiplication: with M = ceil(2^64 / d) and c < 2^32,
    // c M / 2^64 = c / d + c e / (d 2^64) with e = M d - 2^64 < d, an excess
    // below 1 / d, so the floor is floor(c / d)
    const unsigned long long dx = (unsigned long long)(g->nc[0] > 0 ? g->nc[0] : 1);
    const unsigned long long dxy = dx * (unsigned long long)(g->nc[1] > 0 ? g->nc[1] : 1);
    g->divx = ~0ull / dx + 1;
    g->divxy = ~0ull / dxy + 1;
}

void make_box(BoxDev *b, const double box[3], double rc, int cell_off, int part_off, int n) {
    make_grid(&b->g, box, rc);
    for (int oi = 0; oi < 27; ++oi) {
        const int o[3] = {oi % 3 - 1, (oi / 3) % 3 - 1, oi / 9 - 1};
        for (int d = 0; d < 3; ++d) {
            const double S = (double)o[d] * b->g.h[d];
            const float Sh = (float)S;
            b->sh[oi][d] = Sh;
            b->sl[oi][d] = (float)(S - (double)Sh);
        }
    }
    b->cell_off = cell_off;
    b->part_off = part_off;
    b->n = n;
    b->pad = 0;
}

}  // namespace lc

using namespace lc;

struct lc_ctx : public Ctx {};

static lc_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return LC_OK;
    if (e == cudaErrorMemoryAllocation) return LC_ERR_OOM;
    return LC_ERR_CUDA;
}

#define LC_TRY(expr)                              \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) {                  \
            cudaGetLastError();                   \
            return from_cuda(_e);                 \
        }                                         \
    } while (0)

#define LC_TRY_ST(expr)                           \
    do {                                          \
        lc_status _s = (expr);                    \
        if (_s != LC_OK) return _s;               \
    } while (0)

template <typename T>
static cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, sizeof(T) * count);
}

static void free_ctx(Ctx *c) {
    if (!c) return;
    void *ptrs[] = {c->cur.x, c->cur.vx, c->cur.id, c->nxt.x, c->nxt.vx, c->nxt.id, c->d_cell, c->d_rank,
                    c->d_count, c->d_start, c->d_src, c->d_key, c->d_cellt, c->d_blocksums, c->d_colour, c->d_p4, c->fx, c->kx,
                    c->d_warp_acc, c->d_warp_pairs, c->d_kin_part, c->d_result,
                    c->d_stamp, c->d_visit, c->d_counters, c->d_boxes, c->d_cell_box, c->d_slot_box,
                    c->d_box_acc, c->d_box_pairs, c->d_box_out, c->d_fbuf, c->d_nbr, c->d_nn, c->d_q4,
                    c->d_list_stats, c->d_cs_done, c->d_cs_ctrl, c->d_cell_acc, c->d_cell_pairs, c->d_cs_items,
                    c->d_cs_cell, c->d_cs_rank, c->d_cs_dep};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int k = 0; k < kNumGraphs; ++k)
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
    for (DagDev *d : c->dag) free_dag(d);
    for (cudaGraphExec_t gx : c->list_graph)
        if (gx) cudaGraphExecDestroy(gx);
    for (int k = 0; k < 2; ++k) {
        if (c->d_stage[k]) cudaFree(c->d_stage[k]);
        if (c->ev_staged[k]) cudaEventDestroy(c->ev_staged[k]);
        if (c->ev_consumed[k]) cudaEventDestroy(c->ev_consumed[k]);
    }
    if (c->h_out) cudaFreeHost(c->h_out);
    free(c->h_boxes);
    delete static_cast<lc_ctx *>(c);
}

static cudaError_t alloc_state(State *st, int64_t n) {
    cudaError_t e;
    double *xs, *vs;
    if ((e = dalloc(&xs, 3 * (size_t)n))) return e;
    st->x = xs; st->y = xs + n; st->z = xs + 2 * n;
    if ((e = dalloc(&vs, 3 * (size_t)n))) return e;
    st->vx = vs; st->vy = vs + n; st->vz = vs + 2 * n;
    return dalloc(&st->id, (size_t)n);
}

// Device buffers shared by single-box and batch contexts (c->n particles,
// c->g.ncell cells in total).
static cudaError_t alloc_common(Ctx *c) {
    cudaError_t e;
    Stencil st, st2;
    make_stencil(&st, 3);
    make_stencil(&st2, 2);
    const int64_t n = c->n;
    const size_t N = (size_t)n, NC = (size_t)c->g.ncell;
    const int ntiles = (c->g.ncell + 4095) / 4096;
    c->nwarp_max = c->num_sms * 64;
    if ((e = upload_stencil(st, st2)) || (e = alloc_state(&c->cur, n)) || (e = alloc_state(&c->nxt, n)) ||
        (e = dalloc(&c->d_cell, N)) || (e = dalloc(&c->d_rank, N)) || (e = dalloc(&c->d_count, NC)) ||
        (e = dalloc(&c->d_start, 2 * (NC + 1))) || (e = dalloc(&c->d_src, N)) || (e = dalloc(&c->d_key, N)) || (e = dalloc(&c->d_cellt, N)) ||
        (e = dalloc(&c->d_blocksums, (size_t)ntiles + 1)) || (e = dalloc(&c->d_colour, NC)) ||
        (e = dalloc(&c->d_p4, N)) || (e = dalloc(&c->fx, 3 * N)) || (e = dalloc(&c->kx, 3 * N)) ||
        (e = dalloc(&c->d_warp_acc, 4 * (size_t)c->nwarp_max)) || (e = dalloc(&c->d_warp_pairs, (size_t)c->nwarp_max)) ||
        (e = dalloc(&c->d_kin_part, (size_t)kinetic_blocks(c))) || (e = dalloc(&c->d_result, 8)) ||
        (e = dalloc(&c->d_cs_done, NC)) || (e = dalloc(&c->d_cs_ctrl, 2)) ||
        (e = dalloc(&c->d_cell_acc, 4 * NC)) || (e = dalloc(&c->d_cell_pairs, NC)) ||
        (e = cudaHostAlloc(&c->h_out, 64, cudaHostAllocDefault)))
        return e;
    c->d_npairs = reinterpret_cast<long long *>(c->d_result + 4);
    c->d_err = reinterpret_cast<int *>(c->d_result + 5);
    c->d_kin_ticket = reinterpret_cast<unsigned *>(c->d_result + 6);
    c->state_a = c->cur.x;
    if ((e = init_force_kernels())) return e;
    c->fy = c->fx + N; c->fz = c->fx + 2 * N;
    c->ky = c->kx + N; c->kz = c->kx + 2 * N;
    cudaStream_t s = 0;
    if ((e = cudaMemsetAsync(c->d_result, 0, 8 * sizeof(double), s)) ||   // energies, pair count, flags
        (e = cudaMemsetAsync(c->d_blocksums, 0, ((size_t)ntiles + 1) * sizeof(int), s)) ||   // scan ticket
        (e = cudaMemsetAsync(c->fx, 0, 3 * N * sizeof(double), s)))
        return e;
    return cudaSuccess;
}

static lc_status read_err(lc_ctx *c, cudaStream_t s) {
    int err = 0;
    LC_TRY(cudaMemcpyAsync(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    LC_TRY(cudaStreamSynchronize(s));
    if (err & kErrNonfinite) return LC_ERR_NONFINITE;
    if (err & kErrTimeout) return LC_ERR_TIMEOUT;
    return LC_OK;
}

extern "C" {

const char *lc_status_str(lc_status s) {
    switch (s) {
        case LC_OK: return "ok";
        case LC_ERR_INVALID_ARG: return "invalid argument";
        case LC_ERR_BOX_TOO_SMALL: return "box too small: fewer than 3 cells of side >= rc in some dimension";
        case LC_ERR_CUDA: return "CUDA runtime error";
        case LC_ERR_OOM: return "device out of memory";
        case LC_ERR_NONFINITE: return "non-finite position or velocity";
        case LC_ERR_TIMEOUT: return "bounded device wait expired";
        case LC_ERR_STATE: return "call order violated";
        case LC_ERR_RACE: return "colour phase wrote a cell twice";
        case LC_ERR_TOO_LARGE: return "size beyond the supported maximum";
    }
    return "unknown status";
}

// Colour-queue tables of one box's grid: the colour (rank) of every cell,
// and the cells in queue order (colour-major, ascending cell index inside a
// colour), offset by the box's first global cell.
// dep: per cell, bit e set when the cell at the stencil's dependence offset
// e has an earlier colour (the cells a task waits for).
static void colour_tables(const Grid &g, int cell_off, int8_t *rank, int *cell_of_pos, unsigned long long *dep) {
    std::vector<int> fill(g.cs_first, g.cs_first + g.cs_ncolours);
    for (int c = 0; c < g.ncell; ++c) {
        const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
        const int raw = cs_class(cx, g.nc[0], g.cs_p[0]) + 5 * cs_class(cy, g.nc[1], g.cs_p[1]) +
                        25 * cs_class(cz, g.nc[2], g.cs_p[2]);
        const int r = g.cs_colour_of_raw[raw];
        rank[c] = (int8_t)r;
        cell_of_pos[fill[r]++] = cell_off + c;
    }
    Stencil st;
    make_stencil(&st, g.dims);
    for (int c = 0; c < g.ncell; ++c) {
        const int cc[3] = {c % g.nc[0], (c / g.nc[0]) % g.nc[1], c / (g.nc[0] * g.nc[1])};
        unsigned long long m = 0;
        for (int e = 0; e < st.ndep; ++e) {
            int n[3];
            for (int d = 0; d < 3; ++d) n[d] = ((cc[d] + st.dep[e][d]) % g.nc[d] + g.nc[d]) % g.nc[d];
            if (rank[n[0] + g.nc[0] * (n[1] + g.nc[1] * n[2])] < rank[c]) m |= 1ull << e;
        }
        dep[c] = m;
    }
}

static cudaError_t upload_colour_tables(Ctx *c) {
    std::vector<int8_t> rank((size_t)c->g.ncell);
    std::vector<int> cells((size_t)c->g.ncell);
    std::vector<unsigned long long> dep((size_t)c->g.ncell);
    colour_tables(c->g, 0, rank.data(), cells.data(), dep.data());
    cudaError_t e = cudaMemcpy(c->d_cs_rank, rank.data(), rank.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(c->d_cs_cell, cells.data(), sizeof(int) * cells.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(c->d_cs_dep, dep.data(), sizeof(unsigned long long) * dep.size(), cudaMemcpyHostToDevice);
    return e;
}

static lc_status create_single(const double box[3], double rc, int64_t n, lc_precision prec, int dims, lc_ctx **out) {
    if (!out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!box || !(rc > 0.0) || !isfinite(rc) || n < 0 || (prec != LC_PREC_FP64 && prec != LC_PREC_MIXED))
        return LC_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d)
        if (!(box[d] > 0.0) || !isfinite(box[d])) return LC_ERR_INVALID_ARG;
    if (n >= kMaxParticles) return LC_ERR_TOO_LARGE;
    for (int d = 0; d < dims; ++d)
        if (floor(box[d] / rc) < 3.0) return LC_ERR_BOX_TOO_SMALL;
    const double nz = dims == 2 ? 1.0 : floor(box[2] / rc);
    if (floor(box[0] / rc) * floor(box[1] / rc) * nz > 1.0e9) return LC_ERR_TOO_LARGE;

    lc_ctx *c = new lc_ctx();
    memset(static_cast<Ctx *>(c), 0, sizeof(Ctx));
    make_grid(&c->g, box, rc, dims);
    c->skin = 0.4;
    c->cs_wait_s = 2.0;
    c->n = n;
    c->prec = prec;
    c->ni = 16;
    c->warps = 8;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) { cudaGetLastError(); free_ctx(c); return from_cuda(e); }
    cudaError_t e2 = alloc_common(c);
    if (e2) { cudaGetLastError(); free_ctx(c); return from_cuda(e2); }
    if ((e = launch_colour(c, 0)) || (e = cudaStreamSynchronize(0))) {
        cudaGetLastError();
        free_ctx(c);
        return from_cuda(e);
    }
    *out = c;
    return LC_OK;
}

lc_status lc_create(const double box[3], double rc, int64_t n, lc_precision prec, lc_ctx **out) {
    return create_single(box, rc, n, prec, 3, out);
}

lc_status lc_create_2d(const double box[2], double rc, int64_t n, lc_precision prec, lc_ctx **out) {
    if (!box) {
        if (out) *out = nullptr;
        return LC_ERR_INVALID_ARG;
    }
    const double b3[3] = {box[0], box[1], rc};   // one cell layer of side rc in z
    return create_single(b3, rc, n, prec, 2, out);
}

lc_status lc_batch_create(int32_t nbox, const double *box, const double *rc, const int64_t *n, lc_precision prec,
                          lc_ctx **out) {
    if (!out) return LC_ERR_INVALID_ARG;
    *out = nullptr;
    if (nbox <= 0 || !box || !rc || !n || (prec != LC_PREC_FP64 && prec != LC_PREC_MIXED)) return LC_ERR_INVALID_ARG;
    if (nbox > 65535) return LC_ERR_TOO_LARGE;
    int64_t ntot = 0;
    double ctot = 0.0;
    for (int b = 0; b < nbox; ++b) {
        if (!(rc[b] > 0.0) || n[b] < 0) return LC_ERR_INVALID_ARG;
        for (int d = 0; d < 3; ++d) {
            if (!(box[3 * b + d] > 0.0) || !isfinite(box[3 * b + d])) return LC_ERR_INVALID_ARG;
            if (floor(box[3 * b + d] / rc[b]) < 3.0) return LC_ERR_BOX_TOO_SMALL;
        }
        ntot += n[b];
        ctot += floor(box[3 * b] / rc[b]) * floor(box[3 * b + 1] / rc[b]) * floor(box[3 * b + 2] / rc[b]);
    }
    if (ntot >= kMaxParticles || ctot > 1.0e9) return LC_ERR_TOO_LARGE;

    lc_ctx *c = new lc_ctx();
    memset(static_cast<Ctx *>(c), 0, sizeof(Ctx));
    c->nbox = nbox;
    c->h_boxes = (BoxDev *)calloc((size_t)nbox, sizeof(BoxDev));
    if (!c->h_boxes) { delete c; return LC_ERR_OOM; }
    int coff = 0, poff = 0;
    for (int b = 0; b < nbox; ++b) {
        make_box(&c->h_boxes[b], box + 3 * b, rc[b], coff, poff, (int)n[b]);
        coff += c->h_boxes[b].g.ncell;
        poff += (int)n[b];
    }
    c->g = c->h_boxes[0].g;   // scalar fields of box 0; totals below
    c->g.ncell = coff;
    c->cs_wait_s = 2.0;
    c->n = ntot;
    c->prec = prec;
    c->ni = 16;
    c->warps = 8;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (!e) e = alloc_common(c);
    if (!e) e = dalloc(&c->d_boxes, (size_t)nbox);
    if (!e) e = dalloc(&c->d_cell_box, (size_t)coff);
    if (!e) e = dalloc(&c->d_slot_box, (size_t)(ntot > 0 ? ntot : 1));
    if (!e) e = dalloc(&c->d_box_acc, 2 * (size_t)nbox);
    if (!e) e = dalloc(&c->d_box_pairs, (size_t)nbox);
    if (!e) e = dalloc(&c->d_box_out, 4 * (size_t)nbox);
    if (e) { cudaGetLastError(); free_ctx(c); return from_cuda(e); }
    unsigned short *cb = (unsigned short *)malloc(sizeof(unsigned short) * (size_t)(coff > 0 ? coff : 1));
    unsigned short *sb = (unsigned short *)malloc(sizeof(unsigned short) * (size_t)(ntot > 0 ? ntot : 1));
    if (!cb || !sb) { free(cb); free(sb); free_ctx(c); return LC_ERR_OOM; }
    for (int b = 0; b < nbox; ++b) {
        const BoxDev &bd = c->h_boxes[b];
        for (int k = 0; k < bd.g.ncell; ++k) cb[bd.cell_off + k] = (unsigned short)b;
        for (int k = 0; k < bd.n; ++k) sb[bd.part_off + k] = (unsigned short)b;
    }
    // colour-queue items, one cell each.  A box's colours form a chain (a
    // cell waits for its earlier-coloured neighbours), and boxes have from 8
    // to 48 colours: the (box, colour) groups are ordered by the colour's
    // position within its box's chain, k / colours(box), so every box's chain
    // advances at the same pace through the queue and the long chains of the
    // many-coloured small boxes do not end up alone at its tail.  Within a
    // box the order stays colour-major, so a waited-for task was claimed
    // earlier (no deadlock).
    std::vector<std::pair<double, std::pair<int, int>>> groups;
    int64_t nitems = 0;
    for (int b = 0; b < nbox; ++b) {
        const Grid &gb = c->h_boxes[b].g;
        for (int k = 0; k < gb.cs_ncolours; ++k) {
            groups.push_back({(double)k / gb.cs_ncolours, {b, k}});
            nitems += gb.cs_first[k + 1] - gb.cs_first[k];
        }
    }
    std::stable_sort(groups.begin(), groups.end(),
                     [](const std::pair<double, std::pair<int, int>> &x,
                        const std::pair<double, std::pair<int, int>> &y) { return x.first < y.first; });
    int4 *items = (int4 *)malloc(sizeof(int4) * (size_t)(nitems > 0 ? nitems : 1));
    if (!items) { free(cb); free(sb); free_ctx(c); return LC_ERR_OOM; }
    // per box: the colour of every cell (at the box's global cells) and its
    // cells in colour order
    std::vector<int8_t> rank((size_t)(coff > 0 ? coff : 1));
    std::vector<int> cell_of_pos((size_t)(coff > 0 ? coff : 1));
    std::vector<unsigned long long> dep((size_t)(coff > 0 ? coff : 1));
    for (int b = 0; b < nbox; ++b) {
        const BoxDev &bd = c->h_boxes[b];
        colour_tables(bd.g, bd.cell_off, rank.data() + bd.cell_off, cell_of_pos.data() + bd.cell_off,
                      dep.data() + bd.cell_off);
    }
    int64_t q = 0;
    for (const auto &gr : groups) {
        const int b = gr.second.first, k = gr.second.second;
        const BoxDev &bd = c->h_boxes[b];
        for (int t = bd.g.cs_first[k]; t < bd.g.cs_first[k + 1]; ++t)
            items[q++] = make_int4(b, k, cell_of_pos[(size_t)bd.cell_off + t], 1);
    }
    c->cs_nitems = (int)nitems;
    e = dalloc(&c->d_cs_items, (size_t)(nitems > 0 ? nitems : 1));
    if (!e && nitems > 0) e = cudaMemcpy(c->d_cs_items, items, sizeof(int4) * (size_t)nitems, cudaMemcpyHostToDevice);
    free(items);
    if (!e) e = cudaMemcpy(c->d_boxes, c->h_boxes, sizeof(BoxDev) * (size_t)nbox, cudaMemcpyHostToDevice);
    if (!e) e = dalloc(&c->d_cs_rank, (size_t)(coff > 0 ? coff : 1));
    if (!e) e = dalloc(&c->d_cs_dep, (size_t)(coff > 0 ? coff : 1));
    if (!e && coff > 0) e = cudaMemcpy(c->d_cs_rank, rank.data(), (size_t)coff, cudaMemcpyHostToDevice);
    if (!e && coff > 0)
        e = cudaMemcpy(c->d_cs_dep, dep.data(), sizeof(unsigned long long) * (size_t)coff, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(c->d_cell_box, cb, sizeof(unsigned short) * (size_t)coff, cudaMemcpyHostToDevice);
    if (!e && ntot > 0) e = cudaMemcpy(c->d_slot_box, sb, sizeof(unsigned short) * (size_t)ntot, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(c->d_box_out, 0, sizeof(double) * 4 * (size_t)nbox);
    free(cb);
    free(sb);
    if (e) { cudaGetLastError(); free_ctx(c); return from_cuda(e); }
    *out = c;
    return LC_OK;
}

lc_status lc_batch_energies(lc_ctx *c, double *u_pot, double *k_kin, double *virial, int64_t *npairs, void *stream) {
    if (!c || c->nbox <= 0) return LC_ERR_INVALID_ARG;
    if (!c->have_state) return LC_ERR_STATE;
    if ((u_pot || virial || npairs) && !c->forces_valid) return LC_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    LC_TRY(launch_box_kinetic(c, s));
    double *h = (double *)malloc(sizeof(double) * 4 * (size_t)c->nbox);
    if (!h) return LC_ERR_OOM;
    cudaError_t e = cudaMemcpyAsync(h, c->d_box_out, sizeof(double) * 4 * (size_t)c->nbox, cudaMemcpyDeviceToHost, s);
    lc_status st = e ? from_cuda(e) : read_err(c, s);
    if (st == LC_OK) {
        for (int b = 0; b < c->nbox; ++b) {
            if (u_pot) u_pot[b] = h[4 * b + 0];
            if (virial) virial[b] = h[4 * b + 1];
            if (npairs) npairs[b] = (int64_t)h[4 * b + 2];
            if (k_kin) k_kin[b] = h[4 * b + 3];
        }
    }
    free(h);
    cudaGetLastError();
    return st;
}

lc_status lc_batch_info(const lc_ctx *c, int32_t *nbox, int64_t *total_particles, int64_t *total_cells) {
    if (!c) return LC_ERR_INVALID_ARG;
    if (nbox) *nbox = c->nbox;
    if (total_particles) *total_particles = c->n;
    if (total_cells) *total_cells = c->g.ncell;
    return LC_OK;
}

void lc_destroy(lc_ctx *ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    free_ctx(ctx);
}

// Device address of a page-locked, device-mapped host array, or nullptr.
static const double *mapped_host(const double *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || !at.devicePointer) return nullptr;
    return static_cast<const double *>(at.devicePointer);
}

lc_status lc_set_state(lc_ctx *c, const double *pos, const double *vel, const int32_t *id, int on_device,
                       void *stream) {
    if (!c || (!pos && c->n > 0) || id) return LC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * 3 * (size_t)c->n;
    const double *dpos = pos, *dvel = vel;
    if (c->n > 0 && !on_device) {
        // Page-locked host arrays are read in place by the set-up kernel
        // (device-mapped; over NVLink-C2C on GB300); other host memory is
        // staged through the force buffer and the next-state buffer.
        const double *mp = mapped_host(pos), *mv = vel ? mapped_host(vel) : nullptr;
        if (mp) {
            dpos = mp;
        } else {
            LC_TRY(cudaMemcpyAsync(c->fx, pos, bytes, cudaMemcpyHostToDevice, s));
            dpos = c->fx;
        }
        if (vel && mv) {
            dvel = mv;
        } else if (vel) {
            LC_TRY(cudaMemcpyAsync(c->nxt.x, vel, bytes, cudaMemcpyHostToDevice, s));
            dvel = c->nxt.x;
        }
    }
    LC_TRY(launch_set_state(c, dpos, dvel, s));
    LC_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
    if (!on_device) LC_TRY(cudaStreamSynchronize(s));  // host buffers are the caller's again on return
    c->have_state = true;
    c->binned = false;
    c->forces_valid = false;
    c->list_valid = false;
    return LC_OK;
}

lc_status lc_stage_state(lc_ctx *c, const double *pos, const double *vel, int32_t slot, void *copy_stream) {
    if (!c || (slot != 0 && slot != 1) || (!pos && c->n > 0)) return LC_ERR_INVALID_ARG;
    cudaStream_t cs = (cudaStream_t)copy_stream;
    const size_t bytes = sizeof(double) * 3 * (size_t)c->n;
    // first use of the slot: buffers and events (each created once)
    if (!c->d_stage[slot]) LC_TRY(dalloc(&c->d_stage[slot], 6 * (size_t)(c->n > 0 ? c->n : 1)));
    if (!c->ev_staged[slot]) LC_TRY(cudaEventCreateWithFlags(&c->ev_staged[slot], cudaEventDisableTiming));
    if (!c->ev_consumed[slot]) {
        LC_TRY(cudaEventCreateWithFlags(&c->ev_consumed[slot], cudaEventDisableTiming));
        LC_TRY(cudaEventRecord(c->ev_consumed[slot], cs));
    }
    // the slot's previous content must have been consumed before it is overwritten
    LC_TRY(cudaStreamWaitEvent(cs, c->ev_consumed[slot], 0));
    if (c->n > 0) {
        LC_TRY(cudaMemcpyAsync(c->d_stage[slot], pos, bytes, cudaMemcpyHostToDevice, cs));
        if (vel) LC_TRY(cudaMemcpyAsync(c->d_stage[slot] + 3 * (size_t)c->n, vel, bytes, cudaMemcpyHostToDevice, cs));
    }
    c->stage_has_vel[slot] = vel != nullptr;
    LC_TRY(cudaEventRecord(c->ev_staged[slot], cs));
    return LC_OK;
}

lc_status lc_set_state_staged(lc_ctx *c, int32_t slot, void *stream) {
    if (!c || (slot != 0 && slot != 1)) return LC_ERR_INVALID_ARG;
    if (!c->d_stage[slot] || !c->ev_staged[slot] || !c->ev_consumed[slot]) return LC_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    LC_TRY(cudaStreamWaitEvent(s, c->ev_staged[slot], 0));
    const double *pos = c->d_stage[slot];
    const double *vel = c->stage_has_vel[slot] ? c->d_stage[slot] + 3 * (size_t)c->n : nullptr;
    LC_TRY(launch_set_state(c, pos, vel, s));
    LC_TRY(cudaEventRecord(c->ev_consumed[slot], s));
    LC_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
    c->have_state = true;
    c->binned = false;
    c->forces_valid = false;
    c->list_valid = false;
    return LC_OK;
}

lc_status lc_bin(lc_ctx *c, void *stream) {
    if (!c) return LC_ERR_INVALID_ARG;
    if (!c->have_state) return LC_ERR_STATE;
    int launches = 0;
    LC_TRY(launch_bin(c, (cudaStream_t)stream, &launches));
    c->binned = true;
    return LC_OK;
}

// The buffer schedule's private buffers, allocated on its first use (before
// any stream capture, so that a captured step never allocates).
// The colour queue's tables of a single box (queue position -> cell, cell
// colour, wait masks), built on the schedule's first use: before any stream
// capture, and contexts that never use the colour schedule hold none.
static lc_status ensure_colour_tables(lc_ctx *c, lc_schedule sched) {
    if (sched != LC_SCHED_COLOUR || c->nbox > 0 || c->d_cs_rank) return LC_OK;
    const size_t NC = (size_t)c->g.ncell;
    cudaError_t e;
    if ((e = dalloc(&c->d_cs_cell, NC)) || (e = dalloc(&c->d_cs_rank, NC)) || (e = dalloc(&c->d_cs_dep, NC)) ||
        (e = upload_colour_tables(c))) {
        cudaGetLastError();
        cudaFree(c->d_cs_cell); cudaFree(c->d_cs_rank); cudaFree(c->d_cs_dep);
        c->d_cs_cell = nullptr; c->d_cs_rank = nullptr; c->d_cs_dep = nullptr;
        return e == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA;
    }
    return LC_OK;
}

static lc_status ensure_fbuf(lc_ctx *c, lc_schedule sched) {
    if (sched != LC_SCHED_BUFFER || c->d_fbuf) return LC_OK;
    const size_t elem = c->prec == LC_PREC_MIXED ? sizeof(float) : sizeof(double);
    const size_t bytes = elem * 3 * (size_t)kNumFbuf * (size_t)(c->n > 0 ? c->n : 1);
    cudaError_t e = cudaMalloc(&c->d_fbuf, bytes);
    if (e) { cudaGetLastError(); c->d_fbuf = nullptr; return e == cudaErrorMemoryAllocation ? LC_ERR_OOM : LC_ERR_CUDA; }
    return LC_OK;
}

static lc_status do_forces(lc_ctx *c, lc_schedule sched, cudaStream_t s, int *launches) {
    LC_TRY_ST(ensure_fbuf(c, sched));
    LC_TRY_ST(ensure_colour_tables(c, sched));
    if (!c->binned) {
        LC_TRY(launch_bin(c, s, launches));
        c->binned = true;
    }
    LC_TRY(launch_forces(c, sched, s, launches));
    c->forces_valid = true;
    return LC_OK;
}

// ---- Verlet neighbour lists ------------------------------------------------
static void drop_list_graphs(lc_ctx *c) {
    for (int k = 0; k < 4; ++k)
        if (c->list_graph[k]) { cudaGraphExecDestroy(c->list_graph[k]); c->list_graph[k] = nullptr; }
}

// List grid, buffers and row capacity on first use (a counting build of the
// current state sizes the rows unless lc_set_skin fixed kmax).
static lc_status ensure_list(lc_ctx *c, cudaStream_t s) {
    if (c->d_nbr) return LC_OK;
    if (!make_list_grid(c)) return LC_ERR_BOX_TOO_SMALL;
    const size_t N = (size_t)(c->n > 0 ? c->n : 1);
    if (!c->d_nn) LC_TRY(dalloc(&c->d_nn, N));
    if (!c->d_q4) LC_TRY(dalloc(&c->d_q4, 2 * N));
    if (!c->d_list_stats) {
        LC_TRY(dalloc(&c->d_list_stats, 6));   // 5 counters + 2 control words
        LC_TRY(cudaMemsetAsync(c->d_list_stats, 0, 6 * sizeof(unsigned long long), s));
    }
    int64_t kmax = c->list_kmax_req;
    if (kmax == 0) {
        int l = 0;
        const Grid saved = c->g;
        c->g = c->gl;
        cudaError_t e = launch_bin(c, s, &l, 0, 0.0);
        c->g = saved;
        LC_TRY(e);
        c->list_kmax = 0;
        LC_TRY(launch_list_build(c, s, false));
        unsigned long long longest = 0;
        LC_TRY(cudaMemcpyAsync(&longest, c->d_list_stats + 2, sizeof(longest), cudaMemcpyDeviceToHost, s));
        LC_TRY(cudaStreamSynchronize(s));
        LC_TRY(cudaMemsetAsync(c->d_list_stats + 2, 0, sizeof(longest), s));
        kmax = (int64_t)(longest + longest / 4 + 8);
    }
    if (kmax * (int64_t)N > (int64_t(1) << 36)) return LC_ERR_TOO_LARGE;
    c->list_kmax = (int)kmax;
    LC_TRY(dalloc(&c->d_nbr, (size_t)kmax * N));
    return LC_OK;
}

// Forces from the lists, built first when they are stale (new state, or a
// link-cell binning re-sorted the particles); lists kept valid by list
// steps are used as they are.
static lc_status list_forces(lc_ctx *c, cudaStream_t s, int *launches) {
    if (c->prec != LC_PREC_MIXED || c->nbox > 0) return LC_ERR_INVALID_ARG;
    if (!c->list_valid || !c->d_nbr) {
        LC_TRY_ST(ensure_list(c, s));
        LC_TRY(launch_list_rebuild(c, s, false, launches));
    }
    LC_TRY(launch_list_forces(c, s, true, launches));
    c->binned = false;   // the cells are the list grid's
    c->forces_valid = true;
    c->list_valid = true;
    return LC_OK;
}

static lc_status list_verlet(lc_ctx *c, double dt, int nsteps, cudaStream_t s) {
    if (c->prec != LC_PREC_MIXED || c->nbox > 0) return LC_ERR_INVALID_ARG;
    int launches = 0;
    if (!c->list_valid || !c->forces_valid) LC_TRY_ST(list_forces(c, s, &launches));
    const int par = c->cur.x == c->state_a ? 0 : 1;   // the graphs keep the buffers in place
    int done = 0;
    while (done < nsteps) {
        const int k = nsteps - done >= 2 ? 2 : 1;
        const int gi = 2 * (k - 1) + par;
        if (!c->list_graph[gi] || c->list_graph_dt[gi] != dt) {
            if (c->list_graph[gi]) { cudaGraphExecDestroy(c->list_graph[gi]); c->list_graph[gi] = nullptr; }
            int per = 0;
            LC_TRY(capture_list_steps(c, dt, k, &c->list_graph[gi], &per));
            c->list_graph_dt[gi] = dt;
            c->launches_step = per / k;
            c->list_graph_launches[gi] = per;
        }
        LC_TRY(cudaGraphLaunch(c->list_graph[gi], s));
        if (k == 2) c->launches_two = c->list_graph_launches[gi];
        else c->launches_one = c->list_graph_launches[gi];
        done += k;
    }
    c->binned = false;
    c->forces_valid = true;
    c->list_valid = true;
    return LC_OK;
}

lc_status lc_set_skin(lc_ctx *c, double skin, int32_t kmax) {
    if (!c || !(skin >= 0.0) || !isfinite(skin) || kmax < 0) return LC_ERR_INVALID_ARG;
    LC_TRY(cudaDeviceSynchronize());   // no list step in flight past this point
    drop_list_graphs(c);
    if (c->d_nbr) { cudaFree(c->d_nbr); c->d_nbr = nullptr; }
    c->skin = skin;
    c->list_kmax_req = kmax;
    c->list_kmax = 0;
    c->list_valid = false;
    if (c->d_list_stats) LC_TRY(cudaMemset(c->d_list_stats, 0, 6 * sizeof(unsigned long long)));
    return LC_OK;
}

lc_status lc_list_info(lc_ctx *c, int64_t *builds, int64_t *long_rows, int64_t *longest_row, int64_t *rebuild_steps,
                       int64_t *entries, int32_t *kmax, void *stream) {
    if (!c) return LC_ERR_INVALID_ARG;
    unsigned long long v[5] = {0, 0, 0, 0, 0};
    if (c->d_list_stats) {
        cudaStream_t s = (cudaStream_t)stream;
        LC_TRY(cudaMemcpyAsync(v, c->d_list_stats, sizeof(v), cudaMemcpyDeviceToHost, s));
        LC_TRY(cudaStreamSynchronize(s));
    }
    if (builds) *builds = (int64_t)v[0];
    if (long_rows) *long_rows = (int64_t)v[1];
    if (longest_row) *longest_row = (int64_t)v[2];
    if (rebuild_steps) *rebuild_steps = (int64_t)v[3];
    if (entries) *entries = (int64_t)v[4];
    if (kmax) *kmax = c->list_kmax;
    return LC_OK;
}

lc_status lc_forces(lc_ctx *c, lc_schedule sched, void *stream) {
    if (!c || sched < LC_SCHED_COLOUR || sched > LC_SCHED_LIST) return LC_ERR_INVALID_ARG;
    if (!c->have_state) return LC_ERR_STATE;
    int launches = 0;
    lc_status st = sched == LC_SCHED_LIST ? list_forces(c, (cudaStream_t)stream, &launches)
                                          : do_forces(c, sched, (cudaStream_t)stream, &launches);
    c->launches_force = launches;
    return st;
}

// One Verlet step as a sequence of stream-ordered launches.  stats: the
// force evaluation also produces energy, virial and pair count (the last
// step of every lc_verlet_step call does, so lc_energy_virial stays valid).
// The kick + drift that opens the step is fused into the binning's cell
// pass; `pending`: the previous step's closing kick was left out and is
// fused there too (same arithmetic); `close`: end with the closing kick.
static cudaError_t step_launches(lc_ctx *c, double dt, lc_schedule sched, cudaStream_t s, int *launches,
                                 bool stats, bool pending = false, bool close = true, bool kin = false) {
    cudaError_t e;
    bool pot = false;   // the statistics' final sum left to the kick
    if ((e = launch_bin(c, s, launches, pending ? 2 : 1, dt))) return e;
    if ((e = launch_forces(c, sched, s, launches, stats, close ? &pot : nullptr))) return e;
    if (close) {
        if ((e = launch_kick(c, dt, s, kin, pot))) return e;
        ++*launches;
    }
    return cudaSuccess;
}

// The instantiated graph of nst (1 or 2) steps from the current state
// buffers into slot k, captured on first use and again when dt changes.
// Capture leaves the buffers where they were (a launch of the one-step graph
// swaps them afterwards, as the binning does).  The one-step graph's closing
// kick also forms K (a call of one step is usually followed by a read of
// its energies); the two-step graph's does not.
static cudaError_t ensure_step_graph(lc_ctx *c, double dt, lc_schedule sched, int nst, int k) {
    if (c->graph[k] && c->graph_dt[k] == dt) return cudaSuccess;
    if (c->graph[k]) { cudaGraphExecDestroy(c->graph[k]); c->graph[k] = nullptr; }
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e) return e;
    const State saved_cur = c->cur, saved_nxt = c->nxt;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int per = 0;
    if (nst == 2) {
        if (!e) e = step_launches(c, dt, sched, cap, &per, false, false, false);
        if (!e) e = step_launches(c, dt, sched, cap, &per, true, true, true);
    } else {
        if (!e) e = step_launches(c, dt, sched, cap, &per, true, false, true, true);
    }
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    c->cur = saved_cur; c->nxt = saved_nxt;
    if (!e) e = e2;
    if (!e) e = cudaGraphInstantiate(&c->graph[k], graph, 0);
    if (graph && !e2) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (e) { cudaGetLastError(); c->graph[k] = nullptr; return e; }
    c->graph_dt[k] = dt;
    if (nst == 2) c->launches_step = per / 2;
    c->graph_launches[k] = per;
    return cudaSuccess;
}

lc_status lc_verlet_step(lc_ctx *c, double dt, int nsteps, lc_schedule sched, void *stream) {
    if (!c || nsteps < 0 || !isfinite(dt) || sched < LC_SCHED_COLOUR || sched > LC_SCHED_LIST)
        return LC_ERR_INVALID_ARG;
    if (!c->have_state) return LC_ERR_STATE;
    if (nsteps > 0) c->kin_valid = c->kin_final = false;   // the steps change the velocities
    if (sched == LC_SCHED_LIST) return list_verlet(c, dt, nsteps, (cudaStream_t)stream);
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    if (!c->forces_valid) {
        lc_status st = do_forces(c, sched, s, &launches);
        if (st) return st;
    }
    if (nsteps == 0) return LC_OK;
    LC_TRY_ST(ensure_fbuf(c, sched));
    LC_TRY_ST(ensure_colour_tables(c, sched));
    // The step swaps the two state buffers once (in the binning), so one
    // graph holds two steps and returns the buffers to where they were; a
    // separate graph serves each buffer parity.  An odd count ends with a
    // graph of one step (its own per parity), after which the buffers are
    // swapped.
    const int par = c->cur.x == c->state_a ? 0 : 1;
    if (nsteps >= 2) LC_TRY(ensure_step_graph(c, dt, sched, 2, 2 * (int)sched + par));
    const int k1 = 2 * kNumSched + 2 * (int)sched + par;
    if (nsteps & 1) LC_TRY(ensure_step_graph(c, dt, sched, 1, k1));
    int done = 0;
    while (done + 2 <= nsteps) {
        LC_TRY(cudaGraphLaunch(c->graph[2 * (int)sched + par], s));
        c->launches_two = c->graph_launches[2 * (int)sched + par];
        done += 2;
    }
    if (done < nsteps) {
        LC_TRY(cudaGraphLaunch(c->graph[k1], s));
        c->launches_one = c->graph_launches[k1];
        const State t = c->cur; c->cur = c->nxt; c->nxt = t;
        ++done;
    }
    c->binned = true;
    c->forces_valid = true;
    if (c->n > 0 && (nsteps & 1)) c->kin_valid = c->kin_final = true;   // the one-step graph formed K
    return LC_OK;
}

lc_status lc_batch_step(lc_ctx *c, double dt, int32_t nsteps, void *stream) {
    if (!c || c->nbox <= 0) return LC_ERR_INVALID_ARG;
    return lc_verlet_step(c, dt, nsteps, LC_SCHED_COLOUR, stream);
}

lc_status lc_set_queue_wait(lc_ctx *c, double seconds, int32_t flags) {
    if (!c || !(seconds > 0.0) || !isfinite(seconds) || seconds > 1.0e6 || (flags & ~LC_QUEUE_WITHHOLD))
        return LC_ERR_INVALID_ARG;
    LC_TRY(cudaDeviceSynchronize());   // no captured step in flight: the graphs hold the old values
    for (int k = 0; k < kNumGraphs; ++k)
        if (c->graph[k]) { cudaGraphExecDestroy(c->graph[k]); c->graph[k] = nullptr; }
    c->cs_wait_s = seconds;
    c->cs_withhold = (flags & LC_QUEUE_WITHHOLD) ? 1 : 0;
    return LC_OK;
}


lc_status lc_energy_virial(lc_ctx *c, double *u_pot, double *k_kin, double *virial, int64_t *npairs, void *stream) {
    if (!c) return LC_ERR_INVALID_ARG;
    if (!c->have_state) return LC_ERR_STATE;
    if ((u_pot || virial || npairs) && !c->forces_valid) return LC_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->nbox > 0) {   // a batch: sums over its boxes
        double *u = (double *)malloc(sizeof(double) * 4 * (size_t)c->nbox);
        if (!u) return LC_ERR_OOM;
        double *k = u + c->nbox, *w = u + 2 * c->nbox;
        int64_t *p = (int64_t *)(u + 3 * c->nbox);
        lc_status st = lc_batch_energies(c, u, k, w, p, stream);
        if (st == LC_OK) {
            double su = 0, sk = 0, sw = 0;
            int64_t sp = 0;
            for (int b = 0; b < c->nbox; ++b) { su += u[b]; sk += k[b]; sw += w[b]; sp += p[b]; }
            if (u_pot) *u_pot = su;
            if (k_kin) *k_kin = sk;
            if (virial) *virial = sw;
            if (npairs) *npairs = sp;
        }
        free(u);
        return st;
    }
    LC_TRY(launch_kinetic(c, s));
    // one read-back of the result block: energies, pair count, error flags
    LC_TRY(cudaMemcpyAsync(c->h_out, c->d_result, 48, cudaMemcpyDeviceToHost, s));
    LC_TRY(cudaStreamSynchronize(s));
    const double *r = static_cast<const double *>(c->h_out);
    const long long np = *reinterpret_cast<const long long *>(r + 4);
    const int err = *reinterpret_cast<const int *>(r + 5);
    if (err & kErrNonfinite) return LC_ERR_NONFINITE;
    if (err & kErrTimeout) return LC_ERR_TIMEOUT;
    if (u_pot) *u_pot = r[0];
    if (virial) *virial = r[1];
    if (npairs) *npairs = (int64_t)np;
    if (k_kin) *k_kin = r[3];
    return LC_OK;
}

lc_status lc_energy_virial_async(lc_ctx *c, void *out, void *stream) {
    if (!c || !out || c->nbox > 0) return LC_ERR_INVALID_ARG;
    if (!c->have_state || !c->forces_valid) return LC_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    LC_TRY(launch_kinetic(c, s));
    LC_TRY(cudaMemcpyAsync(out, c->d_result, 48, cudaMemcpyDeviceToHost, s));
    return LC_OK;
}

// Layout of the result block: U, W, pairs (as double), K, then the pair
// count as int64 and the error flags as int32.
lc_status lc_result_decode(const void *out, double *u_pot, double *k_kin, double *virial, int64_t *npairs) {
    if (!out) return LC_ERR_INVALID_ARG;
    const double *r = static_cast<const double *>(out);
    long long np;
    int err;
    memcpy(&np, r + 4, sizeof(np));
    memcpy(&err, r + 5, sizeof(err));
    if (err & kErrNonfinite) return LC_ERR_NONFINITE;
    if (err & kErrTimeout) return LC_ERR_TIMEOUT;
    if (u_pot) *u_pot = r[0];
    if (virial) *virial = r[1];
    if (npairs) *npairs = (int64_t)np;
    if (k_kin) *k_kin = r[3];
    return LC_OK;
}

lc_status lc_get(lc_ctx *c, lc_get_what what, void *dst, int on_device, void *stream) {
    if (!c || !dst) return LC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = (size_t)c->n, NC = (size_t)c->g.ncell;
    const void *src = nullptr;
    size_t bytes = 0;
    switch (what) {
        case LC_GET_CELL_COUNT: if (!c->binned) return LC_ERR_STATE; src = c->d_count; bytes = 4 * NC; break;
        case LC_GET_CELL_START: if (!c->binned) return LC_ERR_STATE; src = c->d_start; bytes = 4 * NC; break;
        case LC_GET_PERM: if (!c->binned) return LC_ERR_STATE; src = c->cur.id; bytes = 4 * N; break;
        case LC_GET_COLOUR: if (c->nbox > 0) return LC_ERR_INVALID_ARG; src = c->d_colour; bytes = NC; break;
        case LC_GET_FORCES:
        case LC_GET_POS:
        case LC_GET_VEL: {
            if (!c->have_state) return LC_ERR_STATE;
            if (what == LC_GET_FORCES && !c->forces_valid) return LC_ERR_STATE;
            double *tmp = c->nxt.x;   // 3n doubles of scratch between binnings
            if (what == LC_GET_FORCES) LC_TRY(launch_unsort_vec(c, c->fx, c->fy, c->fz, tmp, s, 0));
            else if (what == LC_GET_POS) LC_TRY(launch_unsort_vec(c, c->cur.x, c->cur.y, c->cur.z, tmp, s, 1));
            else LC_TRY(launch_unsort_vec(c, c->cur.vx, c->cur.vy, c->cur.vz, tmp, s, 0));
            src = tmp;
            bytes = 3 * N * sizeof(double);
            break;
        }
        default: return LC_ERR_INVALID_ARG;
    }
    if (bytes == 0) return LC_OK;
    LC_TRY(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!on_device) return read_err(c, s);
    return LC_OK;
}

lc_status lc_grid(const lc_ctx *c, int32_t nc[3], int32_t *ncolours, int32_t *nphases) {
    if (!c) return LC_ERR_INVALID_ARG;
    if (nc) for (int d = 0; d < 3; ++d) nc[d] = c->g.nc[d];
    if (ncolours) *ncolours = c->g.ncolours;
    if (nphases) *nphases = c->g.cs_ncolours;   // colours of LC_SCHED_COLOUR
    return LC_OK;
}

lc_status lc_schedule_check(lc_ctx *c, lc_schedule sched, int64_t *conflicts, int64_t *coverage_errors, void *stream) {
    if (!c || sched < LC_SCHED_COLOUR || sched > LC_SCHED_BUFFER || c->nbox > 0) return LC_ERR_INVALID_ARG;
    LC_TRY_ST(ensure_colour_tables(c, sched));
    if (!c->d_visit) {   // the check's buffers (27 counters per cell) on first use
        const size_t NC = (size_t)c->g.ncell;
        if (!c->d_stamp) LC_TRY(dalloc(&c->d_stamp, NC));
        if (!c->d_counters) LC_TRY(dalloc(&c->d_counters, 4));
        LC_TRY(dalloc(&c->d_visit, 27 * NC));
    }
    cudaStream_t s = (cudaStream_t)stream;
    LC_TRY(launch_schedule_check(c, sched, s));
    unsigned long long cnt[4];
    LC_TRY(cudaMemcpyAsync(cnt, c->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, s));
    LC_TRY(cudaStreamSynchronize(s));
    if (conflicts) *conflicts = cnt[0];
    if (coverage_errors) *coverage_errors = cnt[1];
    return cnt[0] ? LC_ERR_RACE : LC_OK;
}

static lc_status ensure_dag(lc_ctx *c, lc_order order) {
    if (c->dag[order]) return LC_OK;
    if (14 * (int64_t)c->g.ncell > (int64_t(1) << 29)) return LC_ERR_TOO_LARGE;
    Stencil st;
    make_stencil(&st, c->g.dims);
    DagDev *d = nullptr;
    LC_TRY(build_dag(c, st, (int)order, &d));
    c->dag[order] = d;
    return LC_OK;
}

lc_status lc_dag_build(lc_ctx *c, lc_order order, int64_t *ntasks, int64_t *nedges, int64_t *critical_path) {
    if (!c || (order != LC_ORDER_CELL && order != LC_ORDER_LOOPEX) || c->nbox > 0) return LC_ERR_INVALID_ARG;
    LC_TRY_ST(ensure_dag(c, order));
    const DagDev *d = c->dag[order];
    if (ntasks) *ntasks = d->ntasks;
    if (nedges) *nedges = d->nedges;
    if (critical_path) *critical_path = d->critical_path;
    return LC_OK;
}

// perm: a permutation of 0 .. nh (nh = 13 in 3D, 4 in 2D)?
static bool valid_stencil_perm(const int32_t *perm, int32_t nperm, int dims) {
    Stencil st;
    make_stencil(&st, dims);
    if (nperm != st.nh + 1) return false;
    bool seen[14] = {};
    for (int q = 0; q < nperm; ++q) {
        if (perm[q] < 0 || perm[q] > st.nh || seen[perm[q]]) return false;
        seen[perm[q]] = true;
    }
    return true;
}

lc_status lc_dag_plan(const int32_t nc[3], lc_order order, const int32_t *perm, int32_t nperm, int64_t *ntasks,
                      int64_t *nedges, int64_t *critical_path) {
    if (!nc || (order != LC_ORDER_CELL && order != LC_ORDER_LOOPEX)) return LC_ERR_INVALID_ARG;
    const int dims = nc[2] == 1 ? 2 : 3;
    for (int d = 0; d < dims; ++d)
        if (nc[d] < 3) return LC_ERR_BOX_TOO_SMALL;
    if (perm && !valid_stencil_perm(perm, nperm, dims)) return LC_ERR_INVALID_ARG;
    if (14 * (int64_t)nc[0] * nc[1] * nc[2] > (int64_t(1) << 29)) return LC_ERR_TOO_LARGE;
    const int n3[3] = {nc[0], nc[1], nc[2]};
    const int64_t cp = dag_plan_host(n3, (int)order, perm, perm ? nperm : 0, ntasks, nedges);
    if (critical_path) *critical_path = cp;
    return LC_OK;
}

lc_status lc_dag_stencil_order(lc_ctx *c, const int32_t *perm, int32_t nperm) {
    if (!c || c->nbox > 0) return LC_ERR_INVALID_ARG;
    if (perm && !valid_stencil_perm(perm, nperm, c->g.dims)) return LC_ERR_INVALID_ARG;
    c->dag_perm_n = perm ? nperm : 0;
    for (int q = 0; q < c->dag_perm_n; ++q) c->dag_perm[q] = perm[q];
    free_dag(c->dag[LC_ORDER_CELL]);     // rebuilt with the new order on its next use
    c->dag[LC_ORDER_CELL] = nullptr;
    return LC_OK;
}

lc_status lc_dag_forces(lc_ctx *c, lc_order order, double wait_seconds, int flags, int32_t *trace, void *stream) {
    if (!c || (order != LC_ORDER_CELL && order != LC_ORDER_LOOPEX) || c->nbox > 0 || !(wait_seconds == wait_seconds) ||
        (flags & ~LC_DAG_WITHHOLD))
        return LC_ERR_INVALID_ARG;
    if (!c->have_state) return LC_ERR_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    LC_TRY_ST(ensure_dag(c, order));
    int launches = 0;
    if (!c->binned) {
        LC_TRY(launch_bin(c, s, &launches));
        c->binned = true;
    }
    LC_TRY_ST(read_err(c, s));                 // a non-finite input stops here
    c->forces_valid = false;
    const double ws = wait_seconds > 0 ? (wait_seconds < 60.0 ? wait_seconds : 60.0) : 2.0;
    LC_TRY(launch_forces_dag(c, c->dag[order], (long long)(ws * 1e9), flags & LC_DAG_WITHHOLD, trace, s, &launches));
    lc_status st = read_err(c, s);
    if (st == LC_ERR_TIMEOUT) {                // clear the flag: the context stays usable
        LC_TRY(cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
        LC_TRY(cudaStreamSynchronize(s));
        return st;
    }
    if (st) return st;
    c->launches_force = launches;
    c->forces_valid = true;
    return LC_OK;
}

lc_status lc_set_tile(lc_ctx *c, int ni, int warps) {
    if (!c) return LC_ERR_INVALID_ARG;
    if (ni && ni != 8 && ni != 16) return LC_ERR_INVALID_ARG;
    // 1 .. 8 warps per block; 16: the atomic schedule's row-group kernel
    if (warps < 0 || (warps > 8 && warps != 16)) return LC_ERR_INVALID_ARG;
    if (ni) c->ni = ni;
    if (warps) c->warps = warps;
    for (int k = 0; k < kNumGraphs; ++k)
        if (c->graph[k]) { cudaGraphExecDestroy(c->graph[k]); c->graph[k] = nullptr; }
    return LC_OK;
}

lc_status lc_launch_counts(const lc_ctx *c, int32_t *per_force, int32_t *per_step) {
    if (!c) return LC_ERR_INVALID_ARG;
    if (per_force) *per_force = c->launches_force;
    if (per_step) *per_step = c->launches_step;
    return LC_OK;
}

lc_status lc_launch_counts_graphs(const lc_ctx *c, int32_t *one_step, int32_t *two_steps) {
    if (!c) return LC_ERR_INVALID_ARG;
    if (one_step) *one_step = c->launches_one;
    if (two_steps) *two_steps = c->launches_two;
    return LC_OK;
}

}  // extern "C"
