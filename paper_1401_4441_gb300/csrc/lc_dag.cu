// Task dependency DAG of the link-cell force sweep, built on the host for
// the device task queue (k_force_dag).
//
// The paper's model (Sec. III, Sec. V): a StarSs runtime turns the sequence
// of task creations into a DAG by comparing the addresses of the tasks'
// parameters; a cell-cell interaction task declares both of its cells inout
// (Sec. IV), so it depends on the last earlier task that touched either cell.
// Two creation orders are built:
//   LC_ORDER_CELL    outer loop over the cells (x fastest), inner loop over
//                    the stencil: the intra-cell task, then the 13 half-shell
//                    offsets in table order (the literature order, Sec. IV/V);
//   LC_ORDER_LOOPEX  loop exchange with 2-strided colouring (Sec. VI,
//                    Strategy 1, Fig. 6): outer loop over the stencil entries
//                    (intra first), then over the colours, inner loop over the
//                    cells of that colour (x fastest).
// With equal task durations the critical path counted in tasks bounds the
// speedup (Eq. 1): S = tasks / critical path.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lc_internal.cuh"

namespace lc {

namespace {

int wrap_cell(int c, int n) { return c >= n ? c - n : (c < 0 ? c + n : c); }

// Creation order of the (nh + 1) * ncell tasks, each coded A << 4 | k.
// perm: the order of the stencil entries inside a cell for LC_ORDER_CELL
// (k values, a permutation of 0 .. nh), or empty for table order.
std::vector<int> creation_order(const Grid &g, const Stencil &st, int order, const std::vector<int> &perm) {
    const int ncell = g.ncell;
    const int per = st.nh + 1;
    std::vector<int> task;
    task.reserve((size_t)ncell * per);
    if (order == LC_ORDER_CELL) {
        for (int A = 0; A < ncell; ++A)
            for (int q = 0; q < per; ++q) task.push_back(A << 4 | (perm.empty() ? q : perm[q]));
    } else {
        std::vector<int> colour(ncell);
        for (int A = 0; A < ncell; ++A) {
            const int c[3] = {A % g.nc[0], (A / g.nc[0]) % g.nc[1], A / (g.nc[0] * g.nc[1])};
            int raw = 0, mul = 1;
            for (int d = 0; d < 3; ++d, mul *= 3) {
                const int cls = (g.nc[d] % 2 == 1 && c[d] == g.nc[d] - 1) ? 2 : (c[d] & 1);
                raw += cls * mul;
            }
            colour[A] = g.colour_of_raw[raw];
        }
        for (int k = 0; k < per; ++k)
            for (int col = 0; col < g.ncolours; ++col)
                for (int A = 0; A < ncell; ++A)
                    if (colour[A] == col) task.push_back(A << 4 | k);
    }
    return task;
}

}  // namespace

// The DAG of one creation order on the host (successor lists in CSR).
struct DagHost {
    std::vector<int> task, pred_count, succ_start, succ, queue_init;
    int nroots = 0;
    int64_t nedges = 0, critical_path = 0;
};

void plan_dag(const Grid &g, const Stencil &st, int order, const std::vector<int> &perm, DagHost &h) {
    h.task = creation_order(g, st, order, perm);
    const std::vector<int> &task = h.task;
    const int T = (int)task.size();
    std::vector<int> last(g.ncell, -1);
    std::vector<int> pred_count(T, 0), depth(T, 0), outdeg(T, 0);
    std::vector<int> preds(2 * (size_t)T, -1);
    int64_t cp = 0;
    for (int t = 0; t < T; ++t) {
        const int A = task[t] >> 4, k = task[t] & 15;
        int B = A;
        if (k > 0) {
            const int cA[3] = {A % g.nc[0], (A / g.nc[0]) % g.nc[1], A / (g.nc[0] * g.nc[1])};
            int cB[3];
            for (int d = 0; d < 3; ++d) cB[d] = wrap_cell(cA[d] + st.hs[k - 1][d], g.nc[d]);
            B = cB[0] + g.nc[0] * (cB[1] + g.nc[1] * cB[2]);
        }
        int p0 = last[A], p1 = (B != A) ? last[B] : -1;
        if (p1 == p0) p1 = -1;
        int dep = 0;
        if (p0 >= 0) { preds[2 * (size_t)t] = p0; ++outdeg[p0]; dep = std::max(dep, depth[p0]); ++pred_count[t]; }
        if (p1 >= 0) { preds[2 * (size_t)t + 1] = p1; ++outdeg[p1]; dep = std::max(dep, depth[p1]); ++pred_count[t]; }
        depth[t] = dep + 1;
        cp = std::max<int64_t>(cp, depth[t]);
        last[A] = t;
        last[B] = t;
    }
    std::vector<int> succ_start(T + 1, 0);
    for (int t = 0; t < T; ++t) succ_start[t + 1] = succ_start[t] + outdeg[t];
    const int64_t E = succ_start[T];
    std::vector<int> succ(std::max<int64_t>(E, 1)), fill(succ_start.begin(), succ_start.end() - 1);
    for (int t = 0; t < T; ++t)     // successors listed in creation order
        for (int q = 0; q < 2; ++q) {
            const int p = preds[2 * (size_t)t + q];
            if (p >= 0) succ[fill[p]++] = t;
        }
    std::vector<int> queue_init(T, -1);
    int nroots = 0;
    for (int t = 0; t < T; ++t)
        if (pred_count[t] == 0) queue_init[nroots++] = t;
    h.pred_count.swap(pred_count);
    h.succ_start.swap(succ_start);
    h.succ.swap(succ);
    h.queue_init.swap(queue_init);
    h.nroots = nroots;
    h.nedges = E;
    h.critical_path = cp;
}

// Builds the DAG of one creation order and uploads it.  Host work is
// O(tasks); device memory: about 9 ints per task.
cudaError_t build_dag(const Ctx *c, const Stencil &st, int order, DagDev **out) {
    *out = nullptr;
    DagHost h;
    std::vector<int> perm;
    if (order == LC_ORDER_CELL && c->dag_perm_n > 0) perm.assign(c->dag_perm, c->dag_perm + c->dag_perm_n);
    plan_dag(c->g, st, order, perm, h);
    const int T = (int)h.task.size();
    const int64_t E = h.nedges;
    const int nroots = h.nroots;
    const std::vector<int> &task = h.task, &succ_start = h.succ_start, &succ = h.succ,
                           &pred_count = h.pred_count, &queue_init = h.queue_init;
    const int ctrl_init[4] = {0, nroots, 0, 0};

    DagDev *d = new DagDev();
    d->ntasks = T;
    d->nroots = nroots;
    d->nedges = E;
    d->critical_path = h.critical_path;
    // one allocation: task, succ_start, succ, pred_count, cnt, queue, queue_init, ctrl, ctrl_init
    const size_t words = (size_t)T * 6 + (size_t)(T + 1) + (size_t)std::max<int64_t>(E, 1) + 8;
    int *base = nullptr;
    cudaError_t e = cudaMalloc(&base, sizeof(int) * words);
    if (e) { delete d; return e; }
    int *p = base;
    d->task = p; p += T;
    d->succ_start = p; p += T + 1;
    d->succ = p; p += std::max<int64_t>(E, 1);
    d->pred_count = p; p += T;
    d->cnt = p; p += T;
    d->queue = p; p += T;
    d->queue_init = p; p += T;
    d->ctrl = p; p += 4;
    d->ctrl_init = p; p += 4;
    struct { int *dst; const void *src; size_t n; } up[] = {
        {d->task, task.data(), (size_t)T}, {d->succ_start, succ_start.data(), (size_t)T + 1},
        {d->succ, succ.data(), (size_t)E}, {d->pred_count, pred_count.data(), (size_t)T},
        {d->queue_init, queue_init.data(), (size_t)T}, {d->ctrl_init, ctrl_init, 4}};
    for (auto &u : up)
        if (!e && u.n) e = cudaMemcpy(u.dst, u.src, sizeof(int) * u.n, cudaMemcpyHostToDevice);
    if (e) { cudaFree(base); delete d; return e; }
    *out = d;
    return cudaSuccess;
}

int64_t dag_plan_host(const int nc[3], int order, const int *perm, int nperm, int64_t *ntasks, int64_t *nedges) {
    Grid g;
    const int dims = nc[2] == 1 ? 2 : 3;
    const double box[3] = {(double)nc[0], (double)nc[1], (double)nc[2]};
    make_grid(&g, box, 1.0, dims);
    Stencil st;
    make_stencil(&st, dims);
    DagHost h;
    std::vector<int> p;
    if (order == LC_ORDER_CELL && perm && nperm > 0) p.assign(perm, perm + nperm);
    plan_dag(g, st, order, p, h);
    if (ntasks) *ntasks = (int64_t)h.task.size();
    if (nedges) *nedges = h.nedges;
    return h.critical_path;
}

void free_dag(DagDev *d) {
    if (!d) return;
    cudaFree(d->task);    // the start of the single allocation
    delete d;
}

}  // namespace lc
