/*
 * CPU baseline: the paper's Strategy 1 for the link-cell force sweep with
 * Newton's third law, on all host cores (OpenMP).
 *
 * Sec. VI, Strategy 1 and Fig. 6: the loops over cells and over the stencil
 * are exchanged, so that the outer loop runs over the stencil entries (the
 * intra-cell interaction and the 13 forward half-shell offsets o) and, for
 * each entry, over the 2-strided colour classes of the cells; the cells of one
 * class are processed in parallel.  Two cells of one class differ by an even
 * number of cells in every dimension while o has an odd component, so the
 * tasks (A, A + o) of one (entry, class) phase write pairwise different cells:
 * plain writes, no atomics, one barrier per phase.  An odd-sized periodic
 * dimension gives its last cell a class of its own (its neighbour across the
 * boundary, cell 0, has the same parity).
 *
 * This is a measured baseline for bench.py, not the oracle: it is written
 * independently of oracle/ and of the CUDA library (tests check it against
 * the oracle's serial link-cell sums).  FP64 throughout; Lennard-Jones with
 * sigma = epsilon = 1, truncated (unshifted) at r_c; cells nc_d =
 * floor(L_d / r_c); within a cell the particles are kept in ID order.
 * Build: gcc -O3 -fopenmp -fPIC -shared.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int wrapi(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }

static double wrapx(double x, double L)
{
    double y = x - L * floor(x / L);
    if (y >= L) y -= L;
    if (y < 0.0) y += L;
    if (y >= L) y = 0.0;
    return y;
}

static int cls(int c, int n) { return ((n & 1) && c == n - 1) ? 2 : (c & 1); }

int s1_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Forces (n x 3, by particle ID), potential energy *U, virial *W and the
 * number of pairs inside r_c of positions xyz (n x 3).  Returns 0, or 1 if
 * a dimension has fewer than 3 cells, 2 if memory runs out.
 */
int s1_forces(int64_t n, const double *xyz, const double L[3], double rc, double *f, double *U, double *W,
              int64_t *npairs)
{
    int nc[3];
    for (int d = 0; d < 3; ++d) {
        nc[d] = (int)floor(L[d] / rc);
        if (nc[d] < 3) return 1;
    }
    const int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int *cell = malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int64_t *start = calloc((size_t)ncell + 1, sizeof(int64_t));
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)ncell);
    double *p = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));   /* wrapped, cell order */
    double *fs = calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));   /* forces, cell order */
    int64_t *id = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cell || !start || !fill || !p || !fs || !id) {
        free(cell); free(start); free(fill); free(p); free(fs); free(id);
        return 2;
    }
    /* counting sort by cell, ID order inside a cell */
    for (int64_t i = 0; i < n; ++i) {
        int c3[3];
        for (int d = 0; d < 3; ++d) {
            const double x = wrapx(xyz[3 * i + d], L[d]);
            int c = (int)(x * ((double)nc[d] / L[d]));
            c3[d] = c > nc[d] - 1 ? nc[d] - 1 : (c < 0 ? 0 : c);
        }
        cell[i] = c3[0] + nc[0] * (c3[1] + nc[1] * c3[2]);
        start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    memcpy(fill, start, sizeof(int64_t) * (size_t)ncell);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t s = fill[cell[i]]++;
        id[s] = i;
        for (int d = 0; d < 3; ++d) p[3 * s + d] = wrapx(xyz[3 * i + d], L[d]);
    }
    /* the stencil: entry 0 intra, entries 1..13 the forward half-shell */
    int st[14][3] = {{0, 0, 0}};
    int k = 1;
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox)
                if (oz > 0 || (oz == 0 && oy > 0) || (oz == 0 && oy == 0 && ox > 0)) {
                    st[k][0] = ox; st[k][1] = oy; st[k][2] = oz;
                    ++k;
                }
    const double rc2 = rc * rc;
    double u6 = 0.0, u12 = 0.0, wsum = 0.0;
    int64_t pairs = 0;
    /* cells of colour class a along each dimension, in order */
    int *ccell[3][3], ncls[3][3];
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a) {
            ccell[d][a] = malloc(sizeof(int) * (size_t)nc[d]);
            ncls[d][a] = 0;
        }
    for (int d = 0; d < 3; ++d)
        for (int c = 0; c < nc[d]; ++c) {
            const int a = cls(c, nc[d]);
            ccell[d][a][ncls[d][a]++] = c;
        }
    for (int e = 0; e < 14; ++e) {                          /* stencil entry: outer (loop exchange) */
        for (int a = 0; a < 27; ++a) {                      /* colour class (ax, ay, az) */
            const int ac[3] = {a % 3, (a / 3) % 3, a / 9};
            const int64_t ntask = (int64_t)ncls[0][ac[0]] * ncls[1][ac[1]] * ncls[2][ac[2]];
            if (ntask == 0) continue;
            #pragma omp parallel for schedule(dynamic, 8) reduction(+ : u6, u12, wsum, pairs)
            for (int64_t t = 0; t < ntask; ++t) {
                const int cA[3] = {ccell[0][ac[0]][t % ncls[0][ac[0]]],
                                   ccell[1][ac[1]][(t / ncls[0][ac[0]]) % ncls[1][ac[1]]],
                                   ccell[2][ac[2]][t / ((int64_t)ncls[0][ac[0]] * ncls[1][ac[1]])]};
                const int64_t A = cA[0] + nc[0] * ((int64_t)cA[1] + nc[1] * (int64_t)cA[2]);
                int cB[3];
                double sh[3];
                for (int d = 0; d < 3; ++d) {
                    const int c = cA[d] + st[e][d];
                    cB[d] = wrapi(c, nc[d]);
                    sh[d] = c >= nc[d] ? L[d] : (c < 0 ? -L[d] : 0.0);   /* image of B seen from A */
                }
                const int64_t B = cB[0] + nc[0] * ((int64_t)cB[1] + nc[1] * (int64_t)cB[2]);
                for (int64_t i = start[A]; i < start[A + 1]; ++i) {
                    const int64_t j0 = e == 0 ? i + 1 : start[B];
                    for (int64_t j = j0; j < start[B + 1]; ++j) {
                        const double dx = p[3 * i] - (p[3 * j] + sh[0]);
                        const double dy = p[3 * i + 1] - (p[3 * j + 1] + sh[1]);
                        const double dz = p[3 * i + 2] - (p[3 * j + 2] + sh[2]);
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        if (!(r2 < rc2)) continue;
                        const double s2 = 1.0 / r2, s6 = s2 * s2 * s2;
                        const double fr = 24.0 * s6 * (2.0 * s6 - 1.0) * s2;
                        fs[3 * i] += fr * dx; fs[3 * i + 1] += fr * dy; fs[3 * i + 2] += fr * dz;
                        fs[3 * j] -= fr * dx; fs[3 * j + 1] -= fr * dy; fs[3 * j + 2] -= fr * dz;
                        u6 += s6;
                        u12 += s6 * s6;
                        wsum += fr * r2;
                        ++pairs;
                    }
                }
            }
        }
    }
    for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 3; ++a) free(ccell[d][a]);
    for (int64_t s = 0; s < n; ++s)
        for (int d = 0; d < 3; ++d) f[3 * id[s] + d] = fs[3 * s + d];
    *U = 4.0 * (u12 - u6);
    *W = wsum;
    *npairs = pairs;
    free(cell); free(start); free(fill); free(p); free(fs); free(id);
    return 0;
}
