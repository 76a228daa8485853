/*
 * Plain FP64 CPU oracle for the link-cell Lennard-Jones force sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path: every quantity here
 * (grid size, wrap, cell index, colours, half-shell table, pair force) is
 * written out from its definition.  Build: gcc -O2 -ffp-contract=off -fPIC
 * -shared (no FMA contraction, so every product and sum is rounded once).
 *
 * Definitions and where they come from:
 *  - Link-cell method, cells of side >= r_c, partners only in the own and the
 *    neighbouring cells: paper Sec. IV ("Example: Molecular Dynamics").
 *  - Newton's third law, half-shell stencil (centre + 13 neighbours in 3D),
 *    each pair computed once and both particles updated: Sec. IV, Fig. 3.
 *  - Cell-cell interaction (intra / inter) as the unit of work: Sec. IV.
 *  - Literature loop order: per cell the intra-cell interaction first, then
 *    the inter-cell interactions, cells visited x fastest, then y, then z:
 *    Sec. IV and Sec. V.
 *  - Loop exchange with 2-strided colouring (Strategy 1): Sec. VI, Fig. 6.
 *  The paper states no potential; the Lennard-Jones form with
 *  sigma = epsilon = m = 1, truncated (unshifted) at r_c, is the workload's:
 *    U(r) = 4 (r^-12 - r^-6),  F_i = sum_j 24 (2 r^-12 - r^-6) / r^2 (r_i - r_j).
 *
 * Parity pins (tests/test_oracle_*.py): two-particle closed form, perfect FCC
 * lattice shell sums (forces vanish by symmetry), Newton's third law (sum of
 * forces = 0), O(N^2) == link-cell, finite-difference gradient of U, energy
 * conservation under velocity Verlet, binning invariants, colour-phase write
 * disjointness and exact coverage of every half-shell cell pair.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- grid --- */

/* Number of cells per dimension: the largest count whose side is >= r_c,
 * nc_d = floor(L_d / r_c) in IEEE FP64 (cells "of the size of the cutoff
 * radius", Sec. IV).  Returns 0 on success, 1 if any nc_d < 3 (a periodic
 * grid with 2 cells would make the +1 and -1 neighbour the same cell). */
int orc_grid(const double L[3], double rc, int32_t nc[3])
{
    int bad = 0;
    for (int d = 0; d < 3; ++d) {
        double q = floor(L[d] / rc);
        nc[d] = (int32_t)q;
        if (nc[d] < 3) bad = 1;
    }
    return bad;
}

/* Periodic wrap into [0, L): x - L*floor(x/L), each operation rounded once,
 * then one correction step for the rounding edge cases. */
double orc_wrap(double x, double L)
{
    double q = floor(x / L);
    double p = q * L;
    double y = x - p;
    if (y >= L) y = y - L;
    if (y < 0.0) y = y + L;
    if (y >= L) y = 0.0;
    return y;
}

/* Cell coordinate of a wrapped coordinate: (int)(x * (nc / L)), clamped to
 * nc - 1 (the factor nc/L is one FP64 division). */
static int32_t cell_coord(double xw, int32_t nc, double L)
{
    double inv = (double)nc / L;
    double t = xw * inv;
    int32_t c = (int32_t)t;
    if (c > nc - 1) c = nc - 1;
    if (c < 0) c = 0;
    return c;
}

/* Colour class of one cell coordinate for 2-strided colouring (Fig. 6):
 * parity of c, except that the last cell of an odd-sized periodic dimension
 * gets its own class 2 (its +1 neighbour is cell 0, which has the same parity). */
static int colour_class(int32_t c, int32_t nc)
{
    if ((nc & 1) && c == nc - 1) return 2;
    return (int)(c & 1);
}

/* The 13 forward offsets of the 3D half-shell, in (z, y, x) lexicographic
 * order.  Forward: oz > 0, or oz == 0 and oy > 0, or oz == oy == 0 and ox > 0.
 * Any half of the 26 neighbours works (Fig. 3b shows one); this is the one
 * used throughout. */
static void half_shell(int off[13][3])
{
    int k = 0;
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                int fwd = (oz > 0) || (oz == 0 && oy > 0) || (oz == 0 && oy == 0 && ox > 0);
                if (!fwd) continue;
                off[k][0] = ox; off[k][1] = oy; off[k][2] = oz; ++k;
            }
}

/* Loop exchange with colouring (Strategy 1, Sec. VI): a phase runs one
 * colour of cells against a set of stencil offsets, and the writes of one
 * phase must be disjoint.  Two cells of one colour differ by an even number of
 * cells (or are equal) in every dimension, so the neighbours A + o and A' + o'
 * of two same-colour cells can only coincide when o and o' have the same
 * parity pattern (|o_x|, |o_y|, |o_z|).  Offsets with pairwise different
 * patterns may therefore share a phase.  group_of[k] assigns each half-shell
 * offset (table order) to the first of the groups 0..3 that does not yet hold
 * its pattern; the intra-cell interaction belongs to group 0.  Phases are
 * (group g, colour k) for g = 0..3, k = 0..ncolours-1, in that order. */
void orc_offset_groups(int32_t group_of[13])
{
    int off[13][3];
    half_shell(off);
    int used[4][8];
    for (int g = 0; g < 4; ++g) for (int p = 0; p < 8; ++p) used[g][p] = 0;
    for (int k = 0; k < 13; ++k) {
        int pat = (off[k][0] != 0) + 2 * (off[k][1] != 0) + 4 * (off[k][2] != 0);
        int g = 0;
        while (used[g][pat]) ++g;
        used[g][pat] = 1;
        group_of[k] = g;
    }
}

void orc_half_shell(int32_t out[39])
{
    int off[13][3];
    half_shell(off);
    for (int k = 0; k < 13; ++k)
        for (int d = 0; d < 3; ++d) out[3 * k + d] = off[k][d];
}

/* ---------------------------------------------------------------- binning */

/* Counting sort of particles into cells.
 *  pos: x[n], y[n], z[n] by particle ID (index = ID), any real values
 *  out: cell_of[n] (by ID), count[ncell], start[ncell] (exclusive prefix sum),
 *       perm[n] (slot -> ID; within a cell ascending ID), colour[ncell]
 *       (rank of the raw colour cx + 3 cy + 9 cz among the raw colours that
 *       occur), *ncolours.
 * Cells are numbered x fastest: cell = cx + nc_x (cy + nc_y cz). */
int orc_bin(int64_t n, const double *x, const double *y, const double *z,
            const double L[3], double rc,
            int32_t *cell_of, int32_t *count, int32_t *start, int32_t *perm,
            int8_t *colour, int32_t *ncolours)
{
    int32_t nc[3];
    if (orc_grid(L, rc, nc)) return 1;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    for (int64_t c = 0; c < ncell; ++c) count[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t cx = cell_coord(orc_wrap(x[i], L[0]), nc[0], L[0]);
        int32_t cy = cell_coord(orc_wrap(y[i], L[1]), nc[1], L[1]);
        int32_t cz = cell_coord(orc_wrap(z[i], L[2]), nc[2], L[2]);
        int32_t c = cx + nc[0] * (cy + nc[1] * cz);
        cell_of[i] = c;
        count[c] += 1;
    }
    int32_t run = 0;
    for (int64_t c = 0; c < ncell; ++c) { start[c] = run; run += count[c]; }
    /* visiting IDs in ascending order makes the placement stable by ID */
    int32_t *fill = (int32_t *)calloc((size_t)ncell, sizeof(int32_t));
    if (!fill) return 2;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c = cell_of[i];
        perm[start[c] + fill[c]] = (int32_t)i;
        fill[c] += 1;
    }
    free(fill);
    /* colours: raw id per cell, then rank among the raw ids present */
    int present[27];
    for (int k = 0; k < 27; ++k) present[k] = 0;
    for (int32_t cz = 0; cz < nc[2]; ++cz)
        for (int32_t cy = 0; cy < nc[1]; ++cy)
            for (int32_t cx = 0; cx < nc[0]; ++cx)
                present[colour_class(cx, nc[0]) + 3 * colour_class(cy, nc[1]) + 9 * colour_class(cz, nc[2])] = 1;
    int rank[27];
    int r = 0;
    for (int k = 0; k < 27; ++k) { rank[k] = present[k] ? r : -1; if (present[k]) ++r; }
    *ncolours = r;
    for (int32_t cz = 0; cz < nc[2]; ++cz)
        for (int32_t cy = 0; cy < nc[1]; ++cy)
            for (int32_t cx = 0; cx < nc[0]; ++cx) {
                int raw = colour_class(cx, nc[0]) + 3 * colour_class(cy, nc[1]) + 9 * colour_class(cz, nc[2]);
                colour[cx + nc[0] * (cy + nc[1] * cz)] = (int8_t)rank[raw];
            }
    return 0;
}

/* ------------------------------------------------------------ pair force */

/* One Lennard-Jones pair at displacement d = r_i - r_j.  Returns 1 and the
 * scalar f (force on i is f * d), the pair energy u and the pair virial
 * w = f * r^2 if r^2 < r_c^2 (strict; truncated, unshifted potential). */
static int lj_pair(double dx, double dy, double dz, double rc2,
                   double *f, double *u, double *w)
{
    double r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 < rc2)) return 0;
    double inv = 1.0 / r2;
    double s6 = inv * inv * inv;
    *f = 24.0 * s6 * (2.0 * s6 - 1.0) * inv;
    *u = 4.0 * s6 * (s6 - 1.0);
    *w = *f * r2;
    return 1;
}

/* Minimum-image displacement along one axis for wrapped coordinates:
 * t = xi - xj, then t - s L with s the nearest integer image (s in {-1,0,1}). */
static double min_image(double xi, double xj, double L)
{
    double t = xi - xj;
    double s = nearbyint(t / L);
    if (s == 0.0) return t;
    return t - s * L;
}

/* O(N^2) sum over all pairs i < j under the minimum image convention
 * (the plain definition of the forces the link-cell method computes).
 * f: [3n] interleaved (fx, fy, fz) by ID.  *npairs: pairs inside r_c. */
void orc_nsq_forces(int64_t n, const double *x, const double *y, const double *z,
                    const double L[3], double rc,
                    double *f, double *u_pot, double *virial, int64_t *npairs)
{
    double rc2 = rc * rc;
    double U = 0.0, W = 0.0;
    int64_t np = 0;
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        xw[3 * i + 0] = orc_wrap(x[i], L[0]);
        xw[3 * i + 1] = orc_wrap(y[i], L[1]);
        xw[3 * i + 2] = orc_wrap(z[i], L[2]);
        f[3 * i + 0] = f[3 * i + 1] = f[3 * i + 2] = 0.0;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx = min_image(xw[3 * i + 0], xw[3 * j + 0], L[0]);
            double dy = min_image(xw[3 * i + 1], xw[3 * j + 1], L[1]);
            double dz = min_image(xw[3 * i + 2], xw[3 * j + 2], L[2]);
            double fs, u, w;
            if (!lj_pair(dx, dy, dz, rc2, &fs, &u, &w)) continue;
            f[3 * i + 0] += fs * dx; f[3 * i + 1] += fs * dy; f[3 * i + 2] += fs * dz;
            f[3 * j + 0] -= fs * dx; f[3 * j + 1] -= fs * dy; f[3 * j + 2] -= fs * dz;
            U += u; W += w; ++np;
        }
    free(xw);
    *u_pot = U; *virial = W; *npairs = np;
}

/* Serial link-cell sweep in the literature order (Sec. IV / V): cells x
 * fastest; per cell A the intra-cell pairs (i < j in slot order) first, then
 * the 13 half-shell neighbours B = A + o in table order, all i in A against
 * all j in B.  Both particles of a pair are updated (Newton's third law).
 * The periodic image of B is chosen by the cell wrap: if c_A + o leaves the
 * grid on the high side the image sits at +L, on the low side at -L, and the
 * displacement is (x_i - x_j) - s L.  Same outputs as orc_nsq_forces. */
int orc_lc_forces(int64_t n, const double *x, const double *y, const double *z,
                  const double L[3], double rc,
                  double *f, double *u_pot, double *virial, int64_t *npairs)
{
    int32_t nc[3];
    if (orc_grid(L, rc, nc)) return 1;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int8_t *colour = (int8_t *)malloc((size_t)ncell);
    double *xs = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *fs_ = (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t ncol;
    int rcb = orc_bin(n, x, y, z, L, rc, cell_of, count, start, perm, colour, &ncol);
    if (rcb) {
        free(cell_of); free(count); free(start); free(perm); free(colour); free(xs); free(fs_);
        return rcb;
    }
    for (int64_t s = 0; s < n; ++s) {
        int32_t id = perm[s];
        xs[3 * s + 0] = orc_wrap(x[id], L[0]);
        xs[3 * s + 1] = orc_wrap(y[id], L[1]);
        xs[3 * s + 2] = orc_wrap(z[id], L[2]);
    }
    int off[13][3];
    half_shell(off);
    double rc2 = rc * rc;
    double U = 0.0, W = 0.0;
    int64_t np = 0;
    for (int32_t cz = 0; cz < nc[2]; ++cz)
        for (int32_t cy = 0; cy < nc[1]; ++cy)
            for (int32_t cx = 0; cx < nc[0]; ++cx) {
                int32_t A = cx + nc[0] * (cy + nc[1] * cz);
                int32_t a0 = start[A], a1 = start[A] + count[A];
                /* intra-cell interaction */
                for (int32_t i = a0; i < a1; ++i)
                    for (int32_t j = i + 1; j < a1; ++j) {
                        double dx = xs[3 * i + 0] - xs[3 * j + 0];
                        double dy = xs[3 * i + 1] - xs[3 * j + 1];
                        double dz = xs[3 * i + 2] - xs[3 * j + 2];
                        double fsc, u, w;
                        if (!lj_pair(dx, dy, dz, rc2, &fsc, &u, &w)) continue;
                        fs_[3 * i + 0] += fsc * dx; fs_[3 * i + 1] += fsc * dy; fs_[3 * i + 2] += fsc * dz;
                        fs_[3 * j + 0] -= fsc * dx; fs_[3 * j + 1] -= fsc * dy; fs_[3 * j + 2] -= fsc * dz;
                        U += u; W += w; ++np;
                    }
                /* inter-cell interactions with the half-shell neighbours */
                for (int k = 0; k < 13; ++k) {
                    int32_t c[3] = {cx + off[k][0], cy + off[k][1], cz + off[k][2]};
                    double sh[3];
                    for (int d = 0; d < 3; ++d) {
                        sh[d] = 0.0;
                        if (c[d] >= nc[d]) { c[d] -= nc[d]; sh[d] = L[d]; }
                        else if (c[d] < 0) { c[d] += nc[d]; sh[d] = -L[d]; }
                    }
                    int32_t B = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
                    int32_t b0 = start[B], b1 = start[B] + count[B];
                    for (int32_t i = a0; i < a1; ++i)
                        for (int32_t j = b0; j < b1; ++j) {
                            double dx = xs[3 * i + 0] - xs[3 * j + 0];
                            double dy = xs[3 * i + 1] - xs[3 * j + 1];
                            double dz = xs[3 * i + 2] - xs[3 * j + 2];
                            if (sh[0] != 0.0) dx = dx - sh[0];
                            if (sh[1] != 0.0) dy = dy - sh[1];
                            if (sh[2] != 0.0) dz = dz - sh[2];
                            double fsc, u, w;
                            if (!lj_pair(dx, dy, dz, rc2, &fsc, &u, &w)) continue;
                            fs_[3 * i + 0] += fsc * dx; fs_[3 * i + 1] += fsc * dy; fs_[3 * i + 2] += fsc * dz;
                            fs_[3 * j + 0] -= fsc * dx; fs_[3 * j + 1] -= fsc * dy; fs_[3 * j + 2] -= fsc * dz;
                            U += u; W += w; ++np;
                        }
                }
            }
    for (int64_t s = 0; s < n; ++s) {
        int32_t id = perm[s];
        f[3 * id + 0] = fs_[3 * s + 0];
        f[3 * id + 1] = fs_[3 * s + 1];
        f[3 * id + 2] = fs_[3 * s + 2];
    }
    free(cell_of); free(count); free(start); free(perm); free(colour); free(xs); free(fs_);
    *u_pot = U; *virial = W; *npairs = np;
    return 0;
}

/* Pair-force scale of every particle: S_i = sum over j within r_c of
 * |F_ij| (the magnitudes of the pair forces, not of their sum).  Any
 * arithmetic that rounds each pair force to relative precision eps errs by
 * at most about eps S_i on F_i, whatever cancellation the sum has; tests
 * normalise force errors by it where forces cancel strongly.  scale: [n] by
 * ID.  Same loops and pair test as orc_nsq_forces. */
void orc_force_scale(int64_t n, const double *x, const double *y, const double *z,
                     const double L[3], double rc, double *scale)
{
    double rc2 = rc * rc;
    double *xw = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int32_t nc[3];
    orc_grid(L, rc, nc);
    for (int64_t i = 0; i < n; ++i) {
        xw[3 * i + 0] = orc_wrap(x[i], L[0]);
        xw[3 * i + 1] = orc_wrap(y[i], L[1]);
        xw[3 * i + 2] = orc_wrap(z[i], L[2]);
        scale[i] = 0.0;
    }
    /* bucket by cell to keep it O(N) */
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *head = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int32_t c3[3];
        for (int d = 0; d < 3; ++d) c3[d] = cell_coord(xw[3 * i + d], nc[d], L[d]);
        int32_t c = c3[0] + nc[0] * (c3[1] + nc[1] * c3[2]);
        next[i] = head[c];
        head[c] = (int32_t)i;
    }
    for (int64_t i = 0; i < n; ++i) {
        int32_t ci[3];
        for (int d = 0; d < 3; ++d) ci[d] = cell_coord(xw[3 * i + d], nc[d], L[d]);
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    int32_t c[3] = {ci[0] + ox, ci[1] + oy, ci[2] + oz};
                    for (int d = 0; d < 3; ++d) { if (c[d] >= nc[d]) c[d] -= nc[d]; else if (c[d] < 0) c[d] += nc[d]; }
                    for (int32_t j = head[c[0] + nc[0] * (c[1] + nc[1] * c[2])]; j >= 0; j = next[j]) {
                        if (j == i) continue;
                        double dx = min_image(xw[3 * i + 0], xw[3 * j + 0], L[0]);
                        double dy = min_image(xw[3 * i + 1], xw[3 * j + 1], L[1]);
                        double dz = min_image(xw[3 * i + 2], xw[3 * j + 2], L[2]);
                        double fs, u, w;
                        if (!lj_pair(dx, dy, dz, rc2, &fs, &u, &w)) continue;
                        scale[i] += fabs(fs) * sqrt(dx * dx + dy * dy + dz * dz);
                    }
                }
    }
    free(head); free(next); free(xw);
}

/* Force on selected particles only (sampled checks at sizes where a full
 * sweep is too slow): for each requested ID, the sum over all j != i within
 * r_c, found by scanning the 27 cells around the particle's cell.  Same pair
 * arithmetic and image rule as orc_lc_forces; the sum order differs. */
int orc_forces_sample(int64_t n, const double *x, const double *y, const double *z,
                      const double L[3], double rc, int64_t nsample, const int64_t *ids,
                      double *f, int64_t *nneigh)
{
    int32_t nc[3];
    if (orc_grid(L, rc, nc)) return 1;
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int8_t *colour = (int8_t *)malloc((size_t)ncell);
    int32_t ncol;
    int rcb = orc_bin(n, x, y, z, L, rc, cell_of, count, start, perm, colour, &ncol);
    if (rcb) {
        free(cell_of); free(count); free(start); free(perm); free(colour);
        return rcb;
    }
    double rc2 = rc * rc;
    for (int64_t s = 0; s < nsample; ++s) {
        int64_t i = ids[s];
        double xi = orc_wrap(x[i], L[0]), yi = orc_wrap(y[i], L[1]), zi = orc_wrap(z[i], L[2]);
        int32_t ci[3] = {cell_coord(xi, nc[0], L[0]), cell_coord(yi, nc[1], L[1]), cell_coord(zi, nc[2], L[2])};
        double fx = 0.0, fy = 0.0, fz = 0.0;
        int64_t nn = 0;
        for (int oz = -1; oz <= 1; ++oz)
            for (int oy = -1; oy <= 1; ++oy)
                for (int ox = -1; ox <= 1; ++ox) {
                    int32_t c[3] = {ci[0] + ox, ci[1] + oy, ci[2] + oz};
                    for (int d = 0; d < 3; ++d) { if (c[d] >= nc[d]) c[d] -= nc[d]; else if (c[d] < 0) c[d] += nc[d]; }
                    int32_t B = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
                    for (int32_t sl = start[B]; sl < start[B] + count[B]; ++sl) {
                        int32_t j = perm[sl];
                        if (j == i) continue;
                        double dx = min_image(xi, orc_wrap(x[j], L[0]), L[0]);
                        double dy = min_image(yi, orc_wrap(y[j], L[1]), L[1]);
                        double dz = min_image(zi, orc_wrap(z[j], L[2]), L[2]);
                        double fsc, u, w;
                        if (!lj_pair(dx, dy, dz, rc2, &fsc, &u, &w)) continue;
                        fx += fsc * dx; fy += fsc * dy; fz += fsc * dz; ++nn;
                    }
                }
        f[3 * s + 0] = fx; f[3 * s + 1] = fy; f[3 * s + 2] = fz;
        nneigh[s] = nn;
    }
    free(cell_of); free(count); free(start); free(perm); free(colour);
    return 0;
}

/* --------------------------------------------------------- integration --- */

/* Velocity Verlet (m = 1): v += dt/2 F; x += dt v; x wrapped; F = F(x);
 * v += dt/2 F.  x, v: [3n] interleaved by ID, updated in place; f holds the
 * forces of the current x on entry (computed here if *have_f == 0) and on
 * exit.  e_out[3*(s)] = (U, K, W) after step s for s = 0..nsteps (s = 0 is
 * the initial state; its U and W are NaN when have_f != 0).  Forces by
 * orc_lc_forces. */
int orc_verlet(int64_t n, double *xyz, double *v, double *f, int have_f,
               const double L[3], double rc, double dt, int nsteps, double *e_out)
{
    double *px = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *py = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *pz = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double U = NAN, W = NAN;
    int64_t np;
    int rc_ = 0;
    for (int64_t i = 0; i < n; ++i) { px[i] = xyz[3 * i]; py[i] = xyz[3 * i + 1]; pz[i] = xyz[3 * i + 2]; }
    if (!have_f) {  /* else f already holds F(x); U, W of step 0 stay NaN */
        rc_ = orc_lc_forces(n, px, py, pz, L, rc, f, &U, &W, &np);
        if (rc_) return rc_;
    }
    double half = 0.5 * dt;
    for (int s = 0; s <= nsteps; ++s) {
        if (s > 0) {
            for (int64_t i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) {
                    v[3 * i + d] = v[3 * i + d] + half * f[3 * i + d];
                    double xn = xyz[3 * i + d] + dt * v[3 * i + d];
                    xyz[3 * i + d] = orc_wrap(xn, L[d]);
                }
            for (int64_t i = 0; i < n; ++i) { px[i] = xyz[3 * i]; py[i] = xyz[3 * i + 1]; pz[i] = xyz[3 * i + 2]; }
            rc_ = orc_lc_forces(n, px, py, pz, L, rc, f, &U, &W, &np);
            if (rc_) return rc_;
            for (int64_t i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) v[3 * i + d] = v[3 * i + d] + half * f[3 * i + d];
        }
        double K = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) K += v[3 * i + d] * v[3 * i + d];
        K = 0.5 * K;
        if (e_out) { e_out[3 * s + 0] = U; e_out[3 * s + 1] = K; e_out[3 * s + 2] = W; }
    }
    free(px); free(py); free(pz);
    return 0;
}
