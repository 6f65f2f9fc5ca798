/*
 * CPU FP64 oracle for the weight function and the weighted K-means of the
 * complex-valued K-means ISDF (arXiv 2208.07731).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never does.
 * It shares no code with the CUDA library.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no fast-math), so
 * that every floating-point operation below is one IEEE-rounded operation in
 * the written order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* |z|^alpha for z = re + i im, via m = |z|^2 = re*re + im*im (Eq. weight
 * function 2), for alpha != 2. The values of alpha the paper studies besides
 * 2 (SM, SCM, SQM: alpha = 1, 3, 4) use sqrt and products only; any other
 * alpha uses pow. */
static double modpow(double re, double im, double alpha)
{
    double m = re * re;
    m = m + im * im;
    if (alpha == 1.0) return sqrt(m);
    if (alpha == 3.0) return m * sqrt(m);
    if (alpha == 4.0) return m * m;
    return pow(m, 0.5 * alpha);
}

/* floor(log2|x|) for x != 0 */
static int log2_floor(double x)
{
    int e = 0;
    frexp(x, &e);
    return e - 1;
}

/* round-to-nearest-even of an unsigned 128-bit integer, times 2^scale */
static double u128_scaled(u128 acc, int scale)
{
    return ldexp((double)acc, scale);
}

/*
 * Exact sum of the squared real components x = Re z, Im z of the n columns of
 * one or two rows (a, na) and (b, nb): every x^2 is exact as a rational, the
 * row's window top is E = max floor(log2|x|) over its non-zero components, and
 *     sum = RN( sum_x floor(x^2 2^(110 - 2E)) ) * 2^(2E - 110),
 * i.e. the squares are truncated 2^-110 below 2^(2E) (at most 2^14 of them,
 * so the integer sum stays below 2^127), summed exactly, and rounded once.
 * Each x = m 2^(e - 53) with an integer m < 2^53 (frexp), so x^2 = m^2 2^(2e-106)
 * and the term is floor(m^2 2^(2e + 4 - 2E)). Returns 0 for an all-zero row.
 */
static double exact_square_sum(const double *a, int32_t na, const double *b, int32_t nb)
{
    int E = -100000;
    for (int32_t i = 0; i < 2 * na; ++i) if (a[i] != 0.0 && log2_floor(a[i]) > E) E = log2_floor(a[i]);
    for (int32_t j = 0; j < 2 * nb; ++j) if (b[j] != 0.0 && log2_floor(b[j]) > E) E = log2_floor(b[j]);
    if (E == -100000) return 0.0;
    u128 acc = 0;
    for (int32_t k = 0; k < 2 * (na + nb); ++k) {
        const double x = k < 2 * na ? a[k] : b[k - 2 * na];
        if (x == 0.0) continue;
        int e = 0;
        const double f = frexp(fabs(x), &e);
        const u128 m = (u128)(uint64_t)ldexp(f, 53);      /* |x| = m 2^(e - 53), m < 2^53 exact */
        const int sh = 2 * e + 4 - 2 * E;                   /* <= 6 */
        const u128 sq = m * m;
        if (sh >= 0) acc += sq << sh;
        else if (sh > -128) acc += sq >> (-sh);
    }
    return u128_scaled(acc, 2 * E - 110);
}

/*
 * Exact sum of non-negative FP64 terms t_k: window top E = max floor(log2 t),
 *     sum = RN( sum_k floor(t_k 2^(110 - E)) ) * 2^(E - 110)
 * (at most 2^13 terms, each below 2^111, so the integer sum stays below 2^127).
 */
static double exact_term_sum(const double *t, int64_t n)
{
    int E = -100000;
    for (int64_t k = 0; k < n; ++k) if (t[k] != 0.0 && log2_floor(t[k]) > E) E = log2_floor(t[k]);
    if (E == -100000) return 0.0;
    u128 acc = 0;
    for (int64_t k = 0; k < n; ++k) acc += (u128)ldexp(t[k], 110 - E);
    return u128_scaled(acc, E - 110);
}

/*
 * Weight function, Sec. 2.2.
 *   kind 0 (SSM family, Eq. weight function 2): w(r) = sum_i |phi_i(r)|^a + sum_j |psi_j(r)|^a
 *   kind 1 (PSM, Eq. weight function):          w(r) = (sum_i |phi_i(r)|^2)(sum_j |psi_j(r)|^2)
 * Each sum runs over all columns of its orbital set(s) and is the exact sum of
 * its terms rounded once (the reading of these sums used on both sides; any
 * summation order gives the same bits):
 *   alpha = 2: the terms are the exact squares of the real components
 *              (exact_square_sum over both sets for SSM, over each set for PSM);
 *   alpha != 2: the terms are |z|^alpha in FP64 (modpow), summed exactly over
 *              both sets (exact_term_sum).
 * PSM multiplies its two sums once. phi, psi: interleaved complex128, row r
 * at phi + 2*r*ld.
 */
int oracle_weights(const double *phi, int64_t ld_phi, int32_t n_phi,
                   const double *psi, int64_t ld_psi, int32_t n_psi,
                   int64_t n_r, int32_t kind, double alpha, double *w)
{
    if (kind == 1) alpha = 2.0;
#pragma omp parallel
    {
        double *t = (alpha == 2.0) ? NULL : (double *)malloc(sizeof(double) * (size_t)(n_phi + n_psi));
#pragma omp for schedule(static)
        for (int64_t r = 0; r < n_r; ++r) {
            const double *a = phi + 2 * r * ld_phi;
            const double *b = psi + 2 * r * ld_psi;
            if (kind == 1) {
                w[r] = exact_square_sum(a, n_phi, b, 0) * exact_square_sum(b, n_psi, a, 0);
            } else if (alpha == 2.0) {
                w[r] = exact_square_sum(a, n_phi, b, n_psi);
            } else {
                for (int32_t i = 0; i < n_phi; ++i) t[i] = modpow(a[2 * i], a[2 * i + 1], alpha);
                for (int32_t j = 0; j < n_psi; ++j) t[n_phi + j] = modpow(b[2 * j], b[2 * j + 1], alpha);
                w[r] = exact_term_sum(t, n_phi + n_psi);
            }
        }
        free(t);
    }
    return 0;
}

/* squared Euclidean distance, Eq. opt (second form): ((dx^2 + dy^2) + dz^2) */
static inline double dist2(double x, double y, double z, const double *c)
{
    double dx = x - c[0], dy = y - c[1], dz = z - c[2];
    double d = dx * dx;
    d = d + dy * dy;
    d = d + dz * dz;
    return d;
}

static int bits_of(uint64_t v) { int b = 0; while (v) { ++b; v >>= 1; } return b; }

/*
 * Weighted Lloyd K-means on the real-space grid, Algorithm 1 with Eq. opt
 * (second form) and Eq. r_k.
 *
 * Grid: x_r = h*(ix, iy, iz), h_k = cell[k]/n_k, r = (ix*ny + iy)*nz + iz.
 * Start: c_0 = x[init_idx]. For t = 0 .. max_iter-1:
 *   (i)   a_t(r) = argmin_mu |x_r - c_mu|^2, ties to the lowest mu;
 *         J_t = sum_r w(r) |x_r - c_{a_t(r)}|^2 (ascending r);
 *   (ii)  c_{t+1,mu} = sum_{a_t(r)=mu} w x_r / sum_{a_t(r)=mu} w, where each
 *         product w*x_r is rounded to FP64 and then taken as the integer
 *         floor(w*x_r * 2^s) in 128 bits; the integer sums are exact, and each
 *         is rounded to FP64 before one IEEE division. An empty cluster keeps
 *         its centroid.
 *   early_stop: stop once a_t equals a_{t-1} (then c_{t+1} = c_t exactly).
 * Final: a_T from c_T, J_T, and idx_mu = the member of cluster mu nearest to
 * c_mu (ties to the lowest r); -1 for an empty cluster.
 *
 * near_ties counts, over all assignment passes, points whose two smallest
 * distances d1 <= d2 satisfy d2 - d1 <= 1e-12 * max(d1, hmin^2).
 * Returns 0, -1 for invalid arguments, or the number of empty clusters
 * (as a positive count) after writing all outputs.
 */
int oracle_kmeans(const double *w, int32_t nx, int32_t ny, int32_t nz, const double *cell,
                  int32_t n_mu, const int64_t *init_idx, int32_t max_iter, int32_t early_stop,
                  int64_t *idx_out, double *centroids_out, double *objective,
                  int32_t *n_iter_out, int64_t *near_ties_out, int32_t *labels_out)
{
    const int64_t n_r = (int64_t)nx * ny * nz;
    if (n_mu <= 0 || n_r <= 0 || max_iter < 0) return -1;
    const double hx = cell[0] / nx, hy = cell[1] / ny, hz = cell[2] / nz;
    double hmin = hx < hy ? hx : hy; hmin = hmin < hz ? hmin : hz;
    const double tie_floor = hmin * hmin;

    /* fixed-point scale: N_r * w_max * max(L, 1) < 2^(126 - s) */
    double wmax = 0.0;
    for (int64_t r = 0; r < n_r; ++r) {
        if (!(w[r] >= 0.0) || isinf(w[r])) return -1;
        if (w[r] > wmax) wmax = w[r];
    }
    double lmax = 1.0;
    for (int k = 0; k < 3; ++k) if (cell[k] > lmax) lmax = cell[k];
    int ew = 0, el = 0;
    if (wmax > 0.0) frexp(wmax, &ew);
    frexp(lmax, &el);
    const int s = 126 - (bits_of((uint64_t)n_r) + ew + el);
    if (s < 0) return -1;

    double *c = (double *)malloc(sizeof(double) * 3 * n_mu);
    int32_t *lab = (int32_t *)malloc(sizeof(int32_t) * n_r);
    int32_t *prev = (int32_t *)malloc(sizeof(int32_t) * n_r);
    double *d1 = (double *)malloc(sizeof(double) * n_r);
    u128 *S = (u128 *)malloc(sizeof(u128) * 4 * n_mu);
    for (int32_t m = 0; m < n_mu; ++m) {
        int64_t r = init_idx[m];
        if (r < 0 || r >= n_r) { free(c); free(lab); free(prev); free(d1); free(S); return -1; }
        int64_t ix = r / ((int64_t)ny * nz), iy = (r / nz) % ny, iz = r % nz;
        c[3 * m + 0] = (double)ix * hx;
        c[3 * m + 1] = (double)iy * hy;
        c[3 * m + 2] = (double)iz * hz;
    }

    int64_t ties = 0;
    int32_t t = 0;
    int stopped = 0;
    for (int pass = 0; pass <= max_iter; ++pass) {
        /* (i) assignment with the current centroids */
        int64_t pass_ties = 0;
#pragma omp parallel for schedule(static) reduction(+ : pass_ties)
        for (int64_t r = 0; r < n_r; ++r) {
            int64_t ix = r / ((int64_t)ny * nz), iy = (r / nz) % ny, iz = r % nz;
            double x = (double)ix * hx, y = (double)iy * hy, z = (double)iz * hz;
            double best = INFINITY, second = INFINITY;
            int32_t arg = 0;
            for (int32_t m = 0; m < n_mu; ++m) {
                double d = dist2(x, y, z, c + 3 * m);
                if (d < best) { second = best; best = d; arg = m; }
                else if (d < second) second = d;
            }
            lab[r] = arg;
            d1[r] = best;
            double fl = best > tie_floor ? best : tie_floor;
            if (n_mu > 1 && second - best <= 1e-12 * fl) pass_ties += 1;
        }
        ties += pass_ties;
        double J = 0.0;
        for (int64_t r = 0; r < n_r; ++r) J = J + w[r] * d1[r];
        if (objective) objective[pass] = J;
        if (pass == max_iter) break;
        if (early_stop && pass > 0 && memcmp(lab, prev, sizeof(int32_t) * n_r) == 0) {
            for (int p = pass + 1; p <= max_iter; ++p) if (objective) objective[p] = J;
            stopped = 1;
            break;
        }
        memcpy(prev, lab, sizeof(int32_t) * n_r);

        /* (ii) weighted centroid update, Eq. r_k, with exact integer sums */
        memset(S, 0, sizeof(u128) * 4 * n_mu);
        for (int64_t r = 0; r < n_r; ++r) {
            int64_t ix = r / ((int64_t)ny * nz), iy = (r / nz) % ny, iz = r % nz;
            double x = (double)ix * hx, y = (double)iy * hy, z = (double)iz * hz;
            u128 *q = S + 4 * (int64_t)lab[r];
            q[0] += (u128)ldexp(w[r], s);
            q[1] += (u128)ldexp(w[r] * x, s);
            q[2] += (u128)ldexp(w[r] * y, s);
            q[3] += (u128)ldexp(w[r] * z, s);
        }
        for (int32_t m = 0; m < n_mu; ++m) {
            u128 *q = S + 4 * (int64_t)m;
            if (q[0] == 0) continue;
            double sw = (double)q[0];
            c[3 * m + 0] = (double)q[1] / sw;
            c[3 * m + 1] = (double)q[2] / sw;
            c[3 * m + 2] = (double)q[3] / sw;
        }
        t += 1;
    }
    (void)stopped;

    /* snap: nearest member of each cluster, ties to the lowest r */
    int empty = 0;
    for (int32_t m = 0; m < n_mu; ++m) idx_out[m] = -1;
    double *best = (double *)malloc(sizeof(double) * n_mu);
    for (int32_t m = 0; m < n_mu; ++m) best[m] = INFINITY;
    for (int64_t r = 0; r < n_r; ++r) {
        int32_t m = lab[r];
        if (d1[r] < best[m]) { best[m] = d1[r]; idx_out[m] = r; }
    }
    for (int32_t m = 0; m < n_mu; ++m) if (idx_out[m] < 0) ++empty;
    if (centroids_out) memcpy(centroids_out, c, sizeof(double) * 3 * n_mu);
    if (labels_out) memcpy(labels_out, lab, sizeof(int32_t) * n_r);
    if (n_iter_out) *n_iter_out = t;
    if (near_ties_out) *near_ties_out = ties;
    free(best); free(c); free(lab); free(prev); free(d1); free(S);
    return empty;
}

/* the fixed-point exponent s used above, exposed for tests */
int oracle_fixed_point_scale(int64_t n_r, double wmax, const double *cell)
{
    double lmax = 1.0;
    for (int k = 0; k < 3; ++k) if (cell[k] > lmax) lmax = cell[k];
    int ew = 0, el = 0;
    if (wmax > 0.0) frexp(wmax, &ew);
    frexp(lmax, &el);
    return 126 - (bits_of((uint64_t)n_r) + ew + el);
}

/*
 * Single steps of Algorithm 1, for checking a long K-means run one step at a
 * time (a lock-step check) without repeating all its passes on the CPU.
 * They restate the same formulas as oracle_kmeans above.
 */

/* fixed-point exponent of the centroid sums for these weights (as in oracle_kmeans) */
static int kmeans_scale(const double *w, int64_t n_r, const double *cell, int *s_out)
{
    double wmax = 0.0;
    for (int64_t r = 0; r < n_r; ++r) {
        if (!(w[r] >= 0.0) || isinf(w[r])) return -1;
        if (w[r] > wmax) wmax = w[r];
    }
    *s_out = oracle_fixed_point_scale(n_r, wmax, cell);
    return *s_out < 0 ? -1 : 0;
}

/*
 * One centroid update, Eq. r_k: c_out[mu] = sum_{lab(r)=mu} w x_r / sum w, with
 * each FP64 product w*x taken as floor(w*x*2^s) in 128 bits, the integer sums
 * rounded to FP64, one IEEE division; a cluster without weight keeps
 * c_in[mu]. labels: n_r entries in [0, n_mu). Returns 0, or -1 for invalid
 * input.
 */
int oracle_kmeans_update(const double *w, int32_t nx, int32_t ny, int32_t nz, const double *cell, int32_t n_mu,
                         const int32_t *labels, const double *c_in, double *c_out)
{
    const int64_t n_r = (int64_t)nx * ny * nz;
    int s = 0;
    if (n_mu <= 0 || kmeans_scale(w, n_r, cell, &s) < 0) return -1;
    const double hx = cell[0] / nx, hy = cell[1] / ny, hz = cell[2] / nz;
    u128 *S = (u128 *)calloc((size_t)4 * n_mu, sizeof(u128));
    for (int64_t r = 0; r < n_r; ++r) {
        const int32_t m = labels[r];
        if (m < 0 || m >= n_mu) { free(S); return -1; }
        int64_t ix = r / ((int64_t)ny * nz), iy = (r / nz) % ny, iz = r % nz;
        double x = (double)ix * hx, y = (double)iy * hy, z = (double)iz * hz;
        u128 *q = S + 4 * (int64_t)m;
        q[0] += (u128)ldexp(w[r], s);
        q[1] += (u128)ldexp(w[r] * x, s);
        q[2] += (u128)ldexp(w[r] * y, s);
        q[3] += (u128)ldexp(w[r] * z, s);
    }
    for (int32_t m = 0; m < n_mu; ++m) {
        const u128 *q = S + 4 * (int64_t)m;
        if (q[0] == 0) {
            c_out[3 * m + 0] = c_in[3 * m + 0];
            c_out[3 * m + 1] = c_in[3 * m + 1];
            c_out[3 * m + 2] = c_in[3 * m + 2];
            continue;
        }
        double sw = (double)q[0];
        c_out[3 * m + 0] = (double)q[1] / sw;
        c_out[3 * m + 1] = (double)q[2] / sw;
        c_out[3 * m + 2] = (double)q[3] / sw;
    }
    free(S);
    return 0;
}

/*
 * Assignment, Eq. opt (second form), of the listed grid points only:
 * labels[i] = argmin_mu |x_{points[i]} - c_mu|^2 (lowest mu on ties) and
 * dist[i] its squared distance (nullable). Brute force over all centroids.
 */
int oracle_kmeans_assign(int32_t nx, int32_t ny, int32_t nz, const double *cell, int32_t n_mu,
                         const double *centroids, const int64_t *points, int64_t count, int32_t *labels,
                         double *dist)
{
    const int64_t n_r = (int64_t)nx * ny * nz;
    if (n_mu <= 0) return -1;
    const double hx = cell[0] / nx, hy = cell[1] / ny, hz = cell[2] / nz;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < count; ++i) {
        const int64_t r = points[i];
        if (r < 0 || r >= n_r) { bad |= 1; continue; }
        int64_t ix = r / ((int64_t)ny * nz), iy = (r / nz) % ny, iz = r % nz;
        double x = (double)ix * hx, y = (double)iy * hy, z = (double)iz * hz;
        double best = INFINITY;
        int32_t arg = 0;
        for (int32_t m = 0; m < n_mu; ++m) {
            double d = dist2(x, y, z, centroids + 3 * m);
            if (d < best) { best = d; arg = m; }
        }
        labels[i] = arg;
        if (dist) dist[i] = best;
    }
    return bad ? -1 : 0;
}

/*
 * Snap, the last step of Algorithm 1 (reading: each centroid's nearest member):
 * idx[mu] = the grid point r with labels[r] = mu nearest to c_mu, ties to the
 * lowest r, or -1 when the cluster has no member. Returns the number of empty
 * clusters, or -1 for invalid labels.
 */
int oracle_kmeans_snap(int32_t nx, int32_t ny, int32_t nz, const double *cell, int32_t n_mu,
                       const double *centroids, const int32_t *labels, int64_t *idx)
{
    const int64_t n_r = (int64_t)nx * ny * nz;
    const double hx = cell[0] / nx, hy = cell[1] / ny, hz = cell[2] / nz;
    double *best = (double *)malloc(sizeof(double) * n_mu);
    for (int32_t m = 0; m < n_mu; ++m) { best[m] = INFINITY; idx[m] = -1; }
    for (int64_t r = 0; r < n_r; ++r) {
        const int32_t m = labels[r];
        if (m < 0 || m >= n_mu) { free(best); return -1; }
        int64_t ix = r / ((int64_t)ny * nz), iy = (r / nz) % ny, iz = r % nz;
        double d = dist2((double)ix * hx, (double)iy * hy, (double)iz * hz, centroids + 3 * m);
        if (d < best[m]) { best[m] = d; idx[m] = r; }
    }
    int empty = 0;
    for (int32_t m = 0; m < n_mu; ++m) if (idx[m] < 0) ++empty;
    free(best);
    return empty;
}
