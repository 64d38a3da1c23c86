/*
 * FP64 CPU oracle for the DPD step loop of arxiv 1804.06205 (CAMUS).
 * TEST INFRASTRUCTURE ONLY -- see dpd_oracle.h for what it computes, which
 * passages of the paper each part follows and the readings taken.
 *
 * Built with -ffp-contract=off so that no multiply-add is fused: the cell
 * keys and the wrap must come out of exactly the IEEE operations written here.
 */
#include "dpd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  One round: two 32x32->64 products of counter   */
/* words 0 and 2 with the published multipliers; the high halves are mixed  */
/* with the other two counter words and the round key, the low halves pass  */
/* through; the key is advanced by the published Weyl increments between     */
/* rounds.                                                                   */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_u01(uint32_t x) {
    /* odd multiple of 2^-24: never 0 or 1, exact in binary32 and binary64 */
    return (double)(2u * (x >> 9) + 1u) * ldexp(1.0, -24);
}

double orc_theta(uint64_t seed, int64_t i, int64_t j, int64_t s, int32_t noise) {
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    uint32_t ctr[4] = {(uint32_t)lo, (uint32_t)hi, (uint32_t)((uint64_t)s & 0xffffffffu),
                       (uint32_t)((uint64_t)s >> 32)};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    double u0 = orc_u01(out[0]);
    double u1 = orc_u01(out[1]);
    if (noise == 1) return sqrt(3.0) * (2.0 * u0 - 1.0);
    const double two_pi = 6.283185307179586476925286766559;
    return sqrt(-2.0 * log(u0)) * cos(two_pi * u1);
}

/* ------------------------------------------------------------------------ */
/* Pair terms of eq. 3 for one ordered pair (force on i).                    */
/* ------------------------------------------------------------------------ */
static inline double min_image(double d, double L) { return d - L * nearbyint(d / L); }

/* The pair terms for bead i (position pi, predicted velocity vi, type ti,
 * id idi) and bead j: returns 1 and fills F (force on i), the conservative
 * virial d.F^C and the pair energy if 0 < r < 1, else returns 0. */
static int pair_terms(const orc_sys *sys, const double *pi, const double *pj, const double *vi,
                      const double *vj, int32_t ti, int32_t tj, int64_t idi, int64_t idj,
                      int64_t s, double F[3], double *wc, double *ep) {
    double d[3];
    for (int k = 0; k < 3; ++k) d[k] = min_image(pi[k] - pj[k], sys->L[k]);
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 >= 1.0 || r2 == 0.0) return 0;
    double r = sqrt(r2);
    double e[3] = {d[0] / r, d[1] / r, d[2] / r};
    double w = 1.0 - r;                                      /* w^R(r) */
    double a = sys->a[ti * sys->ntypes + tj];
    double ev = e[0] * (vi[0] - vj[0]) + e[1] * (vi[1] - vj[1]) + e[2] * (vi[2] - vj[2]);
    double sigma = sqrt(2.0 * sys->gamma * sys->kT);
    double theta = orc_theta(sys->seed, idi, idj, s, sys->noise);
    double fc = a * w;                                       /* eq. 4 */
    double fd = -sys->gamma * w * w * ev;                    /* w^D = (w^R)^2 */
    double fr = sigma * w * theta / sqrt(sys->dt);           /* random term */
    double mag = fc + fd + fr;
    F[0] = mag * e[0];
    F[1] = mag * e[1];
    F[2] = mag * e[2];
    *wc = r * fc;
    *ep = 0.5 * a * w * w;
    return 1;
}

/* Bead index = bead id: the system's own arrays. */
static int pair_core(const orc_sys *sys, const double *pos, const double *vt, int64_t i,
                     int64_t j, int64_t s, double F[3], double *wc, double *ep) {
    return pair_terms(sys, pos + 3 * i, pos + 3 * j, vt + 3 * i, vt + 3 * j, sys->types[i],
                      sys->types[j], i, j, s, F, wc, ep);
}

void orc_pair_force_one(const orc_sys *sys, const double *pos, const double *vt, int64_t i,
                        int64_t j, int64_t s, double F[3]) {
    double wc, ep;
    F[0] = F[1] = F[2] = 0.0;
    if (i == j) return;
    if (!pair_core(sys, pos, vt, i, j, s, F, &wc, &ep)) F[0] = F[1] = F[2] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Cells (used by the cell-list mode and for the canonical sort order).      */
/* ------------------------------------------------------------------------ */
void orc_cell_dims(const orc_sys *sys, int64_t nc[3], double inv_h[3]) {
    for (int k = 0; k < 3; ++k) {
        nc[k] = (int64_t)floor(sys->L[k]);     /* cell edge h = L/n_c >= r_c = 1 */
        if (nc[k] < 1) nc[k] = 1;
        inv_h[k] = (double)nc[k] / sys->L[k];
    }
}

static double wrap_one(double x, double L) {
    double y = x - L * floor(x / L);
    if (y < 0.0) y += L;
    if (y >= L) y -= L;
    return y;
}

void orc_wrap(const orc_sys *sys, double *pos) {
    for (int64_t i = 0; i < sys->n; ++i)
        for (int k = 0; k < 3; ++k) pos[3 * i + k] = wrap_one(pos[3 * i + k], sys->L[k]);
}

void orc_cell_keys(const orc_sys *sys, const double *pos, uint32_t *key) {
    int64_t nc[3];
    double inv_h[3];
    orc_cell_dims(sys, nc, inv_h);
    for (int64_t i = 0; i < sys->n; ++i) {
        int64_t c[3];
        for (int k = 0; k < 3; ++k) {
            double q = floor(pos[3 * i + k] * inv_h[k]);
            int64_t ck = (int64_t)q;
            if (ck < 0) ck = 0;
            if (ck > nc[k] - 1) ck = nc[k] - 1;
            c[k] = ck;
        }
        key[i] = (uint32_t)((c[2] * nc[1] + c[1]) * nc[0] + c[0]);
    }
}

void orc_cell_sort(const orc_sys *sys, const uint32_t *key, int64_t *order, int64_t *cell_start) {
    int64_t nc[3];
    double inv_h[3];
    orc_cell_dims(sys, nc, inv_h);
    int64_t ncell = nc[0] * nc[1] * nc[2];
    memset(cell_start, 0, sizeof(int64_t) * (size_t)(ncell + 1));
    for (int64_t i = 0; i < sys->n; ++i) cell_start[key[i] + 1]++;
    for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    memcpy(fill, cell_start, sizeof(int64_t) * (size_t)ncell);
    /* stable counting sort over ids in ascending order: (cell, id) order */
    for (int64_t i = 0; i < sys->n; ++i) order[fill[key[i]]++] = i;
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Pair forces.                                                              */
/* ------------------------------------------------------------------------ */
int orc_pair_forces(const orc_sys *sys, const double *pos, const double *vt, int64_t s,
                    int32_t mode, double *f, orc_terms *t) {
    const int64_t n = sys->n;
    double *wci = (double *)calloc((size_t)n, sizeof(double));
    double *epi = (double *)calloc((size_t)n, sizeof(double));
    if (!wci || !epi) { free(wci); free(epi); return -1; }
    int rc = 0;
    if (mode == 0) {
        /* plain definition: for every i, all j != i in ascending order */
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t i = 0; i < n; ++i) {
            double fi[3] = {0, 0, 0}, wsum = 0, esum = 0;
            for (int64_t j = 0; j < n; ++j) {
                if (j == i) continue;
                double F[3], wc, ep;
                if (pair_core(sys, pos, vt, i, j, s, F, &wc, &ep)) {
                    fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
                    wsum += wc; esum += ep;
                }
            }
            f[3 * i] = fi[0]; f[3 * i + 1] = fi[1]; f[3 * i + 2] = fi[2];
            wci[i] = wsum; epi[i] = esum;
        }
    } else {
        /* cell list with edge h >= r_c, rebuilt from scratch (the CAMUS design) */
        int64_t nc[3];
        double inv_h[3];
        orc_cell_dims(sys, nc, inv_h);
        if (nc[0] < 3 || nc[1] < 3 || nc[2] < 3) { free(wci); free(epi); return -2; }
        int64_t ncell = nc[0] * nc[1] * nc[2];
        double *wp = (double *)malloc(sizeof(double) * (size_t)(3 * n));
        uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
        int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncell + 1));
        if (!wp || !key || !order || !start) {
            free(wp); free(key); free(order); free(start); free(wci); free(epi);
            return -1;
        }
        memcpy(wp, pos, sizeof(double) * (size_t)(3 * n));
        orc_wrap(sys, wp);
        orc_cell_keys(sys, wp, key);
        orc_cell_sort(sys, key, order, start);
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = key[i];
            int64_t cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / (nc[0] * nc[1]);
            double fi[3] = {0, 0, 0}, wsum = 0, esum = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int64_t x = (cx + dx + nc[0]) % nc[0];
                        int64_t y = (cy + dy + nc[1]) % nc[1];
                        int64_t z = (cz + dz + nc[2]) % nc[2];
                        int64_t cc = (z * nc[1] + y) * nc[0] + x;
                        for (int64_t q = start[cc]; q < start[cc + 1]; ++q) {
                            int64_t j = order[q];
                            if (j == i) continue;
                            double F[3], wc, ep;
                            if (pair_core(sys, pos, vt, i, j, s, F, &wc, &ep)) {
                                fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
                                wsum += wc; esum += ep;
                            }
                        }
                    }
            f[3 * i] = fi[0]; f[3 * i + 1] = fi[1]; f[3 * i + 2] = fi[2];
            wci[i] = wsum; epi[i] = esum;
        }
        free(wp); free(key); free(order); free(start);
    }
    if (t) {
        double ws = 0, es = 0;
        for (int64_t i = 0; i < n; ++i) { ws += wci[i]; es += epi[i]; }
        t->wc = 0.5 * ws;  /* every unique pair was visited from both ends */
        t->ep = 0.5 * es;
    }
    free(wci);
    free(epi);
    return rc;
}

int orc_pair_forces_subset(const orc_sys *sys, const double *pos, const double *vt, int64_t s,
                           const int64_t *idx, int64_t m, double *f) {
    for (int64_t q = 0; q < m; ++q)
        if (idx[q] < 0 || idx[q] >= sys->n) return -3;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx[q];
        double fi[3] = {0, 0, 0};
        for (int64_t j = 0; j < sys->n; ++j) {
            if (j == i) continue;
            double F[3], wc, ep;
            if (pair_core(sys, pos, vt, i, j, s, F, &wc, &ep)) {
                fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
            }
        }
        f[3 * q] = fi[0]; f[3 * q + 1] = fi[1]; f[3 * q + 2] = fi[2];
    }
    return 0;
}

/* Pair forces on the first m of n beads given by their own arrays (positions,
 * predicted velocities, types and global ids), summed over all n beads j != q
 * in the order given: the same terms as orc_pair_forces for any subset of a
 * system that holds every bead within r_c of the targets (a domain and its
 * ghosts). */
int orc_pair_forces_ids(const orc_sys *sys, int64_t n, const double *pos, const double *vt,
                        const int32_t *types, const int64_t *ids, int64_t m, int64_t s,
                        double *f) {
    if (m < 0 || m > n) return -3;
    for (int64_t q = 0; q < n; ++q)
        if (types[q] < 0 || types[q] >= sys->ntypes) return -3;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; ++q) {
        double fi[3] = {0, 0, 0};
        for (int64_t j = 0; j < n; ++j) {
            if (j == q) continue;
            double F[3], wc, ep;
            if (pair_terms(sys, pos + 3 * q, pos + 3 * j, vt + 3 * q, vt + 3 * j, types[q],
                           types[j], ids[q], ids[j], s, F, &wc, &ep)) {
                fi[0] += F[0]; fi[1] += F[1]; fi[2] += F[2];
            }
        }
        f[3 * q] = fi[0]; f[3 * q + 1] = fi[1]; f[3 * q + 2] = fi[2];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Bonded terms, eqs. 6-8 and Fig. 3a.                                       */
/* ------------------------------------------------------------------------ */
void orc_bond_one(int32_t kind, double r0, double k, double alpha, const double d[3],
                  double Fi[3], double *energy) {
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double r = sqrt(r2);
    double coef = 0.0;  /* Fi = coef * d */
    double U = 0.0;
    if (kind == 1) {
        /* harmonic, U = k/2 (r - r0)^2, restoring */
        if (r0 == 0.0) {
            coef = -k;
            U = 0.5 * k * r2;
        } else {
            U = 0.5 * k * (r - r0) * (r - r0);
            if (r > 0.0) coef = -k * (r - r0) / r;
        }
    } else if (kind == 2) {
        /* modified Morse of eq. 7 with the alpha of Fig. 3a: the same
         * direction (towards the partner) on both sides of r0 */
        double e = exp(-alpha * fabs(r - r0));
        U = k * (1.0 - e) * (1.0 - e);
        if (r > 0.0) coef = -2.0 * k * alpha * e * (1.0 - e) / r;
    } else if (kind == 3) {
        /* standard Morse, U = D[(1 - e^{-alpha (r - r0)})^2 - 1] */
        double x = exp(-alpha * (r - r0));
        U = k * ((1.0 - x) * (1.0 - x) - 1.0);
        double dUdr = 2.0 * k * alpha * x * (1.0 - x);
        if (r > 0.0) coef = -dUdr / r;
    }
    Fi[0] = coef * d[0];
    Fi[1] = coef * d[1];
    Fi[2] = coef * d[2];
    *energy = U;
}

int orc_bond_forces(const orc_sys *sys, const double *pos, double *f, orc_terms *t) {
    double wb = 0, eb = 0;
    for (int64_t b = 0; b < sys->nbonds; ++b) {
        int64_t i = sys->bi[b], j = sys->bj[b];
        if (i < 0 || j < 0 || i >= sys->n || j >= sys->n) return -3;
        double d[3], Fi[3], U;
        for (int k = 0; k < 3; ++k) d[k] = min_image(pos[3 * i + k] - pos[3 * j + k], sys->L[k]);
        orc_bond_one(sys->bkind[b], sys->br0[b], sys->bk[b], sys->balpha[b], d, Fi, &U);
        for (int k = 0; k < 3; ++k) {
            f[3 * i + k] += Fi[k];
            f[3 * j + k] -= Fi[k];
        }
        wb += d[0] * Fi[0] + d[1] * Fi[1] + d[2] * Fi[2];
        eb += U;
    }
    if (t) { t->wb = wb; t->eb = eb; }
    return 0;
}

int orc_forces(const orc_sys *sys, const double *pos, const double *vt, int64_t s,
               int32_t mode, double *f, orc_terms *t) {
    orc_terms tt = {0, 0, 0, 0};
    int rc = orc_pair_forces(sys, pos, vt, s, mode, f, &tt);
    if (rc) return rc;
    rc = orc_bond_forces(sys, pos, f, &tt);
    if (t) *t = tt;
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Observables.                                                              */
/* ------------------------------------------------------------------------ */
void orc_observables(const orc_sys *sys, const double *vel, const orc_terms *t, int64_t step,
                     double out[12]) {
    double p[3] = {0, 0, 0}, v2 = 0;
    for (int64_t i = 0; i < sys->n; ++i)
        for (int k = 0; k < 3; ++k) {
            double v = vel[3 * i + k];
            p[k] += v;
            v2 += v * v;
        }
    double V = sys->L[0] * sys->L[1] * sys->L[2];
    out[0] = (double)step;
    out[1] = p[0]; out[2] = p[1]; out[3] = p[2];
    out[4] = v2 / (3.0 * (double)sys->n - 3.0);
    out[6] = v2 / (3.0 * V);
    out[7] = t ? t->wc / (3.0 * V) : 0.0;
    out[8] = t ? t->wb / (3.0 * V) : 0.0;
    out[5] = out[6] + out[7] + out[8];
    out[9] = t ? t->ep : 0.0;
    out[10] = t ? t->eb : 0.0;
    out[11] = v2;
}

/* ------------------------------------------------------------------------ */
/* Fig. 1: Groot's modified velocity-Verlet.                                 */
/* ------------------------------------------------------------------------ */
int orc_run(const orc_sys *sys, double *pos, double *vel, double *f, int64_t *step,
            int64_t nsteps, int32_t mode, int32_t sample_every, double *samples,
            orc_terms *last) {
    const int64_t n = sys->n;
    const double dt = sys->dt, lam = sys->lambda;
    double *vt = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    double *f2 = (double *)malloc(sizeof(double) * (size_t)(3 * n));
    if (!vt || !f2) { free(vt); free(f2); return -1; }
    int64_t ns = 0;
    orc_terms t = {0, 0, 0, 0};
    for (int64_t it = 0; it < nsteps; ++it) {
        int64_t s = *step + 1;
        /* 1. position update and boundary check */
        for (int64_t q = 0; q < 3 * n; ++q) pos[q] = pos[q] + dt * vel[q] + 0.5 * dt * dt * f[q];
        orc_wrap(sys, pos);
        /* 2. velocity predictor */
        for (int64_t q = 0; q < 3 * n; ++q) vt[q] = vel[q] + lam * dt * f[q];
        /* 3.-4. cell division and force (cell division is internal to mode 1) */
        int rc = orc_forces(sys, pos, vt, s, mode, f2, &t);
        if (rc) { free(vt); free(f2); return rc; }
        /* 5. velocity update */
        for (int64_t q = 0; q < 3 * n; ++q) {
            vel[q] = vel[q] + 0.5 * dt * (f[q] + f2[q]);
            f[q] = f2[q];
        }
        *step = s;
        if (samples && sample_every > 0 && (s % sample_every) == 0) {
            orc_observables(sys, vel, &t, s, samples + 12 * ns);
            ++ns;
        }
    }
    if (last) *last = t;
    free(vt);
    free(f2);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* g(r) pair-distance histogram.                                             */
/* ------------------------------------------------------------------------ */
void orc_gr_counts(const orc_sys *sys, const double *pos, double rmax, int32_t nbins,
                   uint64_t *counts) {
    memset(counts, 0, sizeof(uint64_t) * (size_t)nbins);
    double dr = rmax / (double)nbins;
    for (int64_t i = 0; i < sys->n; ++i)
        for (int64_t j = i + 1; j < sys->n; ++j) {
            double d[3];
            for (int k = 0; k < 3; ++k)
                d[k] = min_image(pos[3 * i + k] - pos[3 * j + k], sys->L[k]);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (r < rmax) {
                int64_t b = (int64_t)floor(r / dr);
                if (b < nbins) counts[b]++;
            }
        }
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
