/*
 * FP64 CPU oracle for the DPD step loop of arxiv 1804.06205 (CAMUS).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the correctness reference for the
 * CUDA engine: only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header or constant generator with
 * the CUDA path.
 *
 * What it computes (paper section "Summary of DPD simulation" and Fig. 1):
 *   eq. 3   f_i = sum_{j != i} (F^C_ij + F^D_ij + F^R_ij + F^S_ij)
 *   eq. 4   F^C = a_ij (1 - r) e_ij for r < r_c = 1 (soft repulsion)
 *   F^D, F^R  Groot-Warren forms (the paper names them only): w^R = 1 - r,
 *           w^D = (w^R)^2, sigma^2 = 2 gamma kT, random term theta/sqrt(dt)
 *   eqs. 6-8  bonded terms: harmonic, the paper's modified Morse, and a
 *           standard Morse kind
 *   Fig. 1  Groot's modified velocity-Verlet with lambda
 * The pair sum is the plain definition: every j != i, minimum image, no
 * cell list ("brute" mode).  A cell-list mode (the CAMUS design, section
 * "Design concept of CAMUS") gives the same pair set and exists to time the
 * CPU baseline on large systems.
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *   - theta_ij: Philox4x32-10 (Salmon et al., SC'11) with counter
 *     (min id, max id, s_lo, s_hi) and key (seed_lo, seed_hi); uniforms
 *     u = (2*(x>>9)+1) * 2^-24; Gaussian by Box-Muller from outputs 0 and 1,
 *     theta = sqrt(-2 ln u0) cos(2 pi u1); optional uniform noise
 *     theta = sqrt(3) (2 u0 - 1).
 *   - bond kind 1 (eq. 6): restoring spring derived from U = k/2 (r - r0)^2.
 *   - bond kind 2 (eq. 7 with the alpha factor of Fig. 3a): magnitude
 *     2 k alpha e (1 - e), e = exp(-alpha |r - r0|), pointing from i towards
 *     j on both sides of r0; energy k (1 - e)^2.
 *   - bond kind 3: standard Morse U = D[(1 - exp(-alpha (r - r0)))^2 - 1].
 *   - mass 1 for all beads; pairs at r == 0 contribute nothing.
 */
#ifndef DPD_ORACLE_H
#define DPD_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double L[3];            /* periodic box edges */
    int64_t n;              /* beads */
    int32_t ntypes;
    const int32_t *types;   /* [n] */
    const double *a;        /* [ntypes*ntypes] eq. 4 repulsion a_ij */
    double gamma, kT, dt, lambda;
    uint64_t seed;          /* Philox key */
    int32_t noise;          /* 0 = Gaussian (Box-Muller), 1 = uniform */
    int64_t nbonds;         /* bonded records, eqs. 6-8 */
    const int32_t *bi, *bj, *bkind;
    const double *br0, *bk, *balpha;
} orc_sys;

/* Virial and energy sums of one force evaluation. */
typedef struct {
    double wc;   /* sum over unique pairs of d_ij . F^C_ij */
    double wb;   /* sum over bond records of d_ij . F^S_ij */
    double ep;   /* sum over unique pairs of a w^2 / 2 */
    double eb;   /* bond energies (Fig. 3a accumulation) */
} orc_terms;

/* Philox4x32 with 10 rounds, from the published definition. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Uniform in (0,1) from one 32-bit word: (2*(x>>9)+1) * 2^-24. */
double orc_u01(uint32_t x);
/* Pair noise theta_ij for evaluation counter s (symmetric in i, j). */
double orc_theta(uint64_t seed, int64_t i, int64_t j, int64_t s, int32_t noise);

/* Force on bead i from bead j alone (pair terms of eq. 3), 0 if r >= 1. */
void orc_pair_force_one(const orc_sys *sys, const double *pos, const double *vt,
                        int64_t i, int64_t j, int64_t s, double F[3]);

/* Pair forces f[n*3] (overwritten).  mode 0 = brute force, 1 = cell list. */
int orc_pair_forces(const orc_sys *sys, const double *pos, const double *vt,
                    int64_t s, int32_t mode, double *f, orc_terms *t);
/* Pair forces on the m beads idx[] only (plain definition, all j != i);
 * f[m*3] overwritten.  For spot checks of very large systems. */
int orc_pair_forces_subset(const orc_sys *sys, const double *pos, const double *vt, int64_t s,
                           const int64_t *idx, int64_t m, double *f);
/* Bond forces added into f[n*3]. */
int orc_pair_forces_ids(const orc_sys *sys, int64_t n, const double *pos, const double *vt,
                        const int32_t *types, const int64_t *ids, int64_t m, int64_t s,
                        double *f);
int orc_bond_forces(const orc_sys *sys, const double *pos, double *f, orc_terms *t);
/* Force and energy of one bond record on bead i (F_j = -F_i). */
void orc_bond_one(int32_t kind, double r0, double k, double alpha, const double d[3],
                  double Fi[3], double *energy);

/* Periodic wrap into [0, L). */
void orc_wrap(const orc_sys *sys, double *pos);
/* Cell geometry: n_c = floor(L), inv_h = n_c / L. */
void orc_cell_dims(const orc_sys *sys, int64_t nc[3], double inv_h[3]);
/* Cell key per bead: (cz*ny + cy)*nx + cx, c = min(floor(x*inv_h), n_c-1). */
void orc_cell_keys(const orc_sys *sys, const double *pos, uint32_t *key);
/* Canonical (cell, id) order: order[slot] = id, cell_start[ncells+1]. */
void orc_cell_sort(const orc_sys *sys, const uint32_t *key, int64_t *order, int64_t *cell_start);

/* Full force f = pair + bond at (pos, vt), counter s. */
int orc_forces(const orc_sys *sys, const double *pos, const double *vt, int64_t s,
               int32_t mode, double *f, orc_terms *t);

/* Fig. 1 loop.  On entry f holds the force at (pos, vel); *step the counter
 * of that evaluation.  Advances nsteps steps.  If samples != NULL, every
 * sample_every steps 12 doubles are appended (see orc_observables). */
int orc_run(const orc_sys *sys, double *pos, double *vel, double *f, int64_t *step,
            int64_t nsteps, int32_t mode, int32_t sample_every, double *samples,
            orc_terms *last);

/* out[12]: step, px, py, pz, kT, p_total, p_ideal, p_cons, p_bond, e_pair,
 * e_bond, sum v^2.  kT = sum v^2 / (3n - 3); p = (sum v^2 + W_C + W_B)/(3V). */
void orc_observables(const orc_sys *sys, const double *vel, const orc_terms *t,
                     int64_t step, double out[12]);

/* Pair-distance histogram, bins of width rmax/nbins, unique pairs, minimum
 * image.  counts[nbins] (overwritten). */
void orc_gr_counts(const orc_sys *sys, const double *pos, double rmax, int32_t nbins,
                   uint64_t *counts);

/* Threads OpenMP will use. */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
