/*
 * hemeoracle.c -- FP64 CPU oracle for the sparse D3Q19 LBGK hot path of
 * "Towards Blood Flow in the Virtual Human: Efficient Self-Coupling of HemeLB"
 * (arXiv 2010.04144).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is loaded by the test suite, the
 * package smoke check and the CPU-baseline leg of the benchmark, nowhere else.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * It is plain and slow on purpose: double precision, loops in the order the
 * method states them, compiled with -ffp-contract=off so each product and sum
 * is rounded as written.  OpenMP, when present, only splits the independent
 * per-site loops across threads; it changes no arithmetic.  Reductions run
 * sequentially in canonical site order.
 *
 * What the paper fixes (Section 2): D3Q19 velocity set, single-relaxation-time
 * (LBGK) collision, rigid walls, pressure and velocity boundary conditions at
 * inlets/outlets, Newtonian fluid with nu = (tau - 1/2)/3 in lattice units
 * (Section 3.3, stability rules).  What it leaves open is filled by these
 * readings (each repeated where it is used):
 *   R1 velocity ordering and weights: textbook D3Q19, rest first, then the 6
 *      axis directions (+x,-x,+y,-y,+z,-z), then the 12 diagonals in
 *      opposite pairs; weights 1/3, 1/18, 1/36.
 *   R2 canonical site order: ascending 3-D Morton key, x in the lowest bit.
 *   R3 a non-fluid lattice point q belongs to iolet k when it lies beyond the
 *      iolet's cut plane by at most 2 lattice units and within the iolet
 *      radius of its axis; exact integer test on 2^-10 fixed point; the
 *      lowest k wins; everything else is wall.
 *   R4 state is stored as the deviation f~ = f - w from the lattice weights;
 *      equilibrium is the standard second-order one,
 *      f~eq_i = w_i [drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u.u)].
 *   R5 walls: half-way bounce-back.  Pressure iolets: anti-bounce-back
 *      f~_i = -f~*_opp + 2 w_i drho_k.  Velocity iolets: moving-wall
 *      bounce-back f~_i = f~*_opp + 6 w_i (c_i . u_w), rho0 = 1, with u_w the
 *      inward profile velocity at the link midpoint.
 *   R6 time: step t (t = 1, 2, ...) streams the post-collision state F_{t-1}
 *      into G_t using the boundary values of time t, then collides G_t into
 *      F_t.  Iolet means M_t are taken over the moments of G_t.
 *   R7 body force (Section 3, reverse coupling direction, which names the
 *      forcing of Guo, Zheng and Shi, Phys. Rev. E 65, 046308, 2002): at a
 *      site with force density F the velocity is u = (j + F/2)/rho, the
 *      equilibrium is taken at that u, and the collision adds
 *      (1 - 1/(2 tau)) w_i [3 (c_i - u) + 9 (c_i . u) c_i] . F.  Collision
 *      then conserves mass and raises the momentum by exactly F.  Sites
 *      without a force run the unforced update bit for bit.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ERR_RANGE (-1)
#define OR_ERR_DUPLICATE (-2)
#define OR_ERR_ALLOC (-3)

#define OR_PRESSURE 0
#define OR_VELOCITY 1
#define OR_PLUG 0
#define OR_PARABOLIC 1

/* R1: the D3Q19 velocity set. */
static const int CV[19][3] = {
    {0, 0, 0},
    {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},   {0, -1, 0}, {0, 0, 1},   {0, 0, -1},
    {1, 1, 0},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1},
    {1, 0, -1},  {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static double weight(int i) {
    int s = abs(CV[i][0]) + abs(CV[i][1]) + abs(CV[i][2]);
    if (s == 0) return 1.0 / 3.0;
    if (s == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* Opposite direction, found by search so that it follows from the table. */
static int opposite(int i) {
    for (int j = 0; j < 19; ++j)
        if (CV[j][0] == -CV[i][0] && CV[j][1] == -CV[i][1] && CV[j][2] == -CV[i][2]) return j;
    return -1;
}

/* Iolet descriptor (fixed point: 1 lattice unit = 1024). */
typedef struct {
    int32_t kind;     /* OR_PRESSURE / OR_VELOCITY */
    int32_t profile;  /* OR_PLUG / OR_PARABOLIC (velocity iolets) */
    int32_t pulse;    /* time modulation, applied by the caller */
    int32_t pad;
    double value;
    double period;
    int64_t centre[3];
    int64_t axis[3];  /* outward, any length */
    int64_t radius;
} or_iolet;

void or_lattice(int32_t *c_out, double *w_out, int32_t *opp_out) {
    for (int i = 0; i < 19; ++i) {
        for (int d = 0; d < 3; ++d) c_out[3 * i + d] = CV[i][d];
        w_out[i] = weight(i);
        opp_out[i] = opposite(i);
    }
}

/* R4: the equilibrium in deviation form. */
static void equilibrium(double drho, const double u[3], double feq[19]) {
    double rho = 1.0 + drho;
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < 19; ++i) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = weight(i) * (drho + rho * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
    }
}

void or_feq(double drho, double ux, double uy, double uz, double *out) {
    double u[3] = {ux, uy, uz};
    equilibrium(drho, u, out);
}

/* R2: 3-D Morton key, 21 bits per axis, x in bit 0, y in bit 1, z in bit 2. */
uint64_t or_morton(int32_t x, int32_t y, int32_t z) {
    uint64_t key = 0;
    for (int b = 0; b < 21; ++b) {
        key |= (uint64_t)((x >> b) & 1) << (3 * b);
        key |= (uint64_t)((y >> b) & 1) << (3 * b + 1);
        key |= (uint64_t)((z >> b) & 1) << (3 * b + 2);
    }
    return key;
}

#define COORD_LIMIT (1 << 21)

static int iolet_in_range(const or_iolet *io) {
    const int64_t lim = (int64_t)1 << 31;
    for (int d = 0; d < 3; ++d) {
        if (io->centre[d] < -lim || io->centre[d] > lim) return 0;
        if (io->axis[d] < -(1 << 20) || io->axis[d] > (1 << 20)) return 0;
    }
    if (io->axis[0] == 0 && io->axis[1] == 0 && io->axis[2] == 0) return 0;
    if (io->radius < 0 || io->radius > lim) return 0;
    return 1;
}

/* R3: does lattice point q lie in the opening of iolet io?  Exact integers. */
static int in_iolet(const int64_t q[3], const or_iolet *io) {
    __int128 d[3], a[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = (__int128)q[k] * 1024 - io->centre[k];
        a[k] = io->axis[k];
    }
    __int128 dot = d[0] * a[0] + d[1] * a[1] + d[2] * a[2];
    if (dot <= 0) return 0; /* not beyond the cut plane */
    __int128 aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    __int128 depth = 2 * 1024;
    if (dot * dot > depth * depth * aa) return 0; /* more than 2 units beyond it */
    __int128 x0 = d[1] * a[2] - d[2] * a[1];
    __int128 x1 = d[2] * a[0] - d[0] * a[2];
    __int128 x2 = d[0] * a[1] - d[1] * a[0];
    __int128 cc = x0 * x0 + x1 * x1 + x2 * x2; /* |d x a|^2 = dist^2 |a|^2 */
    __int128 r = io->radius;
    return cc <= r * r * aa;
}

int or_classify(int32_t x, int32_t y, int32_t z, const or_iolet *io, int32_t nio) {
    int64_t q[3] = {x, y, z};
    for (int k = 0; k < nio; ++k)
        if (in_iolet(q, &io[k])) return -(2 + k);
    return -1;
}

typedef struct {
    uint64_t key;
    int64_t idx;
} keyidx;

static int cmp_keyidx(const void *a, const void *b) {
    const keyidx *p = (const keyidx *)a, *q = (const keyidx *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return 0;
}

static int64_t find_key(const uint64_t *keys, int64_t n, uint64_t k) {
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (keys[mid] == k) return mid;
        if (keys[mid] < k) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* One row of the neighbour table for the site at (x, y, z): entry i-1 is the
 * canonical index of the fluid site at x - c_i (the pull source), else the
 * iolet code -(2+k), else -1 (wall). */
static void nbr_row(const uint64_t *keys, int64_t n, const int32_t p[3], const or_iolet *io,
                    int32_t nio, int32_t out[18]) {
    for (int i = 1; i < 19; ++i) {
        int64_t q[3] = {(int64_t)p[0] - CV[i][0], (int64_t)p[1] - CV[i][1],
                        (int64_t)p[2] - CV[i][2]};
        int64_t found = -1;
        if (q[0] >= 0 && q[1] >= 0 && q[2] >= 0 && q[0] < COORD_LIMIT && q[1] < COORD_LIMIT &&
            q[2] < COORD_LIMIT)
            found = find_key(keys, n, or_morton((int32_t)q[0], (int32_t)q[1], (int32_t)q[2]));
        if (found >= 0) {
            out[i - 1] = (int32_t)found;
        } else {
            int32_t code = -1;
            for (int k = 0; k < nio; ++k)
                if (in_iolet(q, &io[k])) {
                    code = -(2 + k);
                    break;
                }
            out[i - 1] = code;
        }
    }
}

/* Canonical ordering (R2) and, if nbr != NULL, the neighbour table nbr[18][n].
 * perm[s] = input index of canonical site s; xyz_sorted = coordinates in
 * canonical order; keys_sorted (optional) = their Morton keys. */
int or_build(const int32_t *xyz, int64_t n, const or_iolet *io, int32_t nio, int64_t *perm,
             int32_t *xyz_sorted, uint64_t *keys_sorted, int32_t *nbr) {
    for (int k = 0; k < nio; ++k)
        if (!iolet_in_range(&io[k])) return OR_ERR_RANGE;
    for (int64_t s = 0; s < n; ++s)
        for (int d = 0; d < 3; ++d)
            if (xyz[3 * s + d] < 0 || xyz[3 * s + d] >= COORD_LIMIT) return OR_ERR_RANGE;
    keyidx *ki = (keyidx *)malloc(sizeof(keyidx) * (size_t)(n > 0 ? n : 1));
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    if (!ki || !keys) {
        free(ki);
        free(keys);
        return OR_ERR_ALLOC;
    }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        ki[s].key = or_morton(xyz[3 * s], xyz[3 * s + 1], xyz[3 * s + 2]);
        ki[s].idx = s;
    }
    qsort(ki, (size_t)n, sizeof(keyidx), cmp_keyidx);
    int rc = OR_OK;
    for (int64_t s = 0; s < n; ++s) {
        if (s > 0 && ki[s].key == ki[s - 1].key) rc = OR_ERR_DUPLICATE;
        keys[s] = ki[s].key;
        perm[s] = ki[s].idx;
        for (int d = 0; d < 3; ++d) xyz_sorted[3 * s + d] = xyz[3 * ki[s].idx + d];
    }
    free(ki);
    if (rc != OR_OK) {
        free(keys);
        return rc;
    }
    if (keys_sorted) memcpy(keys_sorted, keys, sizeof(uint64_t) * (size_t)n);
    if (nbr) {
#pragma omp parallel for schedule(dynamic, 4096)
        for (int64_t s = 0; s < n; ++s) {
            int32_t row[18];
            nbr_row(keys, n, &xyz_sorted[3 * s], io, nio, row);
            for (int i = 0; i < 18; ++i) nbr[(int64_t)i * n + s] = row[i];
        }
    }
    free(keys);
    return OR_OK;
}

/* Neighbour-table rows for selected sites only (sampled checks at full size). */
void or_nbr_rows(const uint64_t *keys_sorted, int64_t n, const or_iolet *io, int32_t nio,
                 const int32_t *pts, int64_t npts, int32_t *out) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < npts; ++p) nbr_row(keys_sorted, n, &pts[3 * p], io, nio, &out[18 * p]);
}

/* R5 velocity profile: inward wall velocity at the midpoint of the link that
 * leaves site x in direction -c_i (towards x - c_i).  Parabolic: peak U on the
 * axis, zero at the iolet radius; plug: U everywhere. */
static void wall_velocity(const or_iolet *io, const int32_t x[3], int i, double U, double uw[3]) {
    double a[3] = {(double)io->axis[0], (double)io->axis[1], (double)io->axis[2]};
    double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    double ah[3] = {a[0] / an, a[1] / an, a[2] / an};
    double phi = 1.0;
    if (io->profile == OR_PARABOLIC) {
        double rel[3];
        for (int d = 0; d < 3; ++d)
            rel[d] = ((double)x[d] - 0.5 * CV[i][d]) - (double)io->centre[d] / 1024.0;
        double along = rel[0] * ah[0] + rel[1] * ah[1] + rel[2] * ah[2];
        double perp2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double p = rel[d] - along * ah[d];
            perp2 += p * p;
        }
        double r = (double)io->radius / 1024.0;
        phi = 1.0 - perp2 / (r * r);
        if (phi < 0.0) phi = 0.0;
    }
    for (int d = 0; d < 3; ++d) uw[d] = -ah[d] * U * phi;
}

/* BGK collision of the streamed values g (R4); with force density F != NULL
 * the Guo forcing of R7.  mom receives (drho, ux, uy, uz). */
static void collide(const double g[19], double tau, const double *F, double out[19], double mom[4]) {
    double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 19; ++i) {
        drho += g[i];
        for (int d = 0; d < 3; ++d) j[d] += CV[i][d] * g[i];
    }
    double rho = 1.0 + drho;
    double u[3];
    for (int d = 0; d < 3; ++d) u[d] = F ? (j[d] + 0.5 * F[d]) / rho : j[d] / rho;
    double feq[19];
    equilibrium(drho, u, feq);
    for (int i = 0; i < 19; ++i) out[i] = g[i] - (g[i] - feq[i]) / tau;
    if (F) {
        double pref = 1.0 - 0.5 / tau;
        double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
        for (int i = 0; i < 19; ++i) {
            double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
            double cF = CV[i][0] * F[0] + CV[i][1] * F[1] + CV[i][2] * F[2];
            out[i] += pref * weight(i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
        }
    }
    mom[0] = drho;
    mom[1] = u[0];
    mom[2] = u[1];
    mom[3] = u[2];
}

/* The collision alone, for checks of its conservation laws. */
void or_collide(const double *g, double tau, const double *F, double *out, double *mom) {
    collide(g, tau, F, out, mom);
}

/* One site of step t (R5, R6): stream into g (pull from x - c_i, boundary
 * rules on non-fluid links), moments, BGK collision.  bcval[k] is the iolet's
 * value at time t (density deviation or speed); force (NULL = none) holds a
 * force density per site, [n][3]. */
static void site_update(int64_t n, int64_t s, const int32_t *nbr, const int32_t *xyz,
                        const double *Fin, double tau, const or_iolet *io, const double *bcval,
                        const double *force, double out[19], double mom[4]) {
    double g[19];
    g[0] = Fin[s];
    for (int i = 1; i < 19; ++i) {
        int32_t v = nbr[(int64_t)(i - 1) * n + s];
        int o = opposite(i);
        double own = Fin[(int64_t)o * n + s]; /* post-collision value leaving x towards x - c_i */
        if (v >= 0) {
            g[i] = Fin[(int64_t)i * n + v];
        } else if (v == -1) {
            g[i] = own;
        } else {
            const or_iolet *k = &io[-v - 2];
            if (k->kind == OR_PRESSURE) {
                g[i] = -own + 2.0 * weight(i) * bcval[-v - 2];
            } else {
                double uw[3];
                wall_velocity(k, &xyz[3 * s], i, bcval[-v - 2], uw);
                double cu = CV[i][0] * uw[0] + CV[i][1] * uw[1] + CV[i][2] * uw[2];
                g[i] = own + 6.0 * weight(i) * cu;
            }
        }
    }
    const double *F = force ? &force[3 * s] : NULL;
    if (F && F[0] == 0.0 && F[1] == 0.0 && F[2] == 0.0) F = NULL;
    collide(g, tau, F, out, mom);
}

/* Step t over all sites: Fin = F_{t-1} (SoA [19][n]) -> Fout = F_t; mom (if
 * non-NULL) receives (drho, ux, uy, uz) of G_t per site; force as above. */
void or_step(int64_t n, const int32_t *nbr, const int32_t *xyz, const double *Fin, double *Fout,
             double tau, const or_iolet *io, const double *bcval, const double *force, double *mom) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        double out[19], m[4];
        site_update(n, s, nbr, xyz, Fin, tau, io, bcval, force, out, m);
        for (int i = 0; i < 19; ++i) Fout[(int64_t)i * n + s] = out[i];
        if (mom)
            for (int c = 0; c < 4; ++c) mom[4 * s + c] = m[c];
    }
}

/* The same update for a list of sites only: out[p][19], mom[p][4]. */
void or_step_sites(int64_t n, const int32_t *nbr, const int32_t *xyz, const double *Fin,
                   double tau, const or_iolet *io, const double *bcval, const double *force,
                   const int64_t *sites, int64_t nsites, double *out, double *mom) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < nsites; ++p)
        site_update(n, sites[p], nbr, xyz, Fin, tau, io, bcval, force, &out[19 * p], &mom[4 * p]);
}

/* Moments (drho, ux, uy, uz) of a stored state F (SoA [19][n]). */
void or_moments(int64_t n, const double *F, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < n; ++s) {
        double drho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 19; ++i) {
            double f = F[(int64_t)i * n + s];
            drho += f;
            for (int d = 0; d < 3; ++d) j[d] += CV[i][d] * f;
        }
        double rho = 1.0 + drho;
        out[4 * s] = drho;
        for (int d = 0; d < 3; ++d) out[4 * s + 1 + d] = j[d] / rho;
    }
}

/* Iolet means (Section 2.3: only averages cross a coupled boundary).  For each
 * iolet k, over the sites with at least one link coded -(2+k), in canonical
 * order: out[3k] = mean of u . n_k (n_k the unit outward axis), out[3k+1] =
 * mean drho, out[3k+2] = number of sites.  Means of an empty set are 0. */
void or_iolet_means(int64_t n, const int32_t *nbr, const double *mom, const or_iolet *io,
                    int32_t nio, double *out) {
    if (nio <= 0) return;
    double *nh = (double *)calloc((size_t)nio * 3, sizeof(double));
    double *su = (double *)calloc((size_t)nio, sizeof(double));
    double *sr = (double *)calloc((size_t)nio, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)nio, sizeof(int64_t));
    for (int k = 0; k < nio; ++k) {
        double a[3] = {(double)io[k].axis[0], (double)io[k].axis[1], (double)io[k].axis[2]};
        double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
        for (int d = 0; d < 3; ++d) nh[3 * k + d] = a[d] / an;
    }
    /* one pass in canonical order: each iolet's sums take its sites in that order */
    for (int64_t s = 0; s < n; ++s) {
        int seen[18], n_seen = 0;
        for (int i = 0; i < 18; ++i) {
            int32_t v = nbr[(int64_t)i * n + s];
            if (v >= -1) continue;
            int k = -v - 2, dup = 0;
            for (int q = 0; q < n_seen; ++q) dup |= seen[q] == k;
            if (!dup) seen[n_seen++] = k;
        }
        const double *m = &mom[4 * s];
        for (int q = 0; q < n_seen; ++q) {
            int k = seen[q];
            su[k] += m[1] * nh[3 * k] + m[2] * nh[3 * k + 1] + m[3] * nh[3 * k + 2];
            sr[k] += m[0];
            cnt[k] += 1;
        }
    }
    for (int k = 0; k < nio; ++k) {
        out[3 * k] = cnt[k] ? su[k] / (double)cnt[k] : 0.0;
        out[3 * k + 1] = cnt[k] ? sr[k] / (double)cnt[k] : 0.0;
        out[3 * k + 2] = (double)cnt[k];
    }
    free(nh);
    free(su);
    free(sr);
    free(cnt);
}

/* Total mass deviation: sum over sites and directions, canonical order. */
double or_mass(int64_t n, const double *F) {
    double m = 0.0;
    for (int64_t s = 0; s < n; ++s)
        for (int i = 0; i < 19; ++i) m += F[(int64_t)i * n + s];
    return m;
}

int or_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the per-site loops (timing of one core vs all cores). */
void or_set_threads(int n) {
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
