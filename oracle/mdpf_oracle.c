/*
 * mdpf_oracle.c -- plain, slow FP64 CPU oracle for the per-step energy/force
 * evaluation and integrator update.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path links,
 * loads or calls this file; only the tests, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header or constant
 * table with the CUDA sources.
 *
 * The method: the force provider receives positions and hands energy and
 * forces back to the MD engine, which then advances the state (paper,
 * Methods section and the usage listing there; the integrator runs are the
 * NVE runs of the Results section, "Example: Ethanol").  The paper does not
 * fix the potential; the force field evaluated here is the plain analytic one
 * of the benchmark workloads (harmonic bonds and angles, all-pairs LJ +
 * Coulomb with 1-2/1-3 exclusions, no cutoff, no periodic images).
 *
 * Every function below is the direct definition: O(N^2) pair loops in i<j
 * order, analytic derivatives written out, no blocking or reordering.
 *
 * Units: A, fs, amu, e, kcal/mol.  Forces are -dE/dx.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_ACC 4.184e-4 /* kcal/mol/A/amu -> A/fs^2 (1 kcal/mol = 4.184e-4 amu A^2/fs^2) */

/*
 * Threads of the O(N^2) and per-atom loops (1 = the serial loops as written;
 * only the CPU-baseline timing asks for more).  With T > 1 the i loop is split
 * over T OpenMP threads, cyclically, each with its own force or gradient
 * accumulator; the accumulators are then added in thread order, so results
 * differ from the serial ones by rounding only.
 */
static int g_threads = 1;

int orc_set_threads(int32_t t) {
#ifdef _OPENMP
    g_threads = t < 1 ? 1 : t;
#else
    (void)t;
    g_threads = 1;
#endif
    return g_threads;
}

typedef struct {
    int32_t n;
    const int32_t *element;  /* [n] 0=H 1=C 2=N 3=O */
    const double *mass;      /* [n] amu */
    const double *charge;    /* [n] e */
    int32_t n_bonds;
    const int32_t *bonds;    /* [n_bonds][2] */
    const double *bond_r0;   /* [n_bonds] A */
    const double *bond_k;    /* [n_bonds] kcal/mol/A^2, E = k/2 (r - r0)^2 */
    int32_t n_angles;
    const int32_t *angles;   /* [n_angles][3] (a, vertex, b) */
    double angle_k;          /* kcal/mol/rad^2, E = k/2 (theta - theta0)^2 */
    double angle_theta0;     /* rad */
    double lj_sigma[4];      /* per element, Lorentz-Berthelot mixing */
    double lj_eps[4];
    double coulomb_k;        /* kcal A / (mol e^2) */
    const int32_t *excl_offset; /* [n+1] CSR of excluded partners, each row ascending */
    const int32_t *excl_idx;
} orc_system;

/* ---------------------------------------------------------------- topology */

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Neighbour lists of the bond graph, each row ascending. */
static void bond_graph(int n, int nb, const int32_t *bonds, int **off_out, int **adj_out) {
    int *deg = (int *)calloc((size_t)n + 1, sizeof(int));
    for (int b = 0; b < nb; ++b) { deg[bonds[2 * b]]++; deg[bonds[2 * b + 1]]++; }
    int *off = (int *)malloc(((size_t)n + 1) * sizeof(int));
    off[0] = 0;
    for (int i = 0; i < n; ++i) off[i + 1] = off[i] + deg[i];
    int *fill = (int *)calloc((size_t)n + 1, sizeof(int));
    int *adj = (int *)malloc(((size_t)off[n] + 1) * sizeof(int));
    for (int b = 0; b < nb; ++b) {
        int a = bonds[2 * b], c = bonds[2 * b + 1];
        adj[off[a] + fill[a]++] = c;
        adj[off[c] + fill[c]++] = a;
    }
    for (int i = 0; i < n; ++i) qsort(adj + off[i], (size_t)(off[i + 1] - off[i]), sizeof(int), cmp_int);
    free(deg);
    free(fill);
    *off_out = off;
    *adj_out = adj;
}

/*
 * Exclusions: j != i is excluded from i's nonbonded sum when j is bonded to i
 * (1-2) or j and i share a bonded neighbour (1-3).  Output as CSR rows sorted
 * ascending with duplicates removed.  Returns the total number of entries, or
 * -1 when it exceeds cap.
 */
int orc_exclusions(int32_t n, int32_t nb, const int32_t *bonds, int32_t *offset, int32_t *idx, int32_t cap) {
    int *off, *adj;
    bond_graph(n, nb, bonds, &off, &adj);
    int total = 0;
    int *tmp = (int *)malloc(((size_t)n + 1) * sizeof(int));
    offset[0] = 0;
    for (int i = 0; i < n; ++i) {
        int m = 0;
        for (int p = off[i]; p < off[i + 1]; ++p) {
            int j = adj[p];
            tmp[m++] = j;                                   /* 1-2 */
            for (int q = off[j]; q < off[j + 1]; ++q)       /* 1-3 through j */
                if (adj[q] != i) tmp[m++] = adj[q];
        }
        qsort(tmp, (size_t)m, sizeof(int), cmp_int);
        int u = 0;
        for (int k = 0; k < m; ++k)
            if (u == 0 || tmp[k] != tmp[u - 1]) tmp[u++] = tmp[k];
        if (total + u > cap) { total = -1; break; }
        memcpy(idx + total, tmp, (size_t)u * sizeof(int));
        total += u;
        offset[i + 1] = total;
    }
    free(tmp);
    free(off);
    free(adj);
    return total;
}

/*
 * Angles from the bond graph: one (a, v, b) per vertex v and per pair a < b of
 * v's bonded neighbours; vertices ascending, then a, then b.  Returns the count
 * or -1 when it exceeds cap.
 */
int orc_angles(int32_t n, int32_t nb, const int32_t *bonds, int32_t *angles, int32_t cap) {
    int *off, *adj;
    bond_graph(n, nb, bonds, &off, &adj);
    int na = 0;
    for (int v = 0; v < n && na >= 0; ++v)
        for (int p = off[v]; p < off[v + 1] && na >= 0; ++p)
            for (int q = p + 1; q < off[v + 1]; ++q) {
                if (na >= cap) { na = -1; break; }
                angles[3 * na] = adj[p];
                angles[3 * na + 1] = v;
                angles[3 * na + 2] = adj[q];
                na++;
            }
    free(off);
    free(adj);
    return na;
}

static int is_excluded(const orc_system *s, int i, int j) {
    for (int p = s->excl_offset[i]; p < s->excl_offset[i + 1]; ++p)
        if (s->excl_idx[p] == j) return 1;
    return 0;
}

/* ------------------------------------------------------------ plain forces */

/*
 * Total potential energy and forces of the plain analytic force field.
 * terms (optional) receives {E_bond, E_angle, E_lj, E_coulomb}.
 */
double orc_plain_energy_forces(const orc_system *s, const double *x, double *f, double *terms) {
    const int n = s->n;
    double eb = 0, ea = 0, elj = 0, ec = 0;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);

    /* harmonic bonds: E = k/2 (r - r0)^2 */
    for (int b = 0; b < s->n_bonds; ++b) {
        int i = s->bonds[2 * b], j = s->bonds[2 * b + 1];
        double d[3], r = 0;
        for (int c = 0; c < 3; ++c) { d[c] = x[3 * j + c] - x[3 * i + c]; r += d[c] * d[c]; }
        r = sqrt(r);
        double dr = r - s->bond_r0[b];
        eb += 0.5 * s->bond_k[b] * dr * dr;
        double g = s->bond_k[b] * dr / r;          /* dE/dr / r */
        for (int c = 0; c < 3; ++c) { f[3 * i + c] += g * d[c]; f[3 * j + c] -= g * d[c]; }
    }

    /* harmonic angles: E = k/2 (theta - theta0)^2, theta = angle a-v-b */
    for (int t = 0; t < s->n_angles; ++t) {
        int a = s->angles[3 * t], v = s->angles[3 * t + 1], b = s->angles[3 * t + 2];
        double u[3], w[3], ru = 0, rw = 0, uw = 0;
        for (int c = 0; c < 3; ++c) {
            u[c] = x[3 * a + c] - x[3 * v + c];
            w[c] = x[3 * b + c] - x[3 * v + c];
            ru += u[c] * u[c]; rw += w[c] * w[c]; uw += u[c] * w[c];
        }
        ru = sqrt(ru); rw = sqrt(rw);
        double cs = uw / (ru * rw);
        if (cs > 1.0) cs = 1.0;
        if (cs < -1.0) cs = -1.0;
        double th = acos(cs);
        double dth = th - s->angle_theta0;
        ea += 0.5 * s->angle_k * dth * dth;
        /* dtheta/dcos = -1/sin(theta); F = -dE/dtheta * dtheta/dx = k dth / sin * dcos/dx */
        double pref = s->angle_k * dth / sin(th);
        for (int c = 0; c < 3; ++c) {
            double dca = w[c] / (ru * rw) - cs * u[c] / (ru * ru);   /* dcos/dx_a */
            double dcb = u[c] / (ru * rw) - cs * w[c] / (rw * rw);   /* dcos/dx_b */
            f[3 * a + c] += pref * dca;
            f[3 * b + c] += pref * dcb;
            f[3 * v + c] -= pref * (dca + dcb);
        }
    }

    /* all pairs i < j not excluded: LJ (Lorentz-Berthelot) + Coulomb, no cutoff */
    const int T = g_threads;
    double *ft = T > 1 ? (double *)calloc((size_t)T * 3 * n, sizeof(double)) : f;
    double *et = (double *)calloc(2 * (size_t)T, sizeof(double));
#pragma omp parallel for schedule(static, 1) num_threads(T) if (T > 1)
    for (int i = 0; i < n; ++i) {
#ifdef _OPENMP
        const int tid = T > 1 ? omp_get_thread_num() : 0;
#else
        const int tid = 0;
#endif
        double *fo = T > 1 ? ft + (size_t)tid * 3 * n : f;
        for (int j = i + 1; j < n; ++j) {
            if (is_excluded(s, i, j)) continue;
            double d[3], r2 = 0;
            for (int c = 0; c < 3; ++c) { d[c] = x[3 * j + c] - x[3 * i + c]; r2 += d[c] * d[c]; }
            double r = sqrt(r2);
            double sig = 0.5 * (s->lj_sigma[s->element[i]] + s->lj_sigma[s->element[j]]);
            double eps = sqrt(s->lj_eps[s->element[i]] * s->lj_eps[s->element[j]]);
            double sr6 = pow(sig / r, 6.0);
            double sr12 = sr6 * sr6;
            double e_lj = 4.0 * eps * (sr12 - sr6);
            double e_c = s->coulomb_k * s->charge[i] * s->charge[j] / r;
            et[2 * tid] += e_lj;
            et[2 * tid + 1] += e_c;
            /* dE/dr = (-48 eps sr12 + 24 eps sr6)/r - e_c/r */
            double dedr = (-48.0 * eps * sr12 + 24.0 * eps * sr6) / r - e_c / r;
            double g = dedr / r;                   /* F_i = +dE/dr * d/r, F_j = -F_i */
            for (int c = 0; c < 3; ++c) { fo[3 * i + c] += g * d[c]; fo[3 * j + c] -= g * d[c]; }
        }
    }
    for (int t = 0; t < T; ++t) {
        elj += et[2 * t];
        ec += et[2 * t + 1];
        if (T > 1)
            for (int q = 0; q < 3 * n; ++q) f[q] += ft[(size_t)t * 3 * n + q];
    }
    if (T > 1) free(ft);
    free(et);
    if (terms) { terms[0] = eb; terms[1] = ea; terms[2] = elj; terms[3] = ec; }
    return eb + ea + elj + ec;
}

/* Kinetic energy in kcal/mol of velocities v [n][3] in A/fs. */
double orc_kinetic(int32_t n, const double *mass, const double *v) {
    double k = 0;
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) k += 0.5 * mass[i] * v[3 * i + c] * v[3 * i + c];
    return k / ORC_ACC;
}

/*
 * Velocity Verlet, n_steps of dt fs, in place on x [A] and v [A/fs]:
 *   v <- v + dt/2 a(x);  x <- x + dt v;  v <- v + dt/2 a(x).
 * U[s], K[s] receive the potential and kinetic energy after step s+1.
 * f (optional, [n][3]) receives the forces at the final positions.
 */
void orc_vv_run(const orc_system *s, double dt, int32_t n_steps, double *x, double *v, double *U, double *K,
                double *f_out) {
    const int n = s->n;
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    orc_plain_energy_forces(s, x, f, NULL);
    for (int st = 0; st < n_steps; ++st) {
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) {
                v[3 * i + c] += 0.5 * dt * ORC_ACC * f[3 * i + c] / s->mass[i];
                x[3 * i + c] += dt * v[3 * i + c];
            }
        double u = orc_plain_energy_forces(s, x, f, NULL);
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt * ORC_ACC * f[3 * i + c] / s->mass[i];
        if (U) U[st] = u;
        if (K) K[st] = orc_kinetic(n, s->mass, v);
    }
    if (f_out) memcpy(f_out, f, sizeof(double) * 3 * (size_t)n);
    free(f);
}

/* ====================================================================
 * Learned potential: symmetry-function features + per-element MLP.
 *
 * The paper's force module is an ML force field called from the engine each
 * step (Results, "Example: Ethanol"); its architecture is not given there.
 * The stand-in evaluated here is an ANI-style potential (Smith et al. 2017):
 *   radial    G[i, 16 Zj + k]           = sum_j  exp(-eta_R (r_ij - R_k)^2) fc_R(r_ij)
 *   angular   G[i, 64 + 32 P + 8 m + p] = sum_{j<k} 2^(1-zeta) (1 + cos(theta - theta_p))^zeta
 *                                         * exp(-eta_A ((r_ij + r_ik)/2 - R_m)^2) fc_A(r_ij) fc_A(r_ik)
 *   with theta = acos(0.95 cos(theta_ijk)), P the unordered element pair of
 *   (Zj, Zk) in the order HH HC HN HO CC CN CO NN NO OO, fc(r) = cos(pi r/rc)/2 + 1/2
 *   for r < rc, 0 otherwise.
 *   E = sum_i [ W3 . celu(W2 celu(W1 G_i + b1) + b2) + b3 + e0 ]_{element of i}
 * Forces are -dE/dx through the analytic feature derivatives.
 * ==================================================================== */

#define ORC_NFEAT 384
#define ORC_NRAD 16
#define ORC_RC_R 5.2
#define ORC_RC_A 3.5
#define ORC_ETA_R 16.0
#define ORC_ETA_A 8.0
#define ORC_ZETA 32.0
#define ORC_ANG_SCALE 0.95
#define ORC_PI 3.14159265358979323846

static double orc_rk(int k) { return 0.9 + k * (ORC_RC_R - 0.9) / 16.0; }
static double orc_rm(int m) { return 0.9 + m * (ORC_RC_A - 0.9) / 4.0; }
static double orc_thp(int p) { return (2 * p + 1) * ORC_PI / 16.0; }

static double orc_fc(double r, double rc) { return r < rc ? 0.5 * cos(ORC_PI * r / rc) + 0.5 : 0.0; }
static double orc_dfc(double r, double rc) { return r < rc ? -0.5 * ORC_PI / rc * sin(ORC_PI * r / rc) : 0.0; }

/* unordered element pair index for a <= b: HH HC HN HO CC CN CO NN NO OO */
static int orc_pair(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    static const int base[4] = {0, 4, 7, 9};
    return base[a] + (b - a);
}

/*
 * Neighbour list by brute force with the single-precision predicate
 *   dx = fl(x_j - x_i) (FP32 coordinates), d2 = fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)),
 *   neighbour iff d2 < rc2 (rc2 given in FP32), j != i.
 * Rows ascending.  Returns the total count or -1 if a row exceeds max_per_atom.
 */
int orc_neighbors(int32_t n, const float *x, float rc2, int32_t max_per_atom, int32_t *count, int32_t *idx) {
    int total = 0;
    for (int i = 0; i < n; ++i) {
        int m = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            float dx = x[3 * j] - x[3 * i];
            float dy = x[3 * j + 1] - x[3 * i + 1];
            float dz = x[3 * j + 2] - x[3 * i + 2];
            float sx = dx * dx;
            float sy = dy * dy;
            float sz = dz * dz;
            float d2 = sx + sy;
            d2 = d2 + sz;
            if (d2 < rc2) {
                if (m >= max_per_atom) return -1;
                idx[(size_t)i * max_per_atom + m] = j;
                m++;
            }
        }
        count[i] = m;
        total += m;
    }
    return total;
}

/*
 * Per-term visitor.  For atom i, every term T of feature f that involves atoms
 * (i, j[, k]) is visited with its value and its gradients with respect to the
 * positions of the atoms involved.  mode 0: accumulate G; mode 1: forces
 * F -= w[i,f] dT/dx; mode 2: JVP Gdot[i,f] += dT/dx . u.
 */
static void orc_feature_pass(int n, const int32_t *el, const double *x, int mode, const double *w, const double *u,
                             double *out_all) {
    /* modes 0 and 2 write row i only; mode 1 adds into every atom's force, so each thread has its own */
    const int T = g_threads;
    double *priv = (T > 1 && mode == 1) ? (double *)calloc((size_t)T * 3 * n, sizeof(double)) : NULL;
#pragma omp parallel for schedule(static, 1) num_threads(T) if (T > 1)
    for (int i = 0; i < n; ++i) {
#ifdef _OPENMP
        double *out = priv ? priv + (size_t)omp_get_thread_num() * 3 * n : out_all;
#else
        double *out = out_all;
#endif
        const double *xi = x + 3 * i;
        /* radial */
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double d[3], r = 0;
            for (int c = 0; c < 3; ++c) { d[c] = x[3 * j + c] - xi[c]; r += d[c] * d[c]; }
            r = sqrt(r);
            if (!(r < ORC_RC_R)) continue;
            for (int k = 0; k < ORC_NRAD; ++k) {
                int f = 16 * el[j] + k;
                double e = exp(-ORC_ETA_R * (r - orc_rk(k)) * (r - orc_rk(k)));
                double T = e * orc_fc(r, ORC_RC_R);
                double dT = e * (-2.0 * ORC_ETA_R * (r - orc_rk(k)) * orc_fc(r, ORC_RC_R) + orc_dfc(r, ORC_RC_R));
                /* dT/dx_j = dT * d/r, dT/dx_i = -dT * d/r */
                if (mode == 0) out[(size_t)i * ORC_NFEAT + f] += T;
                else if (mode == 1) {
                    double wf = w[(size_t)i * ORC_NFEAT + f];
                    for (int c = 0; c < 3; ++c) {
                        out[3 * j + c] -= wf * dT * d[c] / r;
                        out[3 * i + c] += wf * dT * d[c] / r;
                    }
                } else {
                    double s = 0;
                    for (int c = 0; c < 3; ++c) s += dT * d[c] / r * (u[3 * j + c] - u[3 * i + c]);
                    out[(size_t)i * ORC_NFEAT + f] += s;
                }
            }
        }
        /* angular: unordered pairs j < k of neighbours within rc_A */
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double dj[3], rj = 0;
            for (int c = 0; c < 3; ++c) { dj[c] = x[3 * j + c] - xi[c]; rj += dj[c] * dj[c]; }
            rj = sqrt(rj);
            if (!(rj < ORC_RC_A)) continue;
            for (int k = j + 1; k < n; ++k) {
                if (k == i) continue;
                double dk[3], rk = 0;
                for (int c = 0; c < 3; ++c) { dk[c] = x[3 * k + c] - xi[c]; rk += dk[c] * dk[c]; }
                rk = sqrt(rk);
                if (!(rk < ORC_RC_A)) continue;
                double uj[3], uk[3], ct = 0;
                for (int c = 0; c < 3; ++c) { uj[c] = dj[c] / rj; uk[c] = dk[c] / rk; ct += uj[c] * uk[c]; }
                /* d cos(theta_ijk) / d x_j, d x_k */
                double dcj[3], dck[3];
                for (int c = 0; c < 3; ++c) {
                    dcj[c] = (uk[c] - ct * uj[c]) / rj;
                    dck[c] = (uj[c] - ct * uk[c]) / rk;
                }
                double cs = ORC_ANG_SCALE * ct;
                double sn = sqrt(1.0 - cs * cs);
                double fj = orc_fc(rj, ORC_RC_A), fk = orc_fc(rk, ORC_RC_A);
                double C = fj * fk;
                double dCj = orc_dfc(rj, ORC_RC_A) * fk, dCk = fj * orc_dfc(rk, ORC_RC_A);
                int P = orc_pair(el[j], el[k]);
                double ravg = 0.5 * (rj + rk);
                for (int m = 0; m < 4; ++m) {
                    double B = exp(-ORC_ETA_A * (ravg - orc_rm(m)) * (ravg - orc_rm(m)));
                    double dB = -ORC_ETA_A * (ravg - orc_rm(m)) * B;  /* dB/dr_ij = dB/dr_ik */
                    for (int p = 0; p < 8; ++p) {
                        int f = 64 + 32 * P + 8 * m + p;
                        double cp = cos(orc_thp(p)), sp = sin(orc_thp(p));
                        double base = 1.0 + cs * cp + sn * sp;      /* 1 + cos(theta - theta_p) */
                        double A = pow(2.0, 1.0 - ORC_ZETA) * pow(base, ORC_ZETA);
                        double dAdcs = pow(2.0, 1.0 - ORC_ZETA) * ORC_ZETA * pow(base, ORC_ZETA - 1.0) * (cp - cs / sn * sp);
                        double T = A * B * C;
                        if (mode == 0) { out[(size_t)i * ORC_NFEAT + f] += T; continue; }
                        /* gradient of T with respect to x_j and x_k; x_i gets minus their sum */
                        double gj[3], gk[3];
                        for (int c = 0; c < 3; ++c) {
                            gj[c] = dAdcs * ORC_ANG_SCALE * dcj[c] * B * C + A * dB * uj[c] * C + A * B * dCj * uj[c];
                            gk[c] = dAdcs * ORC_ANG_SCALE * dck[c] * B * C + A * dB * uk[c] * C + A * B * dCk * uk[c];
                        }
                        if (mode == 1) {
                            double wf = w[(size_t)i * ORC_NFEAT + f];
                            for (int c = 0; c < 3; ++c) {
                                out[3 * j + c] -= wf * gj[c];
                                out[3 * k + c] -= wf * gk[c];
                                out[3 * i + c] += wf * (gj[c] + gk[c]);
                            }
                        } else {
                            double s = 0;
                            for (int c = 0; c < 3; ++c)
                                s += gj[c] * (u[3 * j + c] - u[3 * i + c]) + gk[c] * (u[3 * k + c] - u[3 * i + c]);
                            out[(size_t)i * ORC_NFEAT + f] += s;
                        }
                    }
                }
            }
        }
    }
    if (priv) {
        for (int t = 0; t < T; ++t)
            for (int q = 0; q < 3 * n; ++q) out_all[q] += priv[(size_t)t * 3 * n + q];
        free(priv);
    }
}

/* G [n][384] */
void orc_features(int32_t n, const int32_t *el, const double *x, double *G) {
    memset(G, 0, sizeof(double) * (size_t)n * ORC_NFEAT);
    orc_feature_pass(n, el, x, 0, NULL, NULL, G);
}

/* F [n][3] = -sum_{i,f} w[i,f] dG[i,f]/dx  (w = dE/dG) */
void orc_feature_forces(int32_t n, const int32_t *el, const double *x, const double *w, double *F) {
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    orc_feature_pass(n, el, x, 1, w, NULL, F);
}

/* Gdot [n][384] = sum_a dG[i,f]/dx_a . u_a */
void orc_feature_jvp(int32_t n, const int32_t *el, const double *x, const double *u, double *Gdot) {
    memset(Gdot, 0, sizeof(double) * (size_t)n * ORC_NFEAT);
    orc_feature_pass(n, el, x, 2, NULL, u, Gdot);
}

/* ---------------------------------------------------------------- MLP */

typedef struct {
    int32_t n_feat, h1, h2;
    double alpha;          /* CELU alpha */
    const double *W1[4];   /* [h1][n_feat] */
    const double *b1[4];   /* [h1] */
    const double *W2[4];   /* [h2][h1] */
    const double *b2[4];   /* [h2] */
    const double *W3[4];   /* [h2] */
    double b3[4];
    double e0[4];
} orc_mlp;

static double orc_celu(double z, double a) { return z > 0 ? z : a * (exp(z / a) - 1.0); }
static double orc_dcelu(double z, double a) { return z >= 0 ? 1.0 : exp(z / a); }

/*
 * Per-atom energies E_i (optional) and input gradients dEdG [n][n_feat]
 * (optional); returns sum_i E_i.
 *   h1 = W1 G + b1, a1 = celu(h1); h2 = W2 a1 + b2, a2 = celu(h2); E = W3 . a2 + b3 + e0
 *   dE/dG = W1^T [celu'(h1) * W2^T (celu'(h2) * W3)]
 */
double orc_mlp_energy(const orc_mlp *M, int32_t n, const int32_t *el, const double *G, double *Ei_out,
                      double *dEdG) {
    const int F = M->n_feat, H1 = M->h1, H2 = M->h2;
    const int T = g_threads;
    double *Ei = Ei_out ? Ei_out : (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
#pragma omp parallel num_threads(T) if (T > 1)
    {
    double *h1 = (double *)malloc(sizeof(double) * H1), *a1 = (double *)malloc(sizeof(double) * H1);
    double *h2 = (double *)malloc(sizeof(double) * H2), *a2 = (double *)malloc(sizeof(double) * H2);
    double *d2 = (double *)malloc(sizeof(double) * H2), *d1 = (double *)malloc(sizeof(double) * H1);
#pragma omp for schedule(static, 1)
    for (int i = 0; i < n; ++i) {
        const int e = el[i];
        const double *g = G + (size_t)i * F;
        for (int a = 0; a < H1; ++a) {
            double s = M->b1[e][a];
            for (int f = 0; f < F; ++f) s += M->W1[e][(size_t)a * F + f] * g[f];
            h1[a] = s;
            a1[a] = orc_celu(s, M->alpha);
        }
        for (int b = 0; b < H2; ++b) {
            double s = M->b2[e][b];
            for (int a = 0; a < H1; ++a) s += M->W2[e][(size_t)b * H1 + a] * a1[a];
            h2[b] = s;
            a2[b] = orc_celu(s, M->alpha);
        }
        double E = M->b3[e] + M->e0[e];
        for (int b = 0; b < H2; ++b) E += M->W3[e][b] * a2[b];
        Ei[i] = E;
        if (dEdG) {
            for (int b = 0; b < H2; ++b) d2[b] = M->W3[e][b] * orc_dcelu(h2[b], M->alpha);
            for (int a = 0; a < H1; ++a) {
                double s = 0;
                for (int b = 0; b < H2; ++b) s += M->W2[e][(size_t)b * H1 + a] * d2[b];
                d1[a] = s * orc_dcelu(h1[a], M->alpha);
            }
            for (int f = 0; f < F; ++f) {
                double s = 0;
                for (int a = 0; a < H1; ++a) s += M->W1[e][(size_t)a * F + f] * d1[a];
                dEdG[(size_t)i * F + f] = s;
            }
        }
    }
    free(h1); free(a1); free(h2); free(a2); free(d2); free(d1);
    }
    double total = 0;   /* summed in atom order, whatever the threads */
    for (int i = 0; i < n; ++i) total += Ei[i];
    if (!Ei_out) free(Ei);
    return total;
}

/* Learned energy and forces at x: E returned, F [n][3] = -dE/dx. */
double orc_learned_energy_forces(const orc_mlp *M, int32_t n, const int32_t *el, const double *x, double *F,
                                 double *G_out) {
    double *G = G_out ? G_out : (double *)malloc(sizeof(double) * (size_t)n * ORC_NFEAT);
    double *w = (double *)malloc(sizeof(double) * (size_t)n * ORC_NFEAT);
    orc_features(n, el, x, G);
    double E = orc_mlp_energy(M, n, el, G, NULL, w);
    if (F) orc_feature_forces(n, el, x, w, F);
    free(w);
    if (!G_out) free(G);
    return E;
}

/*
 * Repulsive core of the learned potential: for every pair i < j closer than
 * rc,  E = A (1 - x)^3 / x  with x = r / rc, so E and its first two
 * derivatives vanish at rc and E grows as 1/r towards r = 0.  Returns the
 * energy and adds -dE/dx to F [n][3] (F may be NULL).  dE/dr is written out
 * by hand: dE/dx = -A (1 - x)^2 (3 x + (1 - x)) / x^2 = -A (1 - x)^2 (1 + 2 x) / x^2.
 */
double orc_core_energy_forces(int32_t n, const double *x, double A, double rc, double *F) {
    double E = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (!(r < rc)) continue;
            const double u = r / rc, om = 1.0 - u;
            E += A * om * om * om / u;
            if (F) {
                const double dEdr = -A / rc * om * om * (1.0 + 2.0 * u) / (u * u);
                for (int c = 0; c < 3; ++c) {
                    /* E depends on x_j - x_i through r: dE/dx_j = dEdr d / r, dE/dx_i = -dEdr d / r */
                    F[3 * i + c] += dEdr * d[c] / r;
                    F[3 * j + c] -= dEdr * d[c] / r;
                }
            }
        }
    return E;
}

/* ---------------------------------------------------------------- training gradient */

static double orc_d2celu(double z, double a) { return z >= 0 ? 0.0 : exp(z / a) / a; }

/*
 * Parameter gradient of  J = sum_i [ c_i E_i - D_i ],  D_i = u_i . dE_i/dG_i,
 * accumulated into gW1 [4][h1][F], gb1 [4][h1], gW2 [4][h2][h1], gb2 [4][h2],
 * gW3 [4][h2], gb3 [4].  With c_i the energy-loss weight of atom i's frame and
 * u_i the feature JVP of the force-loss gradient, J's parameter gradient is
 * the force-matching loss gradient (the force term reaches the parameters
 * through the input gradient, so it is reverse mode over the tangent pass):
 *   primal   h1 = W1 G + b1, a1 = s(h1); h2 = W2 a1 + b2, a2 = s(h2); E = W3 . a2 + b3 + e0
 *   tangent  t1 = W1 u, ta1 = s'(h1) t1; t2 = W2 ta1, ta2 = s'(h2) t2; D = W3 . ta2
 * then one reverse sweep over both, last operation first.  s'' is taken as 0
 * for z >= 0 and exp(z/alpha)/alpha below.
 */
void orc_mlp_param_grad(const orc_mlp *M, int32_t n, const int32_t *el, const double *G, const double *U,
                        const double *c, double *gW1_all, double *gb1_all, double *gW2_all, double *gb2_all,
                        double *gW3_all, double *gb3_all) {
    const int F = M->n_feat, H1 = M->h1, H2 = M->h2;
    const double al = M->alpha;
    const int T = g_threads;
    /* per-thread gradient accumulators when threaded (added in thread order at the end) */
    const size_t nW1 = 4 * (size_t)H1 * F, nW2 = 4 * (size_t)H2 * H1;
    const size_t per = nW1 + 4 * (size_t)H1 + nW2 + 4 * (size_t)H2 + 4 * (size_t)H2 + 4;
    double *acc = T > 1 ? (double *)calloc((size_t)T * per, sizeof(double)) : NULL;
#pragma omp parallel num_threads(T) if (T > 1)
    {
#ifdef _OPENMP
    double *mine = acc ? acc + (size_t)omp_get_thread_num() * per : NULL;
#else
    double *mine = NULL;
#endif
    double *gW1 = mine ? mine : gW1_all, *gb1 = mine ? mine + nW1 : gb1_all;
    double *gW2 = mine ? mine + nW1 + 4 * (size_t)H1 : gW2_all;
    double *gb2 = mine ? mine + nW1 + 4 * (size_t)H1 + nW2 : gb2_all;
    double *gW3 = mine ? mine + nW1 + 4 * (size_t)H1 + nW2 + 4 * (size_t)H2 : gW3_all;
    double *gb3 = mine ? mine + nW1 + 4 * (size_t)H1 + nW2 + 8 * (size_t)H2 : gb3_all;
    double *h1 = (double *)malloc(sizeof(double) * H1), *a1 = (double *)malloc(sizeof(double) * H1);
    double *t1 = (double *)malloc(sizeof(double) * H1), *ta1 = (double *)malloc(sizeof(double) * H1);
    double *h2 = (double *)malloc(sizeof(double) * H2), *a2 = (double *)malloc(sizeof(double) * H2);
    double *t2 = (double *)malloc(sizeof(double) * H2), *ta2 = (double *)malloc(sizeof(double) * H2);
    double *bt2 = (double *)malloc(sizeof(double) * H2), *bh2 = (double *)malloc(sizeof(double) * H2);
    double *bt1 = (double *)malloc(sizeof(double) * H1), *bh1 = (double *)malloc(sizeof(double) * H1);
    double *bta1 = (double *)malloc(sizeof(double) * H1), *ba1 = (double *)malloc(sizeof(double) * H1);
#pragma omp for schedule(static, 1)
    for (int i = 0; i < n; ++i) {
        const int e = el[i];
        const double *g = G + (size_t)i * F, *u = U + (size_t)i * F;
        const double *W1 = M->W1[e], *W2 = M->W2[e], *W3 = M->W3[e];
        /* primal and tangent */
        for (int a = 0; a < H1; ++a) {
            double s = M->b1[e][a], t = 0;
            for (int f = 0; f < F; ++f) {
                s += W1[(size_t)a * F + f] * g[f];
                t += W1[(size_t)a * F + f] * u[f];
            }
            h1[a] = s;
            a1[a] = orc_celu(s, al);
            t1[a] = t;
            ta1[a] = orc_dcelu(s, al) * t;
        }
        for (int b = 0; b < H2; ++b) {
            double s = M->b2[e][b], t = 0;
            for (int a = 0; a < H1; ++a) {
                s += W2[(size_t)b * H1 + a] * a1[a];
                t += W2[(size_t)b * H1 + a] * ta1[a];
            }
            h2[b] = s;
            a2[b] = orc_celu(s, al);
            t2[b] = t;
            ta2[b] = orc_dcelu(s, al) * t;
        }
        /* reverse: J = c E - W3 . ta2 */
        const double ci = c[i];
        gb3[e] += ci;
        for (int b = 0; b < H2; ++b) {
            gW3[e * H2 + b] += ci * a2[b] - ta2[b];
            const double bta2 = -W3[b], ba2 = ci * W3[b];
            bt2[b] = orc_dcelu(h2[b], al) * bta2;
            bh2[b] = orc_d2celu(h2[b], al) * t2[b] * bta2 + orc_dcelu(h2[b], al) * ba2;
            gb2[e * H2 + b] += bh2[b];
            for (int a = 0; a < H1; ++a)
                gW2[((size_t)e * H2 + b) * H1 + a] += bt2[b] * ta1[a] + bh2[b] * a1[a];
        }
        for (int a = 0; a < H1; ++a) {
            double s_t = 0, s_h = 0;
            for (int b = 0; b < H2; ++b) {
                s_t += W2[(size_t)b * H1 + a] * bt2[b];
                s_h += W2[(size_t)b * H1 + a] * bh2[b];
            }
            bta1[a] = s_t;
            ba1[a] = s_h;
            bt1[a] = orc_dcelu(h1[a], al) * bta1[a];
            bh1[a] = orc_d2celu(h1[a], al) * t1[a] * bta1[a] + orc_dcelu(h1[a], al) * ba1[a];
            gb1[e * H1 + a] += bh1[a];
            for (int f = 0; f < F; ++f)
                gW1[((size_t)e * H1 + a) * F + f] += bt1[a] * u[f] + bh1[a] * g[f];
        }
    }
    free(h1); free(a1); free(t1); free(ta1); free(h2); free(a2); free(t2); free(ta2);
    free(bt2); free(bh2); free(bt1); free(bh1); free(bta1); free(ba1);
    }
    if (acc) {
        for (int t = 0; t < T; ++t) {
            const double *m = acc + (size_t)t * per;
            for (size_t q = 0; q < nW1; ++q) gW1_all[q] += m[q];
            for (size_t q = 0; q < 4 * (size_t)H1; ++q) gb1_all[q] += m[nW1 + q];
            for (size_t q = 0; q < nW2; ++q) gW2_all[q] += m[nW1 + 4 * (size_t)H1 + q];
            for (size_t q = 0; q < 4 * (size_t)H2; ++q) gb2_all[q] += m[nW1 + 4 * (size_t)H1 + nW2 + q];
            for (size_t q = 0; q < 4 * (size_t)H2; ++q) gW3_all[q] += m[nW1 + 4 * (size_t)H1 + nW2 + 4 * (size_t)H2 + q];
            for (int q = 0; q < 4; ++q) gb3_all[q] += m[nW1 + 4 * (size_t)H1 + nW2 + 8 * (size_t)H2 + q];
        }
        free(acc);
    }
}

/* ---------------------------------------------------------------- Langevin dynamics */

/*
 * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of
 *   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
 * with M0 = 0xD2511F53, M1 = 0xCD9E8D57, the key advanced by the Weyl
 * constants (0x9E3779B9, 0xBB67AE85) before every round after the first.
 */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c[0] = hi1 ^ c[1] ^ k0;
        c[1] = lo1;
        c[2] = hi0 ^ c[3] ^ k1;
        c[3] = lo0;
    }
    for (int q = 0; q < 4; ++q) out[q] = c[q];
}

/*
 * Three standard normal deviates for atom `atom` at step `step`: Philox with
 * counter (atom, step low word, step high word, 0x4C414E47) and key (seed low,
 * seed high); uniforms u = (x + 1/2) 2^-32; Box-Muller on (u0, u1) and (u2, u3).
 */
void orc_langevin_normals(uint64_t seed, int64_t step, int32_t atom, double z[3]) {
    const uint32_t ctr[4] = {(uint32_t)atom, (uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), 0x4C414E47u};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double u[4];
    for (int q = 0; q < 4; ++q) u[q] = ((double)x[q] + 0.5) * (1.0 / 4294967296.0);
    const double two_pi = 6.283185307179586476925286766559;
    const double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    z[0] = r0 * cos(two_pi * u[1]);
    z[1] = r0 * sin(two_pi * u[1]);
    z[2] = r1 * cos(two_pi * u[3]);
}

/*
 * Langevin dynamics, BAOAB splitting (Leimkuhler and Matthews 2013), n_steps of
 * dt fs from step index step0, in place on x and v:
 *   v <- v + dt/2 a(x);  x <- x + dt/2 v;
 *   v <- c1 v + c2 R,  c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kB T / m)  (R from orc_langevin_normals);
 *   x <- x + dt/2 v;  v <- v + dt/2 a(x).
 * gamma in 1/ps, T in K; U[s], K[s] after step s+1.
 */
void orc_langevin_run(const orc_system *s, double dt, int32_t n_steps, double gamma_ps, double temp_K,
                      uint64_t seed, int64_t step0, double *x, double *v, double *U, double *K) {
    const int n = s->n;
    const double kB = 0.0019872041;  /* kcal/mol/K */
    const double c1 = exp(-gamma_ps * 1e-3 * dt);
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    orc_plain_energy_forces(s, x, f, NULL);
    for (int st = 0; st < n_steps; ++st) {
        for (int i = 0; i < n; ++i) {
            const double c2 = sqrt((1.0 - c1 * c1) * kB * temp_K * ORC_ACC / s->mass[i]);
            double z[3];
            orc_langevin_normals(seed, step0 + st, i, z);
            for (int c = 0; c < 3; ++c) {
                double vc = v[3 * i + c] + 0.5 * dt * ORC_ACC * f[3 * i + c] / s->mass[i];
                double xc = x[3 * i + c] + 0.5 * dt * vc;
                vc = c1 * vc + c2 * z[c];
                x[3 * i + c] = xc + 0.5 * dt * vc;
                v[3 * i + c] = vc;
            }
        }
        double u = orc_plain_energy_forces(s, x, f, NULL);
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) v[3 * i + c] += 0.5 * dt * ORC_ACC * f[3 * i + c] / s->mass[i];
        if (U) U[st] = u;
        if (K) K[st] = orc_kinetic(n, s->mass, v);
    }
    free(f);
}

/* ---------------------------------------------------------------- initial velocities */

/*
 * Maxwell-Boltzmann velocities (A/fs) at temperature T for masses m [n] at
 * positions x [n][3], written to v [n][3]:
 *   1. v_i = sqrt(kB T / m_i) z_i, with z_i three standard normals per atom by
 *      Box-Muller from Philox4x32-10 with counter (i, 0, 0, 0x4D425630) and
 *      key (seed low, seed high) (units: kB T / m in kcal/mol/amu, times
 *      ORC_ACC for A^2/fs^2);
 *   2. the centre-of-mass velocity P / M is subtracted;
 *   3. for n >= 3, the rigid rotation w x (x_i - x_com) with I w = L is
 *      subtracted (L the angular momentum about the centre of mass, I the
 *      inertia tensor), unless I is singular (collinear atoms);
 *   4. v is scaled so that K = (3n - 6) kB T / 2 (3n - 6 taken as at least 1).
 */
void orc_init_velocities(int32_t n, const double *mass, const double *x, double T, uint64_t seed, double *v) {
    const double kB = 0.0019872041;  /* kcal/mol/K */
    const double two_pi = 6.283185307179586476925286766559;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int i = 0; i < n; ++i) {
        const uint32_t ctr[4] = {(uint32_t)i, 0u, 0u, 0x4D425630u};
        uint32_t r[4];
        orc_philox4x32_10(ctr, key, r);
        double u[4];
        for (int q = 0; q < 4; ++q) u[q] = ((double)r[q] + 0.5) * (1.0 / 4294967296.0);
        const double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
        const double z[3] = {r0 * cos(two_pi * u[1]), r0 * sin(two_pi * u[1]), r1 * cos(two_pi * u[3])};
        const double sd = sqrt(kB * T * ORC_ACC / mass[i]);
        for (int c = 0; c < 3; ++c) v[3 * i + c] = sd * z[c];
    }
    double M = 0, P[3] = {0, 0, 0}, com[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
        M += mass[i];
        for (int c = 0; c < 3; ++c) {
            P[c] += mass[i] * v[3 * i + c];
            com[c] += mass[i] * x[3 * i + c];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int c = 0; c < 3; ++c) v[3 * i + c] -= P[c] / M;
    if (n >= 3) {
        double L[3] = {0, 0, 0}, I[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int c = 0; c < 3; ++c) com[c] /= M;
        for (int i = 0; i < n; ++i) {
            const double r[3] = {x[3 * i] - com[0], x[3 * i + 1] - com[1], x[3 * i + 2] - com[2]};
            const double *vi = v + 3 * i;
            L[0] += mass[i] * (r[1] * vi[2] - r[2] * vi[1]);
            L[1] += mass[i] * (r[2] * vi[0] - r[0] * vi[2]);
            L[2] += mass[i] * (r[0] * vi[1] - r[1] * vi[0]);
            const double rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) I[a][b] += mass[i] * ((a == b ? rr : 0.0) - r[a] * r[b]);
        }
        /* w = I^-1 L by the adjugate */
        const double det = I[0][0] * (I[1][1] * I[2][2] - I[1][2] * I[2][1]) -
                           I[0][1] * (I[1][0] * I[2][2] - I[1][2] * I[2][0]) +
                           I[0][2] * (I[1][0] * I[2][1] - I[1][1] * I[2][0]);
        const double tr = I[0][0] + I[1][1] + I[2][2];
        if (fabs(det) > 1e-12 * tr * tr * tr) {
            double inv[3][3];
            inv[0][0] = (I[1][1] * I[2][2] - I[1][2] * I[2][1]) / det;
            inv[0][1] = (I[0][2] * I[2][1] - I[0][1] * I[2][2]) / det;
            inv[0][2] = (I[0][1] * I[1][2] - I[0][2] * I[1][1]) / det;
            inv[1][0] = (I[1][2] * I[2][0] - I[1][0] * I[2][2]) / det;
            inv[1][1] = (I[0][0] * I[2][2] - I[0][2] * I[2][0]) / det;
            inv[1][2] = (I[0][2] * I[1][0] - I[0][0] * I[1][2]) / det;
            inv[2][0] = (I[1][0] * I[2][1] - I[1][1] * I[2][0]) / det;
            inv[2][1] = (I[0][1] * I[2][0] - I[0][0] * I[2][1]) / det;
            inv[2][2] = (I[0][0] * I[1][1] - I[0][1] * I[1][0]) / det;
            double w[3];
            for (int a = 0; a < 3; ++a) w[a] = inv[a][0] * L[0] + inv[a][1] * L[1] + inv[a][2] * L[2];
            for (int i = 0; i < n; ++i) {
                const double r[3] = {x[3 * i] - com[0], x[3 * i + 1] - com[1], x[3 * i + 2] - com[2]};
                v[3 * i] -= w[1] * r[2] - w[2] * r[1];
                v[3 * i + 1] -= w[2] * r[0] - w[0] * r[2];
                v[3 * i + 2] -= w[0] * r[1] - w[1] * r[0];
            }
        }
    }
    const double K = orc_kinetic(n, mass, v);
    const int dof = 3 * n - 6 > 1 ? 3 * n - 6 : 1;
    const double target = 0.5 * dof * kB * T;
    if (K > 0) {
        const double sc = sqrt(target / K);
        for (int q = 0; q < 3 * n; ++q) v[q] *= sc;
    }
}
