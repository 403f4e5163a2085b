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

#define ORC_ACC 4.184e-4 /* kcal/mol/A/amu -> A/fs^2 (1 kcal/mol = 4.184e-4 amu A^2/fs^2) */

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
    for (int i = 0; i < n; ++i) {
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
            elj += e_lj;
            ec += e_c;
            /* dE/dr = (-48 eps sr12 + 24 eps sr6)/r - e_c/r */
            double dedr = (-48.0 * eps * sr12 + 24.0 * eps * sr6) / r - e_c / r;
            double g = dedr / r;                   /* F_i = +dE/dr * d/r, F_j = -F_i */
            for (int c = 0; c < 3; ++c) { f[3 * i + c] += g * d[c]; f[3 * j + c] -= g * d[c]; }
        }
    }
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
