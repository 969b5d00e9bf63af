/*
 * FP64 CPU oracle: AutoDock4 scoring function, gradient and ADADELTA local
 * search, written step by step from the definitions (arxiv 2410.10447,
 * Sec. 2.1, and the force field it names: AutoDock4, Morris et al. 1998;
 * ADADELTA, Zeiler 2012).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA library is compared with.
 * Nothing here is tuned; every sum is a plain left-to-right loop in double
 * precision.  See adgb_oracle.h for the data layout.
 *
 * Readings of points the paper leaves open (the paper names the force field
 * but prints none of its formulas):
 *  - genotype (Sec. 2.1): x,y,z translation (A), rotation axis given by the
 *    azimuth phi and polar angle theta, rotation angle alpha, then one
 *    torsion angle per rotatable bond; 6+T genes;
 *  - every rotation is applied in increment form
 *    r' = r + sin(a) (k x v) + (1 - cos(a)) (k x (k x v)), so a zero angle
 *    leaves a coordinate bit-for-bit unchanged;
 *  - intermolecular energy: trilinear interpolation of the atom type's map,
 *    plus q times the electrostatic map, plus |q| times the desolvation map;
 *    a point outside the grid is clamped onto it and pays 10 kcal/mol/A^2
 *    times its squared distance to the grid;
 *  - intramolecular energy: 12-6 van der Waals (12-10 for donor-acceptor
 *    pairs), Coulomb with the Mehler-Solmajer distance-dependent dielectric,
 *    and the AutoDock4 desolvation term; the singular terms use
 *    max(r, 0.5 A), below which their gradient is zero;
 *  - ADADELTA (Zeiler 2012) moves against the gradient; the best (lowest)
 *    energy seen and its genotype are kept, ties keep the earlier one;
 *    torsion genes are wrapped to [-pi, pi) after each update;
 *  - the Lamarckian GA rules, the Solis-Wets search and the early-stopping
 *    test are this project's readings, written out where they are defined
 *    below.
 *
 * Pins beyond the paper: the Philox4x32-10 generator is checked against the
 * known-answer vectors published with it (Salmon et al., SC'11), so the GA
 * decisions and Solis-Wets deviates drawn from it rest on a pinned stream.
 * Parity unpinned: the GA rules and the Solis-Wets constants themselves have
 * no printed values in the paper to compare with (checked by invariants).
 */
#include "adgb_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

static void cross(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* r += sin(ang) (k x v) + (1 - cos(ang)) (k x (k x v)), v = r - centre */
static void rotate_increment(double r[3], const double centre[3],
                             const double k[3], double s, double omc) {
    double v[3] = {r[0] - centre[0], r[1] - centre[1], r[2] - centre[2]};
    double kv[3], kkv[3];
    cross(k, v, kv);
    cross(k, kv, kkv);
    for (int d = 0; d < 3; d++) r[d] += s * kv[d] + omc * kkv[d];
}

static void axis_from_angles(double phi, double theta, double u[3]) {
    u[0] = sin(theta) * cos(phi);
    u[1] = sin(theta) * sin(phi);
    u[2] = cos(theta);
}

/*
 * Torsioned conformation (Sec. 2.1 genotype, torsion genes psi_k).
 * Torsions are applied root to leaf, each about the CURRENT position of its
 * bond (a->b), so that a later (deeper) torsion turns about an axis already
 * moved by its ancestors.
 */
static int torsion_coords(const orc_ligand *L, const double *genes, double *p) {
    const int N = L->n_atoms, T = L->n_tors;
    memcpy(p, L->xyz, sizeof(double) * 3 * (size_t)N);
    for (int k = 0; k < T; k++) {
        const double *pa = p + 3 * L->tors_bond[2 * k];
        const double *pb = p + 3 * L->tors_bond[2 * k + 1];
        double b[3] = {pb[0], pb[1], pb[2]};
        double ax[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        double len = sqrt(dot(ax, ax));
        if (!(len > 0)) return -1;
        for (int d = 0; d < 3; d++) ax[d] /= len;
        double psi = genes[6 + k];
        double s = sin(psi), omc = 1.0 - cos(psi);
        for (int m = L->mov_off[k]; m < L->mov_off[k + 1]; m++)
            rotate_increment(p + 3 * L->mov_atoms[m], b, ax, s, omc);
    }
    return 0;
}

/* Rigid motion: rotation (phi, theta, alpha) about the frame origin, then t. */
static void rigid_motion(int N, const double *genes, const double *p, double *x) {
    double u[3];
    axis_from_angles(genes[3], genes[4], u);
    double s = sin(genes[5]), omc = 1.0 - cos(genes[5]);
    const double zero[3] = {0, 0, 0};
    memcpy(x, p, sizeof(double) * 3 * (size_t)N);
    for (int i = 0; i < N; i++) {
        rotate_increment(x + 3 * i, zero, u, s, omc);
        for (int d = 0; d < 3; d++) x[3 * i + d] += genes[d];
    }
}

/* Pose -> coordinates: torsions, then rotation about the centre, then translation. */
int orc_pose_coords(const orc_ligand *L, const double *genes, double *x) {
    double *p = (double *)malloc(sizeof(double) * 3 * (size_t)L->n_atoms);
    if (!p) return -2;
    int rc = torsion_coords(L, genes, p);
    if (!rc) rigid_motion(L->n_atoms, genes, p, x);
    free(p);
    return rc;
}

/*
 * Trilinear interpolation of map m at the (already clamped) point p, and its
 * gradient with respect to p.  The 8 corner weights are written out as
 * products of (f) and (1-f) per axis.
 */
static double trilinear(const orc_receptor *R, int m, const double p[3],
                        double grad[3]) {
    const int n[3] = {R->nx, R->ny, R->nz};
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; d++) {
        double u = (p[d] - R->origin[d]) / R->spacing;
        int c = (int)floor(u);
        if (c < 0) c = 0;
        if (c > n[d] - 2) c = n[d] - 2;
        i0[d] = c;
        f[d] = u - c;
    }
    const double *map = R->maps + (size_t)m * R->nx * R->ny * R->nz;
    double val = 0, g[3] = {0, 0, 0};
    for (int cz = 0; cz < 2; cz++)
        for (int cy = 0; cy < 2; cy++)
            for (int cx = 0; cx < 2; cx++) {
                size_t idx = ((size_t)(i0[2] + cz) * R->ny + (i0[1] + cy)) * R->nx
                             + (i0[0] + cx);
                double v = map[idx];
                double wx = cx ? f[0] : 1 - f[0];
                double wy = cy ? f[1] : 1 - f[1];
                double wz = cz ? f[2] : 1 - f[2];
                double sx = cx ? 1.0 : -1.0, sy = cy ? 1.0 : -1.0, sz = cz ? 1.0 : -1.0;
                val += wx * wy * wz * v;
                g[0] += sx * wy * wz * v;
                g[1] += wx * sy * wz * v;
                g[2] += wx * wy * sz * v;
            }
    for (int d = 0; d < 3; d++) grad[d] = g[d] / R->spacing;
    return val;
}

/* Intermolecular energy of one atom and its gradient (reading above). */
static double atom_inter(const orc_receptor *R, int type, double q,
                         const double r[3], double g[3]) {
    const int n[3] = {R->nx, R->ny, R->nz};
    double p[3], pen = 0;
    int inside[3];
    for (int d = 0; d < 3; d++) {
        double lo = R->origin[d], hi = R->origin[d] + (n[d] - 1) * R->spacing;
        p[d] = r[d] < lo ? lo : (r[d] > hi ? hi : r[d]);
        inside[d] = (r[d] >= lo && r[d] <= hi);
        pen += (r[d] - p[d]) * (r[d] - p[d]);
    }
    double gt[3], ge[3], gd[3];
    double vt = trilinear(R, type, p, gt);
    double ve = trilinear(R, R->n_type_maps, p, ge);
    double vd = trilinear(R, R->n_type_maps + 1, p, gd);
    double aq = fabs(q);
    for (int d = 0; d < 3; d++) {
        double gi = inside[d] ? gt[d] + q * ge[d] + aq * gd[d] : 0.0;
        g[d] = gi + 2.0 * ORC_W_OUT * (r[d] - p[d]);
    }
    return vt + q * ve + aq * vd + ORC_W_OUT * pen;
}

/* Mehler-Solmajer distance-dependent dielectric and its derivative. */
static double dielectric(double r, double *deps_dr) {
    const double A = -8.5525, eps0 = 78.4, lam = 0.003627, k = 7.7839;
    const double B = eps0 - A;
    double ex = exp(-lam * B * r);
    double den = 1.0 + k * ex;
    *deps_dr = B * k * lam * B * ex / (den * den);
    return A + B / den;
}

/*
 * Energy of one intramolecular pair at separation vector rv = x_i - x_j,
 * and the gradient with respect to x_i (x_j receives the negative).
 */
static double pair_energy(const orc_ligand *L, int i, int j, const double rv[3],
                          double gi[3]) {
    int ti = L->type[i], tj = L->type[j];
    double r = sqrt(dot(rv, rv));
    double rc = r > ORC_R_MIN ? r : ORC_R_MIN;
    int live = r >= ORC_R_MIN;        /* clamped terms have zero gradient below */
    double e = 0, dedr = 0;
    int hb = (L->hb_role[ti] == 1 && L->hb_role[tj] == 2) ||
             (L->hb_role[ti] == 2 && L->hb_role[tj] == 1);
    if (hb) {
        /* 12-10 hydrogen bond: eps [5 (R/r)^12 - 6 (R/r)^10] */
        double Rh = L->hb_R, eh = L->hb_eps;
        e += ORC_W_HB * eh * (5.0 * pow(Rh / rc, 12) - 6.0 * pow(Rh / rc, 10));
        dedr += ORC_W_HB * eh * (-60.0 * pow(Rh / rc, 12) / rc + 60.0 * pow(Rh / rc, 10) / rc);
    } else {
        /* 12-6 van der Waals, Lorentz-Berthelot mixed: eps [(R/r)^12 - 2 (R/r)^6] */
        double Rij = 0.5 * (L->R[ti] + L->R[tj]);
        double eij = sqrt(L->eps[ti] * L->eps[tj]);
        e += ORC_W_VDW * eij * (pow(Rij / rc, 12) - 2.0 * pow(Rij / rc, 6));
        dedr += ORC_W_VDW * eij * (-12.0 * pow(Rij / rc, 12) / rc + 12.0 * pow(Rij / rc, 6) / rc);
    }
    /* Coulomb with eps(r): C / (r eps(r)) */
    double deps;
    double epsr = dielectric(rc, &deps);
    double C = ORC_W_EL * ORC_ELEC * L->charge[i] * L->charge[j];
    e += C / (rc * epsr);
    dedr += -C * (epsr + rc * deps) / ((rc * epsr) * (rc * epsr));
    if (!live) dedr = 0.0;
    /* desolvation: (S_i V_j + S_j V_i) exp(-r^2 / (2 sigma^2)) */
    double Si = L->solpar[ti] + ORC_QSOL * fabs(L->charge[i]);
    double Sj = L->solpar[tj] + ORC_QSOL * fabs(L->charge[j]);
    double s2 = 2.0 * ORC_DS_SIGMA * ORC_DS_SIGMA;
    double eds = ORC_W_DS * (Si * L->vol[tj] + Sj * L->vol[ti]) * exp(-r * r / s2);
    e += eds;
    for (int d = 0; d < 3; d++) {
        double g = 0;
        if (live) g += dedr * rv[d] / r;
        g += -eds * rv[d] / (ORC_DS_SIGMA * ORC_DS_SIGMA);  /* d/dx_i of exp(-r^2/2s^2) */
        gi[d] = g;
    }
    return e;
}

/* Inter + intra energy of a conformation and dE/dx per atom. */
int orc_energy(const orc_receptor *R, const orc_ligand *L, const double *x,
               double *e_inter, double *e_intra, double *atom_grad) {
    const int N = L->n_atoms;
    double ei = 0, ea = 0;
    for (int i = 0; i < 3 * N; i++) atom_grad[i] = 0;
    for (int i = 0; i < N; i++) {
        double g[3];
        ei += atom_inter(R, L->type[i], L->charge[i], x + 3 * i, g);
        for (int d = 0; d < 3; d++) atom_grad[3 * i + d] += g[d];
    }
    for (int p = 0; p < L->n_pairs; p++) {
        int i = L->pairs[2 * p], j = L->pairs[2 * p + 1];
        double rv[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                        x[3 * i + 2] - x[3 * j + 2]};
        double g[3];
        ea += pair_energy(L, i, j, rv, g);
        for (int d = 0; d < 3; d++) {
            atom_grad[3 * i + d] += g[d];
            atom_grad[3 * j + d] -= g[d];
        }
    }
    *e_inter = ei;
    *e_intra = ea;
    return 0;
}

/*
 * Energy and gradient with respect to the genes (Sec. 2.1: translation,
 * rotation and torsion genes).  Chain rule written out per gene:
 *  - translation: sum of atom gradients;
 *  - rotation genes: sum_i g_i . (dR/dgene) p_i with p_i the torsioned
 *    coordinates and R the increment-form rotation written as a function of
 *    (phi, theta, alpha);
 *  - torsion k: sum over its moving atoms of g_i . (a_k x (x_i - x_b)), the
 *    velocity of atom i when the bond turns, a_k the bond's unit vector in
 *    the final pose.
 */
int orc_score(const orc_receptor *R, const orc_ligand *L, const double *genes,
              double *energy, double *gene_grad, double *xyz_out,
              double *atom_grad) {
    const int N = L->n_atoms, T = L->n_tors;
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *g = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *p = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    if (!x || !g || !p) { free(x); free(g); free(p); return -2; }
    if (torsion_coords(L, genes, p)) { free(x); free(g); free(p); return -1; }
    rigid_motion(N, genes, p, x);
    double ei, ea;
    orc_energy(R, L, x, &ei, &ea, g);
    *energy = ei + ea;
    if (gene_grad) {
        double u[3];
        axis_from_angles(genes[3], genes[4], u);
        double al = genes[5];
        double up[3] = {-sin(genes[4]) * sin(genes[3]), sin(genes[4]) * cos(genes[3]), 0.0};
        double ut[3] = {cos(genes[4]) * cos(genes[3]), cos(genes[4]) * sin(genes[3]), -sin(genes[4])};
        double sa = sin(al), omc = 1.0 - cos(al), ca = cos(al);
        for (int k = 0; k < 6 + T; k++) gene_grad[k] = 0.0;
        for (int i = 0; i < N; i++) {
            const double *pi = p + 3 * i, *gi = g + 3 * i;
            for (int d = 0; d < 3; d++) gene_grad[d] += gi[d];
            /* dR/dphi p = sin a (u_phi x p) + (1-cos a)(u_phi x (u x p) + u x (u_phi x p)) */
            double t1[3], t2[3], t3[3], t4[3], v[3];
            cross(up, pi, t1);
            cross(u, pi, t2);
            cross(up, t2, t3);
            cross(u, t1, t4);
            for (int d = 0; d < 3; d++) v[d] = sa * t1[d] + omc * (t3[d] + t4[d]);
            gene_grad[3] += dot(gi, v);
            cross(ut, pi, t1);
            cross(ut, t2, t3);
            cross(u, t1, t4);
            for (int d = 0; d < 3; d++) v[d] = sa * t1[d] + omc * (t3[d] + t4[d]);
            gene_grad[4] += dot(gi, v);
            /* dR/dalpha p = cos a (u x p) + sin a (u x (u x p)) */
            cross(u, t2, t3);
            for (int d = 0; d < 3; d++) v[d] = ca * t2[d] + sa * t3[d];
            gene_grad[5] += dot(gi, v);
        }
        for (int k = 0; k < T; k++) {
            const double *xa = x + 3 * L->tors_bond[2 * k];
            const double *xb = x + 3 * L->tors_bond[2 * k + 1];
            double ax[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
            double len = sqrt(dot(ax, ax));
            for (int d = 0; d < 3; d++) ax[d] /= len;
            double acc = 0;
            for (int m = L->mov_off[k]; m < L->mov_off[k + 1]; m++) {
                int i = L->mov_atoms[m];
                double v[3] = {x[3 * i] - xb[0], x[3 * i + 1] - xb[1], x[3 * i + 2] - xb[2]};
                double vel[3];
                cross(ax, v, vel);
                acc += dot(g + 3 * i, vel);
            }
            gene_grad[6 + k] = acc;
        }
    }
    if (xyz_out) memcpy(xyz_out, x, sizeof(double) * 3 * (size_t)N);
    if (atom_grad) memcpy(atom_grad, g, sizeof(double) * 3 * (size_t)N);
    free(x);
    free(g);
    free(p);
    return 0;
}

/*
 * Magnitude of every gene-gradient component: the chain rule of orc_score
 * applied to the absolute values of all its contributions (each map corner's
 * share of an atom's grid gradient, the out-of-grid wall, every term of every
 * pair force, and every lever arm).  A floating-point evaluation in unit
 * roundoff u of the same sums has an error of order u times this magnitude,
 * so |g_j| / A_j says how many relative digits of g_j survive cancellation
 * (test infrastructure: it sets where a relative tolerance is meaningful).
 */
static void trilinear_abs(const orc_receptor *R, int m, double w, const double p[3],
                          double ag[3]) {
    const int n[3] = {R->nx, R->ny, R->nz};
    int i0[3];
    double f[3];
    for (int d = 0; d < 3; d++) {
        double u = (p[d] - R->origin[d]) / R->spacing;
        int c = (int)floor(u);
        if (c < 0) c = 0;
        if (c > n[d] - 2) c = n[d] - 2;
        i0[d] = c;
        f[d] = u - c;
    }
    const double *map = R->maps + (size_t)m * R->nx * R->ny * R->nz;
    for (int cz = 0; cz < 2; cz++)
        for (int cy = 0; cy < 2; cy++)
            for (int cx = 0; cx < 2; cx++) {
                size_t idx = ((size_t)(i0[2] + cz) * R->ny + (i0[1] + cy)) * R->nx + (i0[0] + cx);
                double v = fabs(w * map[idx]) / R->spacing;
                double wx = cx ? f[0] : 1 - f[0];
                double wy = cy ? f[1] : 1 - f[1];
                double wz = cz ? f[2] : 1 - f[2];
                ag[0] += wy * wz * v;
                ag[1] += wx * wz * v;
                ag[2] += wx * wy * v;
            }
}

/* pos_mag (may be NULL): the same chain rule over the contributions'
 * sensitivity to rounding the coordinates - a coordinate of magnitude |x| is
 * off by about u |x|, which moves every pair force by its derivative times
 * that and every lever arm by that (stiff r^-12 terms amplify it; the
 * forces' errors cancel in the rigid-body sums by Newton's third law but not
 * over a torsion's moving set). */
int orc_score_magnitude(const orc_receptor *R, const orc_ligand *L, const double *genes,
                        double *mag, double *pos_mag) {
    const int N = L->n_atoms, T = L->n_tors;
    double *x = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *p = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    double *ag = (double *)calloc(3 * (size_t)N, sizeof(double));
    double *pg = (double *)calloc((size_t)L->n_pairs + 1, sizeof(double));   /* per pair */
    if (!x || !p || !ag || !pg) { free(x); free(p); free(ag); free(pg); return -2; }
    if (torsion_coords(L, genes, p)) { free(x); free(p); free(ag); free(pg); return -1; }
    rigid_motion(N, genes, p, x);
    const int n[3] = {R->nx, R->ny, R->nz};
    double *xs = (double *)malloc(sizeof(double) * (size_t)N);   /* coordinate scale |x|_inf */
    if (!xs) { free(x); free(p); free(ag); free(pg); return -2; }
    for (int i = 0; i < N; i++) {
        xs[i] = 0.0;
        for (int d = 0; d < 3; d++) xs[i] = fmax(xs[i], fabs(x[3 * i + d]));
    }
    for (int i = 0; i < N; i++) {
        double q = L->charge[i], pc[3];
        int inside[3];
        for (int d = 0; d < 3; d++) {
            double lo = R->origin[d], hi = R->origin[d] + (n[d] - 1) * R->spacing;
            pc[d] = x[3 * i + d] < lo ? lo : (x[3 * i + d] > hi ? hi : x[3 * i + d]);
            inside[d] = (x[3 * i + d] >= lo && x[3 * i + d] <= hi);
        }
        double t[3] = {0, 0, 0};
        trilinear_abs(R, L->type[i], 1.0, pc, t);
        trilinear_abs(R, R->n_type_maps, q, pc, t);
        trilinear_abs(R, R->n_type_maps + 1, fabs(q), pc, t);
        for (int d = 0; d < 3; d++)
            ag[3 * i + d] += (inside[d] ? t[d] : 0.0) + fabs(2.0 * ORC_W_OUT * (x[3 * i + d] - pc[d]));
    }
    for (int k = 0; k < L->n_pairs; k++) {
        int i = L->pairs[2 * k], j = L->pairs[2 * k + 1];
        int ti = L->type[i], tj = L->type[j];
        double rv[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
        double r = sqrt(dot(rv, rv));
        double rc = r > ORC_R_MIN ? r : ORC_R_MIN;
        int hb = (L->hb_role[ti] == 1 && L->hb_role[tj] == 2) ||
                 (L->hb_role[ti] == 2 && L->hb_role[tj] == 1);
        double a = 0;    /* |dE/dr| summed term by term */
        double a2 = 0;   /* |d2E/dr2| summed term by term */
        if (hb) {
            double Rh = L->hb_R, eh = L->hb_eps;
            a += fabs(ORC_W_HB * eh) * (60.0 * pow(Rh / rc, 12) + 60.0 * pow(Rh / rc, 10)) / rc;
            a2 += fabs(ORC_W_HB * eh) * (780.0 * pow(Rh / rc, 12) + 660.0 * pow(Rh / rc, 10)) / (rc * rc);
        } else {
            double Rij = 0.5 * (L->R[ti] + L->R[tj]), eij = sqrt(L->eps[ti] * L->eps[tj]);
            a += fabs(ORC_W_VDW * eij) * (12.0 * pow(Rij / rc, 12) + 12.0 * pow(Rij / rc, 6)) / rc;
            a2 += fabs(ORC_W_VDW * eij) * (156.0 * pow(Rij / rc, 12) + 84.0 * pow(Rij / rc, 6)) / (rc * rc);
        }
        double deps, epsr = dielectric(rc, &deps);
        double C = ORC_W_EL * ORC_ELEC * L->charge[i] * L->charge[j];
        a += fabs(C) * (fabs(epsr) + rc * fabs(deps)) / ((rc * epsr) * (rc * epsr));
        /* C / (r eps): second derivative bounded term by term (eps'' ~ lambda B eps') */
        a2 += fabs(C) * (2.0 / (rc * rc * rc * fabs(epsr)) + 4.0 * fabs(deps) / (rc * rc * epsr * epsr)
                         + 2.0 * deps * deps / (rc * fabs(epsr * epsr * epsr))
                         + 0.003627 * 86.9525 * fabs(deps) / (rc * epsr * epsr));
        if (r < ORC_R_MIN) a = a2 = 0.0;
        double Si = L->solpar[ti] + ORC_QSOL * fabs(L->charge[i]);
        double Sj = L->solpar[tj] + ORC_QSOL * fabs(L->charge[j]);
        double s2 = 2.0 * ORC_DS_SIGMA * ORC_DS_SIGMA;
        double ads = fabs(ORC_W_DS * (Si * L->vol[tj] + Sj * L->vol[ti])) * exp(-r * r / s2);
        const double sg2 = ORC_DS_SIGMA * ORC_DS_SIGMA;
        a2 += ads * (r * r / (sg2 * sg2) + 1.0 / sg2);
        const double X = xs[i] + xs[j];   /* rounding of the separation: about u X */
        for (int d = 0; d < 3; d++) {
            double m = (r > 0 ? a * fabs(rv[d]) / r : 0.0) + ads * fabs(rv[d]) / sg2;
            ag[3 * i + d] += m;
            ag[3 * j + d] += m;
        }
        /* the force's change under that rounding, per component: its
         * magnitude's derivative along the separation plus its turn
         * (|dE/dr| / r), and the desolvation force's own */
        pg[k] = (a2 + (r > 0 ? a / r : 0.0) + ads / sg2) * X;
    }
    /* the chain rule of orc_score with absolute values */
    double u[3];
    axis_from_angles(genes[3], genes[4], u);
    double al = genes[5];
    double up[3] = {-sin(genes[4]) * sin(genes[3]), sin(genes[4]) * cos(genes[3]), 0.0};
    double ut[3] = {cos(genes[4]) * cos(genes[3]), cos(genes[4]) * sin(genes[3]), -sin(genes[4])};
    double sa = sin(al), omc = 1.0 - cos(al), ca = cos(al);
    /* velocity of atom i under each gene (the chain rule's factors) */
    double *vel = (double *)calloc(3 * (size_t)N * (6 + T), sizeof(double));
    if (!vel) { free(x); free(p); free(ag); free(pg); free(xs); return -2; }
#define VEL(i, k) (vel + 3 * ((size_t)(k) * N + (i)))
    for (int i = 0; i < N; i++) {
        const double *pi = p + 3 * i;
        for (int d = 0; d < 3; d++) VEL(i, d)[d] = 1.0;
        double t1[3], t2[3], t3[3], t4[3];
        cross(up, pi, t1);
        cross(u, pi, t2);
        cross(up, t2, t3);
        cross(u, t1, t4);
        for (int d = 0; d < 3; d++) VEL(i, 3)[d] = sa * t1[d] + omc * (t3[d] + t4[d]);
        cross(ut, pi, t1);
        cross(ut, t2, t3);
        cross(u, t1, t4);
        for (int d = 0; d < 3; d++) VEL(i, 4)[d] = sa * t1[d] + omc * (t3[d] + t4[d]);
        cross(u, t2, t3);
        for (int d = 0; d < 3; d++) VEL(i, 5)[d] = ca * t2[d] + sa * t3[d];
    }
    double *axl = (double *)malloc(sizeof(double) * (T > 0 ? T : 1));
    if (!axl) { free(vel); free(x); free(p); free(ag); free(pg); free(xs); return -2; }
    for (int k = 0; k < T; k++) {
        const double *xa = x + 3 * L->tors_bond[2 * k], *xb = x + 3 * L->tors_bond[2 * k + 1];
        double ax[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
        double len = sqrt(dot(ax, ax));
        axl[k] = len;
        for (int d = 0; d < 3; d++) ax[d] /= len;
        for (int m = L->mov_off[k]; m < L->mov_off[k + 1]; m++) {
            int i = L->mov_atoms[m];
            double v[3] = {x[3 * i] - xb[0], x[3 * i + 1] - xb[1], x[3 * i + 2] - xb[2]};
            cross(ax, v, VEL(i, 6 + k));
        }
    }
    /* pass 0: |contribution| sums */
    for (int k = 0; k < 6 + T; k++) {
        double acc = 0;
        for (int i = 0; i < N; i++)
            for (int d = 0; d < 3; d++) acc += ag[3 * i + d] * fabs(VEL(i, k)[d]);
        mag[k] = acc;
    }
    /* pass 1: coordinate rounding - every pair force's change enters a gene
     * through the difference of its atoms' velocities (it cancels in the
     * translation; pairs inside a torsion's moving set see only their
     * separation), the lever arms round by about u |x|, and a torsion's axis
     * turns by about u (|x_a| + |x_b|) / |x_b - x_a| */
    if (pos_mag) {
        for (int k = 0; k < 6 + T; k++) {
            double acc = 0;
            for (int q = 0; q < L->n_pairs; q++) {
                const int i = L->pairs[2 * q], j = L->pairs[2 * q + 1];
                for (int d = 0; d < 3; d++) acc += pg[q] * fabs(VEL(i, k)[d] - VEL(j, k)[d]);
            }
            if (k >= 3) {
                const double xb = k >= 6 ? xs[L->tors_bond[2 * (k - 6) + 1]] : 0.0;
                for (int i = 0; i < N; i++) {
                    const double *vi = VEL(i, k);
                    if (k >= 6 && vi[0] == 0.0 && vi[1] == 0.0 && vi[2] == 0.0) continue;
                    for (int d = 0; d < 3; d++) acc += ag[3 * i + d] * (xs[i] + xb);
                }
            }
            if (k >= 6) {
                const int ka = L->tors_bond[2 * (k - 6)], kb = L->tors_bond[2 * (k - 6) + 1];
                acc += mag[k] * (xs[ka] + xs[kb]) / axl[k - 6];
            }
            pos_mag[k] = acc;
        }
    }
#undef VEL
    free(vel);
    free(axl);
    free(x);
    free(p);
    free(ag);
    free(pg);
    free(xs);
    return 0;
}

static double wrap_angle(double a) {
    return a - 2.0 * PI * floor((a + PI) / (2.0 * PI));
}

/*
 * One ADADELTA update (Zeiler 2012, Algorithm 1; Sec. 2.1 writes it as
 * Omega_{t+1} = Omega_t + eta_t g_t).  The step is taken against the
 * gradient:
 *   E[g^2]  <- rho E[g^2]  + (1-rho) g^2
 *   d       <- -sqrt(E[d^2] + eps) / sqrt(E[g^2] + eps) * g
 *   E[d^2]  <- rho E[d^2]  + (1-rho) d^2
 *   Omega   <- Omega + d      (torsion genes wrapped to [-pi, pi))
 */
int orc_adadelta_step(int G, const double *grad, double rho, double eps,
                      double *genes, double *eg2, double *ed2) {
    for (int j = 0; j < G; j++) {
        eg2[j] = rho * eg2[j] + (1.0 - rho) * grad[j] * grad[j];
        double d = -sqrt(ed2[j] + eps) / sqrt(eg2[j] + eps) * grad[j];
        ed2[j] = rho * ed2[j] + (1.0 - rho) * d * d;
        genes[j] += d;
        if (j >= 6) genes[j] = wrap_angle(genes[j]);
    }
    return 0;
}

/*
 * ADADELTA local search of one genotype: `iters` energy+gradient
 * evaluations, each followed by one update; the lowest energy seen and the
 * genotype it was seen at are returned (genes is overwritten with it).
 * state, if given, is [3][G] = (Omega, E[g^2], E[d^2]) after the last update;
 * with resume != 0 the search starts from state instead of (genes, 0, 0).
 */
int orc_local_search(const orc_receptor *R, const orc_ligand *L, double *genes,
                     int iters, double rho, double eps, int resume,
                     double *state, double *best_energy) {
    const int G = 6 + L->n_tors;
    double *om = (double *)calloc((size_t)G * 5, sizeof(double));
    if (!om) return -2;
    double *eg2 = om + G, *ed2 = om + 2 * G, *grad = om + 3 * G, *best = om + 4 * G;
    if (resume && state) {
        memcpy(om, state, sizeof(double) * G);
        memcpy(eg2, state + G, sizeof(double) * G);
        memcpy(ed2, state + 2 * G, sizeof(double) * G);
    } else {
        memcpy(om, genes, sizeof(double) * G);
    }
    memcpy(best, om, sizeof(double) * G);
    double best_e = INFINITY;
    int rc = 0;
    for (int t = 0; t < iters; t++) {
        double e;
        rc = orc_score(R, L, om, &e, grad, NULL, NULL);
        if (rc) break;
        if (e < best_e) {
            best_e = e;
            memcpy(best, om, sizeof(double) * G);
        }
        orc_adadelta_step(G, grad, rho, eps, om, eg2, ed2);
    }
    memcpy(genes, best, sizeof(double) * G);
    if (state) {
        memcpy(state, om, sizeof(double) * G);
        memcpy(state + G, eg2, sizeof(double) * G);
        memcpy(state + 2 * G, ed2, sizeof(double) * G);
    }
    *best_energy = best_e;
    free(om);
    return rc;
}

/* Independent local searches over n genotypes ([n][G]), spread over threads. */
int orc_local_search_batch(const orc_receptor *R, const orc_ligand *L, int n,
                           double *genes, int iters, double rho, double eps,
                           double *best_energy, int nthreads) {
    const int G = 6 + L->n_tors;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int p = 0; p < n; p++)
        bad |= orc_local_search(R, L, genes + (size_t)p * G, iters, rho, eps, 0,
                                NULL, best_energy + p) != 0;
    (void)nthreads;
    return bad ? -1 : 0;
}

int orc_score_batch(const orc_receptor *R, const orc_ligand *L, int n,
                    const double *genes, double *energy, double *gene_grad,
                    int nthreads) {
    const int G = 6 + L->n_tors;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
#endif
    for (int p = 0; p < n; p++)
        bad |= orc_score(R, L, genes + (size_t)p * G, energy + p,
                         gene_grad ? gene_grad + (size_t)p * G : NULL, NULL, NULL) != 0;
    (void)nthreads;
    return bad ? -1 : 0;
}

/* Plain left-to-right sum (the definition of the reduction, Sec. 4.2). */
double orc_sum_naive(const double *x, long n, long stride) {
    double s = 0;
    for (long i = 0; i < n; i++) s += x[i * stride];
    return s;
}

/*
 * Neumaier's compensated summation (Neumaier 1974): carries the rounding
 * error of every addition in a second accumulator; the result is the exact
 * sum rounded once, up to O(n u^2) effects.
 */
double orc_sum_neumaier(const double *x, long n, long stride) {
    double s = 0, c = 0;
    for (long i = 0; i < n; i++) {
        double v = x[i * stride];
        double t = s + v;
        if (fabs(s) >= fabs(v))
            c += (s - t) + v;
        else
            c += (v - t) + s;
        s = t;
    }
    return s + c;
}

/* ------------------------------------------------------------------------
 * Lamarckian GA (Sec. 2.1: a GA does the global search and every genotype it
 * produces is refined by the local search).  The paper prints none of the
 * GA's rules; this is the project's reading, written once here and once,
 * independently, in the CUDA library:
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed, counter
 *    = (individual, generation, run, call); each call yields four 32-bit
 *    words, consumed in a fixed order; u(x) = (x >> 8) * 2^-24 in [0,1);
 *    an index below n is (x * n) >> 32;
 *  - initial genotype: translation uniform in the central 60% of the grid
 *    box, axis angles phi = 2 pi u - pi, theta = acos(1 - 2u), angle
 *    alpha = 2 pi u, torsions 2 pi u - pi;
 *  - new generation: individual 0 is the previous generation's best
 *    (elitism); every other child takes two binary tournaments (the lower
 *    energy wins, ties to the lower index), two-point crossover with
 *    probability p_cross (cut points c1 <= c2 drawn in 0..G, genes
 *    [c1, c2) from the second parent), then each gene mutates with
 *    probability p_mut by a uniform offset in [-1, 1) times mut_trans (A)
 *    or mut_angle (rad); torsion genes are wrapped to [-pi, pi);
 *  - each individual is locally searched with probability ls_rate
 *    (ls_iters evaluations), otherwise scored once (one evaluation);
 *  - a run stops after max_gens generations or once its evaluations reach
 *    max_evals; its result is the lowest energy ever seen.
 * ------------------------------------------------------------------------ */

static uint32_t mulhilo32(uint32_t a, uint32_t b, uint32_t *hi) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    return (uint32_t)p;
}

/* Philox4x32 with 10 rounds: each round multiplies words 0 and 2 by the
 * two round multipliers, mixes the high halves with the other words and
 * the key, and the key is bumped by the two Weyl constants between rounds. */
void orc_philox4x32_10(const unsigned int ctr[4], const unsigned int key[2], unsigned int out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0, hi1;
        uint32_t lo0 = mulhilo32(0xD2511F53u, c0, &hi0);
        uint32_t lo1 = mulhilo32(0xCD9E8D57u, c2, &hi1);
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* word w of the stream (individual k, generation gen, run) */
static uint32_t draw(unsigned long long seed, int run, int gen, int k, int w) {
    unsigned int ctr[4] = {(unsigned)k, (unsigned)gen, (unsigned)run, (unsigned)(w / 4)};
    unsigned int key[2] = {(unsigned)(seed & 0xffffffffu), (unsigned)(seed >> 32)};
    unsigned int out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[w % 4];
}

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }
static int below(uint32_t x, int n) { return (int)(((uint64_t)x * (uint64_t)n) >> 32); }

#define INIT_GEN 0xFFFFFFFF

int orc_init_individual(const orc_receptor *R, int n_tors, unsigned long long seed, int run,
                        int k, double *genes) {
    const int n[3] = {R->nx, R->ny, R->nz};
    for (int d = 0; d < 3; d++) {
        double ext = (n[d] - 1) * R->spacing;
        genes[d] = R->origin[d] + ext * (0.2 + 0.6 * u01(draw(seed, run, (int)INIT_GEN, k, d)));
    }
    genes[3] = 2.0 * PI * u01(draw(seed, run, (int)INIT_GEN, k, 3)) - PI;
    genes[4] = acos(1.0 - 2.0 * u01(draw(seed, run, (int)INIT_GEN, k, 4)));
    genes[5] = 2.0 * PI * u01(draw(seed, run, (int)INIT_GEN, k, 5));
    for (int j = 0; j < n_tors; j++)
        genes[6 + j] = 2.0 * PI * u01(draw(seed, run, (int)INIT_GEN, k, 6 + j)) - PI;
    return 0;
}

/* words of child k: 0-3 tournaments, 4 crossover?, 5-6 cuts, 7 local search?,
 * 8 + 2j mutate gene j?, 9 + 2j its offset */
int orc_ga_generation(int G, int pop, const double *go, const double *eo,
                      const orc_dock_params *p, int run, int gen, double *gn, int *ls_flag) {
    int best = 0;
    for (int k = 1; k < pop; k++)
        if (eo[k] < eo[best]) best = k;
    for (int k = 0; k < pop; k++) {
        double *child = gn + (size_t)k * G;
        if (k == 0) {
            memcpy(child, go + (size_t)best * G, sizeof(double) * G);
        } else {
            int par[2];
            for (int t = 0; t < 2; t++) {
                int a = below(draw(p->seed, run, gen, k, 2 * t), pop);
                int b = below(draw(p->seed, run, gen, k, 2 * t + 1), pop);
                par[t] = (eo[b] < eo[a] || (eo[b] == eo[a] && b < a)) ? b : a;
            }
            const double *A = go + (size_t)par[0] * G, *B = go + (size_t)par[1] * G;
            int c1 = 0, c2 = 0;
            if (u01(draw(p->seed, run, gen, k, 4)) < p->p_cross) {
                c1 = below(draw(p->seed, run, gen, k, 5), G + 1);
                c2 = below(draw(p->seed, run, gen, k, 6), G + 1);
                if (c1 > c2) { int t = c1; c1 = c2; c2 = t; }
            }
            for (int j = 0; j < G; j++) child[j] = (j >= c1 && j < c2) ? B[j] : A[j];
            for (int j = 0; j < G; j++) {
                if (u01(draw(p->seed, run, gen, k, 8 + 2 * j)) < p->p_mut) {
                    double off = 2.0 * u01(draw(p->seed, run, gen, k, 9 + 2 * j)) - 1.0;
                    child[j] += off * (j < 3 ? p->mut_trans : p->mut_angle);
                }
                if (j >= 6) child[j] = wrap_angle(child[j]);
            }
        }
        ls_flag[k] = u01(draw(p->seed, run, gen, k, 7)) < p->ls_rate;
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Solis-Wets local search (Solis and Wets, "Minimization by random search
 * techniques", Math. Oper. Res. 6, 1981; AutoDock's derivative-free local
 * search).  This project's reading, step by step:
 *   x: genotype, E(x) its energy, bias b (zero at the start), scale rho.
 *   One step: d_j = b_j + rho * s_j * z_j with z_j standard normal and
 *   s_j = 1 (translation genes, A) or angle_scale (angles, rad).
 *   If E(x + d) < E(x): x <- x + d, b <- 0.2 b + 0.4 d (success).
 *   Else if E(x - d) < E(x): x <- x - d, b <- b - 0.4 d (success).
 *   Else b <- 0.5 b (failure).
 *   max_succ successes in a row: rho <- 2 rho; max_fail failures in a row:
 *   rho <- rho / 2.  Stop after max_evals evaluations or when rho < rho_min.
 * Torsions are wrapped to [-pi, pi) after every move.  The normal numbers
 * come from Philox4x32-10 (key = seed, counter = (genotype, step,
 * 0x5357 << 16 | call, j / 4)) by the Box-Muller transform of two 24-bit
 * uniforms u1 = ((w >> 8) + 1) 2^-24, u2 = (w' >> 8) 2^-24.
 * ------------------------------------------------------------------------ */
double orc_sw_normal(unsigned long long seed, unsigned int genotype, unsigned int step,
                     unsigned int call, int j) {
    const unsigned int ctr[4] = {genotype, step, 0x53570000u | (call & 0xFFFFu), (unsigned int)j >> 2};
    const unsigned int key[2] = {(unsigned int)seed, (unsigned int)(seed >> 32)};
    unsigned int o[4];
    orc_philox4x32_10(ctr, key, o);
    const int second = (j >> 1) & 1;
    const unsigned int a = second ? o[2] : o[0], b = second ? o[3] : o[1];
    const double u1 = (double)((a >> 8) + 1u) / 16777216.0;
    const double u2 = (double)(b >> 8) / 16777216.0;
    const double r = sqrt(-2.0 * log(u1));
    return (j & 1) ? r * sin(2.0 * PI * u2) : r * cos(2.0 * PI * u2);
}

int orc_sw_search(const orc_receptor *R, const orc_ligand *L, double *genes,
                  const orc_sw_params *p, int genotype, int resume, double *state,
                  double *energy, int *evals_out) {
    const int G = 6 + L->n_tors;
    double *x = (double *)malloc(sizeof(double) * 4 * (size_t)G);
    double *b = x + G, *d = x + 2 * G, *y = x + 3 * G;
    double rho, ex;
    int ns, nf, step, evals = 0, bad = 0;
    if (resume) {
        for (int j = 0; j < G; j++) { x[j] = state[j]; b[j] = state[G + j]; }
        rho = state[2 * G];
        ns = (int)state[2 * G + 1];
        nf = (int)state[2 * G + 2];
        ex = state[2 * G + 3];
        step = (int)state[2 * G + 4];
    } else {
        for (int j = 0; j < G; j++) { x[j] = genes[j]; b[j] = 0.0; }
        rho = p->rho0;
        ns = nf = step = 0;
        ex = INFINITY;
        if (p->max_evals > 0) {
            bad |= orc_score(R, L, x, &ex, NULL, NULL, NULL) != 0;
            evals = 1;
        }
    }
    while (evals < p->max_evals && rho >= p->rho_min) {
        for (int j = 0; j < G; j++) {
            const double z = orc_sw_normal(p->seed, (unsigned int)genotype, (unsigned int)step,
                                           (unsigned int)p->call, j);
            d[j] = b[j] + rho * (j < 3 ? 1.0 : p->angle_scale) * z;
            y[j] = x[j] + d[j];
            if (j >= 6) y[j] = wrap_angle(y[j]);
        }
        double e1;
        bad |= orc_score(R, L, y, &e1, NULL, NULL, NULL) != 0;
        evals++;
        int ok = e1 < ex;
        if (ok) {
            ex = e1;
            for (int j = 0; j < G; j++) { x[j] = y[j]; b[j] = 0.2 * b[j] + 0.4 * d[j]; }
        } else if (evals < p->max_evals) {
            for (int j = 0; j < G; j++) {
                y[j] = x[j] - d[j];
                if (j >= 6) y[j] = wrap_angle(y[j]);
            }
            double e2;
            bad |= orc_score(R, L, y, &e2, NULL, NULL, NULL) != 0;
            evals++;
            ok = e2 < ex;
            if (ok) {
                ex = e2;
                for (int j = 0; j < G; j++) { x[j] = y[j]; b[j] = b[j] - 0.4 * d[j]; }
            }
        }
        if (!ok)
            for (int j = 0; j < G; j++) b[j] *= 0.5;
        if (ok) { ns++; nf = 0; } else { nf++; ns = 0; }
        if (ns >= p->max_succ) { rho *= 2.0; ns = 0; }
        if (nf >= p->max_fail) { rho *= 0.5; nf = 0; }
        step++;
    }
    for (int j = 0; j < G; j++) genes[j] = x[j];
    if (state) {
        for (int j = 0; j < G; j++) { state[j] = x[j]; state[G + j] = b[j]; }
        state[2 * G] = rho;
        state[2 * G + 1] = ns;
        state[2 * G + 2] = nf;
        state[2 * G + 3] = ex;
        state[2 * G + 4] = step;
    }
    *energy = ex;
    if (evals_out) *evals_out = evals;
    free(x);
    return bad ? -1 : 0;
}

/* Early stopping, this project's reading (Sec. 5.3 speaks of runs that do
 * or do not converge without defining the test): the population standard
 * deviation of the `top` lowest energies is below tol.  Written as the
 * definition: sort, take the lowest `top`, mean, mean squared deviation. */
static int cmp_double(const void *a, const void *b) {
    const double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

int orc_converged(int pop, const double *energy, int top, double tol) {
    if (top < 1 || top > pop) return 0;
    for (int k = 0; k < pop; k++)
        if (isnan(energy[k])) return 0;   /* no order, no test */
    double *e = (double *)malloc(sizeof(double) * (size_t)pop);
    memcpy(e, energy, sizeof(double) * (size_t)pop);
    qsort(e, (size_t)pop, sizeof(double), cmp_double);
    int finite_all = 1;
    double mean = 0.0;
    for (int k = 0; k < top; k++) {
        if (!isfinite(e[k])) finite_all = 0;
        mean += e[k];
    }
    mean /= top;
    double var = 0.0;
    for (int k = 0; k < top; k++) var += (e[k] - mean) * (e[k] - mean);
    var /= top;
    free(e);
    return finite_all && var < tol * tol;
}

/* Whole Lamarckian GA of every run (Sec. 2.1); slow, for small cases. */
int orc_dock(const orc_receptor *R, const orc_ligand *L, const orc_dock_params *p,
             double *best_genes, double *best_energy, long long *evals, int nthreads) {
    const int G = 6 + L->n_tors, P = p->pop;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
#endif
    for (int r = 0; r < p->n_runs; r++) {
        double *ga = (double *)malloc(sizeof(double) * (size_t)P * G);
        double *gb = (double *)malloc(sizeof(double) * (size_t)P * G);
        double *e = (double *)malloc(sizeof(double) * (size_t)P);
        int *fl = (int *)malloc(sizeof(int) * (size_t)P);
        double *bg = best_genes + (size_t)r * G;
        double be = INFINITY;
        long long ev = 0;
        for (int k = 0; k < P; k++) {
            orc_init_individual(R, L->n_tors, p->seed, r, k, ga + (size_t)k * G);
            bad |= orc_score(R, L, ga + (size_t)k * G, e + k, NULL, NULL, NULL) != 0;
            ev++;
            if (e[k] < be) { be = e[k]; memcpy(bg, ga + (size_t)k * G, sizeof(double) * G); }
        }
        for (int gen = 1; gen <= p->max_gens && ev < p->max_evals; gen++) {
            orc_ga_generation(G, P, ga, e, p, r, gen, gb, fl);
            for (int k = 0; k < P; k++) {
                double *gk = gb + (size_t)k * G;
                int it = fl[k] ? p->ls_iters : 1;
                if (p->ls_method == 1) {
                    /* Solis-Wets: genotype r * P + k, call = generation mod 2^16 */
                    orc_sw_params sw = {it, p->sw_max_succ, p->sw_max_fail, p->sw_rho0,
                                        p->sw_rho_min, p->sw_angle_scale, p->seed, gen & 0xFFFF};
                    bad |= orc_sw_search(R, L, gk, &sw, r * P + k, 0, NULL, e + k, &it) != 0;
                } else {
                    bad |= orc_local_search(R, L, gk, it, p->rho, p->eps, 0, NULL, e + k) != 0;
                }
                ev += it;
                if (e[k] < be) { be = e[k]; memcpy(bg, gk, sizeof(double) * G); }
            }
            double *t = ga; ga = gb; gb = t;
            if (p->conv_every > 0 && gen % p->conv_every == 0 &&
                orc_converged(P, e, p->conv_top, p->conv_tol))
                break;
        }
        best_energy[r] = be;
        if (evals) evals[r] = ev;
        free(ga); free(gb); free(e); free(fl);
    }
    (void)nthreads;
    return bad ? -1 : 0;
}
