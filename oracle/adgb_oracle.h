/*
 * FP64 CPU oracle for the AutoDock4 scoring function, its gradient and the
 * ADADELTA local search (arxiv 2410.10447, Sec. 2.1).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, plain reference that the CUDA
 * library is checked against.  It shares no code, header, table or helper
 * with the CUDA path, and only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Parity status: every function below is pinned by tests that do not go
 * through the oracle's own formulas (finite differences, closed forms,
 * invariants, brute force).  The GA, serving and rescoring parts are not
 * here: they are built from the same scoring call.
 */
#ifndef ADGB_ORACLE_H
#define ADGB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny, nz;          /* grid points per axis (>= 2) */
    int n_type_maps;         /* affinity maps; map n_type_maps = e, +1 = d */
    double spacing;          /* A between grid points */
    double origin[3];        /* position of grid point (0,0,0) */
    const double *maps;      /* [n_type_maps+2][nz][ny][nx] */
} orc_receptor;

typedef struct {
    int n_atoms, n_tors, n_pairs, n_types;
    const int *type;         /* [N] atom type = affinity map index */
    const double *charge;    /* [N] partial charge (e) */
    const double *xyz;       /* [N][3] reference conformation, rotation centre at 0 */
    const int *tors_bond;    /* [T][2] (a,b): axis a->b, root to leaf order */
    const int *mov_off;      /* [T+1] offsets into mov_atoms */
    const int *mov_atoms;    /* atoms moved by torsion k: mov_atoms[mov_off[k]..] */
    const int *pairs;        /* [n_pairs][2] intramolecular pairs */
    const double *R, *eps, *vol, *solpar; /* [n_types] force-field parameters */
    const int *hb_role;      /* [n_types] 0 none, 1 donor, 2 acceptor */
    double hb_R, hb_eps;     /* 12-10 parameters of donor-acceptor pairs */
} orc_ligand;

/* force-field constants (AutoDock4.2 free-energy model) */
#define ORC_W_VDW 0.1662
#define ORC_W_HB 0.1209
#define ORC_W_EL 0.1406
#define ORC_W_DS 0.1322
#define ORC_ELEC 332.06363
#define ORC_DS_SIGMA 3.6
#define ORC_QSOL 0.01097
#define ORC_R_MIN 0.5
#define ORC_W_OUT 10.0

int orc_pose_coords(const orc_ligand *L, const double *genes, double *xyz_out);
int orc_energy(const orc_receptor *R, const orc_ligand *L, const double *xyz,
               double *e_inter, double *e_intra, double *atom_grad);
int orc_score(const orc_receptor *R, const orc_ligand *L, const double *genes,
              double *energy, double *gene_grad, double *xyz_out,
              double *atom_grad);
/* Magnitude [6+T] of each gene-gradient component: orc_score's chain rule
 * over the absolute values of all contributions (the scale of the rounding
 * error of any floating-point evaluation of the same sums); pos_mag [6+T]
 * (may be NULL): the components' sensitivity to rounding the coordinates
 * (a coordinate off by u |x|), in the same units. */
int orc_score_magnitude(const orc_receptor *R, const orc_ligand *L, const double *genes,
                        double *mag, double *pos_mag);
int orc_adadelta_step(int G, const double *grad, double rho, double eps,
                      double *genes, double *eg2, double *ed2);
int orc_local_search(const orc_receptor *R, const orc_ligand *L, double *genes,
                     int iters, double rho, double eps, int resume,
                     double *state, double *best_energy);
int orc_local_search_batch(const orc_receptor *R, const orc_ligand *L, int n,
                           double *genes, int iters, double rho, double eps,
                           double *best_energy, int nthreads);
int orc_score_batch(const orc_receptor *R, const orc_ligand *L, int n,
                    const double *genes, double *energy, double *gene_grad,
                    int nthreads);
/* Lamarckian GA (Sec. 2.1; rules are this project's reading, see adgb_oracle.c) */
typedef struct {
    int n_runs, pop, max_gens;
    long long max_evals;     /* per run */
    int ls_iters;
    double ls_rate, rho, eps;
    double p_cross, p_mut, mut_trans, mut_angle;
    unsigned long long seed;
    int conv_every, conv_top;  /* early stopping: test every conv_every generations (0: off) */
    double conv_tol;
    int ls_method;             /* 0 ADADELTA, 1 Solis-Wets (sw_* below) */
    double sw_rho0, sw_rho_min;
    int sw_max_succ, sw_max_fail;
    double sw_angle_scale;
} orc_dock_params;

void orc_philox4x32_10(const unsigned int ctr[4], const unsigned int key[2], unsigned int out[4]);
int orc_init_individual(const orc_receptor *R, int n_tors, unsigned long long seed, int run,
                        int k, double *genes);
int orc_ga_generation(int G, int pop, const double *genes_old, const double *energy_old,
                      const orc_dock_params *p, int run, int gen, double *genes_new,
                      int *ls_flag);
int orc_converged(int pop, const double *energy, int top, double tol);
int orc_dock(const orc_receptor *R, const orc_ligand *L, const orc_dock_params *p,
             double *best_genes, double *best_energy, long long *evals, int nthreads);
/* Solis-Wets local search (Solis and Wets, 1981), energy only */
typedef struct {
    int max_evals, max_succ, max_fail;
    double rho0, rho_min, angle_scale;
    unsigned long long seed;
    int call;
} orc_sw_params;
double orc_sw_normal(unsigned long long seed, unsigned int genotype, unsigned int step,
                     unsigned int call, int j);
int orc_sw_search(const orc_receptor *R, const orc_ligand *L, double *genes,
                  const orc_sw_params *p, int genotype, int resume, double *state,
                  double *energy, int *evals);
double orc_sum_naive(const double *x, long n, long stride);
double orc_sum_neumaier(const double *x, long n, long stride);

#ifdef __cplusplus
}
#endif
#endif
