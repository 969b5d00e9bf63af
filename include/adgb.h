/*
 * adgb - GB300-native AutoDock4 scoring function, gradient and ADADELTA
 * local search (the hot path of AutoDock-GPU's Lamarckian GA studied in
 * arxiv 2410.10447, "Accelerating Drug Discovery in AutoDock-GPU with
 * Tensor Cores").
 *
 * C ABI.  Conventions:
 *  - Every call returns an int status: ADGB_OK (0) or a negative ADGB_E*
 *    code.  adgb_last_error(ctx) gives a message for the last failure on
 *    that context.  Nothing is left half-done on an ADGB_EINVAL return.
 *  - Pointers named *_dev are device pointers owned by the caller; the call
 *    enqueues its work on `stream` and returns without synchronising.
 *    Pointers without the suffix are host pointers owned by the caller; the
 *    call copies them to the device, runs, copies results back and returns
 *    when they are in host memory.
 *  - Receptors and ligands are device objects owned by the library,
 *    referenced by integer ids, released explicitly or by adgb_destroy.
 *  - A context is bound to one device.  Calls on one context must not run
 *    concurrently from several host threads (thread-compatible); the
 *    library's only global state is the fixed device array of
 *    dock_noalloc_dev and its per-device address cache (mutex-guarded).
 *  - adgb_stream is the CUDA runtime's cudaStream_t (NULL = legacy default
 *    stream); it is declared here without the CUDA headers.
 *
 * Genotype layout (Sec. 2.1): genes[6+T] = (x, y, z, phi, theta, alpha,
 * psi_0 .. psi_{T-1}) in Angstrom and radians: translation of the ligand's
 * rotation centre, rotation axis (azimuth phi, polar angle theta), rotation
 * angle alpha about that axis, and one angle per rotatable bond.
 */
#ifndef ADGB_H
#define ADGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct adgb_ctx adgb_ctx;
typedef struct CUstream_st *adgb_stream;

enum {
    ADGB_OK = 0,
    ADGB_EINVAL = -1,     /* bad argument, size or ligand description */
    ADGB_ENOMEM = -2,     /* device or host allocation failed */
    ADGB_ENOTFOUND = -3,  /* unknown receptor / ligand / job id */
    ADGB_EDEVICE = -4,    /* CUDA error (message in adgb_last_error) */
    ADGB_ETIMEOUT = -5,   /* a wait ran out of time */
    ADGB_EREJECTED = -6,  /* a job can never fit the device */
    ADGB_ECANCELLED = -7  /* the job was cancelled */
};

/* Block-reduction variants of the (E, dE/dt, torque) vector (Sec. 3-4). */
enum {
    ADGB_REDUCE_SHFL = 0,       /* FP32 warp shuffles (reduce-scatter + all-gather) */
    ADGB_REDUCE_MMA_TF32X2 = 1, /* tensor-core sum, operands split into 2 TF32 terms, FP32 accumulate */
    ADGB_REDUCE_MMA_BF16X3 = 2, /* tensor-core sum, operands split into 3 BF16 terms, FP32 accumulate */
    ADGB_REDUCE_TCGEN05 = 3,    /* fifth-generation tensor cores (tcgen05.mma, accumulator in tensor
                                   memory), operands split into 2 TF32 terms, FP32 accumulate */
    ADGB_REDUCE_N = 4
};

/* Limits of one ligand. */
#define ADGB_MAX_ATOMS 256
#define ADGB_MAX_TORS 40
#define ADGB_MAX_TYPES 16

/* Force-field constants (AutoDock4.2 free-energy weights; Sec. 2.1 names
 * the force field without printing it). */
#define ADGB_W_VDW 0.1662f
#define ADGB_W_HB 0.1209f
#define ADGB_W_EL 0.1406f
#define ADGB_W_DS 0.1322f
#define ADGB_ELEC_KCAL 332.06363f
#define ADGB_DS_SIGMA 3.6f
#define ADGB_QSOL 0.01097f
#define ADGB_R_MIN 0.5f      /* clash clamp of the singular pair terms (A) */
#define ADGB_W_OUT 10.0f     /* out-of-grid penalty (kcal/mol/A^2) */

typedef struct {
    int threads_per_pose;  /* 0 = pick per ligand; else 32, 64 or 128 */
    int poses_per_block;   /* 0 = pick per ligand; else 1..8 (at most 128 threads a block) */
    int reduce_variant;    /* default ADGB_REDUCE_* for calls that do not say */
    int pair_rounds;       /* intramolecular pairs: 0 = matching rounds (ligand_pair_rounds;
                              the default, faster at every size measured), 1 = per-pair
                              force buffer and incidence lists */
    int genotypes_per_warp; /* ligands of at most 32 atoms (with matching rounds, at most 26
                              torsions, one warp a genotype's atoms): 0 = two genotypes a
                              warp, their arithmetic in packed FP32x2 instructions (the
                              default), 1 = one genotype a warp */
} adgb_options;

/* Receptor grid (Sec. 2.1: the receptor is fixed; its interaction with a
 * ligand atom is read from precomputed maps). */
typedef struct {
    int nx, ny, nz;        /* grid points per axis, each >= 2 */
    float spacing;         /* A between neighbouring points, > 0 */
    float origin[3];       /* position of point (0,0,0), A */
    int n_type_maps;       /* affinity maps, one per ligand atom type */
} adgb_grid_desc;

/* Ligand with its torsion tree (Sec. 2.1: torsion angles of rotatable bonds). */
typedef struct {
    int n_atoms;               /* 1..ADGB_MAX_ATOMS */
    int n_types;               /* 1..ADGB_MAX_TYPES */
    int n_tors;                /* 0..ADGB_MAX_TORS */
    int n_pairs;               /* >= 0 */
    const int32_t *type;       /* [n_atoms] type, also the receptor map index */
    const float *charge;       /* [n_atoms] partial charge (e) */
    const float *xyz;          /* [n_atoms][3] reference conformation; the rotation centre is the origin */
    const int32_t *tors_bond;  /* [n_tors][2] bond (a,b): torsion turns the atoms beyond b about a->b; listed root to leaf */
    const int32_t *mov_off;    /* [n_tors+1] offsets into mov_atoms */
    const int32_t *mov_atoms;  /* atoms moved by torsion k: mov_atoms[mov_off[k] .. mov_off[k+1]) (excluding a and b) */
    const int32_t *pairs;      /* [n_pairs][2] intramolecular pairs (i != j) */
    const float *R;            /* [n_types] vdW equilibrium distance (A) */
    const float *eps;          /* [n_types] vdW well depth (kcal/mol) */
    const float *vol;          /* [n_types] atomic volume (A^3) */
    const float *solpar;       /* [n_types] atomic solvation parameter */
    const int32_t *hb_role;    /* [n_types] 0 none, 1 donor, 2 acceptor */
    float hb_R, hb_eps;        /* 12-10 term of donor-acceptor pairs */
} adgb_ligand_desc;

/* ADADELTA local search parameters (Sec. 2.1; Zeiler 2012). */
typedef struct {
    int iters;             /* energy+gradient evaluations per genotype, >= 0 */
    float rho;             /* decay of the running averages, 0 < rho < 1 (0.8) */
    float eps;             /* conditioning constant, > 0 (1e-2) */
    int reduce_variant;    /* ADGB_REDUCE_*, or -1 for the context default */
    int flags;             /* ADGB_LS_* */
} adgb_ls_params;

#define ADGB_LS_RESUME 1   /* start from state (Omega, E[g^2], E[d^2]) instead of (genes, 0, 0) */

/* Context on one CUDA device; opts may be NULL (defaults). */
int adgb_create(adgb_ctx **ctx, int device, const adgb_options *opts);
int adgb_destroy(adgb_ctx *ctx);
/* Message of the last failure on ctx ("" if none); valid until the next call. */
const char *adgb_last_error(const adgb_ctx *ctx);

/*
 * upload_receptor_grids - copy the receptor's grid maps to the device.
 * maps: host float32 [n_type_maps+2][nz][ny][nx] (x fastest): the type
 * affinity maps, then the electrostatic potential map e (kcal/mol/e), then
 * the desolvation map d.  Maps already carry their force-field weights.
 * The library stores them cell-major (the 8 corner values of every map of a
 * grid cell contiguous), so one atom reads 3 x 32 contiguous bytes.
 * Errors: EINVAL (sizes), ENOMEM, EDEVICE.
 */
int upload_receptor_grids(adgb_ctx *ctx, const adgb_grid_desc *grid,
                          const float *maps, int *receptor_id);
int release_receptor(adgb_ctx *ctx, int receptor_id);

/*
 * upload_ligand_torsion_tree - validate and copy a ligand (Sec. 2.1).
 * The torsion tree must be laminar: two moving sets are disjoint or nested;
 * a torsion nested in another is listed after it and its bond atoms lie in
 * the outer moving set (or are its b atom); no torsion moves its own bond
 * atoms.  Errors: EINVAL (limits, indices, tree, n_types > ADGB_MAX_TYPES),
 * ENOMEM, EDEVICE.
 */
int upload_ligand_torsion_tree(adgb_ctx *ctx, const adgb_ligand_desc *lig,
                               int *ligand_id);
int release_ligand(adgb_ctx *ctx, int ligand_id);

/*
 * validate_ligand_torsion_tree - the checks of upload_ligand_torsion_tree
 * without a context or a device.  Returns ADGB_OK or ADGB_EINVAL; the
 * reason is written to msg (NUL-terminated, at most msg_len bytes) if msg
 * is not NULL.
 */
int validate_ligand_torsion_tree(const adgb_ligand_desc *lig, char *msg, int msg_len);

/*
 * ligand_pair_rounds - the host-side schedule of the intramolecular pairs
 * (the pair sum in Sec. 2.1's scoring function) that
 * upload_ligand_torsion_tree builds, without a context or a device: for ligands of at most 32 atoms and of more
 * than 112 (between, the per-pair force buffer is faster and no rounds are
 * built).  Lane a owns internal atom a: lanes = 32 up to 32 atoms (one warp
 * a genotype; positions and forces move by warp shuffles), else the atoms
 * rounded up to 32 (128 threads a genotype with two atoms each at most;
 * forces move through per-round slots in shared memory).  In round r lane a computes at most one pair with atom
 * a first and receives the reaction forces of at most two pairs with atom a
 * second.  The paper has no counterpart (its block-wide kernel sums forces
 * through shared memory).  n_rounds: rounds (0 without pairs or rounds),
 * normally max(ceil(pairs / atoms), ceil(max_degree / 3)); max_degree: the
 * largest number of pairs an atom is in.  words [words_cap]: if words_cap >=
 * lanes * n_rounds, word of lane a in round r at [lanes r + a]: partner lane
 * (bits 0-7; a itself without a pair, 0 for a lane past the last atom), lanes
 * whose pairs' reaction forces lane a receives (bits 8-15 and 16-23), H-bond
 * flag (bit 24), whether each of the two receive slots is used (bits 25,
 * 26).  perm [n_atoms] (may be NULL): caller's index of internal atom a.
 * Errors: EINVAL as validate_ligand_torsion_tree, or words_cap too small for
 * a non-NULL words.
 */
int ligand_pair_rounds(const adgb_ligand_desc *lig, int *n_rounds, int *lanes, int *max_degree,
                       unsigned int *words, int words_cap, int *perm);

/*
 * pose_coords - atom coordinates of n genotypes (Sec. 2.1).
 * genes [n][6+T] -> xyz [n][n_atoms][3], atoms in the caller's order.
 */
int pose_coords_dev(adgb_ctx *ctx, int ligand_id, const float *genes_dev, int n,
                    float *xyz_dev, adgb_stream stream);
int pose_coords(adgb_ctx *ctx, int ligand_id, const float *genes, int n, float *xyz);

/*
 * score_poses - energy and gene gradient of n genotypes (Sec. 2.1, the
 * scoring function evaluated with its gradient; Sec. 3, seven block
 * reductions per evaluation, here one 8-wide reduction).
 * genes [n][6+T]; energy [n] (kcal/mol); grad [n][6+T] or NULL.
 * reduce_variant: ADGB_REDUCE_* or -1 for the context default.
 * Errors: EINVAL (n < 0, unknown variant, ligand type beyond the receptor's
 * maps), ENOTFOUND, EDEVICE.
 */
int score_poses_dev(adgb_ctx *ctx, int receptor_id, int ligand_id,
                    const float *genes_dev, int n, float *energy_dev,
                    float *grad_dev, int reduce_variant, adgb_stream stream);
int score_poses(adgb_ctx *ctx, int receptor_id, int ligand_id, const float *genes,
                int n, float *energy, float *grad, int reduce_variant);

/*
 * local_search - ADADELTA local search of n genotypes (Sec. 2.1).
 * For each genotype: p->iters evaluations, each followed by one update
 *   E[g^2] <- rho E[g^2] + (1-rho) g^2
 *   d      <- -sqrt(E[d^2] + eps) / sqrt(E[g^2] + eps) * g
 *   E[d^2] <- rho E[d^2] + (1-rho) d^2
 *   Omega  <- Omega + d   (torsion genes wrapped to [-pi, pi)).
 * genes [n][6+T] in: the start genotypes; out: the genotype of the lowest
 * energy seen (ties keep the earlier one).  best_energy [n] out (+inf when
 * iters == 0).  state [n][3][6+T] or NULL: out, (Omega, E[g^2], E[d^2])
 * after the last update; with ADGB_LS_RESUME also in, and genes in is then
 * ignored.  The whole search of every genotype runs in one kernel launch.
 * Errors: EINVAL, ENOTFOUND, EDEVICE.
 */
int local_search_dev(adgb_ctx *ctx, int receptor_id, int ligand_id,
                     float *genes_dev, int n, const adgb_ls_params *p,
                     float *best_energy_dev, float *state_dev, adgb_stream stream);
int local_search(adgb_ctx *ctx, int receptor_id, int ligand_id, float *genes,
                 int n, const adgb_ls_params *p, float *best_energy, float *state);

/*
 * local_search_sw - Solis-Wets local search of n genotypes (Solis and Wets,
 * 1981; the derivative-free alternative to the gradient search among the
 * local searches Sec. 2.1 names).  Energy only: each evaluation is the
 * scoring function without its gradient, with one reduction of E.
 * Every step draws d_j = bias_j + rho * s_j * z_j (z_j standard normal from
 * Philox4x32-10 keyed by seed, counter (genotype, step, 0x5357 << 16 | call,
 * j / 4), Box-Muller on two 24-bit uniforms; s_j = 1 A for the translation
 * genes, angle_scale rad for the angle genes; torsions wrapped), tries x + d
 * and, if that is not lower, x - d.  A lower energy moves x (bias <- 0.2 bias
 * + 0.4 d forward, bias - 0.4 d backward), otherwise bias <- bias / 2;
 * max_succ successes in a row double rho, max_fail failures halve it.  A
 * search stops after max_evals evaluations (the start point counts one) or
 * once rho < rho_min.  genes [n][6+T] in: start, out: final genotype (the
 * lowest energy seen, since x only moves downhill); energy [n] out; evals [n]
 * out or NULL; state [n][2(6+T)+5] out or NULL: (x, bias, rho, successes,
 * failures, E(x), steps); with ADGB_LS_RESUME also in (genes in ignored; the
 * call then spends up to max_evals further evaluations).
 * Errors: EINVAL, ENOTFOUND, EDEVICE.
 */
typedef struct {
    int max_evals;           /* evaluations a search may spend, >= 1 */
    float rho0, rho_min;     /* initial step scale, and the scale below which a search stops */
    int max_succ, max_fail;  /* successes / failures in a row before rho doubles / halves */
    float angle_scale;       /* deviation of the angle genes per unit rho (rad) */
    unsigned long long seed;
    int call;                /* random-stream selector, 0..65535 */
    int reduce_variant;      /* ADGB_REDUCE_* or -1 for the context default */
    int flags;               /* ADGB_LS_RESUME */
} adgb_sw_params;

int local_search_sw_dev(adgb_ctx *ctx, int receptor_id, int ligand_id, float *genes_dev, int n,
                        const adgb_sw_params *p, float *energy_dev, int *evals_dev,
                        float *state_dev, adgb_stream stream);
int local_search_sw(adgb_ctx *ctx, int receptor_id, int ligand_id, float *genes, int n,
                    const adgb_sw_params *p, float *energy, int *evals, float *state);

/* Lamarckian GA docking parameters (Sec. 2.1: a GA proposes genotypes and
 * each is refined by the local search).  The paper prints no GA rules; the
 * library's rules: individual 0 of a generation is the previous best; every
 * other child comes from two binary tournaments, two-point crossover with
 * probability p_cross, per-gene mutation with probability p_mut by a
 * uniform offset in [-1, 1) times mut_trans (translation genes, A) or
 * mut_angle (angle genes, rad); each individual is locally searched
 * (ls_iters evaluations) with probability ls_rate, else scored once.
 * Random numbers: Philox4x32-10 keyed by seed, counter (individual,
 * generation, run, call), so results do not depend on launch shapes. */
typedef struct {
    int n_runs;              /* independent runs, >= 1 */
    int pop;                 /* individuals per run, 2..1024 */
    int max_gens;            /* generations after the initial population, >= 0 */
    long long max_evals;     /* evaluation budget of a run, checked after each generation */
    int ls_iters;            /* evaluations of one local search, >= 1 */
    float ls_rate;           /* probability of a local search, 0..1 */
    float rho, eps;          /* ADADELTA parameters */
    float p_cross, p_mut;    /* crossover / per-gene mutation probabilities */
    float mut_trans;         /* translation mutation amplitude (A) */
    float mut_angle;         /* angle mutation amplitude (rad) */
    unsigned long long seed;
    int reduce_variant;      /* ADGB_REDUCE_* or -1 for the context default */
    /* Early stopping (convergence detection; Sec. 5.3 discusses runs that do
     * or do not converge, the paper does not define the test).  The library's
     * test: after every conv_every-th generation a run stops once the
     * population standard deviation of its conv_top lowest energies (the
     * energies of that generation's evaluations) is below conv_tol kcal/mol,
     * computed in double precision from the float energies.  conv_every = 0
     * switches it off; otherwise 2 <= conv_top <= pop and conv_tol > 0. */
    int conv_every;
    int conv_top;
    float conv_tol;
    /* Local search of the LGA: 0 = ADADELTA (rho, eps), 1 = Solis-Wets with the
     * sw_* parameters below (see local_search_sw; each individual's search is
     * keyed by genotype index run * pop + k and call = generation mod 65536,
     * and spends at most ls_iters evaluations; a run counts the evaluations
     * actually spent).  The serving loop runs ADADELTA only. */
    int ls_method;
    float sw_rho0, sw_rho_min;
    int sw_max_succ, sw_max_fail;
    float sw_angle_scale;
} adgb_dock_params;

/*
 * dock - n_runs independent Lamarckian GA runs of one ligand against one
 * receptor (Sec. 2.1; Table 1's kernels: initial population scoring, GA
 * generation, local search, evaluation count).  Every generation is three
 * launches: GA generation, one fused local-search launch over all runs'
 * individuals, run-best and evaluation accounting.  At the end each run's
 * best genotype is rescored in FP64 on the GPU.
 * best_genes [n_runs][6+T] float32 out; best_energy [n_runs] FP64 out;
 * evals [n_runs] out or NULL (evaluations each run spent; a run stopped by
 * the evaluation budget or by early stopping spends no more).
 * The device working set (2 populations, energies, counters, about
 * 8 * n_runs * pop * (7 + T) bytes) is allocated stream-ordered per call.
 * Errors: EINVAL, ENOTFOUND, ENOMEM, EDEVICE.
 */
int dock_dev(adgb_ctx *ctx, int receptor_id, int ligand_id, const adgb_dock_params *p,
             float *best_genes_dev, double *best_energy_dev, long long *evals_dev,
             adgb_stream stream);
int dock(adgb_ctx *ctx, int receptor_id, int ligand_id, const adgb_dock_params *p,
         float *best_genes, double *best_energy, long long *evals);

/*
 * dock_noalloc_dev - dock_dev for callers that must not allocate device
 * memory during a call (programs that reserve the GPU's whole memory budget
 * up front, or serving paths where an allocation's latency or failure is not
 * acceptable).  No counterpart in the paper: it is a deployment variant.
 * Same arguments, results and errors as dock_dev, but the working set lives
 * in one fixed 4 MiB device array built into the library (held on every
 * device that loads it, until the process exits); nothing is allocated or
 * freed.  The working set is 8 * n_runs * pop * (6 + T) + 8 * n_runs * pop +
 * 16 * n_runs bytes plus 256-byte alignment per part; larger requests
 * return ADGB_EINVAL.  All calls share the array: calls whose work overlaps
 * on the GPU (other streams, other contexts, other host threads) race and
 * must be serialised by the caller.  Every part of the array a call reads is
 * first written by that call.  Every call made outside a stream capture
 * looks up the array's device address (so a device reset, which reloads the
 * library's module, leaves no stale address); a call made while `stream` is
 * being captured reuses the address its device's last uncaptured call found,
 * and fails with EDEVICE if there was none: make one uncaptured call on a
 * device (after any reset) before capturing.
 */
int dock_noalloc_dev(adgb_ctx *ctx, int receptor_id, int ligand_id, const adgb_dock_params *p,
                     float *best_genes_dev, double *best_energy_dev, long long *evals_dev,
                     adgb_stream stream);

/*
 * ga_init_population_dev - the initial genotypes dock() starts from:
 * genes [n_runs * pop][6+T] out (translation uniform in the central 60% of
 * the receptor's grid box, axis uniform on the sphere, angles uniform).
 * ga_generation_dev - one GA generation of n_runs populations (the rules
 * of adgb_dock_params; p->n_runs and p->pop give the shapes): genes and
 * energy [n_runs * pop] in, genes_out out, iters_out [n_runs * pop] out
 * (ls_iters for individuals chosen for a local search, else 1).
 * generation >= 1 selects the random stream.  Errors: EINVAL, ENOTFOUND.
 */
int ga_init_population_dev(adgb_ctx *ctx, int receptor_id, int ligand_id, unsigned long long seed,
                           int n_runs, int pop, float *genes_dev, adgb_stream stream);
int ga_generation_dev(adgb_ctx *ctx, int ligand_id, const adgb_dock_params *p, int generation,
                      const float *genes_dev, const float *energy_dev, float *genes_out_dev,
                      int *iters_out_dev, adgb_stream stream);

/*
 * ga_converged_dev - the early-stopping test of adgb_dock_params applied to
 * n_runs populations: energy [n_runs * pop] float32 in, converged [n_runs]
 * out (1 when the population standard deviation of the run's conv_top
 * lowest energies, in double precision, is below conv_tol; 0 otherwise,
 * when one of them is not finite, or when an energy of the run is NaN).  p->n_runs, p->pop, p->conv_top and
 * p->conv_tol are used (conv_every is not).  Errors: EINVAL, EDEVICE.
 */
int ga_converged_dev(adgb_ctx *ctx, const adgb_dock_params *p, const float *energy_dev,
                     int *converged_dev, adgb_stream stream);

/*
 * rescore_fp64_dev - energies of n genotypes recomputed in double precision
 * on the GPU from the same inputs (coordinates, grid and pair terms).
 * genes [n][6+T] float32, energy [n] FP64 out.
 */
int rescore_fp64_dev(adgb_ctx *ctx, int receptor_id, int ligand_id, const float *genes_dev,
                     int n, double *energy_dev, adgb_stream stream);

/*
 * Uneven batches: genotypes of many ligands (of different atom, torsion and
 * pair counts), each against its own receptor, locally searched by ONE
 * persistent multi-ligand launch.  Blocks take work items (up to
 * poses-per-block genotypes of one ligand, longest first) from a device
 * counter, so big and small ligands share the GPU without stragglers.  The
 * launch is captured into a CUDA graph on the first call and replayed by
 * later calls with the same buffers and parameters.
 *
 * batch_create - item i: n_poses[i] genotypes of ligand ligand_ids[i]
 *   against receptor receptor_ids[i].  Genotypes of item i occupy rows
 *   [off_i, off_i + n_poses[i]) of a [total][ADGB_MAX_GENES] float32 array
 *   (the first 6 + T_i entries of a row are used), off_i = sum of n_poses[j]
 *   over j < i.  The batch refers to the ligands and receptors: release the
 *   batch before them.  Errors: EINVAL, ENOTFOUND, ENOMEM.
 * batch_autotune - times the candidate launch shapes (32, 64 or 128 threads
 *   a genotype; poses per block; reduction variant) on this batch with
 *   `iters` evaluations per genotype from genes_dev (read on the context's
 *   own stream after the caller's work is complete; not modified), keeps the
 *   fastest for this batch and for later batches of the same size class
 *   (largest ligand in 32-atom and 512-pair steps), and writes it to chosen
 *   (may be NULL).  Synchronous.
 * batch_local_search_dev - local_search over every genotype of the batch:
 *   genes [total][ADGB_MAX_GENES] in/out, best_energy [total] out, on
 *   `stream`.  p->flags must not ask for resume.
 */
#define ADGB_MAX_GENES (6 + ADGB_MAX_TORS)
int batch_create(adgb_ctx *ctx, int n_items, const int *receptor_ids, const int *ligand_ids,
                 const int *n_poses, int *batch_id);
int batch_autotune(adgb_ctx *ctx, int batch_id, const float *genes_dev, int iters,
                   adgb_options *chosen);
int batch_local_search_dev(adgb_ctx *ctx, int batch_id, float *genes_dev,
                           const adgb_ls_params *p, float *best_energy_dev, adgb_stream stream);
int batch_release(adgb_ctx *ctx, int batch_id);

/*
 * Serving: continuous batching of docking jobs.
 *
 * serve_start creates a server on ctx's device with its own host thread.
 * Every admitted job runs as an independent chain of launches on a stream of
 * its own: initial population, then one Lamarckian-GA generation after
 * another (GA, the generation's local searches - ADADELTA or Solis-Wets as
 * the job's parameters say - run bests and evaluation accounting), in the
 * kernels, launch shape and order of a dock() call of the job, so a served
 * job returns the same bits as dock() and the same bits alone or among other
 * jobs.  The GPU interleaves the active jobs' kernels.  The server thread
 * keeps two generations of each job queued and reads their counters from
 * pinned memory as they land (event queries, no synchronisation); a job is
 * done at its generation limit or once every run reached its evaluation
 * budget or stopped early, and is then rescored in FP64, its results copied
 * to host memory and its device memory released.  Queued jobs are admitted
 * in arrival order while the job fits the device's free memory at that
 * moment (plus what the library's stream-ordered pool holds unused, less a
 * reserve of 1/64 of the device memory, at least 256 MiB), the caller's
 * budget if one is set, and the active-job cap (by default two jobs, and
 * more while their local searches together fill less than twice the GPU:
 * one job's generations then cover the other's gaps, while more large jobs
 * only compete for L2 and SMs).  Populations, ligands and
 * counters stay on the device between generations.
 *
 * dock_submit validates the ligand and parameters on the calling thread and
 * queues the job (ADGB_EREJECTED if it can never fit the budget or the
 * server is stopping).  dock_poll reports a job's state; dock_wait blocks
 * until the job has finished, been cancelled or failed (ADGB_ETIMEOUT after
 * timeout_ms; < 0 waits without limit); dock_result copies a finished job's
 * best genotypes [n_runs][6+T], FP64 best energies [n_runs] and evaluation
 * counts [n_runs] (ADGB_ETIMEOUT while it is queued or running, the job's
 * error status if it did not finish); dock_cancel asks for cancellation
 * (queued: dropped; running: no further generation is queued and the job
 * ends once those in flight have completed);
 * dock_forget frees the host record of a job that is no longer queued or
 * running.  serve_stop cancels all jobs, joins the thread and frees the
 * server.  The submit/poll/wait/result/cancel calls may come from any host
 * threads; receptors must stay uploaded while jobs that use them are
 * pending, and must not be uploaded or released concurrently with
 * dock_submit.
 */
typedef struct adgb_server adgb_server;

typedef struct {
    int max_active_jobs;          /* 0: two jobs, more while their local searches together need
                                     fewer resident warps than two GPU-fulls (16 warps an SM) */
    long long mem_budget_bytes;   /* 0: the device's free memory at each admission (less a reserve) */
    int threads_per_pose;         /* 0: the context's rule (by ligand size unless its options set it) */
    int poses_per_block;          /* 0: the context's rule */
    int reduce_variant;           /* -1: the context default */
} adgb_serve_options;

typedef struct {
    int status;          /* 0 done, 1 queued, 2 running, ADGB_ECANCELLED, ADGB_EDEVICE */
    int n_runs, n_genes; /* n_genes = 6 + T */
    int generations;     /* generations completed */
    long long evals;     /* evaluations of all runs (when done) */
    double submit_s, start_s, finish_s;  /* server clock, seconds; -1 if not yet */
} adgb_job_info;

typedef struct {
    int queued, active;
    long long ticks;       /* generations queued (initial populations included), all jobs */
    long long items_run;   /* genotypes of those generations */
    long long device_bytes_in_use, device_bytes_budget;
    double busy_s, uptime_s;
} adgb_serve_stats;

int serve_start(adgb_ctx *ctx, const adgb_serve_options *opts, adgb_server **server);
int serve_stop(adgb_server *server);
const char *serve_last_error(adgb_server *server);
int serve_stats(adgb_server *server, adgb_serve_stats *stats);
int dock_submit(adgb_server *server, int receptor_id, const adgb_ligand_desc *lig,
                const adgb_dock_params *p, long long *job_id);
int dock_poll(adgb_server *server, long long job_id, adgb_job_info *info);
int dock_wait(adgb_server *server, long long job_id, int timeout_ms, adgb_job_info *info);
int dock_result(adgb_server *server, long long job_id, float *best_genes, double *best_energy,
                long long *evals);
int dock_cancel(adgb_server *server, long long job_id);
int dock_forget(adgb_server *server, long long job_id);

/*
 * reduce4_bench_dev - the reduction test kernel of Sec. 5.2: every thread
 * of a block holds one four-element vector, the block computes the sum and
 * every thread receives it.  in [n_blocks][threads][4] float32, out the same
 * shape (each thread's copy of its block's sum).  The reduction is repeated
 * `reps` times inside the kernel (every repetition reduces the same input),
 * so that its own cost dominates a timing.  variant:
 *   ADGB_REDUCE_SHFL / _MMA_TF32X2 / _MMA_BF16X3 - this library's warp-level
 *     forms (the local search's reductions) applied at warp and block level;
 *   ADGB_REDUCE4_PAPER_FS - the per-component shuffle + shared-memory atomic
 *     reduction that Sec. 3 profiles (three barriers per component);
 *   ADGB_REDUCE4_PAPER_HALF - the matrix form of Sec. 4.2 as the paper runs
 *     it: operands and accumulators V = A.P, W = Q.V in FP16 (about three
 *     significant digits; a total above 65504 in magnitude becomes inf);
 *   ADGB_REDUCE4_TCGEN05_TF32X2 - one block-wide tcgen05.mma chain on the
 *     fifth-generation tensor cores (split TF32 operands, FP32 accumulation
 *     in tensor memory); needs threads to be a multiple of 64.  Should the
 *     wait for the tensor core ever give up, the block's outputs are NaN;
 *   ADGB_REDUCE4_TCGEN05_WAIT_SELFTEST - the same kernel with nothing issued
 *     to the tensor core, so that every completion wait gives up after a
 *     short bounded wait: the outputs are NaN, the tensor memory is released
 *     and the context stays usable (a test of the failure path).
 * threads: 32..1024, a multiple of 32; reps >= 1.
 * Errors: EINVAL, EDEVICE.
 */
#define ADGB_REDUCE4_PAPER_FS 100
#define ADGB_REDUCE4_PAPER_HALF 101
#define ADGB_REDUCE4_TCGEN05_TF32X2 102
#define ADGB_REDUCE4_TCGEN05_WAIT_SELFTEST 103
int reduce4_bench_dev(adgb_ctx *ctx, int variant, const float *in_dev,
                      int threads, int n_blocks, int reps, float *out_dev,
                      adgb_stream stream);

/*
 * alu_bench_dev - throughput probe of the arithmetic units the scoring
 * kernels are bound by (no counterpart in the paper; it measures the
 * roofline's denominator): n_blocks x threads threads each run reps x 128
 * dependent operations in 8 independent chains.  kind 0: FP32 fused
 * multiply-add (2 flops each); 1: ex2.approx; 2: rsqrt.approx (special-
 * function unit); 3: packed FP32x2 fused multiply-add (two FMAs, 4 flops,
 * an instruction).  out [n_blocks * threads] float32 receives a value per
 * thread.  threads: 32..256, a multiple of 32.  Errors: EINVAL, EDEVICE.
 */
int alu_bench_dev(adgb_ctx *ctx, int kind, int n_blocks, int threads, int reps, float *out_dev,
                  adgb_stream stream);

/*
 * l2_bench_dev - read-bandwidth probe of the L2 cache (no counterpart in the
 * paper; it measures the denominator of the grid gathers' roofline, whose
 * maps stay resident in L2 for grids up to ~100 MB).  buf_dev [n_float4]
 * float4 (16-byte aligned; the caller sizes it to stay resident in L2 and
 * reads it once before timing) is read by n_blocks x threads threads, reps
 * times each.  kind 0: coalesced streaming reads, 16 bytes a thread and
 * repetition.  kind 1: the scoring kernels' gathers - per repetition a
 * pseudo-random cell of cell_float4 float4 (even, >= 6; the grid's cells are
 * maps x 2 float4) and 96 bytes of it: two float4 of one leading map and the
 * four trailing float4.  out_dev [n_blocks * threads] float32 receives each
 * thread's sum of the x components read (with a buffer of ones: 1 a float4
 * read).  threads: 32..256, a multiple of 32.  Errors: EINVAL, EDEVICE.
 */
int l2_bench_dev(adgb_ctx *ctx, int kind, const float *buf_dev, long long n_float4,
                 int cell_float4, int n_blocks, int threads, int reps, float *out_dev,
                 adgb_stream stream);

/*
 * device_status - tensor-core failure report (no counterpart in the paper).
 * Every wait of the tcgen05 local-search kernels for the tensor core is
 * bounded; a wait that gives up makes that warp's sums NaN for the rest of
 * its launch, frees its tensor memory and is counted on the device.  The
 * synchronous calls (score_poses, local_search, local_search_sw, dock)
 * return ADGB_EDEVICE when the count grew during the call or since the last
 * report; the asynchronous *_dev calls cannot, and device_status reports it
 * for them: it waits for the context's stream and returns ADGB_EDEVICE
 * (once) if any wait gave up on ctx's device since the context last
 * reported one, else ADGB_OK.  The count is device-wide: a give-up in any
 * caller's kernels on the device is reported.  (A served job is failed with
 * ADGB_EDEVICE by the same rule, between its first and last launch.)
 * Errors: EINVAL, EDEVICE.
 */
int device_status(adgb_ctx *ctx);

/*
 * ls_ablation_dev - measurement aid with no counterpart in the paper: the
 * two-genotypes-a-warp local search of local_search_dev with some of its
 * steps left out at compile time, so that a step's share of the time is the
 * difference to the whole search.  The outputs are NOT energies or searched
 * genotypes.  skip_mask (values built): 0 (nothing left out), 1 (pair
 * rounds), 2 (grid terms), 12 (the reduce-and-broadcast and the torsions'
 * moving-set sums: each lane keeps its own partials), 8 (the moving-set sums
 * of the shuffle form), 16 (the torsion-tree walk of the coordinates), 32
 * (the gene-gradient formulas), 64 (sines and cosines: zero angles), 3
 * (pairs and grid), 128 (the pair terms' arithmetic, the exchanges kept),
 * 256 (the pair rounds' shuffles, the arithmetic kept); 512 (nothing left
 * out: the tcgen05 variant with ONE tensor-core product a block over all its
 * warps' partials, after a block barrier, instead of one a warp - the other
 * design of the reduction on tensor cores, kept for measurement; needs n a
 * multiple of the genotypes a block); 1024 (a test of the failure path: the
 * tcgen05 variant with nothing issued to the tensor core, so that every
 * warp's first completion wait gives up after a short bounded wait; its sums
 * are NaN, its tensor memory is released, the give-up is counted and the
 * next synchronous call or device_status reports ADGB_EDEVICE once).
 * variant: ADGB_REDUCE_SHFL or ADGB_REDUCE_TCGEN05.  genes_dev [n][6+T]
 * in/out, best_energy_dev [n] out, on `stream`.  The ligand must run two
 * genotypes a warp (at most 32 atoms with matching rounds, at most 26
 * torsions, the context's default launch shape).  Errors: EINVAL (other
 * masks, variants or ligands), ENOTFOUND, EDEVICE.
 */
int ls_ablation_dev(adgb_ctx *ctx, int receptor_id, int ligand_id, float *genes_dev, int n,
                    int iters, int variant, int skip_mask, float *best_energy_dev,
                    adgb_stream stream);

/*
 * philox4x32_10_dev - the counter-based generator every random decision of
 * the library draws from (GA selection, crossover and mutation, initial
 * genotypes, Solis-Wets deviates): Philox4x32 with 10 rounds, Salmon,
 * Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
 * (SC'11), the generator behind the Lamarckian GA of Sec. 2.1 here.  Exposed
 * so that the device implementation can be checked against the published
 * known-answer vectors.  in_dev [n][6] uint32 = (counter words 0-3, key words
 * 0-1), out_dev [n][4] uint32 receives the four output words; both device
 * buffers are caller-owned and used on `stream`.  n = 0 does nothing.
 * Errors: EINVAL (null buffers with n > 0, n < 0), EDEVICE.
 */
int philox4x32_10_dev(adgb_ctx *ctx, const unsigned int *in_dev, int n, unsigned int *out_dev,
                      adgb_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* ADGB_H */
