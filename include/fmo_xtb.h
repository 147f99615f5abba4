/*
 * fmo_xtb.h - C ABI of the batched FMO-xTB self-consistent-charge library.
 *
 * The library computes the fragment molecular orbital (FMO) energy of a
 * molecular system with GFN1-xTB fragments, as stated in Sec. 2.2-2.3 of
 * Einsele & Mitric, "FMO-xTB: Fragment molecular orbital method with
 * GFN1-xTB":
 *   in:  geometry, fragment partition, element parameter table;
 *   out: monomer energies and shell charges, dimer/trimer interaction
 *        energies, and the FMO1/FMO2/FMO3 totals.
 * All arithmetic runs in CUDA kernels on one GPU (sm_103a); the host code
 * only validates input, plans batches and copies data.
 *
 * Conventions
 *   - Units: bohr and Hartree.  Charges are in electrons, as population
 *     minus reference occupation (positive = excess electrons).
 *   - Every function returns fmo_status; FMO_OK is 0.  On error the context
 *     keeps a message readable through fmo_last_error().  No C++ exception
 *     crosses the ABI.
 *   - Ownership: the caller owns every pointer it passes; the library copies
 *     what it needs during the call and keeps no caller pointer.  Output
 *     arrays are caller-allocated with the sizes stated per call.
 *   - Threading: a context may be used by one host thread at a time.
 */
#ifndef FMO_XTB_H
#define FMO_XTB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FMO_MAX_Z 87     /* element slots 0..86 */
#define FMO_MAX_SHELL 3  /* shells per element */
#define FMO_MAX_PRIM 12  /* Gaussian primitives per shell */

typedef enum {
  FMO_OK = 0,
  FMO_ERR_ARG = 1,           /* invalid argument or input */
  FMO_ERR_CUDA = 2,          /* CUDA runtime error */
  FMO_ERR_OOM = 3,           /* device allocation failed */
  FMO_ERR_NOT_CONVERGED = 4, /* an SCC or the monomer loop hit its limit */
  FMO_ERR_TIMEOUT = 5,       /* deadline passed; kernels stopped early */
  FMO_ERR_NAN = 6,           /* non-finite value in a result */
  FMO_ERR_STATE = 7,         /* call out of order (e.g. run before set_system) */
  FMO_ERR_UNSUPPORTED = 8,   /* feature or size not supported */
  FMO_ERR_EXCHANGE = 9       /* the exchange callback of a sharded run failed */
} fmo_status;

/* Per-n-mer status words written by the SCC kernel. */
enum {
  FMO_SCC_CONVERGED = 0,
  FMO_SCC_MAX_ITER = 1,
  FMO_SCC_NAN = 2,
  FMO_SCC_TIMEOUT = 3,
  FMO_SCC_JACOBI = 4          /* eigensolver sweep limit reached */
};

/*
 * One element of the GFN1-xTB parameter table (Eqs. 2-11 of the paper; the
 * values themselves are not printed in the paper and are an input).
 * Shell k has angular momentum l[k] (0 = s, 1 = p) and the contracted
 * function sum_p coef[k][p] * g(alpha[k][p]) where g is a primitive Gaussian
 * normalised on its own (s: (2a/pi)^(3/4) e^{-a r^2}; p_x: the same times
 * 2 sqrt(a) x).  n_shell == 0 marks an absent element.
 */
typedef struct fmo_element {
  int32_t n_shell;
  int32_t l[FMO_MAX_SHELL];
  int32_t n_prim[FMO_MAX_SHELL];
  int32_t pad_;
  double alpha[FMO_MAX_SHELL][FMO_MAX_PRIM];
  double coef[FMO_MAX_SHELL][FMO_MAX_PRIM];
  double h_l[FMO_MAX_SHELL];     /* H_A^l, Eq. 10 (Eh) */
  double k_cn_l[FMO_MAX_SHELL];  /* k_CN,l, Eq. 10 */
  double k_poly_l[FMO_MAX_SHELL];/* k^poly_{A,l}, Eq. 9 */
  double kappa_l[FMO_MAX_SHELL]; /* kappa_A^l, Eq. 5 */
  double q0_l[FMO_MAX_SHELL];    /* reference shell occupation (e), Eq. 3 */
  double eta;                    /* eta_A, Eq. 5 (Eh) */
  double gamma3;                 /* Gamma_A, third-order term of Eq. 2 (Eh) */
  double en;                     /* electronegativity, Delta EN of Eq. 8 */
  double r_cov;                  /* covalent radius (bohr), Eq. 9 and CN */
  double z_eff;                  /* Z^eff_A, Eq. 11 */
  double alpha_rep;              /* alpha_A, Eq. 11 */
} fmo_element;

/* The whole table plus the global parameters of Eqs. 4, 8, 11 and the CN. */
typedef struct fmo_params {
  fmo_element el[FMO_MAX_Z];
  double k_l[3];                 /* k_l of Eq. 8 for l = s, p, d */
  double k_ab[FMO_MAX_Z][FMO_MAX_Z]; /* K_AB of Eq. 8 */
  double k_en;                   /* k_EN of Eq. 8 */
  double k_g;                    /* k_g of Eq. 4 */
  double k_f;                    /* k_f of Eq. 11 */
  double cn_k1, cn_k2;           /* k_1, k_2 of the CN counting function */
  double cn_cutoff;              /* pairs at R >= cutoff are not counted (bohr) */
  double t_el;                   /* electronic temperature of Eq. 6 (K) */
  double v_hop;                  /* HOP projector strength (Eh) */
} fmo_params;

enum { FMO_PREC_FP64 = 0, FMO_PREC_MIXED = 1 };
enum { FMO_LOOP_GLOBAL = 0, FMO_LOOP_NESTED = 1 };
enum { FMO_NMER_FINISH_ENERGY = 0, FMO_NMER_FINISH_ITERATE = 1 };
enum { FMO_ESP_AUTO = 0, FMO_ESP_PAIRWISE = 1 };

typedef struct fmo_options {
  int32_t level;            /* 1 = FMO1, 2 = FMO2 (Eq. 12), 3 = FMO3 (Eq. 16) */
  int32_t precision;        /* FMO_PREC_FP64 or FMO_PREC_MIXED (FP32 loose
                               iterations, then FP64 to convergence) */
  int32_t all_dimers_scc;   /* 1: every pair gets an SCC dimer (no ES-DIM) */
  int32_t max_iter;         /* SCC iterations per n-mer solve */
  int32_t max_outer;        /* monomer ESP iterations */
  int32_t guess;            /* 0 neutral charges, 1 learned model (fmo_mlp_*;
                               restarts from 0 if the monomer loop does not
                               converge), 2 user charges (fmo_set_guess) */
  int32_t schedule;         /* 0 (default): the global monomer loop runs
                               device-driven in CUDA graphs with conditional
                               while nodes: the FP32 steps after the first (a
                               device-side loop control ends them at the
                               FP32 -> FP64 hand-over), then the FP64 steps
                               after the hand-over step (ended on
                               convergence); 1: one host round trip per step.
                               Results are identical. */
  int32_t monomer_loop;     /* FMO_LOOP_GLOBAL (default): one SCC iteration of
                               every monomer per outer step, then one Broyden
                               step on all monomer charges together;
                               FMO_LOOP_NESTED: every monomer SCC converged in
                               the ESP of the previous outer iterate */
  double dimer_cut;         /* SCC dimer iff closest atom pair < dimer_cut (bohr) */
  double trimer_cut;        /* SCC trimer iff all three pairs < trimer_cut */
  double scc_tol;           /* max |dq_out - dq_in| at SCC convergence (e) */
  double e_tol;             /* |E - E_prev| at SCC convergence (Eh) */
  double outer_tol;         /* monomer loop: max charge change (e) */
  double mixed_switch_tol;  /* mixed: FP32 until max |dq_out - dq_in| < this */
  double deadline_s;        /* wall-clock limit per fmo_run, 0 = none */
  int32_t mixed_finish;     /* nmer_finish = FMO_NMER_FINISH_ITERATE: FP64 SCC
                               iterations of dimers and trimers after the FP32
                               phase (0: converge in FP64 to scc_tol/e_tol) */
  int32_t nmer_finish;      /* mixed precision, dimers and trimers: how the FP32
                               phase ends.  FMO_NMER_FINISH_ENERGY (default):
                               energy and charges of the FP32-converged density
                               evaluated in FP64, its occupied orbitals first
                               made S-orthonormal in FP64.
                               FMO_NMER_FINISH_ITERATE: mixed_finish FP64 SCC
                               iterations.  Either way the n-mer interaction
                               energy is variational in the n-mer density (its
                               ESP is fixed), so it is off only to second order
                               in the FP32 charge error. */
  int32_t want_gradient;    /* 1: keep what fmo_get_gradient needs; in mixed
                               precision the dimers and trimers then converge
                               in FP64 after the FP32 phase (nmer_finish and
                               mixed_finish are ignored).  Precision FP64 runs
                               always allow the gradient. */
  int32_t esp_mode;         /* the supersystem potential phi = gamma dq (Eq. 21)
                               of every monomer-loop step: FMO_ESP_AUTO
                               (default) keeps gamma of all shell pairs in
                               device memory when it fits (<= 32 GB and <= 1/4
                               of the free memory) and forms phi as a matrix-
                               vector product; FMO_ESP_PAIRWISE evaluates gamma
                               pair by pair every step (no n_sh^2 buffer). */
  int32_t shard_rank;       /* sharded run over shard_world processes (one per
                               GPU; Sec. 2.3 and Eqs. 12 and 16 make the
                               monomer steps, dimers and trimers independent
                               given the monomer charges): this process solves
                               the n-mers that fmo_lpt_partition (cost n^3)
                               gives shard_rank in each pass, and every monomer
                               step, pass and result is summed over the ranks
                               through the callback of fmo_set_exchange.
                               Results are those of the unsharded run, bit for
                               bit, on every rank. */
  int32_t shard_world;      /* number of ranks; 0 or 1 = not sharded.  Sharded
                               runs need the global monomer loop and
                               want_gradient = 0, and run the monomer loop
                               host-driven (schedule 1). */
  int32_t nmer_ctas_per_sm; /* schedule of the dimer and trimer passes (the
                               autotuner's knobs; results do not depend on
                               them): 0 (default) the built-in rule, 1 one CTA
                               per SM with 255 registers per thread, 2 two CTAs
                               per SM with 128 registers each and half an SM of
                               shared memory each */
  int32_t nmer_matrix_smem; /* where the dimers' and trimers' n x n eigen-solve
                               matrix lives: 0 (default) the built-in rule
                               (global memory for mixed-precision n-mers that
                               iterate in FP32 only), 1 shared memory where it
                               fits, 2 global memory */
  int32_t monomer_ctas_per_sm;  /* the same two knobs for the monomer pass: 0
                               (default) the built-in rule, 1 or 2 CTAs per SM */
  int32_t monomer_matrix_smem;  /* 0 (default) the rule (shared memory where it
                               fits), 1 shared memory where it fits, 2 global
                               memory, 3 mixed precision: only the FP32 matrix
                               in shared memory (small enough for two CTAs per
                               SM) */
} fmo_options;

/* Element-wise sum over the ranks of a sharded run: replace buf[0 .. n) by
 * the sum of every rank's buf.  fmo_run calls it on every rank with the same
 * n, in the same order (once per monomer-loop step and once after each
 * pass); each entry is non-zero on the rank that owns it only, so the sum is
 * exact.  Return 0 on success; anything else ends fmo_run with
 * FMO_ERR_EXCHANGE.  A torch.distributed all_reduce (gloo, CPU tensor) is
 * one such callback.  The paper has no counterpart (its runs use one GPU). */
typedef int32_t (*fmo_exchange_fn)(void *user, double *buf, int64_t n);

/* Counters of the last fmo_run. */
typedef struct fmo_stats {
  int64_t n_monomer_solves;   /* monomer SCCs brought to self-consistency (nested
                                 loop: summed over outer iterations) */
  int64_t n_dimer_scc;        /* SCC dimers */
  int64_t n_dimer_esdim;      /* ES-DIM pairs (Eq. 15) */
  int64_t n_trimer_scc;       /* SCC trimers */
  int64_t scc_iterations;     /* all SCC iterations of all solves */
  int64_t kernel_launches;    /* CUDA kernels launched by the run */
  int32_t outer_iterations;   /* monomer ESP iterations */
  int32_t n_failed;           /* n-mers whose status is not CONVERGED */
  double ms_setup, ms_monomer, ms_select, ms_dimer, ms_trimer, ms_reduce;
  /* per pass p = 0 monomers (all outer iterations), 1 dimers, 2 trimers */
  double ms_scc[3];           /* SCC kernel launches alone (CUDA events, same stream) */
  int64_t scc_launches[3];    /* SCC kernel launches */
  int64_t iters_fp32[3];      /* SCC iterations run in FP32 (mixed precision) */
  int64_t iters_fp64[3];      /* SCC iterations run in FP64 */
  double flops_fp32[3];       /* algorithmic flops: 15 n^3 per SCC iteration of an */
  double flops_fp64[3];       /* n-AO n-mer (transform 4n^3, density 2n^3, eigen 9n^3) */
  int64_t h2d_bytes;          /* host -> device bytes copied by the run */
  int64_t d2h_bytes;          /* device -> host bytes copied by the run */
  double ms_gradient;         /* last fmo_get_gradient (CUDA events) */
  int32_t zvector_iterations; /* GMRES iterations of its Z-vector solve */
  int32_t guess_restarts;     /* 1: the learned guess's monomer loop did not
                                 converge and the run restarted from neutral */
  double zvector_residual;    /* final ||w - (1 - Gamma chi) z|| / ||w|| */
} fmo_stats;

typedef struct fmo_ctx fmo_ctx;

/* Install the exchange callback of sharded runs (fn = NULL removes it);
 * user is passed back unchanged.  Errors: FMO_ERR_ARG (ctx NULL). */
fmo_status fmo_set_exchange(fmo_ctx *ctx, fmo_exchange_fn fn, void *user);

/* Longest-processing-time-first partition of n work units over world ranks
 * (host only, needs no GPU): units in order of decreasing cost[i] (ties: lower
 * i first) each go to the rank with the least assigned cost so far (ties:
 * lower rank); owner[i] receives the rank.  The makespan is within 4/3 of the
 * optimum (Graham, 1969).  fmo_run shards every pass with it (cost n^3 of the
 * n-mer's basis size).  Errors: FMO_ERR_ARG (NULL with n > 0, n < 0,
 * world < 1, a cost that is negative or not finite). */
fmo_status fmo_lpt_partition(const double *cost, int64_t n, int32_t world, int32_t *owner);

/* Fill *o with the defaults: level 2, FP64, ES-DIM on, cut 4.0 A, tolerances
 * 1e-10, max_iter 300, max_outer 200, switch 1e-5, one FP64 finishing
 * iteration for mixed-precision dimers and trimers, no deadline. */
void fmo_options_default(fmo_options *o);

/* Create a context on CUDA device `device` with a copy of the table *p.
 * Errors: FMO_ERR_ARG (NULL pointers, element with n_prim > FMO_MAX_PRIM or
 * l > 1), FMO_ERR_CUDA (no such device). */
fmo_status fmo_create(fmo_ctx **out, const fmo_params *p, int device);

/*
 * Define the system (Sec. 2.2: N fragments).
 *   Z[n_atoms]             atomic numbers; each must be present in the table
 *   xyz[3*n_atoms]         coordinates (bohr), atom-major (x0,y0,z0,x1,...)
 *   frag_of_atom[n_atoms]  fragment index 0..n_frag-1; every fragment non-empty
 *   frag_charge[n_frag]    net charge of each fragment (e)
 *   n_cut, bda_baa[2*n_cut] covalent bonds cut between fragments: bond
 *                          detachment atom (BDA) and bond attachment atom
 *                          (BAA), input atom indices; the bonds are treated
 *                          by hybrid orbital projection (HOP section of the
 *                          paper): each BDA needs exactly one s and one p
 *                          shell and is detached at most once.  0 / NULL: no
 *                          cut bonds.
 * Each n-mer must hold an even number of electrons (closed shell).
 * Errors: FMO_ERR_ARG on any violation (indices out of range, BDA and BAA in
 * one fragment, open shell), FMO_ERR_UNSUPPORTED (a BDA without one s and one
 * p shell, or detached twice; a fragment of more than 510 basis functions).
 */
fmo_status fmo_set_system(fmo_ctx *ctx, int32_t n_atoms, const int32_t *Z, const double *xyz,
                          int32_t n_frag, const int32_t *frag_of_atom, const int32_t *frag_charge,
                          int32_t n_cut, const int32_t *bda_baa);

/* New coordinates for the same atoms and partition: host array xyz[3*n_atoms]
 * (bohr, input atom order), copied to the device on the context's stream. */
fmo_status fmo_set_coordinates(fmo_ctx *ctx, const double *xyz);

/* The same, from a device array (3*n_atoms doubles, input atom order) that
 * is read on `cuda_stream`.  With a stream, the call only enqueues the gather:
 * run fmo_run on the same stream (or order the two streams).  With NULL the
 * context's stream is used and the call returns when the copy is done. */
fmo_status fmo_set_coordinates_device(fmo_ctx *ctx, const double *xyz_dev, void *cuda_stream);

/* User initial monomer shell charges (options.guess = 2), n_shell values in
 * the output order of fmo_get_monomers. */
fmo_status fmo_set_guess(fmo_ctx *ctx, const double *shell_dq);

/*
 * Learned initial monomer charges (options.guess = 1).  The paper has no
 * learned guess; this model is specific to this library: per-atom radial and
 * angular descriptors within 6 A (32 + 40), the embedding potential of the
 * other fragments' charges, the element one-hot (H, C, N, O), a 77-128-128-2
 * SiLU network with FP16 weights and FP32 accumulation whose two outputs are
 * the atom's two shell charges, shifted per fragment to minus its charge.
 * Prediction takes two passes: zero potential, then the potential of the
 * first pass's charges.  Every atom must have two shells, k_g = 2, no cut
 * bonds; otherwise FMO_ERR_UNSUPPORTED.
 *
 * Weights: FMO_MLP_N_WEIGHTS floats: W1 (128 x 77), b1, W2 (128 x 128), b2,
 * W3 (2 x 128), b3 (all row-major), then the feature mean and scale (77 each;
 * features are standardised as (x - mean) * scale).
 */
#define FMO_MLP_N_WEIGHTS 26908
/* Random initial weights (seeded), mean 0 / scale 1. */
fmo_status fmo_mlp_init(fmo_ctx *ctx, uint64_t seed);
/* Copy n = FMO_MLP_N_WEIGHTS host floats in; the Adam state is cleared. */
fmo_status fmo_mlp_set_weights(fmo_ctx *ctx, const float *w, int64_t n);
/* *n = FMO_MLP_N_WEIGHTS; with w non-NULL the weights are copied out. */
fmo_status fmo_mlp_get_weights(fmo_ctx *ctx, float *w, int64_t *n);
/* Two-pass prediction for the current coordinates: n_shell values in the
 * output order of fmo_get_monomers. */
fmo_status fmo_mlp_predict(fmo_ctx *ctx, double *shell_dq);
/*
 * Train on the GPU against converged monomer charges of the current system
 * (same atoms, fragments and charges) at n_frames geometries:
 *   xyz_frames  [n_frames][n_atoms][3] bohr, input atom order
 *   shell_dq    [n_frames][n_shell], the order of fmo_get_monomers
 * The feature mean and scale are set from the frames, then `epochs` passes
 * of Adam (learning rate lr) over shuffled batches of batch_frames frames
 * minimise the mean squared error of the two-pass prediction (the potential
 * feature from the current model's first pass, held fixed in the gradient).
 * loss_per_epoch (optional, [epochs]) receives the mean loss of each epoch.
 * Device memory: about 2 GB per 1000 frames of 3000 atoms.
 */
fmo_status fmo_mlp_train(fmo_ctx *ctx, int32_t n_frames, const double *xyz_frames, const double *shell_dq,
                         int32_t epochs, int32_t batch_frames, double lr, uint64_t seed, double *loss_per_epoch);

/*
 * Loss and weight gradient of the current model on n_frames frames (same
 * layouts as fmo_mlp_train), without an update and with the current feature
 * mean and scale: *loss = the mean squared error of the two-pass prediction
 * (the potential feature from the first pass, held fixed in the gradient),
 * grad[FMO_MLP_N_TRAINED] (or NULL) its gradient in the flat weight layout
 * (W1, b1, W2, b2, W3, b3).  The GPU backward kernels of the training step.
 */
#define FMO_MLP_N_TRAINED 26754
fmo_status fmo_mlp_loss_grad(fmo_ctx *ctx, int32_t n_frames, const double *xyz_frames, const double *shell_dq,
                             double *loss, float *grad);

/*
 * Run the FMO calculation (Sec. 2.3): coordination numbers of the whole
 * system, monomer SCCs iterated to self-consistency in each other's ESP,
 * n-mer selection, SCC dimers (and trimers) in the frozen ESP, ES-DIM pairs,
 * and the FMO sums of Eqs. 12-19.  Work is issued on `cuda_stream` (NULL: the
 * context's own stream); the call returns after the results are on the host.
 * Returns FMO_ERR_NOT_CONVERGED if any SCC or the monomer loop hit its limit
 * (results are still readable), FMO_ERR_TIMEOUT if the deadline passed.
 */
fmo_status fmo_run(fmo_ctx *ctx, const fmo_options *opt, void *cuda_stream);

/* Totals of the last run: FMO1 = sum E_I, FMO2 (Eq. 12), FMO3 (Eq. 16; NaN
 * unless level 3).  Any pointer may be NULL. */
fmo_status fmo_get_energy(fmo_ctx *ctx, double *e_fmo1, double *e_fmo2, double *e_fmo3);

/* Number of shells of the whole system (length of shell_dq below). */
fmo_status fmo_get_sizes(fmo_ctx *ctx, int32_t *n_shell, int32_t *n_ao);

/* Monomer results: E_I[n_frag] internal energies, shell_dq[n_shell] (fragments
 * in index order, atoms in input order within a fragment, shells in table
 * order), iters[n_frag] SCC iterations of the final outer pass,
 * status[n_frag] FMO_SCC_* words.  Any pointer may be NULL. */
fmo_status fmo_get_monomers(fmo_ctx *ctx, double *E_I, double *shell_dq, int32_t *iters,
                            int32_t *status);

/* Pairs I<J of the last run in lexicographic order; *n receives the count
 * n_frag(n_frag-1)/2.  ij[2n], dE[n] (dE_IJ of Eq. 12 or Eq. 15), e_dimer[n]
 * (internal E_IJ, NaN for ES-DIM), dEV[n] (Eq. 13), scc[n] (1 = SCC dimer),
 * iters[n].  Any array pointer may be NULL. */
fmo_status fmo_get_dimers(fmo_ctx *ctx, int64_t *n, int32_t *ij, double *dE, double *e_dimer,
                          double *dEV, uint8_t *scc, int32_t *iters);

/* SCC trimers I<J<K of the last level-3 run: ijk[3n], dE3[n] (Eq. 17),
 * corr[n] (dE_IJK - dE_IJ - dE_IK - dE_JK). */
fmo_status fmo_get_trimers(fmo_ctx *ctx, int64_t *n, int32_t *ijk, double *dE3, double *corr);

/*
 * Nuclear gradient dE/dxyz (Eh/bohr) of the FMO energy of the last fmo_run at
 * its level (FMO1, FMO2 or FMO3), grad[3*n_atoms] in the input atom order
 * (host memory, caller-owned).  Analytic (Sec. 2.4 of the paper): for every
 * monomer and SCC dimer and trimer, the GFN1-xTB gradient of its converged
 * density in its embedding potential (Eqs. 23-28: P dH0 + W dS + the Coulomb
 * and repulsion terms, the Pi and CN parts of dH0) times its FMO2/FMO3
 * coefficient; the charge-transfer part of dE^V (Eq. 13) and the ES-DIM pairs
 * (Eq. 15); the coordination numbers of the whole system; and the response of
 * the monomer charges through the self-consistent Z-vector, solved in charge
 * space: (1 - Gamma chi) z = w with the monomers' coupled-perturbed
 * susceptibilities chi, by GMRES on the GPU.  All in FP64.
 * Needs a run whose dimer and trimer densities are converged in FP64
 * (precision FP64, or mixed with want_gradient = 1).
 * Fermi occupations (Eq. 6) are taken as they are, fractional ones included.
 * Errors: FMO_ERR_ARG (NULL), FMO_ERR_STATE (no run), FMO_ERR_UNSUPPORTED
 * (cut bonds, a run without FP64 n-mer densities, a trimer holding an
 * ES-DIM pair), FMO_ERR_NOT_CONVERGED (Z-vector or eigen-solve),
 * FMO_ERR_CUDA.
 */
fmo_status fmo_get_gradient(fmo_ctx *ctx, double *grad);

fmo_status fmo_get_stats(fmo_ctx *ctx, fmo_stats *st);

/*
 * SCC solve of one molecule that allocates no device memory.
 *
 * For callers that cannot allocate device memory while they run: real-time
 * loops that forbid allocation after start-up (an allocation may block or
 * fail at any moment), or hosts whose memory manager owns all device memory
 * (a framework's caching allocator would not see a cudaMalloc made behind
 * its back).  The paper has no counterpart; it is a packaging of the
 * library's own kernels.
 *
 * Solves the GFN1-xTB SCC of one closed-shell molecule (one fragment) from a
 * neutral guess, optionally in an external shell potential, with the table
 * *p and the tolerances, iteration limit and precision of *opt.  Results
 * equal those of fmo_run on a one-fragment system (E_I and shell charges).
 *   Z[n_atoms]           host atomic numbers (1 <= n_atoms <= 128)
 *   xyz_dev[3*n_atoms]   device coordinates (bohr), atom-major
 *   charge               net charge of the molecule (e)
 *   esp_dev[n_shell]     device external potential per shell (Eh/e), or NULL;
 *                        it enters the Fock matrix as 1/2 S (v_mu + v_nu)
 *   energy_dev[1]        device output: the internal energy E = E_el + E_rep
 *                        (Eh) of the converged density; the interaction
 *                        sum_s v_s dq_s with the potential is not included
 *   shell_dq_dev[n_shell] device output: shell charges, table order per atom
 *   status_dev[1]        device output (or NULL): FMO_SCC_* word
 *   cuda_stream          stream for all work (NULL: the legacy default stream)
 *   err[err_len]         host buffer for a message (or NULL)
 * Limits: at most 256 basis functions, 128 shells and 128 atoms; larger
 * molecules return FMO_ERR_ARG with a message.  The call enqueues the work
 * and returns; read the outputs after the stream has finished.
 * Memory: all scratch (about 5 MiB) is one fixed device array that every
 * GPU loading the library holds until the process exits.  The first call on
 * a device looks up that array's device address (once per device, guarded
 * against concurrent first calls); a cudaDeviceReset() invalidates it, and
 * calls after a reset are not supported.  All calls share the array and it
 * keeps the last call's contents, so calls that overlap on the GPU (other
 * streams, other host threads) race: serialise them.
 * Errors: FMO_ERR_ARG (NULL pointers, sizes, open shell, more electrons than
 * the basis holds, unknown element), FMO_ERR_UNSUPPORTED, FMO_ERR_CUDA
 * (launch or copy failure).
 */
fmo_status fmo_scc_solve_noalloc(const fmo_params *p, int32_t n_atoms, const int32_t *Z,
                                 const double *xyz_dev, int32_t charge, const double *esp_dev,
                                 const fmo_options *opt, double *energy_dev, double *shell_dq_dev,
                                 int32_t *status_dev, void *cuda_stream, char *err, int32_t err_len);

/*
 * Occupied-subspace projectors of a batch of symmetric matrices by
 * second-order spectral-projection purification (SP2), the matrix-product
 * alternative to the diagonalisation in each SCC iteration (Introduction:
 * diagonalisation is the cubic step; Methodology, GFN1-xTB SCC).  For every
 * b < batch:
 *   D_b = sum_{i < n_occ[b]} c_i c_i^T,  F_b c_i = e_i c_i,  e ascending,
 * the zero-temperature density with occupation one (a closed-shell density
 * is 2 D_b); unique when e_{n_occ-1} < e_{n_occ}.
 *   F_dev      device, batch x n x n doubles, row-major, symmetric (read only)
 *   n_occ_dev  device, batch int32 occupied-orbital counts, 0..n
 *   n          1..FMO_SP2_MAX_N;  batch >= 0 (0: nothing is launched)
 *   max_iter   >= 1, purification steps per matrix (the step count grows
 *              with the logarithm of the spectrum-to-gap ratio: a ratio
 *              of ~11 takes 31-35 steps in FP64)
 *   D_dev      device, batch x n x n doubles, output
 *   work_dev   device, batch x n x n doubles of caller-owned scratch
 *   iters_dev  device, batch int32 output: steps taken, -1 not converged
 *              within max_iter (or no gap at n_occ), -2 n_occ out of range
 *   cuda_stream  stream the kernel is enqueued on (NULL: default stream);
 *              the call returns without waiting.
 * FP64 throughout; one CTA per matrix.  Allocates nothing.  Errors:
 * FMO_ERR_ARG (sizes, NULL pointers), FMO_ERR_CUDA (launch failure).
 */
#define FMO_SP2_MAX_N 2048
fmo_status fmo_sp2_projector(const double *F_dev, const int32_t *n_occ_dev, int32_t n,
                             int32_t batch, int32_t max_iter, double *D_dev, double *work_dev,
                             int32_t *iters_dev, void *cuda_stream);

/*
 * The same projectors in FP32 (float buffers, FP32 products; traces and the
 * step choice in FP64), the precision of the loose iterations of a
 * mixed-precision SCC (Methodology, GFN1-xTB SCC; the FP32 phase before the
 * FP64 finish).  Arguments, layout, ownership and errors as for
 * fmo_sp2_projector.  The stop test is opened once the idempotency error is
 * below 1e-2; the result is idempotent to ~n * 1e-7 and equals the FP64
 * projector to ~1e-5 for well-conditioned gaps.
 */
fmo_status fmo_sp2_projector_f32(const float *F_dev, const int32_t *n_occ_dev, int32_t n,
                                 int32_t batch, int32_t max_iter, float *D_dev, float *work_dev,
                                 int32_t *iters_dev, void *cuda_stream);

/*
 * Measured FMA throughput of CUDA device `device` in TFLOP/s (2 flops per
 * FMA): precision FMO_PREC_MIXED measures FP32, FMO_PREC_FP64 FP64.  A
 * diagnostic for the roofline of the SCC kernel; the paper has no
 * counterpart.  Runs an FMA-loop kernel (8 blocks of 256 threads per SM,
 * eight independent FMA chains per thread) on a private stream and returns
 * the best of five timed launches.  Allocates and frees 8 bytes of device
 * memory.  Errors: FMO_ERR_ARG (NULL, unknown precision), FMO_ERR_CUDA.
 */
fmo_status fmo_fma_peak(int32_t precision, int32_t device, double *tflops);

/* Message of the last error on this context ("" if none). */
const char *fmo_last_error(const fmo_ctx *ctx);

/* Free the context and its device memory.  NULL is allowed. */
void fmo_destroy(fmo_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* FMO_XTB_H */
