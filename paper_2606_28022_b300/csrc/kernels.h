// Launch interface between the host library (capi.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include "fmo_device.cuh"

namespace fmo {

// per-n-mer status words (same values as the FMO_SCC_* enum of fmo_xtb.h)
constexpr int FMO_SCC_CONVERGED_CODE = 0;
constexpr int FMO_SCC_MAX_ITER_CODE = 1;
constexpr int FMO_SCC_NAN_CODE = 2;
constexpr int FMO_SCC_TIMEOUT_CODE = 3;
constexpr int FMO_SCC_JACOBI_CODE = 4;

// Layout of the diagnostic trace buffer (kTraceLen doubles) of the first
// block of an SCC launch: [1, 512) residual per iteration, [512, 1024)
// Jacobi sweeps, [1024, 1536) SM cycles per iteration ([1024] the setup,
// [1535] the FP64 energy finish), then kTraceNParts sums of the cycles of the
// parts of an SCC iteration (Fock, MO-basis transform, occupations and
// rotation generator, rotation or Jacobi, density, populations, energy).
constexpr int kTraceParts = 1536;
constexpr int kTraceNParts = 7;
// two 64-bit counters over all blocks follow: (cycles << 20 | block) of the
// slowest block, and the number of Jacobi eigen-solves
constexpr int kTraceSlowest = kTraceParts + kTraceNParts;
constexpr int kTraceJacobi = kTraceSlowest + 1;
constexpr int kTraceLen = kTraceJacobi + 1;

struct SccLaunch {
  const Nmer* nmers;
  const int* order;
  FragTab ft;
  const double* xyz;
  const int* elem;
  const int* atom_sh0;
  const DevElem* el;
  GParams g;
  const double* S;
  const double* H0;
  const double* gam;
  double* CTd;
  double* W1d;
  double* W2d;
  double* Agd;
  float* CTf;
  float* W1f;
  float* W2f;
  float* Agf;
  const double* phi;
  const double* vhop;   // per-n-mer hybrid orbital projectors (null without cut bonds)
  const double* hop_Qd; // their factors (hop_projector_kernel), or null
  const float* hop_Qf;
  const double* hop_Dd;
  const float* hop_Df;
  const int* hop_nq;
  const double* dq_mono;
  double* esp;
  double* dq;
  double* eps;
  double* hist;
  double* energy;
  double* e_el;
  double* e_rep;
  double* dEV;
  int* iters;
  int* iters32;   // iterations spent in the FP32 phase
  int* status;
  int guess_from_mono;
  int precision;
  int max_iter;
  int fp32_cap;
  int single_step;
  int step_phase;
  int reortho;
  int cold_refine;
  int reortho32;
  const int* step_dev;   // graph-launched FP32 steps: steps done before this one (sets reortho32 on the device)
  double jac_hint;
  const double* jac_hint_dev;
  const float* S32;   // mixed precision: FP32 copies of S and H0 (launch_to_float)
  const float* H32;
  double* trace;
  int fp64_finish;
  int energy_finish;
  int cold_steps;
  int first_rot;
  double first_jac_tol;
  double tol, etol, switch_tol;
  double jacobi_tol_d, jacobi_tol_f;
  const unsigned long long* t0;   // device timestamp of the run start
  unsigned long long budget_ns;   // 0 = no deadline
  int a_smem_d, a_smem_f;
  int ctas_per_sm;   // 0: rule (two CTAs per SM when the eigen-solve matrix is in global memory), 1 or 2
  int max_n, max_nsh, max_nat;
};

cudaError_t launch_cn(cudaStream_t st, int n_atoms, const double* xyz, const int* elem, const DevElem* el,
                      GParams g, double* cn, const int* ghost_src = nullptr);
cudaError_t launch_integrals(cudaStream_t st, int n_nmer, int max_pairs, const Nmer* nmers, FragTab ft,
                             const double* xyz, const int* elem, const int* atom_sh0, const double* cn,
                             const DevElem* el, const double* kab, int ne, GParams g, double* S, double* H0,
                             const Nmer* mono = nullptr, const double* mono_S = nullptr,
                             const double* mono_H0 = nullptr, const PrimPair* prim = nullptr);
cudaError_t launch_gamma(cudaStream_t st, int n_nmer, int max_nsh, const Nmer* nmers, FragTab ft,
                         const double* xyz, const int* elem, const int* sh_atom, const double* sh_inv_eta,
                         GParams g, double* gam);
cudaError_t launch_lowdin(cudaStream_t st, int n_nmer, int max_n, const Nmer* nmers, const double* S,
                          void* CT, void* W, void* Ag, int use_float, int a_in_smem, int* status,
                          void* W2 = nullptr);   // W2: spare n x n per n-mer (FP32: Newton-Schulz start)
size_t scc_smem_size(int max_n, int max_nsh, int max_nat, int a_bytes);
cudaError_t launch_scc(cudaStream_t st, int n_nmer, const SccLaunch& L);
cudaError_t launch_warm_start(cudaStream_t st, int n_nmer, const Nmer* nmers, const Nmer* mono, const float* mono_ct,
                              float* ct);
int phi_chunks(int n_sh);
cudaError_t launch_phi(cudaStream_t st, int n_sh, const double* xyz, const int* sh_atom, const double* sh_inv_eta,
                       const double* dq, GParams g, double* phi, double* part, int use_float = 0);
cudaError_t launch_gamma_full(cudaStream_t st, int n_sh, const double* xyz, const int* sh_atom,
                              const double* sh_inv_eta, GParams g, double* gam);
cudaError_t launch_phi_gemv(cudaStream_t st, int n_sh, const double* gam, const double* dq, double* phi);
// V^HOP (n x n per n-mer) and, with Qd non-null, its factors V = Q^T D Q:
// Qd/Qf kHopCols x n per n-mer at kHopCols * nm.aov, Dd/Df kHopCols^2 per
// n-mer, nq[n-mer] rows used
cudaError_t launch_hop_projector(cudaStream_t st, int n_nmer, const Nmer* nmers, FragTab ft, const double* xyz,
                                 const int* elem, const DevElem* el, double v_hop, const double* S, double* V,
                                 double* Qd = nullptr, float* Qf = nullptr, double* Dd = nullptr, float* Df = nullptr,
                                 int* nq = nullptr);
// FP32 steps of the global monomer loop inside a CUDA graph: the same stall
// and hand-over bookkeeping as the host-driven loop, on the device
struct Phase32State {
  double min32;   // best residual of the FP32 steps
  int stall32;    // steps since its last 10% improvement
  int n32;        // FP32 steps taken
  int hand_over;  // 1: the FP32 phase ended (converged to the switch tolerance, cap, or stall)
};
cudaError_t launch_loop_control32(cudaStream_t st, unsigned long long handle, const void* mix_state,
                                  Phase32State* p32, int* outer, int max_outer, double switch_tol, int cap32,
                                  int stall_limit);
cudaError_t launch_loop_control(cudaStream_t st, unsigned long long handle, const void* mix_state, int* outer,
                                int max_outer);
cudaError_t launch_frag_bounds(cudaStream_t st, int n_frag, FragTab ft, const double* xyz, double* bounds);
cudaError_t launch_pair_distance(cudaStream_t st, int n_frag, FragTab ft, const double* xyz, const double* bounds,
                                 double cut, double* rmin);
cudaError_t launch_esdim(cudaStream_t st, int n_pairs, const int2* pairs, const long long* out_idx, FragTab ft,
                         const double* xyz, const int* sh_atom, const double* sh_inv_eta, const double* dq,
                         GParams g, double* out, const double* gam_full = nullptr, int n_sh = 0);
// ---------------------------------------------------------------------------
// Analytic FMO gradient (fmo_gradient.cu).  Every monomer and SCC n-mer X of
// the FMO energy enters as a term with coefficient m (the FMO2/FMO3
// inclusion-exclusion counts); the charge-space Z-vector z of the monomer
// charges carries the response.

enum { kGradMonomer = 0, kGradNmer = 1, kGradResponse = 2 };

struct GradTerm {
  Nmer nm;              // layout of the n-mer in its pass
  const double* S;      // its overlap, H0 (n x n) and gamma block (nsh x nsh)
  const double* H0;
  const double* gam;
  const double* CT;     // energy terms: FP64 orbital rows of the converged solve
  const double* eps;    //               and their orbital energies
  const double* dq;     // its converged shell charges (nsh)
  const double* esp;    // its embedding potential ESP^{not X} (nsh); null for response terms
  double* Pa;           // n x n: density (energy) or first-order density (response)
  double* W;            // n x n: energy-weighted density, or its first-order change
  const double* Pb;     // response terms: the monomer density (n x n), else null
  double* sa;           // nsh: shell shifts of the converged solve (ESP included)
  const double* sb;     // response terms: first-order shell shifts, else null
  const double* qb;     // response terms: first-order charges, else null (1/2 dq)
  double* work;         // energy terms: 3 n^2 doubles of scratch
  double m;             // coefficient of the term
  double es;            // SCC dimers at level >= 2: 1 (its pair leaves the all-pairs ES-DIM form)
  int kind;             // kGradMonomer, kGradNmer, kGradResponse
  int with_rep;
  long long aslot;      // offset of its per-atom slots (nat x 4: g, F)
  long long sslot;      // offset of its per-shell slots (nsh x 2: w, d)
};

// One monomer's response data (kernels fmo_gradient.cu): canonical orbitals
// and energies at its converged charges, and its susceptibility chi.
struct MonoResp {
  double* C;            // n x n canonical orbital rows
  double* eps;          // n: their orbital energies
  double* focc;         // n: their Fermi occupations (Eq. 6)
  double* chi;          // nsh x nsh
  double* sig;          // nsh: shell shifts (ESP included)
  double* work;         // scratch: 7 n^2 + npad^2 + 3 nsh^2 doubles
};

struct GradLaunch {
  FragTab ft;
  const double* xyz;
  const int* elem;
  const int* atom_sh0;
  const DevElem* el;
  const double* kab;
  int ne;
  const PrimPair* prim;
  const double* cn;
  GParams g;
  const double* dq_mono;  // converged monomer charges, global shell order
  int max_n, max_nsh, max_nat;
};

// energy terms: occupations, density P, shifts, energy-weighted density W~
cudaError_t launch_grad_prep(cudaStream_t st, int n_terms, const GradTerm* terms, const GradLaunch& L, int* flag);
// explicit gradient of every term into its slots (sslots may be null for response terms)
cudaError_t launch_grad_explicit(cudaStream_t st, int n_terms, const GradTerm* terms, const GradLaunch& L,
                                 double* aslots, double* sslots);
// per atom (and shell), fixed order: sum of the slots of the entries of its
// fragment (frag_ptr CSR; ent_aoff / ent_soff slot offsets of the fragment's
// first atom / shell, ent_soff < 0: no shell slots); g_atom[n_atoms][4],
// w[n_sh], d[n_sh]; accumulate: add to the outputs instead of overwriting
cudaError_t launch_grad_gather(cudaStream_t st, int n_atoms, int n_sh, const GradLaunch& L, const int* atom_frag,
                               const int* sh_frag, const int* frag_ptr, const long long* ent_aoff,
                               const long long* ent_soff, const double* aslots, const double* sslots,
                               double* g_atom, double* w, double* d, int accumulate);
// monomers: canonical orbitals, susceptibility chi (flag |= 2: eigen-solve
// not converged)
cudaError_t launch_grad_mono_response(cudaStream_t st, int n_mono, const GradTerm* mono_terms, MonoResp* mr,
                                      const GradLaunch& L, int* flag);
// Z-vector operator pieces: y = chi z (block diagonal); out = the monomers'
// own gamma blocks times v (sh0: first global shell of each monomer)
cudaError_t launch_chi_apply(cudaStream_t st, int n_mono, const GradTerm* mono_terms, const MonoResp* mr,
                             const int* sh0, const double* z, double* y);
cudaError_t launch_intra_gamma(cudaStream_t st, int n_mono, const GradTerm* mono_terms, const int* sh0,
                               const double* v, double* out);
// out[j] = V_j . u (j < k, rows of V ldv apart); u -= sum_j h_j V_j;
// out = a x + b y + c z (y, z may be null)
cudaError_t launch_vec_dots(cudaStream_t st, int n, int k, const double* V, long long ldv, const double* u,
                            double* out);
cudaError_t launch_vec_update(cudaStream_t st, int n, int k, const double* V, long long ldv, const double* h,
                              double* u);
cudaError_t launch_vec_lincomb3(cudaStream_t st, int n, double a, const double* x, double b, const double* y,
                                double c, const double* z, double* out);
// monomers: first-order P, W~ and shifts along the Z-vector potential z
// (y = chi z), into the response terms
cudaError_t launch_grad_first_order(cudaStream_t st, int n_mono, const GradTerm* resp_terms, const MonoResp* mr,
                                    const GradLaunch& L, const double* z, const double* y);
// per atom: gathered term gradient + CN chain rule sum_A F_A dCN_A + the
// inter-fragment Coulomb sum over (a_s q_t + q_s a_t) dgamma_st
cudaError_t launch_grad_cn_coulomb(cudaStream_t st, int n_atoms, int n_sh, const GradLaunch& L,
                                   const int* atom_frag, const int* sh_atom, const double* sh_inv_eta,
                                   const double* a, const double* g_atom, double* grad);
// largest dynamic shared memory of the gradient kernels for these maxima
size_t grad_smem_max(const GradLaunch& L);

// out[i] = (float)in[i], i < n
cudaError_t launch_to_float(cudaStream_t st, long long n, const double* in, float* out);
cudaError_t launch_stamp(cudaStream_t st, unsigned long long* t);
cudaError_t launch_global_mix(cudaStream_t st, int n, double* x, const double* xo, int nf, const double* e,
                              double* hist, void* state, double tol, double etol, int allow_converge);
size_t mix_state_bytes();
// number of kernels launched by this library so far (all threads and contexts)
long long launch_count();
void note_launch();
cudaError_t launch_maxdiff(cudaStream_t st, int n, const double* a, const double* b, double* out);
cudaError_t launch_fmo_sum(cudaStream_t st, int n_frag, const double* e_mono, long long n_pair, const int* pair_scc,
                           const double* e_dim, const double* dEV_dim, double* dE_pair, int n_tri,
                           const int* tri_frag, const double* e_tri, const double* dEV_tri, double* dE3,
                           double* corr, double* totals);
cudaError_t launch_gather_xyz(cudaStream_t st, int n_atoms, const int* perm, const double* in, double* out);

}  // namespace fmo
