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
cudaError_t launch_hop_projector(cudaStream_t st, int n_nmer, const Nmer* nmers, FragTab ft, const double* xyz,
                                 const int* elem, const DevElem* el, double v_hop, const double* S, double* V);
cudaError_t launch_loop_control(cudaStream_t st, unsigned long long handle, const void* mix_state, int* outer,
                                int max_outer);
cudaError_t launch_frag_bounds(cudaStream_t st, int n_frag, FragTab ft, const double* xyz, double* bounds);
cudaError_t launch_pair_distance(cudaStream_t st, int n_frag, FragTab ft, const double* xyz, const double* bounds,
                                 double cut, double* rmin);
cudaError_t launch_esdim(cudaStream_t st, int n_pairs, const int2* pairs, const long long* out_idx, FragTab ft,
                         const double* xyz, const int* sh_atom, const double* sh_inv_eta, const double* dq,
                         GParams g, double* out, const double* gam_full = nullptr, int n_sh = 0);
// Analytic gradient of the GFN1-xTB energy of one n-mer that is one fragment
// without hybrid-orbital projection (gradient.cu): grad[nat][3] in the
// fragment's atom order; work holds 4 n^2 doubles; *frac (zeroed by the
// caller) is set to 1 if an occupation is fractional.
cudaError_t launch_xtb_gradient(cudaStream_t st, const Nmer* nm, int n, int nsh, int nat, FragTab ft,
                                const double* xyz, const int* elem, const int* atom_sh0, const DevElem* el,
                                const double* kab, int ne, const PrimPair* prim, const double* cn, GParams g,
                                const double* S, const double* H0, const double* CT, const double* eps,
                                const double* gam, double* work, double* grad, int* frac);
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
