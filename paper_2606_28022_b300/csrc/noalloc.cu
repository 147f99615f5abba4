// fmo_scc_solve_noalloc: the SCC solve of one molecule with no device
// allocation at all.
//
// Some callers cannot allocate device memory while they run: real-time or
// embedded loops that forbid allocation after start-up (an allocation can
// block or fail at any time), and hosts whose memory manager hands out every
// byte ahead of time (for example a framework's caching allocator, which
// would see a cudaMalloc behind its back as memory it cannot account for).
// For them this file keeps all the scratch that the SCC kernels need (the
// n x n matrices, gamma block, charge vectors, Broyden history and index
// tables) in one fixed device array that exists from library load until
// process exit.
//
// The kernels are the library's own (kernels.cu); only where their scratch
// lives differs from fmo_run.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/fmo_xtb.h"
#include "kernels.h"

using namespace fmo;

namespace {

constexpr int kNaMaxAO = 256;      // basis functions of the molecule
constexpr int kNaMaxShell = 128;   // shells
constexpr int kNaMaxAtom = 128;    // atoms
constexpr size_t kNaBytes = 5120 * 1024;   // 5 MiB

// The scratch of every call, on every device that loads the library.  Host
// code must not pass this symbol to a kernel (on the host it is only a
// stand-in); it uses the device address from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of the array, looked up once per device (with that device
// current) by the first call on it.  The lookup is guarded: host threads may
// make their first calls at the same time.  A cudaDeviceReset() destroys the
// context the address belongs to; calls after a reset are not supported.
constexpr int kNaMaxDevices = 64;
void* g_noalloc_addr[kNaMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

void set_error(char* buf, int len, const char* msg) {
  if (buf && len > 0) {
    std::strncpy(buf, msg, (size_t)len - 1);
    buf[len - 1] = '\0';
  }
}

// Bump layout of the scratch array (256-byte aligned regions).
struct Layout {
  unsigned char* base;
  size_t used = 0;
  template <typename T> T* take(size_t count) {
    used = (used + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + used);
    used += sizeof(T) * count;
    return p;
  }
};

}  // namespace

extern "C" fmo_status fmo_scc_solve_noalloc(const fmo_params* p, int32_t n_atoms, const int32_t* Z,
                                            const double* xyz_dev, int32_t charge, const double* esp_dev,
                                            const fmo_options* opt, double* energy_dev,
                                            double* shell_dq_dev, int32_t* status_dev, void* cuda_stream,
                                            char* err, int32_t err_len) {
  if (!p || !Z || !xyz_dev || !opt || !energy_dev || !shell_dq_dev) {
    set_error(err, err_len, "NULL argument");
    return FMO_ERR_ARG;
  }
  if (n_atoms < 1 || n_atoms > kNaMaxAtom) {
    set_error(err, err_len, "n_atoms out of range: this entry point takes 1..128 atoms");
    return FMO_ERR_ARG;
  }
  const fmo_options o = *opt;
  if (o.precision != FMO_PREC_FP64 && o.precision != FMO_PREC_MIXED) {
    set_error(err, err_len, "unknown precision mode");
    return FMO_ERR_ARG;
  }
  if (o.max_iter < 1 || !(o.scc_tol > 0) || !(o.e_tol > 0)) {
    set_error(err, err_len, "iteration limit and tolerances must be positive");
    return FMO_ERR_ARG;
  }
  // ---- host-side tables (no device allocation)
  int ez[kMaxElem];
  int z_to_e[FMO_MAX_Z];
  for (int z = 0; z < FMO_MAX_Z; ++z) z_to_e[z] = -1;
  int ne = 0;
  std::vector<int> elem(n_atoms), atom_sh0(n_atoms), sh_atom;
  std::vector<double> inv_eta;
  int nsh = 0, nao = 0;
  double nel = -double(charge);
  for (int i = 0; i < n_atoms; ++i) {
    const int z = Z[i];
    if (z <= 0 || z >= FMO_MAX_Z || p->el[z].n_shell == 0) {
      set_error(err, err_len, "element not in the table");
      return FMO_ERR_ARG;
    }
    if (z_to_e[z] < 0) {
      if (ne >= kMaxElem) { set_error(err, err_len, "too many distinct elements"); return FMO_ERR_UNSUPPORTED; }
      z_to_e[z] = ne;
      ez[ne++] = z;
    }
    const fmo_element& e = p->el[z];
    elem[i] = z_to_e[z];
    atom_sh0[i] = nsh;
    for (int s = 0; s < e.n_shell; ++s) {
      if (e.l[s] < 0 || e.l[s] > 1 || e.n_prim[s] < 1 || e.n_prim[s] > FMO_MAX_PRIM) {
        set_error(err, err_len, "unsupported shell in the table");
        return FMO_ERR_ARG;
      }
      sh_atom.push_back(i);
      inv_eta.push_back(1.0 / ((1.0 + e.kappa_l[s]) * e.eta));
      nao += 2 * e.l[s] + 1;
      nel += e.q0_l[s];
      ++nsh;
    }
  }
  if (nao > kNaMaxAO || nsh > kNaMaxShell) {
    set_error(err, err_len, "molecule too large: this entry point takes at most 256 basis functions and 128 shells");
    return FMO_ERR_ARG;
  }
  if (std::fabs(nel - std::round(nel)) > 1e-9 || (long long)std::llround(nel) % 2 != 0 || nel <= 0) {
    set_error(err, err_len, "not a closed-shell molecule");
    return FMO_ERR_ARG;
  }
  if (nel > 2.0 * nao) {
    set_error(err, err_len, "more electrons than the basis holds (charge too negative)");
    return FMO_ERR_ARG;
  }
  std::vector<DevElem> h_el(ne);
  for (int k = 0; k < ne; ++k) {
    const fmo_element& src = p->el[ez[k]];
    DevElem d{};
    d.nsh = src.n_shell;
    for (int s = 0; s < src.n_shell; ++s) {
      d.l[s] = src.l[s];
      d.nprim[s] = src.n_prim[s];
      for (int q = 0; q < src.n_prim[s]; ++q) {
        const double a = src.alpha[s][q];
        double norm = std::pow(2.0 * a / M_PI, 0.75);
        if (src.l[s] == 1) norm *= 2.0 * std::sqrt(a);
        d.alpha[s][q] = a;
        d.cn[s][q] = src.coef[s][q] * norm;
      }
      d.h[s] = src.h_l[s];
      d.kcn[s] = src.k_cn_l[s];
      d.kpoly[s] = src.k_poly_l[s];
      d.eta_sh[s] = (1.0 + src.kappa_l[s]) * src.eta;
      d.q0[s] = src.q0_l[s];
    }
    d.gamma3 = src.gamma3; d.en = src.en; d.rcov = src.r_cov; d.zeff = src.z_eff; d.arep = src.alpha_rep;
    h_el[k] = d;
  }
  std::vector<double> kab((size_t)ne * ne);
  for (int a = 0; a < ne; ++a)
    for (int b = 0; b < ne; ++b) kab[(size_t)a * ne + b] = p->k_ab[ez[a]][ez[b]];
  GParams g;
  for (int l = 0; l < 3; ++l) g.k_l[l] = p->k_l[l];
  g.k_en = p->k_en; g.k_g = p->k_g; g.k_f = p->k_f;
  g.cn_k1 = p->cn_k1; g.cn_k2 = p->cn_k2; g.cn_cutoff = p->cn_cutoff;
  g.kT = 3.166811563e-6 * p->t_el;
  if (!(g.kT > 0)) { set_error(err, err_len, "electronic temperature must be positive"); return FMO_ERR_ARG; }

  // ---- once per device: the device address of the scratch array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    set_error(err, err_len, "no usable CUDA device");
    return FMO_ERR_CUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
      void* addr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr) {
        set_error(err, err_len, cudaGetErrorString(e));
        return FMO_ERR_CUDA;
      }
      g_noalloc_addr[dev] = addr;
    }
    base = g_noalloc_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // ---- scratch layout
  Layout L{reinterpret_cast<unsigned char*>(base)};
  const int n = nao, npad = n + (n & 1);
  double* S = L.take<double>((size_t)n * n);
  double* H0 = L.take<double>((size_t)n * n);
  double* CTd = L.take<double>((size_t)n * n);
  double* W1d = L.take<double>((size_t)n * n);
  double* W2d = L.take<double>((size_t)n * n);
  double* Agd = L.take<double>((size_t)npad * npad);
  float* CTf = L.take<float>((size_t)n * n);
  float* W1f = L.take<float>((size_t)n * n);
  float* W2f = L.take<float>((size_t)n * n);
  float* Agf = L.take<float>((size_t)npad * npad);
  float* S32 = L.take<float>((size_t)n * n);
  float* H32 = L.take<float>((size_t)n * n);
  double* gam = L.take<double>((size_t)nsh * nsh);
  double* espv = L.take<double>(nsh);
  double* dqv = L.take<double>(nsh);
  double* dq0 = L.take<double>(nsh);
  double* hist = L.take<double>((size_t)(2 * kHist + 2) * nsh);
  double* eps = L.take<double>(npad);
  double* outs = L.take<double>(4);
  double* cn = L.take<double>(n_atoms);
  double* d_inv_eta = L.take<double>(nsh);
  double* d_kab = L.take<double>((size_t)ne * ne);
  int* d_elem = L.take<int>(n_atoms);
  int* d_atom_sh0 = L.take<int>(n_atoms);
  int* d_sh_atom = L.take<int>(nsh);
  int* d_ft = L.take<int>(8);
  int* d_order = L.take<int>(1);
  int* d_it = L.take<int>(2);
  int* d_status = L.take<int>(1);
  DevElem* d_el = L.take<DevElem>(ne);
  Nmer* d_nm = L.take<Nmer>(1);
  if (L.used > kNaBytes) {
    set_error(err, err_len, "scratch layout exceeds the fixed array");
    return FMO_ERR_UNSUPPORTED;
  }
  Nmer nm{};
  nm.nfrag = 1;
  nm.frag[0] = 0; nm.frag[1] = -1; nm.frag[2] = -1;
  nm.n = n; nm.nsh = nsh; nm.nat = n_atoms; nm.npad = npad; nm.nel = nel;
  nm.mat = 0; nm.shv = 0; nm.gam = 0; nm.aov = 0; nm.hist = 0; nm.apad = 0;
  const int ft_h[8] = {0, n_atoms, 0, nsh, 0, n, 0, 0};
  const int zero_i = 0;
#define NA_CK(x)                                                        \
  do {                                                                  \
    const cudaError_t e_ = (x);                                         \
    if (e_ != cudaSuccess) { set_error(err, err_len, cudaGetErrorString(e_)); return FMO_ERR_CUDA; } \
  } while (0)
  // small tables: copies from pageable host memory, which the runtime stages
  // before each call returns (nothing is allocated)
  NA_CK(cudaMemcpyAsync(d_el, h_el.data(), sizeof(DevElem) * ne, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_kab, kab.data(), sizeof(double) * ne * ne, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_elem, elem.data(), sizeof(int) * n_atoms, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_atom_sh0, atom_sh0.data(), sizeof(int) * n_atoms, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_sh_atom, sh_atom.data(), sizeof(int) * nsh, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_inv_eta, inv_eta.data(), sizeof(double) * nsh, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_ft, ft_h, sizeof(ft_h), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_order, &zero_i, sizeof(int), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(d_nm, &nm, sizeof(Nmer), cudaMemcpyHostToDevice, st));
  // what must start at zero: the neutral guess, the status word
  NA_CK(cudaMemsetAsync(dq0, 0, sizeof(double) * nsh, st));
  NA_CK(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  FragTab ft{d_ft + 0, d_ft + 1, d_ft + 2, d_ft + 3, d_ft + 4, d_ft + 5};

  // ---- the SCC of the molecule: the library's kernels on the fixed scratch
  NA_CK(launch_cn(st, n_atoms, xyz_dev, d_elem, d_el, g, cn));
  NA_CK(launch_integrals(st, 1, n_atoms * (n_atoms + 1) / 2, d_nm, ft, xyz_dev, d_elem, d_atom_sh0, cn, d_el,
                         d_kab, ne, g, S, H0));
  NA_CK(launch_gamma(st, 1, nsh, d_nm, ft, xyz_dev, d_elem, d_sh_atom, d_inv_eta, g, gam));
  const bool use_f = (o.precision == FMO_PREC_MIXED);
  if (use_f) {   // FP32 copies of S and H0 for the FP32 iterations
    NA_CK(launch_to_float(st, (long long)n * n, S, S32));
    NA_CK(launch_to_float(st, (long long)n * n, H0, H32));
  }
  NA_CK(launch_lowdin(st, 1, n, d_nm, S, use_f ? (void*)CTf : (void*)CTd, use_f ? (void*)W1f : (void*)W1d,
                      use_f ? (void*)Agf : (void*)Agd, use_f ? 1 : 0, 0, d_status));
  SccLaunch sl{};
  sl.nmers = d_nm; sl.order = d_order; sl.ft = ft; sl.xyz = xyz_dev; sl.elem = d_elem; sl.atom_sh0 = d_atom_sh0;
  sl.el = d_el; sl.g = g; sl.S = S; sl.H0 = H0; sl.gam = gam;
  sl.CTd = CTd; sl.W1d = W1d; sl.W2d = W2d; sl.Agd = Agd; sl.CTf = CTf; sl.W1f = W1f; sl.W2f = W2f; sl.Agf = Agf;
  if (use_f) { sl.S32 = S32; sl.H32 = H32; }
  sl.phi = esp_dev;          // with zero monomer charges the ESP is exactly esp_dev
  sl.dq_mono = dq0;          // neutral guess, and nothing to subtract from the ESP
  sl.esp = espv; sl.dq = dqv; sl.eps = eps; sl.hist = hist;
  sl.energy = outs; sl.e_el = outs + 1; sl.e_rep = outs + 2; sl.dEV = outs + 3;
  sl.iters = d_it; sl.iters32 = d_it + 1; sl.status = d_status;
  sl.guess_from_mono = 1; sl.precision = o.precision; sl.max_iter = o.max_iter;
  sl.fp32_cap = std::max(4, o.max_iter / 2); sl.single_step = 0; sl.step_phase = 1; sl.reortho = 0;
  sl.cold_refine = 1; sl.reortho32 = 0; sl.jac_hint = 1.0; sl.trace = nullptr;
  sl.cold_steps = 2; sl.first_rot = 0;
  sl.tol = o.scc_tol; sl.etol = o.e_tol; sl.switch_tol = o.mixed_switch_tol;
  sl.jacobi_tol_d = 1e-14; sl.jacobi_tol_f = 2e-7;
  sl.t0 = nullptr; sl.budget_ns = 0;
  sl.a_smem_d = 0; sl.a_smem_f = 0;     // the eigen-solve matrix lives in the fixed scratch
  sl.max_n = n; sl.max_nsh = nsh; sl.max_nat = n_atoms;
  NA_CK(launch_scc(st, 1, sl));
  NA_CK(cudaMemcpyAsync(energy_dev, outs, sizeof(double), cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaMemcpyAsync(shell_dq_dev, dqv, sizeof(double) * nsh, cudaMemcpyDeviceToDevice, st));
  if (status_dev) NA_CK(cudaMemcpyAsync(status_dev, d_status, sizeof(int), cudaMemcpyDeviceToDevice, st));
#undef NA_CK
  set_error(err, err_len, "");
  return FMO_OK;
}
