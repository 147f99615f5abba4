// Host side of the C ABI declared in include/fmo_xtb.h: validation, the
// fragment/n-mer bookkeeping, device memory, and the order of the passes of
// Sec. 2.3 of the paper (monomer loop in the ESP, then dimers and trimers in
// the frozen ESP, then the FMO sums).  Every arithmetic step of the method
// runs in the kernels of kernels.cu.
#include <algorithm>
#include <random>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fmo_xtb.h"
#include "kernels.h"
#include "mlp.h"
#include <nvtx3/nvToolsExt.h>

using namespace fmo;

namespace {

// Grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) { p = nullptr; return e; }
    cap = want;
    return cudaSuccess;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
  void release() { if (p) cudaFree(p); p = nullptr; cap = 0; }
};

struct Pass {
  std::vector<Nmer> nm;
  std::vector<int> order;
  int max_n = 0, max_nsh = 0, max_nat = 0, max_pairs = 0;
  long long tot_mat = 0, tot_sh = 0, tot_gam = 0, tot_ao = 0, tot_hist = 0, tot_apad = 0;
  DevBuf d_nm, d_order, S, H0, S32, H32, gam, CTd, W1d, W2d, Agd, CTf, W1f, W2f, Agf, esp, dq, eps, hist;
  DevBuf energy, e_el, e_rep, dEV, iters, iters32, status;
  DevBuf V;                               // hybrid orbital projectors (n x n per n-mer)
  DevBuf hQd, hQf, hDd, hDf, hnq;         // their factors V = Q^T D Q (mixed precision)
  int max_healed_sh = 0, max_projected = 0;
  std::vector<int> h_iters, h_iters32;
  std::vector<int> owner;                 // sharded runs: rank of every n-mer (empty: all here)
  void release() {
    for (DevBuf* b : {&d_nm, &d_order, &S, &H0, &gam, &CTd, &W1d, &W2d, &Agd, &CTf, &W1f, &W2f, &Agf, &esp, &dq,
                      &eps, &hist, &energy, &e_el, &e_rep, &dEV, &iters, &iters32, &status, &V, &hQd, &hQf, &hDd,
                      &hDf, &hnq})
      b->release();
  }
};

// Pinned staging for every host <-> device copy (no pageable transfers).
// Regions are handed out from page-locked chunks; device->host results are
// copied to their destination after the stream is synchronised (flush), and
// all regions are recycled at that point.
struct Staging {
  struct Chunk { char* p; size_t cap; size_t used; };
  struct Pending { void* dst; const void* src; size_t bytes; };
  std::vector<Chunk> chunks;
  std::vector<Pending> pend;
  void* take(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    for (auto& c : chunks)
      if (c.cap - c.used >= bytes) { void* r = c.p + c.used; c.used += bytes; return r; }
    const size_t cap = std::max<size_t>(bytes, size_t(8) << 20);
    char* p = nullptr;
    if (cudaMallocHost((void**)&p, cap) != cudaSuccess) return nullptr;
    chunks.push_back({p, cap, bytes});
    return p;
  }
  void flush() {
    for (auto& q : pend) std::memcpy(q.dst, q.src, q.bytes);
    pend.clear();
    for (auto& c : chunks) c.used = 0;
  }
  void release() {
    for (auto& c : chunks) cudaFreeHost(c.p);
    chunks.clear();
    pend.clear();
  }
};

}  // namespace

struct fmo_ctx {
  int device = 0;
  // sharded runs: this rank, the number of ranks and the exchange callback
  int shard_rank = 0, shard_world = 1;
  fmo_exchange_fn ex_fn = nullptr;
  DevBuf d_p32;                           // FP32-phase bookkeeping of the graph-driven monomer loop
  void* ex_user = nullptr;
  cudaStream_t own_stream = nullptr;
  std::string err;
  fmo_params params;
  // compact element table
  int ne = 0;
  int z_to_e[FMO_MAX_Z];
  std::vector<DevElem> h_el;
  std::vector<double> h_kab;
  std::vector<PrimPair> h_prim;           // geometry-free primitive-pair factors
  DevBuf d_el, d_kab, d_prim;
  GParams g;
  int smem_optin = 0;
  // system
  bool have_system = false;
  int n_atoms = 0, n_frag = 0, n_sh = 0, n_ao = 0;
  // hybrid orbital projection: cut bonds, and the internal atom list (real
  // atoms, then per fragment the ghosts of the bonds whose BAA it holds)
  int n_cut = 0, n_int = 0;
  std::vector<int> h_ghost_frag, h_ghost_src, h_bda_baa_frag, h_hop_baa;
  struct GhostInfo { int bda_frag, nsh, nao; };
  std::vector<std::vector<GhostInfo>> f_ghosts;   // per hosting fragment
  std::vector<std::vector<int>> f_bda_baa_frag;   // per fragment: BAA fragment of each of its BDAs
  DevBuf d_ghost_frag, d_ghost_src, d_bda_baa_frag, d_hop_baa;
  // learned initial charges: weights (FP32 master + feature mean/scale, FP16
  // copy), Adam moments, per-system tables and inference buffers
  bool mlp_ready = false, mlp_tables_ok = false;
  DevBuf d_mlp_W, d_mlp_W16, d_mlp_m, d_mlp_v;
  DevBuf d_mlp_elem4, d_mlp_atom_frag, d_mlp_atom_ie, d_mlp_sh_ie, d_mlp_fcharge, d_mlp_err;
  DevBuf d_mlp_X, d_mlp_y, d_mlp_q;
  std::vector<int> perm;                  // internal atom i <- input atom perm[i]
  std::vector<int> h_elem, h_atom_sh0, h_sh_atom;
  std::vector<int> f_atom0, f_nat, f_sh0, f_nsh, f_ao0, f_nao;
  std::vector<double> f_nel, h_sh_inv_eta;
  std::vector<int> f_charge;
  DevBuf d_xyz, d_xyz_in, d_perm, d_elem, d_cn, d_atom_sh0, d_sh_atom, d_sh_inv_eta;
  DevBuf d_f_atom0, d_f_nat, d_f_sh0, d_f_nsh, d_f_ao0, d_f_nao;
  DevBuf d_gam_full;                      // gamma of all shell pairs (when it fits)
  bool gam_full_ok = false;
  DevBuf d_trace, d_dq_mono, d_phi, d_phi_part, d_bounds, d_rmin, d_scalar, d_t0, d_mix_hist, d_mix_state;
  DevBuf d_pair_scc, d_dE_pair, d_esdim_pairs, d_esdim_idx, d_tri_frag, d_dE3, d_corr, d_totals;
  std::vector<double> guess;
  bool have_guess = false;
  Pass mono, dim, tri;
  // results of the last run
  bool have_result = false;
  int last_level = 0;
  int last_precision = 0;
  bool grad_ready = false;                // the last run's n-mer densities are converged in FP64
  bool last_cuts_ok = false;              // trimers hold only SCC pairs (gradient bookkeeping)
  std::vector<int> r_pair_k;              // SCC-dimer index of every pair, -1 for ES-DIM
  DevBuf d_grad_work, d_grad;
  DevBuf d_gt, d_gslots_a, d_gslots_s, d_gpair, d_gfrag_ptr, d_gent_a, d_gent_s, d_gatom_frag, d_gsh_frag,
      d_gatom, d_gw, d_gd, d_gmono_terms, d_gmr, d_gmr_mem, d_gresp_terms, d_gresp_mem, d_gflag, d_gsh0,
      d_gkrylov, d_gz, d_gy, d_ga, d_gout;
  double totals[3] = {0, 0, 0};
  std::vector<double> r_e_mono, r_dq_mono, r_dE_pair, r_e_dim_pair, r_dEV_pair;
  std::vector<int> r_mono_iters, r_mono_status, r_pair_iters;
  std::vector<uint8_t> r_pair_scc;
  std::vector<int> r_tri;
  std::vector<double> r_dE3, r_corr;
  fmo_stats stats;
  Staging stg;
  int64_t h2d_bytes = 0, d2h_bytes = 0;

  FragTab ftab() const {
    FragTab t{d_f_atom0.as<int>(), d_f_nat.as<int>(), d_f_sh0.as<int>(),
              d_f_nsh.as<int>(), d_f_ao0.as<int>(), d_f_nao.as<int>()};
    if (n_cut > 0) {
      t.ghost_frag = d_ghost_frag.as<int>();
      t.ghost_src = d_ghost_src.as<int>();
      t.bda_baa_frag = d_bda_baa_frag.as<int>();
      t.hop_baa = d_hop_baa.as<int>();
    }
    return t;
  }
};

namespace {

fmo_status fail(fmo_ctx* c, fmo_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

#define CK(x)                                                                             \
  do {                                                                                    \
    cudaError_t e_ = (x);                                                                 \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? FMO_ERR_OOM : FMO_ERR_CUDA,     \
                  std::string(#x) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

// host <-> device copies through pinned staging, counted in the run statistics
fmo_ctx* g_ctx = nullptr;   // context of the current call (one host thread per context)

cudaError_t h2d(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  void* s = g_ctx->stg.take(bytes);
  if (!s) return cudaErrorMemoryAllocation;
  std::memcpy(s, src, bytes);
  g_ctx->h2d_bytes += (int64_t)bytes;
  return cudaMemcpyAsync(dst, s, bytes, cudaMemcpyHostToDevice, st);
}
// The host destination is written at the next sync_stream().
cudaError_t d2h(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  void* s = g_ctx->stg.take(bytes);
  if (!s) return cudaErrorMemoryAllocation;
  g_ctx->d2h_bytes += (int64_t)bytes;
  g_ctx->stg.pend.push_back({dst, s, bytes});
  return cudaMemcpyAsync(s, src, bytes, cudaMemcpyDeviceToHost, st);
}
cudaError_t sync_stream(cudaStream_t st) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) g_ctx->stg.flush();
  return e;
}

template <typename T>
cudaError_t upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
  cudaError_t e = b.ensure(sizeof(T) * std::max<size_t>(v.size(), 1));
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  return h2d(b.p, v.data(), sizeof(T) * v.size(), st);
}

// Geometry-free factors of every pair of primitives of the element table
// (layout of prim_pair_index), from the normalised contraction coefficients.
void build_prim_table(const std::vector<DevElem>& el, std::vector<PrimPair>& t) {
  const int ne = int(el.size());
  t.assign((size_t)ne * ne * kMaxShell * kMaxShell * kMaxPrim * kMaxPrim, PrimPair{0, 0, 0, 0, 0});
  for (int ea = 0; ea < ne; ++ea)
    for (int eb = 0; eb < ne; ++eb)
      for (int sa = 0; sa < el[ea].nsh; ++sa)
        for (int sb = 0; sb < el[eb].nsh; ++sb)
          for (int pa = 0; pa < el[ea].nprim[sa]; ++pa)
            for (int pb = 0; pb < el[eb].nprim[sb]; ++pb) {
              const double a = el[ea].alpha[sa][pa], b = el[eb].alpha[sb][pb];
              PrimPair q;
              q.ip = 1.0 / (a + b);
              q.abp = a * b * q.ip;
              q.ap = a * q.ip;
              q.bp = b * q.ip;
              q.pref = el[ea].cn[sa][pa] * el[eb].cn[sb][pb] * std::pow(M_PI * q.ip, 1.5);
              t[prim_pair_index(ne, ea, eb, sa, sb, pa, pb)] = q;
            }
}

int elem_nao(const DevElem& e) {
  int n = 0;
  for (int s = 0; s < e.nsh; ++s) n += 2 * e.l[s] + 1;
  return n;
}

// Longest-processing-time-first partition: units by decreasing cost (ties:
// lower index), each to the least loaded rank (ties: lower rank).
std::vector<int> lpt_owner(const std::vector<double>& cost, int world) {
  const size_t n = cost.size();
  std::vector<int> idx(n), owner(n, 0);
  for (size_t i = 0; i < n; ++i) idx[i] = int(i);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<double> load(std::max(world, 1), 0.0);
  for (int i : idx) {
    int r = 0;
    for (int q = 1; q < world; ++q)
      if (load[q] < load[r]) r = q;
    owner[i] = r;
    load[r] += cost[i];
  }
  return owner;
}

// Lay out a pass of n-mers (tuples of fragments) and size its buffers.
cudaError_t plan_pass(fmo_ctx* ctx, Pass& P, const std::vector<std::array<int, 3>>& tuples,
                      const std::vector<int>& nf, bool monomer_layout, int precision, cudaStream_t st) {
  P.nm.clear();
  P.max_n = P.max_nsh = P.max_nat = P.max_pairs = 0;
  P.max_healed_sh = P.max_projected = 0;
  long long mat = 0, sh = 0, gam = 0, ao = 0, hist = 0, apad = 0;
  for (size_t t = 0; t < tuples.size(); ++t) {
    Nmer m{};
    m.nfrag = nf[t];
    int n = 0, ns = 0, na = 0;
    double nel = 0.0;
    for (int k = 0; k < 3; ++k) m.frag[k] = (k < m.nfrag) ? tuples[t][k] : -1;
    int healed_sh = 0, projected = 0;
    for (int k = 0; k < m.nfrag; ++k) {
      const int f = tuples[t][k];
      n += ctx->f_nao[f];
      ns += ctx->f_nsh[f];
      na += ctx->f_nat[f];
      nel += ctx->f_nel[f];
      if (ctx->n_cut == 0) continue;
      // ghosts of bonds healed here leave the n-mer; healing moves the
      // ghost's electron back to the BDA, so the electron count is unchanged
      for (const auto& gh : ctx->f_ghosts[f]) {
        const bool healed = std::find(m.frag, m.frag + m.nfrag, gh.bda_frag) != m.frag + m.nfrag;
        if (healed) { n -= gh.nao; ns -= gh.nsh; na -= 1; healed_sh += gh.nsh; }
        else ++projected;
      }
      for (int baa_f : ctx->f_bda_baa_frag[f])
        if (std::find(m.frag, m.frag + m.nfrag, baa_f) == m.frag + m.nfrag) ++projected;
    }
    P.max_healed_sh = std::max(P.max_healed_sh, healed_sh);
    P.max_projected = std::max(P.max_projected, projected);
    m.n = n; m.nsh = ns; m.nat = na; m.npad = n + (n & 1); m.nel = nel;
    m.mat = mat; m.gam = gam; m.aov = ao; m.hist = hist; m.apad = apad;
    m.shv = monomer_layout ? ctx->f_sh0[tuples[t][0]] : sh;
    mat += (long long)n * n;
    sh += ns;
    gam += (long long)ns * ns;
    ao += m.npad;
    hist += (long long)(2 * kHist + 2) * ns;
    apad += (long long)m.npad * m.npad;
    P.max_n = std::max(P.max_n, n);
    P.max_nsh = std::max(P.max_nsh, ns);
    P.max_nat = std::max(P.max_nat, na);
    P.max_pairs = std::max(P.max_pairs, na * (na + 1) / 2);
    P.nm.push_back(m);
  }
  if (monomer_layout) sh = ctx->n_sh;
  P.tot_mat = mat; P.tot_sh = sh; P.tot_gam = gam; P.tot_ao = ao; P.tot_hist = hist; P.tot_apad = apad;
  // longest-processing-time-first order of the blocks
  P.order.resize(P.nm.size());
  for (size_t i = 0; i < P.order.size(); ++i) P.order[i] = int(i);
  std::stable_sort(P.order.begin(), P.order.end(), [&](int a, int b) { return P.nm[a].n > P.nm[b].n; });
  const size_t nn = std::max<size_t>(P.nm.size(), 1);
  cudaError_t e;
#define ENS(buf, bytes) if ((e = (buf).ensure(bytes)) != cudaSuccess) return e
  ENS(P.S, sizeof(double) * mat);
  ENS(P.H0, sizeof(double) * mat);
  ENS(P.gam, sizeof(double) * gam);
  ENS(P.CTd, sizeof(double) * mat);
  ENS(P.W1d, sizeof(double) * mat);
  ENS(P.W2d, sizeof(double) * mat);
  if (precision == FMO_PREC_MIXED) {
    ENS(P.S32, sizeof(float) * mat);
    ENS(P.H32, sizeof(float) * mat);
    ENS(P.CTf, sizeof(float) * mat);
    ENS(P.W1f, sizeof(float) * mat);
    ENS(P.W2f, sizeof(float) * mat);
  }
  ENS(P.esp, sizeof(double) * std::max<long long>(sh, 1));
  ENS(P.dq, sizeof(double) * std::max<long long>(sh, 1));
  ENS(P.eps, sizeof(double) * ao);
  ENS(P.hist, sizeof(double) * hist);
  ENS(P.energy, sizeof(double) * nn);
  ENS(P.e_el, sizeof(double) * nn);
  ENS(P.e_rep, sizeof(double) * nn);
  ENS(P.dEV, sizeof(double) * nn);
  ENS(P.iters, sizeof(int) * nn);
  ENS(P.iters32, sizeof(int) * nn);
  ENS(P.status, sizeof(int) * nn);
  if (ctx->n_cut > 0) ENS(P.V, sizeof(double) * std::max<long long>(mat, 1));
  if (ctx->n_cut > 0 && precision == FMO_PREC_MIXED) {
    ENS(P.hQd, sizeof(double) * kHopCols * std::max<long long>(ao, 1));
    ENS(P.hQf, sizeof(float) * kHopCols * std::max<long long>(ao, 1));
    ENS(P.hDd, sizeof(double) * kHopCols * kHopCols * nn);
    ENS(P.hDf, sizeof(float) * kHopCols * kHopCols * nn);
    ENS(P.hnq, sizeof(int) * nn);
  }
#undef ENS
  P.owner.clear();
  if (ctx->shard_world > 1 && !P.nm.empty()) {
    // this rank launches its own n-mers only (LPT partition by n^3), in the
    // pass's largest-first order
    std::vector<double> cost(P.nm.size());
    for (size_t i = 0; i < P.nm.size(); ++i) cost[i] = double(P.nm[i].n) * P.nm[i].n * P.nm[i].n;
    P.owner = lpt_owner(cost, ctx->shard_world);
    std::vector<int> mine;
    for (int i : P.order)
      if (P.owner[i] == ctx->shard_rank) mine.push_back(i);
    P.order.swap(mine);
  }
  if ((e = upload(P.d_nm, P.nm, st)) != cudaSuccess) return e;
  if ((e = upload(P.d_order, P.order, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Entries of a device array that a sharded run sums over its ranks: entry e
// belongs to n-mer item_of(e); other ranks' entries are zeroed before the sum.
struct ExPart {
  void* dev;
  int type;        // 0 double, 1 int, 2 float
  long long n;
  std::vector<int> item;   // n-mer of every entry
};

// ExPart for per-n-mer arrays (one entry per n-mer)
ExPart ex_per_nmer(DevBuf& b, int type, size_t nn) {
  ExPart x{b.p, type, (long long)nn, std::vector<int>(nn)};
  for (size_t i = 0; i < nn; ++i) x.item[i] = int(i);
  return x;
}

// Sum of the parts over the ranks, in place, through the exchange callback.
fmo_status shard_exchange(fmo_ctx* ctx, const Pass& P, std::vector<ExPart>& parts, cudaStream_t st) {
  long long total = 0;
  for (auto& x : parts) total += x.n;
  std::vector<double> buf(std::max<long long>(total, 1), 0.0);
  std::vector<std::vector<char>> raw(parts.size());
  const size_t esz[3] = {sizeof(double), sizeof(int), sizeof(float)};
  for (size_t k = 0; k < parts.size(); ++k) {
    raw[k].resize(std::max<size_t>(esz[parts[k].type] * parts[k].n, 1));
    if (parts[k].n) CK(d2h(raw[k].data(), parts[k].dev, esz[parts[k].type] * parts[k].n, st));
  }
  CK(sync_stream(st));
  long long o = 0;
  for (size_t k = 0; k < parts.size(); ++k) {
    const ExPart& x = parts[k];
    for (long long e = 0; e < x.n; ++e, ++o) {
      if (P.owner[x.item[e]] != ctx->shard_rank) continue;
      if (x.type == 0) buf[o] = reinterpret_cast<const double*>(raw[k].data())[e];
      else if (x.type == 1) buf[o] = double(reinterpret_cast<const int*>(raw[k].data())[e]);
      else buf[o] = double(reinterpret_cast<const float*>(raw[k].data())[e]);
    }
  }
  if (ctx->ex_fn(ctx->ex_user, buf.data(), total) != 0) return fail(ctx, FMO_ERR_EXCHANGE, "exchange callback failed");
  o = 0;
  for (size_t k = 0; k < parts.size(); ++k) {
    const ExPart& x = parts[k];
    for (long long e = 0; e < x.n; ++e, ++o) {
      if (x.type == 0) reinterpret_cast<double*>(raw[k].data())[e] = buf[o];
      else if (x.type == 1) reinterpret_cast<int*>(raw[k].data())[e] = int(buf[o]);
      else reinterpret_cast<float*>(raw[k].data())[e] = float(buf[o]);
    }
    if (x.n) CK(h2d(x.dev, raw[k].data(), esz[x.type] * x.n, st));
  }
  CK(sync_stream(st));
  return FMO_OK;
}

// The results of a dimer or trimer pass on every rank of a sharded run.
fmo_status shard_exchange_pass(fmo_ctx* ctx, Pass& P, cudaStream_t st) {
  const size_t nn = P.nm.size();
  if (ctx->shard_world <= 1 || nn == 0) return FMO_OK;
  std::vector<ExPart> parts{ex_per_nmer(P.energy, 0, nn), ex_per_nmer(P.dEV, 0, nn), ex_per_nmer(P.iters, 1, nn),
                            ex_per_nmer(P.status, 1, nn)};
  return shard_exchange(ctx, P, parts, st);
}

struct SmemPlan {
  int a_d, a_f;
  size_t bytes;
};

// Limits of the fixed-size index maps of the integral and gamma kernels.
bool pass_fits(const Pass& P) {
  return P.max_nat <= 512 && P.max_nsh <= 1024 && P.max_n <= 4000 && P.max_healed_sh <= kMaxHealedShells &&
         P.max_projected <= kMaxProjected;
}

// fp32_only: mixed-precision dimers or trimers that iterate in FP32 only (they
// end with the FP64 energy of their FP32 density); with 64 or more basis
// functions their matrices stay in global memory, so that two CTAs share an
// SM and the FP32 eigen-solves use the tridiagonal solver.
SmemPlan plan_smem(fmo_ctx* ctx, const Pass& P, int precision, bool fp32_only = false, int placement = 0) {
  const int npad = P.max_n + (P.max_n & 1);
  SmemPlan sp{0, 0, 0};
  const size_t lim = (size_t)ctx->smem_optin;
  const size_t with_d = scc_smem_size(P.max_n, P.max_nsh, P.max_nat, 8 * npad * npad);
  const size_t with_f = scc_smem_size(P.max_n, P.max_nsh, P.max_nat, 4 * npad * npad);
  // placement: 0 the rule above, 1 shared memory where it fits, 2 global
  // memory, 3 (mixed precision) only the FP32 matrix in shared memory
  const bool global = placement == 2 || (placement == 0 && fp32_only && precision == FMO_PREC_MIXED && P.max_n >= 64);
  if (global) {
    // global memory (sp stays {0, 0})
  } else if (placement == 3 && precision == FMO_PREC_MIXED) {
    if (with_f <= lim) sp.a_f = 1;
  } else if (with_d <= lim) { sp.a_d = 1; sp.a_f = (precision == FMO_PREC_MIXED); }
  else if (precision == FMO_PREC_MIXED && with_f <= lim) { sp.a_f = 1; }
  sp.bytes = scc_smem_size(P.max_n, P.max_nsh, P.max_nat, (sp.a_d ? 8 : (sp.a_f ? 4 : 0)) * npad * npad);
  return sp;
}

// S, H0, gamma and the Loewdin start of every n-mer of a pass.
// warm_from: in mixed precision, start the n-mers from the final monomer
// rows of this pass instead of the Loewdin orthogonaliser.
fmo_status setup_pass(fmo_ctx* ctx, Pass& P, int precision, const SmemPlan& sp, cudaStream_t st,
                      const Pass* warm_from = nullptr) {
  const int nn = int(P.nm.size());
  if (nn == 0) return FMO_OK;
  const SmemPlan& s = sp;
  // the monomer S/H0 blocks are reused in the n-mers unless ghost atoms make
  // the fragment blocks of the two passes differ
  const bool reuse = warm_from != nullptr && ctx->n_cut == 0;
  if (!s.a_d) CK(P.Agd.ensure(sizeof(double) * P.tot_apad));
  if (precision == FMO_PREC_MIXED && !s.a_f) CK(P.Agf.ensure(sizeof(float) * P.tot_apad));
  CK(launch_integrals(st, nn, P.max_pairs, P.d_nm.as<Nmer>(), ctx->ftab(), ctx->d_xyz.as<double>(),
                      ctx->d_elem.as<int>(), ctx->d_atom_sh0.as<int>(), ctx->d_cn.as<double>(),
                      ctx->d_el.as<DevElem>(), ctx->d_kab.as<double>(), ctx->ne, ctx->g, P.S.as<double>(),
                      P.H0.as<double>(), reuse ? warm_from->d_nm.as<Nmer>() : nullptr,
                      reuse ? warm_from->S.as<double>() : nullptr,
                      reuse ? warm_from->H0.as<double>() : nullptr, ctx->d_prim.as<PrimPair>()));
  if (precision == FMO_PREC_MIXED) {   // FP32 copies for the FP32 iterations
    CK(launch_to_float(st, P.tot_mat, P.S.as<double>(), P.S32.as<float>()));
    CK(launch_to_float(st, P.tot_mat, P.H0.as<double>(), P.H32.as<float>()));
  }
  if (ctx->n_cut > 0) {
    const bool fac = (precision == FMO_PREC_MIXED);   // mixed: the factors as well
    CK(launch_hop_projector(st, nn, P.d_nm.as<Nmer>(), ctx->ftab(), ctx->d_xyz.as<double>(), ctx->d_elem.as<int>(),
                            ctx->d_el.as<DevElem>(), ctx->params.v_hop, P.S.as<double>(), P.V.as<double>(),
                            fac ? P.hQd.as<double>() : nullptr, fac ? P.hQf.as<float>() : nullptr,
                            fac ? P.hDd.as<double>() : nullptr, fac ? P.hDf.as<float>() : nullptr,
                            fac ? P.hnq.as<int>() : nullptr));
  }
  CK(launch_gamma(st, nn, P.max_nsh, P.d_nm.as<Nmer>(), ctx->ftab(), ctx->d_xyz.as<double>(),
                  ctx->d_elem.as<int>(), ctx->d_sh_atom.as<int>(), ctx->d_sh_inv_eta.as<double>(), ctx->g,
                  P.gam.as<double>()));
  CK(cudaMemsetAsync(P.status.p, 0, sizeof(int) * nn, st));
  const bool use_f = (precision == FMO_PREC_MIXED);
  const int npad = P.max_n + (P.max_n & 1);
  const size_t lim = (size_t)ctx->smem_optin;
  const int elb = use_f ? 4 : 8;
  const int a_in = ((size_t)elb * npad * npad + 64 * 1024 <= lim) ? 1 : 0;
  if (!a_in) {
    if (use_f) CK(P.Agf.ensure(sizeof(float) * P.tot_apad));
    else CK(P.Agd.ensure(sizeof(double) * P.tot_apad));
  }
  if (warm_from && use_f && ctx->n_cut == 0) {
    // warm start in mixed precision only, and only where every n-mer's basis
    // is its monomers' bases side by side (no healed ghost atoms)
    CK(launch_warm_start(st, nn, P.d_nm.as<Nmer>(), warm_from->d_nm.as<Nmer>(), warm_from->CTf.as<float>(),
                         P.CTf.as<float>()));
  } else {
    CK(launch_lowdin(st, nn, P.max_n, P.d_nm.as<Nmer>(), P.S.as<double>(),
                     use_f ? P.CTf.p : P.CTd.p, use_f ? P.W1f.p : P.W1d.p, use_f ? P.Agf.p : P.Agd.p,
                     use_f ? 1 : 0, a_in, P.status.as<int>(), use_f ? P.W2f.p : nullptr));
  }
  return FMO_OK;
}

// FMO_DEBUG=1 in the environment: synchronise after each stage of fmo_run and
// report it on stderr (diagnostics only; the computation is unchanged).
int debug_level() {
  static int v = -1;
  if (v < 0) { const char* e = getenv("FMO_DEBUG"); v = (e && e[0] >= '1' && e[0] <= '9') ? e[0] - '0' : 0; }
  return v;
}
bool debug_on() { return debug_level() >= 1; }
void stage(cudaStream_t st, const char* what, int k = -1) {
  if (!debug_on()) return;
  cudaError_t e = sync_stream(st);
  fprintf(stderr, "[fmo] %s %d: %s\n", what, k, cudaGetErrorString(e));
  fflush(stderr);
}

// Supersystem potential phi = gamma dq_mono of the current monomer charges:
// a matrix-vector product over the stored gamma of all shell pairs when it is
// held, else evaluated pair by pair (use_float: FP32 estimate).
constexpr size_t kGammaFullMaxBytes = size_t(32) << 30;
constexpr int kStall32 = 8;   // monomer-loop steps without a 10% gain before FP32 gives up

cudaError_t compute_phi(fmo_ctx* ctx, cudaStream_t st, int use_float) {
  if (ctx->gam_full_ok)
    return launch_phi_gemv(st, ctx->n_sh, ctx->d_gam_full.as<double>(), ctx->d_dq_mono.as<double>(),
                           ctx->d_phi.as<double>());
  return launch_phi(st, ctx->n_sh, ctx->d_xyz.as<double>(), ctx->d_sh_atom.as<int>(), ctx->d_sh_inv_eta.as<double>(),
                    ctx->d_dq_mono.as<double>(), ctx->g, ctx->d_phi.as<double>(), ctx->d_phi_part.as<double>(),
                    use_float);
}

fmo_status run_scc(fmo_ctx* ctx, Pass& P, const fmo_options& o, const SmemPlan& sp, bool with_phi,
                   int pass_id, cudaStream_t st, int single_step = 0, int step_phase = 1, int reortho = 0,
                   int cold = 1, int reortho32 = 0, double jac_hint = 1.0, bool capture = false,
                   const int* step_dev = nullptr) {
  const int nn = int(P.nm.size());
  if (nn == 0) return FMO_OK;
  SccLaunch L{};
  L.nmers = P.d_nm.as<Nmer>(); L.order = P.d_order.as<int>(); L.ft = ctx->ftab();
  L.xyz = ctx->d_xyz.as<double>(); L.elem = ctx->d_elem.as<int>(); L.atom_sh0 = ctx->d_atom_sh0.as<int>();
  L.el = ctx->d_el.as<DevElem>(); L.g = ctx->g; L.S = P.S.as<double>(); L.H0 = P.H0.as<double>();
  L.gam = P.gam.as<double>();
  L.CTd = P.CTd.as<double>(); L.W1d = P.W1d.as<double>(); L.W2d = P.W2d.as<double>(); L.Agd = P.Agd.as<double>();
  L.CTf = P.CTf.as<float>(); L.W1f = P.W1f.as<float>(); L.W2f = P.W2f.as<float>(); L.Agf = P.Agf.as<float>();
  L.phi = with_phi ? ctx->d_phi.as<double>() : nullptr;
  L.vhop = ctx->n_cut > 0 ? P.V.as<double>() : nullptr;
  if (ctx->n_cut > 0 && o.precision == FMO_PREC_MIXED) {
    L.hop_Qd = P.hQd.as<double>(); L.hop_Qf = P.hQf.as<float>();
    L.hop_Dd = P.hDd.as<double>(); L.hop_Df = P.hDf.as<float>(); L.hop_nq = P.hnq.as<int>();
  }
  if (o.precision == FMO_PREC_MIXED) { L.S32 = P.S32.as<float>(); L.H32 = P.H32.as<float>(); }
  L.dq_mono = ctx->d_dq_mono.as<double>();
  L.esp = P.esp.as<double>(); L.dq = P.dq.as<double>(); L.eps = P.eps.as<double>(); L.hist = P.hist.as<double>();
  L.energy = P.energy.as<double>(); L.e_el = P.e_el.as<double>(); L.e_rep = P.e_rep.as<double>();
  L.dEV = P.dEV.as<double>(); L.iters = P.iters.as<int>(); L.iters32 = P.iters32.as<int>();
  L.status = P.status.as<int>();
  L.guess_from_mono = 1;
  L.precision = o.precision;
  L.max_iter = o.max_iter;
  L.fp32_cap = std::max(4, o.max_iter / 2);
  L.single_step = single_step;
  L.step_phase = step_phase;
  L.reortho = reortho;
  L.cold_refine = cold;
  L.reortho32 = reortho32;
  L.step_dev = step_dev;
  L.jac_hint = jac_hint;
  // a gradient needs FP64-converged n-mer densities: then the FP32 phase of a
  // mixed-precision n-mer hands over to FP64 iterations run to convergence
  // (cut bonds, too: an FP32 phase cannot resolve the 1e6 Eh projector to
  // the accuracy of the FP64 energy finish)
  const bool grad_nmer = (o.want_gradient || ctx->n_cut > 0) && pass_id >= 1;
  L.fp64_finish = (pass_id >= 1 && o.precision == FMO_PREC_MIXED && !grad_nmer) ? std::max(0, o.mixed_finish) : 0;
  L.energy_finish = (pass_id >= 1 && o.precision == FMO_PREC_MIXED && o.nmer_finish == FMO_NMER_FINISH_ENERGY &&
                     !grad_nmer);
  const bool warm_nmer = (pass_id >= 1 && o.precision == FMO_PREC_MIXED && ctx->n_cut == 0);
  L.cold_steps = warm_nmer ? 12 : 2;
  L.first_rot = warm_nmer ? 1 : 0;
  L.first_jac_tol = warm_nmer ? 1e-3 : 0.0;
  L.trace = nullptr;
  // FMO_DEBUG=2 traces the first (largest) dimer, FMO_DEBUG=3 the first
  // trimer, FMO_DEBUG=4 the first monomer (every launch of the monomer loop)
  const int dl = debug_level();
  const bool tracing = (dl == 2 && pass_id == 1) || (dl == 3 && pass_id == 2) || (dl == 4 && pass_id == 0);
  if (tracing) {
    CK(ctx->d_trace.ensure(sizeof(double) * kTraceLen));
    CK(cudaMemsetAsync(ctx->d_trace.p, 0, sizeof(double) * kTraceLen, st));
    L.trace = ctx->d_trace.as<double>();
  }
  L.tol = o.scc_tol; L.etol = o.e_tol; L.switch_tol = o.mixed_switch_tol;
  L.jacobi_tol_d = 1e-14;
  L.jacobi_tol_f = 2e-7;
  L.t0 = ctx->d_t0.as<unsigned long long>();
  L.budget_ns = o.deadline_s > 0 ? (unsigned long long)(o.deadline_s * 1e9) : 0ULL;
  L.a_smem_d = sp.a_d; L.a_smem_f = sp.a_f;
  L.ctas_per_sm = pass_id >= 1 ? o.nmer_ctas_per_sm : o.monomer_ctas_per_sm;
  L.max_n = P.max_n; L.max_nsh = P.max_nsh; L.max_nat = P.max_nat;
  if (!sp.a_d) CK(P.Agd.ensure(sizeof(double) * P.tot_apad));
  if (o.precision == FMO_PREC_MIXED && !sp.a_f) CK(P.Agf.ensure(sizeof(float) * P.tot_apad));
  L.Agd = P.Agd.as<double>(); L.Agf = P.Agf.as<float>();
  if (capture) {
    // recorded into a CUDA graph: the previous step's residual is read on the
    // device (mixer state), no timing or read-back
    L.trace = nullptr;
    L.jac_hint_dev = reinterpret_cast<const double*>(ctx->d_mix_state.p) + 1;
    CK(launch_scc(st, nn, L));
    return FMO_OK;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  CK(launch_scc(st, int(P.order.size()), L));
  cudaEventRecord(e1, st);
  // iteration counts of this launch -> algorithmic flops of the pass
  P.h_iters.resize(nn);
  P.h_iters32.resize(nn);
  CK(d2h(P.h_iters.data(), P.iters.p, sizeof(int) * nn, st));
  CK(d2h(P.h_iters32.data(), P.iters32.p, sizeof(int) * nn, st));
  CK(sync_stream(st));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->stats.ms_scc[pass_id] += ms;
  if (tracing) {
    std::vector<double> tr(kTraceLen);
    CK(d2h(tr.data(), ctx->d_trace.p, sizeof(double) * kTraceLen, st));
    CK(sync_stream(st));
    int last = 1;
    while (last < 511 && tr[last + 1] != 0.0) ++last;
    fprintf(stderr, "[fmo] pass %d, first n-mer (n = %d): residual per iteration (negative = FP32):", pass_id,
            P.nm[P.order[0]].n);
    for (int i = 1; i <= last; ++i) fprintf(stderr, " %.1e", tr[i]);
    fprintf(stderr, "\n[fmo] Jacobi sweeps per iteration (-1 = rotation step):");
    for (int i = 1; i <= last; ++i) fprintf(stderr, " %d", int(tr[512 + i]));
    fprintf(stderr, "\n[fmo] Mcycles: start %.2f, per iteration:", tr[1024] * 1e-6);
    for (int i = 1; i <= last; ++i) fprintf(stderr, " %.2f", tr[1024 + i] * 1e-6);
    fprintf(stderr, ", FP64 energy finish %.2f\n", tr[1535] * 1e-6);
    fprintf(stderr, "[fmo] Mcycles summed over iterations: Fock %.2f, transform %.2f, occupations %.2f, "
            "rotation/Jacobi %.2f, density %.2f, populations %.2f, energy %.2f\n",
            tr[kTraceParts] * 1e-6, tr[kTraceParts + 1] * 1e-6, tr[kTraceParts + 2] * 1e-6,
            tr[kTraceParts + 3] * 1e-6, tr[kTraceParts + 4] * 1e-6, tr[kTraceParts + 5] * 1e-6,
            tr[kTraceParts + 6] * 1e-6);
    unsigned long long slow = 0, njac = 0;
    std::memcpy(&slow, &tr[kTraceSlowest], 8);
    std::memcpy(&njac, &tr[kTraceJacobi], 8);
    const int sb = int(slow & 0xFFFFF);
    fprintf(stderr, "[fmo] slowest block %d (n = %d): %.2f Mcycles; Jacobi eigen-solves in the launch: %llu\n", sb,
            sb < (int)P.order.size() ? P.nm[P.order[sb]].n : -1, double(slow >> 20) * 1e-6, njac);
  }
  ctx->stats.scc_launches[pass_id] += 1;
  for (int i : P.order) {
    const double n3 = 15.0 * double(P.nm[i].n) * P.nm[i].n * P.nm[i].n;
    const int i32 = P.h_iters32[i], i64 = P.h_iters[i] - P.h_iters32[i];
    ctx->stats.iters_fp32[pass_id] += i32;
    ctx->stats.iters_fp64[pass_id] += i64;
    ctx->stats.flops_fp32[pass_id] += n3 * i32;
    ctx->stats.flops_fp64[pass_id] += n3 * i64;
    if (L.energy_finish) {
      // C_o S, C_o H0 and two C_o S C_o^T products in FP64
      const double nn_ = P.nm[i].n, no = 0.5 * P.nm[i].nel;
      ctx->stats.flops_fp64[pass_id] += 4.0 * no * nn_ * nn_ + 4.0 * no * no * nn_;
    }
  }
  return FMO_OK;
}

// NVTX range of the current stage of fmo_run (closed on every return path).
struct StageRange {
  bool open = false;
  void set(const char* name) { end(); nvtxRangePushA(name); open = true; }
  void end() { if (open) nvtxRangePop(); open = false; }
  ~StageRange() { end(); }
};

double now_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

// The FP64 steps of the global monomer loop as one CUDA graph: a while node
// whose body is phi, one single-step SCC launch of every monomer, the global
// mixer and a control kernel that counts the step and clears the node's
// condition on convergence, a NaN residual or the step limit.  No host round
// trip per step.  `done` steps have run; on return *outer is the last step.
cudaError_t run_monomer_graph(fmo_ctx* ctx, const fmo_options& o, const SmemPlan& sp, cudaStream_t st, int done,
                              int* outer, int phase = 1, Phase32State* p32 = nullptr, int cap32 = 0) {
  const int nf = ctx->n_frag;
  int* d_outer = reinterpret_cast<int*>(ctx->d_scalar.p);
  cudaError_t e = h2d(d_outer, &done, sizeof(int), st);
  if (e != cudaSuccess) return e;
  cudaGraph_t g = nullptr, body = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t cs = nullptr;
  cudaGraphConditionalHandle h;
  cudaGraphNodeParams cp{};
  cudaGraphNode_t node;
  const long long l0 = launch_count();
  long long per_step = 0;
  auto cleanup = [&]() {
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
  };
#define GK(x) do { e = (x); if (e != cudaSuccess) { cleanup(); return e; } } while (0)
  GK(cudaGraphCreate(&g, 0));
  GK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  GK(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  body = cp.conditional.phGraph_out[0];
  GK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  GK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  {
    // one step: the FP32 phase works with an FP32 estimate of the potential
    // and orthonormalises every fourth step (decided from the device step count)
    cudaError_t ce = compute_phi(ctx, cs, phase == 0 ? 1 : 0);
    fmo_status fs = (ce == cudaSuccess) ? run_scc(ctx, ctx->mono, o, sp, true, 0, cs, 1, phase, 0, 0, 0, 1.0, true,
                                                  phase == 0 ? d_outer : nullptr)
                                        : FMO_ERR_CUDA;
    if (ce == cudaSuccess && fs == FMO_OK)
      ce = launch_global_mix(cs, ctx->n_sh, ctx->d_dq_mono.as<double>(), ctx->mono.dq.as<double>(), nf,
                             ctx->mono.energy.as<double>(), ctx->d_mix_hist.as<double>(), ctx->d_mix_state.p,
                             o.outer_tol, o.e_tol, phase == 1);
    if (ce == cudaSuccess && fs == FMO_OK)
      ce = (phase == 0) ? launch_loop_control32(cs, h, ctx->d_mix_state.p, p32, d_outer, o.max_outer,
                                                o.mixed_switch_tol, cap32, kStall32)
                        : launch_loop_control(cs, h, ctx->d_mix_state.p, d_outer, o.max_outer);
    cudaGraph_t captured = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(cs, &captured);
    if (ce == cudaSuccess && fs != FMO_OK) ce = cudaErrorUnknown;
    GK(ce);
    GK(ee);
  }
  per_step = launch_count() - l0;
  GK(cudaGraphInstantiate(&ge, g, 0));
  GK(cudaGraphLaunch(ge, st));
  GK(d2h(outer, d_outer, sizeof(int), st));
  GK(sync_stream(st));
  // the captured launches ran once per step
  for (long long k = 0; k < per_step * (long long)(*outer - done - 1); ++k) note_launch();
  const int steps = *outer - done;
  for (const Nmer& m : ctx->mono.nm) {
    const double n3 = 15.0 * double(m.n) * m.n * m.n;
    if (phase == 0) {
      ctx->stats.iters_fp32[0] += steps;
      ctx->stats.flops_fp32[0] += n3 * steps;
    } else {
      ctx->stats.iters_fp64[0] += steps;
      ctx->stats.flops_fp64[0] += n3 * steps;
    }
  }
  ctx->stats.scc_launches[0] += steps;
  cleanup();
  return cudaSuccess;
#undef GK
}

// Per-system tables of the learned-guess model: element index (H, C, N, O),
// fragment and 1/eta of the first shell of every atom, 1/eta of every shell,
// fragment charges.  The model takes two shells per atom and k_g = 2.
fmo_status mlp_tables(fmo_ctx* ctx) {
  if (ctx->mlp_tables_ok) return FMO_OK;
  if (ctx->n_cut > 0) return fail(ctx, FMO_ERR_UNSUPPORTED, "the learned guess takes no cut bonds");
  if (ctx->g.k_g != 2.0) return fail(ctx, FMO_ERR_UNSUPPORTED, "the learned guess needs k_g = 2");
  static const int kZ[4] = {1, 6, 7, 8};
  std::vector<int> e4(ctx->n_int), afrag(ctx->n_int);
  std::vector<float> aie(ctx->n_int), shie(ctx->h_sh_inv_eta.begin(), ctx->h_sh_inv_eta.end());
  std::vector<int> ez(ctx->ne, -1);
  for (int z = 0; z < FMO_MAX_Z; ++z)
    if (ctx->z_to_e[z] >= 0)
      for (int k = 0; k < 4; ++k)
        if (kZ[k] == z) ez[ctx->z_to_e[z]] = k;
  for (int f = 0; f < ctx->n_frag; ++f)
    for (int i = ctx->f_atom0[f]; i < ctx->f_atom0[f] + ctx->f_nat[f]; ++i) {
      const int e = ctx->h_elem[i];
      if (ez[e] < 0) return fail(ctx, FMO_ERR_UNSUPPORTED, "the learned guess covers H, C, N and O only");
      if (ctx->h_el[e].nsh != 2) return fail(ctx, FMO_ERR_UNSUPPORTED, "the learned guess needs two shells per atom");
      e4[i] = ez[e];
      afrag[i] = f;
      aie[i] = float(1.0 / ctx->h_el[e].eta_sh[0]);
    }
  cudaStream_t st = ctx->own_stream;
  CK(upload(ctx->d_mlp_elem4, e4, st));
  CK(upload(ctx->d_mlp_atom_frag, afrag, st));
  CK(upload(ctx->d_mlp_atom_ie, aie, st));
  CK(upload(ctx->d_mlp_sh_ie, shie, st));
  CK(upload(ctx->d_mlp_fcharge, ctx->f_charge, st));
  CK(ctx->d_mlp_err.ensure(sizeof(int)));
  CK(sync_stream(st));
  ctx->mlp_tables_ok = true;
  return FMO_OK;
}

// Two-pass prediction (pass 0 with ESP = 0, pass 1 with the ESP of the pass-0
// charges) for the current coordinates into out (double, internal shell order).
fmo_status mlp_predict_device(fmo_ctx* ctx, cudaStream_t st, double* out) {
  fmo_status fs = mlp_tables(ctx);
  if (fs != FMO_OK) return fs;
  const int n = ctx->n_int;
  CK(ctx->d_mlp_X.ensure(sizeof(float) * (size_t)n * kMlpStride));
  CK(ctx->d_mlp_y.ensure(sizeof(float) * 2 * (size_t)n));
  CK(ctx->d_mlp_q.ensure(sizeof(float) * 2 * (size_t)n));
  CK(cudaMemsetAsync(ctx->d_mlp_err.p, 0, sizeof(int), st));
  const float* W = ctx->d_mlp_W.as<float>();
  const __half* W16 = ctx->d_mlp_W16.as<__half>();
  const MlpCache none{nullptr, nullptr, nullptr, nullptr, nullptr};
  CK(mlp_descriptors(st, 1, n, ctx->d_xyz.as<double>(), ctx->d_mlp_elem4.as<int>(), ctx->d_mlp_X.as<float>(),
                     ctx->d_mlp_err.as<int>()));
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1)
      CK(mlp_esp(st, 1, n, ctx->n_sh, ctx->d_xyz.as<double>(), ctx->d_mlp_atom_frag.as<int>(),
                 ctx->d_mlp_atom_ie.as<float>(), ctx->d_sh_atom.as<int>(), ctx->d_mlp_sh_ie.as<float>(),
                 ctx->d_mlp_q.as<float>(), ctx->d_mlp_X.as<float>()));
    CK(mlp_forward(st, n, ctx->d_mlp_X.as<float>(), W16, W + kMlpOffMean, W + kMlpOffScale, ctx->d_mlp_y.as<float>(),
                   none));
    CK(mlp_project(st, 1, ctx->n_frag, n, ctx->d_f_atom0.as<int>(), ctx->d_f_nat.as<int>(),
                   ctx->d_mlp_fcharge.as<int>(), ctx->d_mlp_y.as<float>(), ctx->d_mlp_q.as<float>(), nullptr, 0.0,
                   nullptr, nullptr));
  }
  CK(mlp_to_double(st, 2 * n, ctx->d_mlp_q.as<float>(), out));
  return FMO_OK;
}


// ---------------------------------------------------------------------------
// Analytic FMO gradient (Sec. 2.4; kernels in fmo_gradient.cu).

// y = Op(v) = v - Gamma_inter chi v (the Z-vector operator; Gamma_inter: gamma
// between shells of different fragments).
cudaError_t zvector_op(fmo_ctx* ctx, cudaStream_t st, int nf, const GradTerm* mt, const MonoResp* mr,
                       const int* sh0, const double* v, double* out, double* t1, double* t2, double* t3) {
  cudaError_t e;
  if ((e = launch_chi_apply(st, nf, mt, mr, sh0, v, t1)) != cudaSuccess) return e;
  if (ctx->gam_full_ok) e = launch_phi_gemv(st, ctx->n_sh, ctx->d_gam_full.as<double>(), t1, t2);
  else e = launch_phi(st, ctx->n_sh, ctx->d_xyz.as<double>(), ctx->d_sh_atom.as<int>(), ctx->d_sh_inv_eta.as<double>(),
                      t1, ctx->g, t2, ctx->d_phi_part.as<double>(), 0);
  if (e != cudaSuccess) return e;
  if ((e = launch_intra_gamma(st, nf, mt, sh0, t1, t3)) != cudaSuccess) return e;
  return launch_vec_lincomb3(st, ctx->n_sh, 1.0, v, -1.0, t2, 1.0, t3, out);
}

// GMRES(m) with classical Gram-Schmidt applied twice for (1 - Gamma chi) z = w.
// Stops at ||w - Op z|| <= rtol ||w||.  Returns iterations (-1: not converged).
fmo_status zvector_gmres(fmo_ctx* ctx, cudaStream_t st, int nf, const GradTerm* mt, const MonoResp* mr,
                         const int* sh0, const double* w, double* z, double rtol, int* iters, double* relres) {
  const int n = ctx->n_sh;
  const int m = 40, max_restart = 12;
  const long long ldv = (n + 31) / 32 * 32;
  CK(ctx->d_gkrylov.ensure(sizeof(double) * (size_t)ldv * (m + 1 + 5) + sizeof(double) * (m + 1) * 2));
  double* V = ctx->d_gkrylov.as<double>();
  double* u = V + (size_t)ldv * (m + 1);
  double* t1 = u + ldv;
  double* t2 = t1 + ldv;
  double* t3 = t2 + ldv;
  double* r = t3 + ldv;
  double* dh = r + ldv;
  double* dh2 = dh + (m + 1);
  std::vector<double> H((size_t)(m + 1) * m), gv(m + 1), cs(m), sn(m), hh(m + 1), hh2(m + 1);
  auto norm = [&](const double* x, double* out) -> cudaError_t {
    cudaError_t e = launch_vec_dots(st, n, 1, x, ldv, x, dh);
    if (e != cudaSuccess) return e;
    e = d2h(out, dh, sizeof(double), st);
    if (e != cudaSuccess) return e;
    e = sync_stream(st);
    *out = std::sqrt(*out);
    return e;
  };
  CK(cudaMemsetAsync(z, 0, sizeof(double) * n, st));
  CK(cudaMemcpyAsync(r, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
  double beta0 = 0.0;
  CK(norm(r, &beta0));
  *iters = 0;
  *relres = 0.0;
  if (!(beta0 > 0.0)) return FMO_OK;
  double beta = beta0;
  int total = 0;
  for (int rs = 0; rs < max_restart; ++rs) {
    CK(launch_vec_lincomb3(st, n, 1.0 / beta, r, 0.0, nullptr, 0.0, nullptr, V));
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    double res = beta;
    for (int j = 0; j < m; ++j) {
      double* vj1 = V + (size_t)ldv * (j + 1);
      CK(zvector_op(ctx, st, nf, mt, mr, sh0, V + (size_t)ldv * j, vj1, t1, t2, t3));
      // h = V^T u, u -= V h, twice
      CK(launch_vec_dots(st, n, j + 1, V, ldv, vj1, dh));
      CK(launch_vec_update(st, n, j + 1, V, ldv, dh, vj1));
      CK(launch_vec_dots(st, n, j + 1, V, ldv, vj1, dh2));
      CK(launch_vec_update(st, n, j + 1, V, ldv, dh2, vj1));
      CK(launch_vec_dots(st, n, 1, vj1, ldv, vj1, dh2 + j + 1));
      CK(d2h(hh.data(), dh, sizeof(double) * (j + 1), st));
      CK(d2h(hh2.data(), dh2, sizeof(double) * (j + 2), st));
      CK(sync_stream(st));
      const double hn = std::sqrt(std::max(hh2[j + 1], 0.0));
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i] + hh2[i];
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) CK(launch_vec_lincomb3(st, n, 1.0 / hn, vj1, 0.0, nullptr, 0.0, nullptr, vj1));
      // Givens rotations on column j
      for (int i = 0; i < j; ++i) {
        const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
      const double den = std::hypot(a, b);
      cs[j] = den > 0.0 ? a / den : 1.0;
      sn[j] = den > 0.0 ? b / den : 0.0;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      res = std::fabs(gv[j + 1]);
      k = j + 1;
      ++total;
      if (res <= rtol * beta0 || hn == 0.0) break;
    }
    // y = H^-1 g (upper triangular), z += V y
    std::vector<double> yv(k);
    for (int i = k - 1; i >= 0; --i) {
      double t = gv[i];
      for (int c = i + 1; c < k; ++c) t -= H[(size_t)i * m + c] * yv[c];
      yv[i] = t / H[(size_t)i * m + i];
    }
    for (double& x : yv) x = -x;   // vec_update subtracts
    CK(h2d(dh, yv.data(), sizeof(double) * k, st));
    CK(launch_vec_update(st, n, k, V, ldv, dh, z));
    // true residual
    CK(zvector_op(ctx, st, nf, mt, mr, sh0, z, t1 + 0, u, t2, t3));   // Op z into t1 (u, t2, t3 scratch)
    CK(launch_vec_lincomb3(st, n, 1.0, w, -1.0, t1, 0.0, nullptr, r));
    CK(norm(r, &beta));
    *relres = beta / beta0;
    if (beta <= rtol * beta0 * 10.0 || beta <= rtol * beta0) { *iters = total; return FMO_OK; }
  }
  *iters = -total;
  return FMO_OK;
}

fmo_status compute_gradient(fmo_ctx* ctx, std::vector<double>& gout) {
  cudaStream_t st = ctx->own_stream;
  const int nf = ctx->n_frag, level = ctx->last_level;
  const Pass& M = ctx->mono;
  const Pass& D = ctx->dim;
  const Pass& T = ctx->tri;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  // coefficients of the FMO2/FMO3 sums (Eqs. 12, 16): monomers c_I, SCC dimers m
  std::vector<double> c_mono(nf, 1.0), m_dim(D.nm.size(), 1.0);
  for (const Nmer& x : D.nm) { c_mono[x.frag[0]] -= 1.0; c_mono[x.frag[1]] -= 1.0; }
  auto pidx = [&](long long a, long long b) { return a * (2LL * nf - a - 1) / 2 + (b - a - 1); };
  for (const Nmer& x : T.nm) {
    const int f[3] = {x.frag[0], x.frag[1], x.frag[2]};
    const int pr[3][2] = {{f[0], f[1]}, {f[0], f[2]}, {f[1], f[2]}};
    for (auto& q : pr) {
      const int k = ctx->r_pair_k[pidx(q[0], q[1])];
      if (k < 0) return fail(ctx, FMO_ERR_UNSUPPORTED, "gradient: a trimer holds an ES-DIM pair");
      m_dim[k] -= 1.0;
      c_mono[q[0]] += 1.0;
      c_mono[q[1]] += 1.0;
    }
    for (int I : f) c_mono[I] -= 1.0;
  }
  GradLaunch L{};
  L.ft = ctx->ftab(); L.xyz = ctx->d_xyz.as<double>(); L.elem = ctx->d_elem.as<int>();
  L.atom_sh0 = ctx->d_atom_sh0.as<int>(); L.el = ctx->d_el.as<DevElem>(); L.kab = ctx->d_kab.as<double>();
  L.ne = ctx->ne; L.prim = ctx->d_prim.as<PrimPair>(); L.cn = ctx->d_cn.as<double>(); L.g = ctx->g;
  L.dq_mono = ctx->d_dq_mono.as<double>();
  for (const Pass* P : {&M, &D, &T}) {
    L.max_n = std::max(L.max_n, P->max_n);
    L.max_nsh = std::max(L.max_nsh, P->max_nsh);
    L.max_nat = std::max(L.max_nat, P->max_nat);
  }
  if (grad_smem_max(L) > (size_t)ctx->smem_optin) return fail(ctx, FMO_ERR_UNSUPPORTED, "gradient: n-mer too large");
  // energy terms: monomers (c_I != 0), SCC dimers, SCC trimers
  struct TermRef { const Pass* P; int k; int kind; double m, es; };
  std::vector<TermRef> refs;
  for (int I = 0; I < nf; ++I) if (c_mono[I] != 0.0) refs.push_back({&M, I, kGradMonomer, c_mono[I], 0.0});
  for (size_t k = 0; k < D.nm.size(); ++k) refs.push_back({&D, int(k), kGradNmer, m_dim[k], level >= 2 ? 1.0 : 0.0});
  for (size_t k = 0; k < T.nm.size(); ++k) refs.push_back({&T, int(k), kGradNmer, 1.0, 0.0});
  const int nt = int(refs.size());
  std::vector<GradTerm> terms(nt);
  long long aoff = 0, soff = 0;
  std::vector<std::vector<std::pair<long long, long long>>> ent(nf);   // per fragment: (atom slot, shell slot)
  for (int i = 0; i < nt; ++i) {
    const TermRef& r = refs[i];
    GradTerm& t = terms[i];
    std::memset(&t, 0, sizeof(t));
    t.nm = r.P->nm[r.k];
    t.S = r.P->S.as<double>() + t.nm.mat;
    t.H0 = r.P->H0.as<double>() + t.nm.mat;
    t.gam = r.P->gam.as<double>() + t.nm.gam;
    t.CT = r.P->CTd.as<double>() + t.nm.mat;
    t.eps = r.P->eps.as<double>() + t.nm.aov;
    t.dq = r.P->dq.as<double>() + t.nm.shv;
    t.esp = r.P->esp.as<double>() + t.nm.shv;
    t.m = r.m;
    t.es = r.es;
    t.kind = r.kind;
    t.with_rep = 1;
    t.aslot = aoff;
    t.sslot = soff;
    long long la = 0, ls = 0;
    for (int q = 0; q < t.nm.nfrag; ++q) {
      const int f = t.nm.frag[q];
      ent[f].push_back({aoff + 4 * la, soff + 2 * ls});
      la += ctx->f_nat[f];
      ls += ctx->f_nsh[f];
    }
    aoff += 4LL * t.nm.nat;
    soff += 2LL * t.nm.nsh;
  }
  // per-fragment entry lists (CSR, term order)
  std::vector<int> fptr(nf + 1, 0);
  std::vector<long long> ea, es;
  for (int f = 0; f < nf; ++f) {
    fptr[f] = int(ea.size());
    for (auto& x : ent[f]) { ea.push_back(x.first); es.push_back(x.second); }
  }
  fptr[nf] = int(ea.size());
  std::vector<int> atom_frag(ctx->n_int), sh_frag(ctx->n_sh), sh0(nf);
  for (int f = 0; f < nf; ++f) {
    sh0[f] = ctx->f_sh0[f];
    for (int i = 0; i < ctx->f_nat[f]; ++i) atom_frag[ctx->f_atom0[f] + i] = f;
    for (int i = 0; i < ctx->f_nsh[f]; ++i) sh_frag[ctx->f_sh0[f] + i] = f;
  }
  const int nat = ctx->n_int, nsh_all = ctx->n_sh;
  CK(ctx->d_gslots_a.ensure(sizeof(double) * std::max<long long>(aoff, 1)));
  CK(ctx->d_gslots_s.ensure(sizeof(double) * std::max<long long>(soff, 1)));
  CK(upload(ctx->d_gfrag_ptr, fptr, st));
  CK(upload(ctx->d_gent_a, ea, st));
  CK(upload(ctx->d_gent_s, es, st));
  CK(upload(ctx->d_gatom_frag, atom_frag, st));
  CK(upload(ctx->d_gsh_frag, sh_frag, st));
  CK(upload(ctx->d_gsh0, sh0, st));
  CK(ctx->d_gatom.ensure(sizeof(double) * 4 * (size_t)nat));
  CK(ctx->d_gw.ensure(sizeof(double) * (size_t)nsh_all));
  CK(ctx->d_gd.ensure(sizeof(double) * (size_t)nsh_all));
  CK(ctx->d_gflag.ensure(sizeof(int)));
  CK(cudaMemsetAsync(ctx->d_gflag.p, 0, sizeof(int), st));
  // per-term scratch, in chunks: Pa, W (n^2 each), work (4 n^2), shifts (nsh)
  auto term_bytes = [](const Nmer& x) { return sizeof(double) * (6 * (size_t)x.n * x.n + x.nsh + 16); };
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t budget = std::max<size_t>(size_t(256) << 20, std::min<size_t>(size_t(8) << 30, free_b / 4));
  CK(ctx->d_gt.ensure(sizeof(GradTerm) * std::max(nt, 1)));
  for (int c0 = 0; c0 < nt;) {
    size_t used = 0;
    int c1 = c0;
    while (c1 < nt && (c1 == c0 || used + term_bytes(terms[c1].nm) <= budget)) used += term_bytes(terms[c1++].nm);
    CK(ctx->d_grad_work.ensure(used));
    char* base = reinterpret_cast<char*>(ctx->d_grad_work.p);
    size_t off = 0;
    for (int i = c0; i < c1; ++i) {
      GradTerm& t = terms[i];
      const size_t nn = (size_t)t.nm.n * t.nm.n;
      double* b = reinterpret_cast<double*>(base + off);
      t.Pa = b;
      t.W = b + nn;
      t.work = b + 2 * nn;
      t.sa = b + 6 * nn;
      off += term_bytes(t.nm);
    }
    CK(h2d(ctx->d_gt.as<GradTerm>() + c0, terms.data() + c0, sizeof(GradTerm) * (c1 - c0), st));
    CK(launch_grad_prep(st, c1 - c0, ctx->d_gt.as<GradTerm>() + c0, L, ctx->d_gflag.as<int>()));
    CK(launch_grad_explicit(st, c1 - c0, ctx->d_gt.as<GradTerm>() + c0, L, ctx->d_gslots_a.as<double>(),
                            ctx->d_gslots_s.as<double>()));
    CK(sync_stream(st));   // the scratch is reused by the next chunk
    c0 = c1;
  }
  CK(launch_grad_gather(st, nat, nsh_all, L, ctx->d_gatom_frag.as<int>(), ctx->d_gsh_frag.as<int>(),
                        ctx->d_gfrag_ptr.as<int>(), ctx->d_gent_a.as<long long>(), ctx->d_gent_s.as<long long>(),
                        ctx->d_gslots_a.as<double>(), ctx->d_gslots_s.as<double>(), ctx->d_gatom.as<double>(),
                        ctx->d_gw.as<double>(), ctx->d_gd.as<double>(), 0));
  CK(ctx->d_ga.ensure(sizeof(double) * (size_t)nsh_all));
  CK(ctx->d_gout.ensure(sizeof(double) * 3 * (size_t)nat));
  double* a_vec = ctx->d_ga.as<double>();
  int zit = 0;
  double zres = 0.0;
  if (nf > 1) {
    // ---- response: monomer susceptibilities, Z-vector, first-order gradients
    std::vector<GradTerm> mt(nf);
    std::vector<MonoResp> mr(nf);
    size_t mem = 0;
    std::vector<size_t> moff(nf);
    for (int I = 0; I < nf; ++I) {
      const Nmer& x = M.nm[I];
      moff[I] = mem;
      const size_t nn = (size_t)x.n * x.n, ss = (size_t)x.nsh * x.nsh;
      mem += sizeof(double) * (nn + 2 * (size_t)x.n + ss + x.nsh + 7 * nn + (size_t)x.npad * x.npad + 3 * ss + 64);
    }
    CK(ctx->d_gmr_mem.ensure(mem));
    for (int I = 0; I < nf; ++I) {
      const Nmer& x = M.nm[I];
      GradTerm& t = mt[I];
      std::memset(&t, 0, sizeof(t));
      t.nm = x;
      t.S = M.S.as<double>() + x.mat;
      t.H0 = M.H0.as<double>() + x.mat;
      t.gam = M.gam.as<double>() + x.gam;
      t.CT = M.CTd.as<double>() + x.mat;
      t.eps = M.eps.as<double>() + x.aov;
      t.dq = M.dq.as<double>() + x.shv;
      t.esp = M.esp.as<double>() + x.shv;
      t.kind = kGradMonomer;
      const size_t nn = (size_t)x.n * x.n, ss = (size_t)x.nsh * x.nsh;
      double* b = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->d_gmr_mem.p) + moff[I]);
      mr[I].C = b;
      mr[I].eps = b + nn;
      mr[I].focc = mr[I].eps + x.n;
      mr[I].chi = mr[I].focc + x.n;
      mr[I].sig = mr[I].chi + ss;
      mr[I].work = mr[I].sig + x.nsh;
    }
    CK(upload(ctx->d_gmono_terms, mt, st));
    CK(upload(ctx->d_gmr, mr, st));
    const GradTerm* dmt = ctx->d_gmono_terms.as<GradTerm>();
    MonoResp* dmr = ctx->d_gmr.as<MonoResp>();
    CK(launch_grad_mono_response(st, nf, dmt, dmr, L, ctx->d_gflag.as<int>()));
    // w += gamma d (charge transfer of the SCC n-mers into every other
    // fragment) and, with pairs, the ESP of the all-pairs ES-DIM form
    CK(ctx->d_gz.ensure(sizeof(double) * (size_t)nsh_all));
    CK(ctx->d_gy.ensure(sizeof(double) * (size_t)nsh_all));
    double* z = ctx->d_gz.as<double>();
    double* y = ctx->d_gy.as<double>();
    if (ctx->gam_full_ok) CK(launch_phi_gemv(st, nsh_all, ctx->d_gam_full.as<double>(), ctx->d_gd.as<double>(), y));
    else CK(launch_phi(st, nsh_all, ctx->d_xyz.as<double>(), ctx->d_sh_atom.as<int>(), ctx->d_sh_inv_eta.as<double>(),
                       ctx->d_gd.as<double>(), ctx->g, y, ctx->d_phi_part.as<double>(), 0));
    CK(launch_vec_lincomb3(st, nsh_all, 1.0, ctx->d_gw.as<double>(), 1.0, y, level >= 2 ? 1.0 : 0.0,
                           M.esp.as<double>(), ctx->d_gw.as<double>()));
    int fl = 0;
    CK(d2h(&fl, ctx->d_gflag.p, sizeof(int), st));
    CK(sync_stream(st));
    if (fl & 2) return fail(ctx, FMO_ERR_NOT_CONVERGED, "gradient: monomer eigen-solve did not converge");
    const std::vector<MonoResp>& mr_h = mr;
    fmo_status fs = zvector_gmres(ctx, st, nf, dmt, dmr, ctx->d_gsh0.as<int>(), ctx->d_gw.as<double>(), z, 1e-12,
                                  &zit, &zres);
    if (fs != FMO_OK) return fs;
    if (zit < 0) return fail(ctx, FMO_ERR_NOT_CONVERGED, "gradient: Z-vector GMRES did not converge");
    CK(launch_chi_apply(st, nf, dmt, dmr, ctx->d_gsh0.as<int>(), z, y));
    // response terms: one per monomer, Pa = dP, W = dW~, Pb = P, sb = dsigma
    std::vector<GradTerm> rt(nf);
    size_t rmem = 0;
    std::vector<size_t> roff(nf);
    long long raoff = 0;
    std::vector<int> rptr(nf + 1);
    std::vector<long long> rea(nf), res_(nf, -1);
    for (int I = 0; I < nf; ++I) {
      roff[I] = rmem;
      rmem += sizeof(double) * (3 * (size_t)M.nm[I].n * M.nm[I].n + M.nm[I].nsh + 8);
    }
    CK(ctx->d_gresp_mem.ensure(rmem));
    CK(ctx->d_gslots_a.ensure(sizeof(double) * std::max<long long>(aoff, 1)));
    for (int I = 0; I < nf; ++I) {
      GradTerm t = mt[I];
      const size_t nn = (size_t)t.nm.n * t.nm.n;
      double* b = reinterpret_cast<double*>(reinterpret_cast<char*>(ctx->d_gresp_mem.p) + roff[I]);
      t.kind = kGradResponse;
      t.Pa = b;
      t.W = b + nn;
      t.Pb = b + 2 * nn;
      t.sb = b + 3 * nn;
      t.sa = mr_h[I].sig;
      t.qb = y + ctx->f_sh0[I];
      t.esp = nullptr;
      t.m = 1.0;
      t.es = 0.0;
      t.with_rep = 0;
      t.aslot = raoff;
      t.sslot = 0;
      rptr[I] = I;
      rea[I] = raoff;
      raoff += 4LL * t.nm.nat;
      rt[I] = t;
    }
    rptr[nf] = nf;
    DevBuf rslots;
    CK(rslots.ensure(sizeof(double) * std::max<long long>(raoff, 1)));
    CK(upload(ctx->d_gresp_terms, rt, st));
    CK(launch_grad_first_order(st, nf, ctx->d_gresp_terms.as<GradTerm>(), dmr, L, z, y));
    CK(launch_grad_explicit(st, nf, ctx->d_gresp_terms.as<GradTerm>(), L, rslots.as<double>(), nullptr));
    DevBuf rp, ra;
    CK(upload(rp, rptr, st));
    CK(upload(ra, rea, st));
    CK(launch_grad_gather(st, nat, 0, L, ctx->d_gatom_frag.as<int>(), nullptr, rp.as<int>(), ra.as<long long>(),
                          nullptr, rslots.as<double>(), nullptr, ctx->d_gatom.as<double>(), nullptr, nullptr, 1));
    // a = d + chi z (+ 1/2 q with ES-DIM pairs)
    CK(launch_vec_lincomb3(st, nsh_all, 1.0, ctx->d_gd.as<double>(), 1.0, y, level >= 2 ? 0.5 : 0.0,
                           ctx->d_dq_mono.as<double>(), a_vec));
    CK(sync_stream(st));
    rslots.release();
    rp.release();
    ra.release();
  } else {
    CK(cudaMemsetAsync(a_vec, 0, sizeof(double) * (size_t)nsh_all, st));
  }
  CK(launch_grad_cn_coulomb(st, nat, nsh_all, L, ctx->d_gatom_frag.as<int>(), ctx->d_sh_atom.as<int>(),
                            ctx->d_sh_inv_eta.as<double>(), a_vec, ctx->d_gatom.as<double>(),
                            ctx->d_gout.as<double>()));
  gout.assign(3 * (size_t)nat, 0.0);
  int fl = 0;
  CK(d2h(gout.data(), ctx->d_gout.p, sizeof(double) * gout.size(), st));
  CK(d2h(&fl, ctx->d_gflag.p, sizeof(int), st));
  cudaEventRecord(e1, st);
  CK(sync_stream(st));
  ctx->stats.ms_gradient = now_ms(e0, e1);
  ctx->stats.zvector_iterations = zit;
  ctx->stats.zvector_residual = zres;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (fl) return fail(ctx, FMO_ERR_NOT_CONVERGED, "gradient: monomer eigen-solve did not converge");
  return FMO_OK;
}

}  // namespace

extern "C" {

void fmo_options_default(fmo_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->level = 2;
  o->precision = FMO_PREC_FP64;
  o->all_dimers_scc = 0;
  o->max_iter = 300;
  o->max_outer = 200;
  o->guess = 0;
  o->schedule = 0;
  o->monomer_loop = FMO_LOOP_GLOBAL;
  o->dimer_cut = 4.0 / 0.529177210903;
  o->trimer_cut = 4.0 / 0.529177210903;
  o->scc_tol = 1e-10;
  o->e_tol = 1e-10;
  o->outer_tol = 1e-10;
  o->mixed_switch_tol = 1e-5;
  o->mixed_finish = 1;
  o->deadline_s = 0.0;
  o->shard_rank = 0;
  o->shard_world = 1;
}

fmo_status fmo_create(fmo_ctx** out, const fmo_params* p, int device) {
  if (!out || !p) return FMO_ERR_ARG;
  *out = nullptr;
  for (int z = 0; z < FMO_MAX_Z; ++z) {
    const fmo_element& e = p->el[z];
    if (e.n_shell < 0 || e.n_shell > FMO_MAX_SHELL) return FMO_ERR_ARG;
    for (int s = 0; s < e.n_shell; ++s) {
      if (e.l[s] < 0 || e.l[s] > 1) return FMO_ERR_ARG;
      if (e.n_prim[s] < 1 || e.n_prim[s] > FMO_MAX_PRIM) return FMO_ERR_ARG;
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return FMO_ERR_CUDA;
  fmo_ctx* ctx = new fmo_ctx();
  ctx->device = device;
  ctx->params = *p;
  if (cudaSetDevice(device) != cudaSuccess) { delete ctx; return FMO_ERR_CUDA; }
  if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete ctx;
    return FMO_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  for (int z = 0; z < FMO_MAX_Z; ++z) ctx->z_to_e[z] = -1;
  std::memset(&ctx->stats, 0, sizeof(ctx->stats));
  *out = ctx;
  return FMO_OK;
}

void fmo_destroy(fmo_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (DevBuf* b : {&ctx->d_el, &ctx->d_kab, &ctx->d_prim, &ctx->d_xyz, &ctx->d_xyz_in, &ctx->d_perm, &ctx->d_elem, &ctx->d_cn,
                    &ctx->d_atom_sh0, &ctx->d_sh_atom, &ctx->d_sh_inv_eta, &ctx->d_f_atom0, &ctx->d_f_nat,
                    &ctx->d_f_sh0, &ctx->d_f_nsh, &ctx->d_f_ao0, &ctx->d_f_nao, &ctx->d_trace, &ctx->d_gam_full, &ctx->d_mlp_W, &ctx->d_mlp_W16, &ctx->d_mlp_m, &ctx->d_mlp_v,
                    &ctx->d_mlp_elem4, &ctx->d_mlp_atom_frag, &ctx->d_mlp_atom_ie, &ctx->d_mlp_sh_ie,
                    &ctx->d_mlp_fcharge, &ctx->d_mlp_err, &ctx->d_mlp_X, &ctx->d_mlp_y, &ctx->d_mlp_q, &ctx->d_ghost_frag, &ctx->d_ghost_src, &ctx->d_bda_baa_frag, &ctx->d_hop_baa, &ctx->d_dq_mono, &ctx->d_phi, &ctx->d_phi_part,
                    &ctx->d_bounds, &ctx->d_rmin, &ctx->d_scalar, &ctx->d_t0, &ctx->d_mix_hist, &ctx->d_mix_state, &ctx->d_p32, &ctx->d_pair_scc, &ctx->d_dE_pair,
                    &ctx->d_esdim_pairs, &ctx->d_esdim_idx, &ctx->d_tri_frag, &ctx->d_dE3, &ctx->d_corr,
                    &ctx->d_totals, &ctx->d_grad_work, &ctx->d_grad, &ctx->d_gt, &ctx->d_gslots_a,
                    &ctx->d_gslots_s, &ctx->d_gpair, &ctx->d_gfrag_ptr, &ctx->d_gent_a, &ctx->d_gent_s,
                    &ctx->d_gatom_frag, &ctx->d_gsh_frag, &ctx->d_gatom, &ctx->d_gw, &ctx->d_gd,
                    &ctx->d_gmono_terms, &ctx->d_gmr, &ctx->d_gmr_mem, &ctx->d_gresp_terms, &ctx->d_gresp_mem,
                    &ctx->d_gflag, &ctx->d_gsh0, &ctx->d_gkrylov, &ctx->d_gz, &ctx->d_gy, &ctx->d_ga, &ctx->d_gout})
    b->release();
  ctx->stg.release();
  ctx->mono.release();
  ctx->dim.release();
  ctx->tri.release();
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  delete ctx;
}

const char* fmo_last_error(const fmo_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

fmo_status fmo_set_system(fmo_ctx* ctx, int32_t n_atoms, const int32_t* Z, const double* xyz, int32_t n_frag,
                          const int32_t* frag_of_atom, const int32_t* frag_charge, int32_t n_cut,
                          const int32_t* bda_baa) {
  g_ctx = ctx;
  if (!ctx) return FMO_ERR_ARG;
  if (n_atoms <= 0 || n_frag <= 0 || !Z || !xyz || !frag_of_atom || !frag_charge)
    return fail(ctx, FMO_ERR_ARG, "empty system or NULL input");
  if (n_cut < 0 || (n_cut > 0 && !bda_baa)) return fail(ctx, FMO_ERR_ARG, "cut-bond list missing");
  cudaSetDevice(ctx->device);
  const fmo_params& p = ctx->params;
  // elements present -> compact table
  ctx->ne = 0;
  for (int z = 0; z < FMO_MAX_Z; ++z) ctx->z_to_e[z] = -1;
  ctx->h_el.clear();
  std::vector<int> ez;
  for (int i = 0; i < n_atoms; ++i) {
    const int z = Z[i];
    if (z <= 0 || z >= FMO_MAX_Z || p.el[z].n_shell == 0)
      return fail(ctx, FMO_ERR_ARG, "atom " + std::to_string(i) + ": element not in the table");
    if (!std::isfinite(xyz[3 * i]) || !std::isfinite(xyz[3 * i + 1]) || !std::isfinite(xyz[3 * i + 2]))
      return fail(ctx, FMO_ERR_ARG, "non-finite coordinate");
    if (frag_of_atom[i] < 0 || frag_of_atom[i] >= n_frag)
      return fail(ctx, FMO_ERR_ARG, "fragment index out of range");
    if (ctx->z_to_e[z] < 0) {
      if (ctx->ne >= kMaxElem) return fail(ctx, FMO_ERR_UNSUPPORTED, "too many distinct elements");
      ctx->z_to_e[z] = ctx->ne++;
      ez.push_back(z);
    }
  }
  for (int k = 0; k < ctx->ne; ++k) {
    const fmo_element& src = p.el[ez[k]];
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
    ctx->h_el.push_back(d);
  }
  ctx->h_kab.assign((size_t)ctx->ne * ctx->ne, 1.0);
  for (int a = 0; a < ctx->ne; ++a)
    for (int b = 0; b < ctx->ne; ++b) ctx->h_kab[a * ctx->ne + b] = p.k_ab[ez[a]][ez[b]];
  for (int l = 0; l < 3; ++l) ctx->g.k_l[l] = p.k_l[l];
  ctx->g.k_en = p.k_en; ctx->g.k_g = p.k_g; ctx->g.k_f = p.k_f;
  ctx->g.cn_k1 = p.cn_k1; ctx->g.cn_k2 = p.cn_k2; ctx->g.cn_cutoff = p.cn_cutoff;
  ctx->g.kT = 3.166811563e-6 * p.t_el;
  if (!(ctx->g.kT > 0)) return fail(ctx, FMO_ERR_ARG, "electronic temperature must be positive");

  // cut bonds (hybrid orbital projection): BDA and BAA in different
  // fragments, the BDA with one s and one p shell, detached at most once
  std::vector<int> bda_bond(n_atoms, -1);
  for (int k = 0; k < n_cut; ++k) {
    const int a = bda_baa[2 * k], b = bda_baa[2 * k + 1];
    if (a < 0 || a >= n_atoms || b < 0 || b >= n_atoms)
      return fail(ctx, FMO_ERR_ARG, "cut bond " + std::to_string(k) + ": atom index out of range");
    if (frag_of_atom[a] == frag_of_atom[b])
      return fail(ctx, FMO_ERR_ARG, "cut bond " + std::to_string(k) + ": both atoms in one fragment");
    if (bda_bond[a] >= 0)
      return fail(ctx, FMO_ERR_UNSUPPORTED, "cut bond " + std::to_string(k) + ": atom is already a BDA");
    bda_bond[a] = k;
    const fmo_element& e = p.el[Z[a]];
    int n_s = 0, n_p = 0;
    for (int sh = 0; sh < e.n_shell; ++sh) { n_s += (e.l[sh] == 0); n_p += (e.l[sh] == 1); }
    if (n_s != 1 || n_p != 1)
      return fail(ctx, FMO_ERR_UNSUPPORTED, "cut bond " + std::to_string(k) + ": the BDA needs one s and one p shell");
  }
  // internal atoms: per fragment its real atoms (input order), then the
  // ghosts (copies of the BDA at its position) of the bonds whose BAA it holds
  ctx->n_atoms = n_atoms;
  ctx->n_frag = n_frag;
  ctx->f_charge.assign(frag_charge, frag_charge + n_frag);
  ctx->n_cut = n_cut;
  ctx->n_int = n_atoms + n_cut;
  const int n_int = ctx->n_int;
  std::vector<std::vector<int>> real_of(n_frag), ghost_of(n_frag);
  for (int i = 0; i < n_atoms; ++i) real_of[frag_of_atom[i]].push_back(i);
  for (int k = 0; k < n_cut; ++k) ghost_of[frag_of_atom[bda_baa[2 * k + 1]]].push_back(k);
  ctx->perm.clear();
  std::vector<int> bond_of(n_int, -1), internal_of(n_atoms, -1);
  for (int f = 0; f < n_frag; ++f) {
    for (int a : real_of[f]) { internal_of[a] = int(ctx->perm.size()); ctx->perm.push_back(a); }
    for (int k : ghost_of[f]) { bond_of[ctx->perm.size()] = k; ctx->perm.push_back(bda_baa[2 * k]); }
  }
  ctx->h_ghost_frag.assign(n_int, -1); ctx->h_ghost_src.assign(n_int, -1);
  ctx->h_bda_baa_frag.assign(n_int, -1); ctx->h_hop_baa.assign(n_int, -1);
  ctx->f_ghosts.assign(n_frag, {});
  ctx->f_bda_baa_frag.assign(n_frag, {});
  for (int i = 0; i < n_int; ++i) {
    const int src = ctx->perm[i];
    if (bond_of[i] >= 0) {
      const int k = bond_of[i];
      ctx->h_ghost_frag[i] = frag_of_atom[bda_baa[2 * k]];
      ctx->h_ghost_src[i] = internal_of[bda_baa[2 * k]];
      ctx->h_hop_baa[i] = internal_of[bda_baa[2 * k + 1]];
    } else if (bda_bond[src] >= 0) {
      const int k = bda_bond[src];
      ctx->h_bda_baa_frag[i] = frag_of_atom[bda_baa[2 * k + 1]];
      ctx->h_hop_baa[i] = internal_of[bda_baa[2 * k + 1]];
      ctx->f_bda_baa_frag[frag_of_atom[src]].push_back(ctx->h_bda_baa_frag[i]);
    }
  }
  ctx->f_atom0.assign(n_frag, 0); ctx->f_nat.assign(n_frag, 0); ctx->f_sh0.assign(n_frag, 0);
  ctx->f_nsh.assign(n_frag, 0); ctx->f_ao0.assign(n_frag, 0); ctx->f_nao.assign(n_frag, 0);
  ctx->f_nel.assign(n_frag, 0.0);
  ctx->h_elem.resize(n_int);
  ctx->h_atom_sh0.resize(n_int);
  ctx->h_sh_atom.clear();
  ctx->h_sh_inv_eta.clear();
  int sh = 0, ao = 0;
  std::vector<double> xyz_int(3 * (size_t)n_int);
  int fprev = -1;
  for (int i = 0; i < n_int; ++i) {
    const int src = ctx->perm[i];
    const bool ghost = bond_of[i] >= 0;
    const int f = ghost ? frag_of_atom[bda_baa[2 * bond_of[i] + 1]] : frag_of_atom[src];
    if (f != fprev) { ctx->f_atom0[f] = i; ctx->f_sh0[f] = sh; ctx->f_ao0[f] = ao; fprev = f; }
    const int e = ctx->z_to_e[Z[src]];
    ctx->h_elem[i] = e;
    ctx->h_atom_sh0[i] = sh;
    const DevElem& d = ctx->h_el[e];
    for (int s2 = 0; s2 < d.nsh; ++s2) {
      ctx->h_sh_atom.push_back(i);
      ctx->h_sh_inv_eta.push_back(1.0 / d.eta_sh[s2]);
      if (!ghost) ctx->f_nel[f] += d.q0[s2];
    }
    if (ghost) {
      ctx->f_nel[f] += 1.0;                                    // the ghost's electron
      ctx->f_nel[frag_of_atom[src]] -= 1.0;                    // taken from the BDA's fragment
      ctx->f_ghosts[f].push_back({frag_of_atom[src], d.nsh, elem_nao(d)});
    }
    ctx->f_nat[f] += 1;
    ctx->f_nsh[f] += d.nsh;
    ctx->f_nao[f] += elem_nao(d);
    sh += d.nsh;
    ao += elem_nao(d);
    for (int c = 0; c < 3; ++c) xyz_int[3 * i + c] = xyz[3 * src + c];
  }
  for (int f = 0; f < n_frag; ++f) {
    if (ctx->f_nat[f] == 0) return fail(ctx, FMO_ERR_ARG, "fragment " + std::to_string(f) + " has no atoms");
    ctx->f_nel[f] -= frag_charge[f];
    const double ne = ctx->f_nel[f];
    if (std::fabs(ne - std::round(ne)) > 1e-9 || (long long)std::llround(ne) % 2 != 0 || ne <= 0)
      return fail(ctx, FMO_ERR_ARG, "fragment " + std::to_string(f) + " is not closed shell");
    if (ctx->f_nao[f] > 510) return fail(ctx, FMO_ERR_UNSUPPORTED, "fragment larger than 510 basis functions");
  }
  ctx->n_sh = sh;
  ctx->n_ao = ao;
  cudaStream_t st = ctx->own_stream;
  build_prim_table(ctx->h_el, ctx->h_prim);
  CK(upload(ctx->d_el, ctx->h_el, st));
  CK(upload(ctx->d_kab, ctx->h_kab, st));
  CK(upload(ctx->d_prim, ctx->h_prim, st));
  CK(upload(ctx->d_xyz, xyz_int, st));
  CK(upload(ctx->d_perm, ctx->perm, st));
  CK(ctx->d_xyz_in.ensure(sizeof(double) * 3 * n_atoms));
  CK(upload(ctx->d_elem, ctx->h_elem, st));
  CK(ctx->d_cn.ensure(sizeof(double) * n_int));
  if (n_cut > 0) {
    CK(upload(ctx->d_ghost_frag, ctx->h_ghost_frag, st));
    CK(upload(ctx->d_ghost_src, ctx->h_ghost_src, st));
    CK(upload(ctx->d_bda_baa_frag, ctx->h_bda_baa_frag, st));
    CK(upload(ctx->d_hop_baa, ctx->h_hop_baa, st));
  }
  CK(upload(ctx->d_atom_sh0, ctx->h_atom_sh0, st));
  CK(upload(ctx->d_sh_atom, ctx->h_sh_atom, st));
  CK(upload(ctx->d_sh_inv_eta, ctx->h_sh_inv_eta, st));
  CK(upload(ctx->d_f_atom0, ctx->f_atom0, st));
  CK(upload(ctx->d_f_nat, ctx->f_nat, st));
  CK(upload(ctx->d_f_sh0, ctx->f_sh0, st));
  CK(upload(ctx->d_f_nsh, ctx->f_nsh, st));
  CK(upload(ctx->d_f_ao0, ctx->f_ao0, st));
  CK(upload(ctx->d_f_nao, ctx->f_nao, st));
  CK(ctx->d_dq_mono.ensure(sizeof(double) * sh));
  CK(ctx->d_phi.ensure(sizeof(double) * sh));
  CK(ctx->d_phi_part.ensure(sizeof(double) * sh * (size_t)(phi_chunks(sh) + 1)));
  CK(ctx->d_bounds.ensure(sizeof(double) * 4 * n_frag));
  CK(ctx->d_scalar.ensure(sizeof(double) * 8));
  CK(ctx->d_t0.ensure(sizeof(unsigned long long)));
  CK(ctx->d_totals.ensure(sizeof(double) * 4));
  CK(sync_stream(st));
  ctx->have_system = true;
  ctx->have_result = false;
  ctx->have_guess = false;
  ctx->mlp_tables_ok = false;
  return FMO_OK;
}

fmo_status fmo_set_coordinates(fmo_ctx* ctx, const double* xyz) {
  g_ctx = ctx;
  if (!ctx || !xyz) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  cudaSetDevice(ctx->device);
  for (int i = 0; i < 3 * ctx->n_atoms; ++i)
    if (!std::isfinite(xyz[i])) return fail(ctx, FMO_ERR_ARG, "non-finite coordinate");
  cudaStream_t st = ctx->own_stream;
  CK(h2d(ctx->d_xyz_in.p, xyz, sizeof(double) * 3 * ctx->n_atoms, st));
  CK(launch_gather_xyz(st, ctx->n_int, ctx->d_perm.as<int>(), ctx->d_xyz_in.as<double>(), ctx->d_xyz.as<double>()));
  CK(sync_stream(st));   // a later fmo_run may use another stream
  ctx->have_result = false;
  return FMO_OK;
}

fmo_status fmo_set_coordinates_device(fmo_ctx* ctx, const double* xyz_dev, void* cuda_stream) {
  g_ctx = ctx;
  if (!ctx || !xyz_dev) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  cudaSetDevice(ctx->device);
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
  CK(launch_gather_xyz(st, ctx->n_int, ctx->d_perm.as<int>(), xyz_dev, ctx->d_xyz.as<double>()));
  if (!cuda_stream) CK(sync_stream(st));
  ctx->have_result = false;
  return FMO_OK;
}

fmo_status fmo_set_guess(fmo_ctx* ctx, const double* shell_dq) {
  if (!ctx || !shell_dq) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  ctx->guess.assign(shell_dq, shell_dq + ctx->n_sh);
  ctx->have_guess = true;
  return FMO_OK;
}

fmo_status fmo_run(fmo_ctx* ctx, const fmo_options* opt, void* cuda_stream) {
  g_ctx = ctx;
  if (!ctx || !opt) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  const fmo_options o = *opt;
  if (o.level < 1 || o.level > 3) return fail(ctx, FMO_ERR_ARG, "level must be 1, 2 or 3");
  if (o.precision != FMO_PREC_FP64 && o.precision != FMO_PREC_MIXED)
    return fail(ctx, FMO_ERR_ARG, "unknown precision mode");
  if (o.max_iter < 1 || o.max_outer < 1 || !(o.scc_tol > 0) || !(o.e_tol > 0) || !(o.outer_tol > 0))
    return fail(ctx, FMO_ERR_ARG, "iteration limits and tolerances must be positive");
  if (o.guess == 2 && !ctx->have_guess) return fail(ctx, FMO_ERR_STATE, "guess = 2 needs fmo_set_guess");
  if (o.guess == 1 && !ctx->mlp_ready) return fail(ctx, FMO_ERR_STATE, "guess = 1 needs model weights");
  if (o.guess != 0 && o.guess != 1 && o.guess != 2) return fail(ctx, FMO_ERR_ARG, "unknown guess");
  if (o.monomer_loop != FMO_LOOP_GLOBAL && o.monomer_loop != FMO_LOOP_NESTED)
    return fail(ctx, FMO_ERR_ARG, "unknown monomer loop");
  if (o.nmer_finish != FMO_NMER_FINISH_ENERGY && o.nmer_finish != FMO_NMER_FINISH_ITERATE)
    return fail(ctx, FMO_ERR_ARG, "unknown n-mer finish");
  if (o.want_gradient != 0 && o.want_gradient != 1) return fail(ctx, FMO_ERR_ARG, "want_gradient must be 0 or 1");
  if (o.esp_mode != FMO_ESP_AUTO && o.esp_mode != FMO_ESP_PAIRWISE) return fail(ctx, FMO_ERR_ARG, "unknown esp_mode");
  if (o.nmer_ctas_per_sm < 0 || o.nmer_ctas_per_sm > 2 || o.nmer_matrix_smem < 0 || o.nmer_matrix_smem > 2 ||
      o.monomer_ctas_per_sm < 0 || o.monomer_ctas_per_sm > 2 || o.monomer_matrix_smem < 0 ||
      o.monomer_matrix_smem > 3)
    return fail(ctx, FMO_ERR_ARG, "schedule knobs out of range");
  const int world = o.shard_world <= 1 ? 1 : o.shard_world;
  if (o.shard_world < 0 || o.shard_rank < 0 || o.shard_rank >= world)
    return fail(ctx, FMO_ERR_ARG, "shard_rank must lie in [0, shard_world)");
  if (world > 1) {
    if (!ctx->ex_fn) return fail(ctx, FMO_ERR_STATE, "a sharded run needs fmo_set_exchange");
    if (o.monomer_loop != FMO_LOOP_GLOBAL) return fail(ctx, FMO_ERR_UNSUPPORTED, "sharded runs use the global monomer loop");
    if (o.want_gradient) return fail(ctx, FMO_ERR_UNSUPPORTED, "sharded runs keep no gradient data");
  }
  ctx->shard_rank = world > 1 ? o.shard_rank : 0;
  ctx->shard_world = world;
  cudaSetDevice(ctx->device);
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
  std::memset(&ctx->stats, 0, sizeof(ctx->stats));
  const long long launches0 = launch_count();
  ctx->have_result = false;
  const int nf = ctx->n_frag;
  ctx->d2h_bytes = 0;
  cudaEvent_t ev[8];
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], st);
  StageRange sr;
  sr.set("fmo_setup");
  CK(launch_stamp(st, ctx->d_t0.as<unsigned long long>()));
  // ---- coordination numbers of the whole system
  CK(launch_cn(st, ctx->n_int, ctx->d_xyz.as<double>(), ctx->d_elem.as<int>(), ctx->d_el.as<DevElem>(), ctx->g,
               ctx->d_cn.as<double>(), ctx->n_cut > 0 ? ctx->d_ghost_src.as<int>() : nullptr));
  stage(st, "cn");
  // gamma of all shell pairs, kept in HBM while it fits the budget
  {
    const size_t gbytes = sizeof(double) * (size_t)ctx->n_sh * (size_t)ctx->n_sh;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    ctx->gam_full_ok = o.esp_mode == FMO_ESP_AUTO && gbytes <= kGammaFullMaxBytes &&
                       (gbytes <= ctx->d_gam_full.cap || gbytes <= free_b / 4);
    if (ctx->gam_full_ok) {
      CK(ctx->d_gam_full.ensure(gbytes));
      CK(launch_gamma_full(st, ctx->n_sh, ctx->d_xyz.as<double>(), ctx->d_sh_atom.as<int>(),
                           ctx->d_sh_inv_eta.as<double>(), ctx->g, ctx->d_gam_full.as<double>()));
    }
  }
  // ---- monomer pass
  {
    std::vector<std::array<int, 3>> tu(nf);
    std::vector<int> nfr(nf, 1);
    for (int f = 0; f < nf; ++f) tu[f] = {f, -1, -1};
    CK(plan_pass(ctx, ctx->mono, tu, nfr, true, o.precision, st));
  }
  const SmemPlan sp_mono = plan_smem(ctx, ctx->mono, o.precision, false, o.monomer_matrix_smem);
  if (sp_mono.bytes > (size_t)ctx->smem_optin || !pass_fits(ctx->mono))
    return fail(ctx, FMO_ERR_UNSUPPORTED, "monomer too large");
  fmo_status fs = setup_pass(ctx, ctx->mono, o.precision, sp_mono, st);
  if (fs != FMO_OK) return fs;
  stage(st, "monomer setup");
  if (o.guess == 2) CK(h2d(ctx->d_dq_mono.p, ctx->guess.data(), sizeof(double) * ctx->n_sh, st));
  else if (o.guess == 1) {
    fs = mlp_predict_device(ctx, st, ctx->d_dq_mono.as<double>());
    if (fs != FMO_OK) return fs;
  }
  else CK(cudaMemsetAsync(ctx->d_dq_mono.p, 0, sizeof(double) * ctx->n_sh, st));
  cudaEventRecord(ev[1], st);
  sr.set("fmo_monomers");
  double change = 1e300;
  int outer = 0;
  double h_change_v = 0.0;
  double* h_change = &h_change_v;
  if (o.monomer_loop == FMO_LOOP_GLOBAL) {
    // one SCC iteration of every monomer per outer step, then one Broyden
    // step on all monomer charges (decided on the device)
    CK(ctx->d_mix_hist.ensure(sizeof(double) * (2 * kHist + 2) * (size_t)ctx->n_sh));
    CK(ctx->d_mix_state.ensure(mix_state_bytes()));
    CK(cudaMemsetAsync(ctx->d_mix_state.p, 0, mix_state_bytes(), st));
    int phase = (o.precision == FMO_PREC_MIXED) ? 0 : 1, reortho = 0, n32 = 0, stall32 = 0;
    const int cap32 = std::max(8, o.max_outer / 2);
    double min32 = 1e300;
    struct { double e_prev, diff, e1; int have_prev, hcount, hhead, converged, count; } hs{};
    bool graph_ok = (o.schedule == 0) && world == 1;
    // sharded: the output charges and energies of every step from all ranks
    std::vector<ExPart> step_parts;
    if (world > 1) {
      ExPart q{ctx->mono.dq.p, 0, (long long)ctx->n_sh, std::vector<int>(ctx->n_sh, 0)};
      for (int f = 0; f < nf; ++f)
        for (int k = 0; k < ctx->mono.nm[f].nsh; ++k) q.item[ctx->mono.nm[f].shv + k] = f;
      step_parts.push_back(std::move(q));
      step_parts.push_back(ex_per_nmer(ctx->mono.energy, 0, nf));
    }
    for (outer = 1; outer <= o.max_outer; ++outer) {
      if (graph_ok && phase == 0 && outer > 1 && outer < o.max_outer) {
        // the FP32 steps after the first run device-driven inside one CUDA
        // graph, which ends on convergence or at the FP32 phase's hand-over
        int last = outer - 1;
        Phase32State p{min32, stall32, n32, 0};
        CK(ctx->d_p32.ensure(sizeof(Phase32State)));
        CK(h2d(ctx->d_p32.p, &p, sizeof(p), st));
        if (run_monomer_graph(ctx, o, sp_mono, st, outer - 1, &last, 0, ctx->d_p32.as<Phase32State>(), cap32) ==
            cudaSuccess) {
          CK(d2h(&hs, ctx->d_mix_state.p, sizeof(hs), st));
          CK(d2h(&p, ctx->d_p32.p, sizeof(p), st));
          CK(sync_stream(st));
          outer = last;
          min32 = p.min32; stall32 = p.stall32; n32 = p.n32;
          change = hs.converged ? 0.0 : hs.diff;
          if (!(hs.diff == hs.diff) || hs.converged) break;
          if (p.hand_over) {
            phase = 1;
            reortho = 1;
            CK(cudaMemsetAsync((char*)ctx->d_mix_state.p + 3 * sizeof(double), 0, sizeof(int), st));
            CK(cudaMemsetAsync((char*)ctx->d_mix_state.p + 3 * sizeof(double) + 4 * sizeof(int), 0, sizeof(int),
                               st));
          }
          continue;
        }
        graph_ok = false;                 // graphs unavailable: host-driven steps
        cudaGetLastError();
      }
      if (graph_ok && phase == 1 && reortho == 0 && outer > 1 && outer < o.max_outer) {
        // the remaining FP64 steps run device-driven inside one CUDA graph
        int last = outer - 1;
        if (run_monomer_graph(ctx, o, sp_mono, st, outer - 1, &last) == cudaSuccess) {
          CK(d2h(&hs, ctx->d_mix_state.p, sizeof(hs), st));
          CK(sync_stream(st));
          outer = last;
          change = hs.converged ? 0.0 : hs.diff;
          break;
        }
        graph_ok = false;                 // graphs unavailable: host-driven steps
        cudaGetLastError();
      }
      // the FP32 phase works with an FP32 estimate of the potential
      CK(compute_phi(ctx, st, phase == 0 ? 1 : 0));
      stage(st, "phi", outer);
      fs = run_scc(ctx, ctx->mono, o, sp_mono, true, 0, st, 1, phase, reortho, outer == 1 ? 1 : 0,
                   (phase == 0 && outer > 1 && outer % 4 == 0) ? 1 : 0, outer == 1 ? 1.0 : hs.diff);
      if (fs != FMO_OK) return fs;
      if (world > 1 && (fs = shard_exchange(ctx, ctx->mono, step_parts, st)) != FMO_OK) return fs;
      reortho = 0;
      CK(launch_global_mix(st, ctx->n_sh, ctx->d_dq_mono.as<double>(), ctx->mono.dq.as<double>(), nf,
                           ctx->mono.energy.as<double>(), ctx->d_mix_hist.as<double>(), ctx->d_mix_state.p,
                           o.outer_tol, o.e_tol, phase == 1));
      CK(d2h(&hs, ctx->d_mix_state.p, sizeof(hs), st));
      CK(sync_stream(st));
      stage(st, "global mix", outer);
      if (debug_level() >= 5)
        fprintf(stderr, "[fmo] outer %d phase %d max|dq_out - dq_in| %.3e E1 %.12f\n", outer, phase, hs.diff, hs.e1);
      change = hs.converged ? 0.0 : hs.diff;
      if (!(hs.diff == hs.diff)) break;
      if (hs.converged) break;
      // the FP32 phase ends when converged, at its cap, or when it stops
      // improving (its rounding floor)
      if (phase == 0) {
        if (hs.diff < 0.9 * min32) { min32 = hs.diff; stall32 = 0; } else { ++stall32; }
      }
      if (phase == 0 && (hs.diff < o.mixed_switch_tol || ++n32 >= cap32 || stall32 >= kStall32)) {
        phase = 1;
        reortho = 1;
        // keep the Broyden history, but form no secant across the hand-over
        // (clear have_prev and the step count of the mixer state)
        CK(cudaMemsetAsync((char*)ctx->d_mix_state.p + 3 * sizeof(double), 0, sizeof(int), st));
        CK(cudaMemsetAsync((char*)ctx->d_mix_state.p + 3 * sizeof(double) + 4 * sizeof(int), 0, sizeof(int), st));
      }
    }
    ctx->stats.n_monomer_solves = nf;
    if (world > 1) {
      // every rank: all monomer results, and the final FP32 rows that start
      // the mixed-precision dimers and trimers
      std::vector<ExPart> parts{ex_per_nmer(ctx->mono.iters, 1, nf), ex_per_nmer(ctx->mono.status, 1, nf)};
      if (o.precision == FMO_PREC_MIXED && ctx->n_cut == 0) {
        ExPart c{ctx->mono.CTf.p, 2, ctx->mono.tot_mat, std::vector<int>(ctx->mono.tot_mat, 0)};
        for (int f = 0; f < nf; ++f) {
          const long long n2 = (long long)ctx->mono.nm[f].n * ctx->mono.nm[f].n;
          for (long long e = 0; e < n2; ++e) c.item[ctx->mono.nm[f].mat + e] = f;
        }
        parts.push_back(std::move(c));
      }
      if ((fs = shard_exchange(ctx, ctx->mono, parts, st)) != FMO_OK) return fs;
    }
  } else {
  for (outer = 1; outer <= o.max_outer; ++outer) {
    CK(compute_phi(ctx, st, 0));
    stage(st, "phi", outer);
    fs = run_scc(ctx, ctx->mono, o, sp_mono, true, 0, st, 0, 1, 0, outer == 1 ? 1 : 0);
    if (fs != FMO_OK) return fs;
    stage(st, "monomer scc", outer);
    CK(launch_maxdiff(st, ctx->n_sh, ctx->mono.dq.as<double>(), ctx->d_dq_mono.as<double>(),
                      ctx->d_scalar.as<double>()));
    CK(cudaMemcpyAsync(ctx->d_dq_mono.p, ctx->mono.dq.p, sizeof(double) * ctx->n_sh, cudaMemcpyDeviceToDevice, st));
    CK(d2h(h_change, ctx->d_scalar.p, sizeof(double), st));
    CK(sync_stream(st));
    ctx->stats.n_monomer_solves += nf;
    change = *h_change;
    if (!(change == change)) break;
    if (change < o.outer_tol) break;
  }
  }
  if (outer > o.max_outer) outer = o.max_outer;
  ctx->stats.outer_iterations = outer;
  if (o.guess == 1 && !(change < o.outer_tol)) {
    // the learned guess did not lead to self-consistent monomers: start
    // again from neutral charges
    for (auto& e : ev) cudaEventDestroy(e);
    fmo_options o2 = o;
    o2.guess = 0;
    const fmo_status rs = fmo_run(ctx, &o2, cuda_stream);
    ctx->stats.guess_restarts = 1;
    return rs;
  }
  // frozen ESP of the final monomer charges
  CK(compute_phi(ctx, st, 0));
  cudaEventRecord(ev[2], st);
  sr.set("fmo_select");
  // ---- n-mer selection
  const long long npair = (long long)nf * (nf - 1) / 2;
  std::vector<double> rmin(npair);
  std::vector<int> pair_scc(std::max<long long>(npair, 1), -1);
  std::vector<std::array<int, 3>> dim_tu, tri_tu;
  std::vector<int> dim_nf, tri_nf;
  std::vector<int2> es_pairs;
  std::vector<long long> es_idx;
  if (o.level >= 2 && npair > 0) {
    CK(ctx->d_rmin.ensure(sizeof(double) * npair));
    CK(launch_frag_bounds(st, nf, ctx->ftab(), ctx->d_xyz.as<double>(), ctx->d_bounds.as<double>()));
    CK(launch_pair_distance(st, nf, ctx->ftab(), ctx->d_xyz.as<double>(), ctx->d_bounds.as<double>(),
                            std::max(o.dimer_cut, o.trimer_cut), ctx->d_rmin.as<double>()));
    CK(d2h(rmin.data(), ctx->d_rmin.p, sizeof(double) * npair, st));
    CK(sync_stream(st));
    long long p = 0;
    for (int I = 0; I < nf; ++I)
      for (int J = I + 1; J < nf; ++J, ++p) {
        if (o.all_dimers_scc || rmin[p] < o.dimer_cut) {
          pair_scc[p] = int(dim_tu.size());
          dim_tu.push_back({I, J, -1});
          dim_nf.push_back(2);
        } else {
          es_pairs.push_back(make_int2(I, J));
          es_idx.push_back(p);
        }
      }
    if (o.level >= 3) {
      // SCC trimer iff all three pair distances < trimer_cut
      std::vector<std::vector<int>> nb(nf);
      p = 0;
      for (int I = 0; I < nf; ++I)
        for (int J = I + 1; J < nf; ++J, ++p)
          if (rmin[p] < o.trimer_cut) nb[I].push_back(J);
      auto near = [&](int a, int b) { return std::binary_search(nb[a].begin(), nb[a].end(), b); };
      for (int I = 0; I < nf; ++I)
        for (size_t x = 0; x < nb[I].size(); ++x)
          for (size_t y = x + 1; y < nb[I].size(); ++y) {
            const int J = nb[I][x], K = nb[I][y];
            if (near(J, K)) { tri_tu.push_back({I, J, K}); tri_nf.push_back(3); }
          }
      std::sort(tri_tu.begin(), tri_tu.end());
    }
  }
  cudaEventRecord(ev[3], st);
  sr.set("fmo_dimers");
  stage(st, "selection", int(dim_tu.size()));
  ctx->stats.n_dimer_scc = (long long)dim_tu.size();
  ctx->stats.n_dimer_esdim = (long long)es_pairs.size();
  ctx->stats.n_trimer_scc = (long long)tri_tu.size();
  // ---- SCC dimers in the frozen ESP
  CK(plan_pass(ctx, ctx->dim, dim_tu, dim_nf, false, o.precision, st));
  // dimers and trimers that iterate in FP32 only: no cut bonds, no gradient,
  // the FP64 energy finish
  const bool nmer_fp32_only = ctx->n_cut == 0 && !o.want_gradient && o.nmer_finish == FMO_NMER_FINISH_ENERGY;
  const SmemPlan sp_dim = plan_smem(ctx, ctx->dim, o.precision, nmer_fp32_only, o.nmer_matrix_smem);
  if (sp_dim.bytes > (size_t)ctx->smem_optin || !pass_fits(ctx->dim))
    return fail(ctx, FMO_ERR_UNSUPPORTED, "dimer too large");
  if (!dim_tu.empty()) {
    fs = setup_pass(ctx, ctx->dim, o.precision, sp_dim, st, &ctx->mono);
    if (fs != FMO_OK) return fs;
    stage(st, "dimer setup");
    fs = run_scc(ctx, ctx->dim, o, sp_dim, true, 1, st);
    if (fs != FMO_OK) return fs;
    if ((fs = shard_exchange_pass(ctx, ctx->dim, st)) != FMO_OK) return fs;
    stage(st, "dimer scc");
  }
  // ---- ES-DIM pairs (Eq. 15)
  CK(ctx->d_dE_pair.ensure(sizeof(double) * std::max<long long>(npair, 1)));
  CK(upload(ctx->d_pair_scc, pair_scc, st));
  if (!es_pairs.empty()) {
    CK(upload(ctx->d_esdim_pairs, es_pairs, st));
    CK(upload(ctx->d_esdim_idx, es_idx, st));
    CK(launch_esdim(st, int(es_pairs.size()), ctx->d_esdim_pairs.as<int2>(), ctx->d_esdim_idx.as<long long>(),
                    ctx->ftab(), ctx->d_xyz.as<double>(), ctx->d_sh_atom.as<int>(), ctx->d_sh_inv_eta.as<double>(),
                    ctx->d_dq_mono.as<double>(), ctx->g, ctx->d_dE_pair.as<double>(),
                    ctx->gam_full_ok ? ctx->d_gam_full.as<double>() : nullptr, ctx->n_sh));
  }
  cudaEventRecord(ev[4], st);
  sr.set("fmo_trimers");
  stage(st, "esdim", int(es_pairs.size()));
  // ---- SCC trimers
  CK(plan_pass(ctx, ctx->tri, tri_tu, tri_nf, false, o.precision, st));
  const SmemPlan sp_tri = plan_smem(ctx, ctx->tri, o.precision, nmer_fp32_only, o.nmer_matrix_smem);
  if (sp_tri.bytes > (size_t)ctx->smem_optin || !pass_fits(ctx->tri))
    return fail(ctx, FMO_ERR_UNSUPPORTED, "trimer too large");
  if (!tri_tu.empty()) {
    fs = setup_pass(ctx, ctx->tri, o.precision, sp_tri, st, &ctx->mono);
    if (fs != FMO_OK) return fs;
    fs = run_scc(ctx, ctx->tri, o, sp_tri, true, 2, st);
    if (fs != FMO_OK) return fs;
    if ((fs = shard_exchange_pass(ctx, ctx->tri, st)) != FMO_OK) return fs;
  }
  std::vector<int> tri_flat;
  for (auto& t : tri_tu) { tri_flat.push_back(t[0]); tri_flat.push_back(t[1]); tri_flat.push_back(t[2]); }
  CK(upload(ctx->d_tri_frag, tri_flat, st));
  CK(ctx->d_dE3.ensure(sizeof(double) * std::max<size_t>(tri_tu.size(), 1)));
  CK(ctx->d_corr.ensure(sizeof(double) * std::max<size_t>(tri_tu.size(), 1)));
  cudaEventRecord(ev[5], st);
  sr.set("fmo_sums");
  // ---- FMO sums
  CK(launch_fmo_sum(st, nf, ctx->mono.energy.as<double>(), o.level >= 2 ? npair : 0, ctx->d_pair_scc.as<int>(),
                    ctx->dim.energy.as<double>(), ctx->dim.dEV.as<double>(), ctx->d_dE_pair.as<double>(),
                    int(tri_tu.size()), ctx->d_tri_frag.as<int>(), ctx->tri.energy.as<double>(),
                    ctx->tri.dEV.as<double>(), ctx->d_dE3.as<double>(), ctx->d_corr.as<double>(),
                    ctx->d_totals.as<double>()));
  stage(st, "fmo sum");
  // ---- results to the host
  ctx->r_e_mono.resize(nf);
  ctx->r_dq_mono.resize(ctx->n_sh);
  ctx->r_mono_iters.resize(nf);
  ctx->r_mono_status.resize(nf);
  CK(d2h(ctx->totals, ctx->d_totals.p, sizeof(double) * 3, st));
  CK(d2h(ctx->r_e_mono.data(), ctx->mono.energy.p, sizeof(double) * nf, st));
  CK(d2h(ctx->r_dq_mono.data(), ctx->d_dq_mono.p, sizeof(double) * ctx->n_sh, st));
  CK(d2h(ctx->r_mono_iters.data(), ctx->mono.iters.p, sizeof(int) * nf, st));
  CK(d2h(ctx->r_mono_status.data(), ctx->mono.status.p, sizeof(int) * nf, st));
  const size_t ndim = dim_tu.size(), ntri = tri_tu.size();
  std::vector<double> e_dim(ndim), dev_dim(ndim);
  std::vector<int> it_dim(ndim), st_dim(ndim), st_tri(ntri), it_tri(ntri);
  if (o.level >= 2) {
    ctx->r_dE_pair.resize(npair);
    if (npair) CK(d2h(ctx->r_dE_pair.data(), ctx->d_dE_pair.p, sizeof(double) * npair, st));
    if (ndim) {
      CK(d2h(e_dim.data(), ctx->dim.energy.p, sizeof(double) * ndim, st));
      CK(d2h(dev_dim.data(), ctx->dim.dEV.p, sizeof(double) * ndim, st));
      CK(d2h(it_dim.data(), ctx->dim.iters.p, sizeof(int) * ndim, st));
      CK(d2h(st_dim.data(), ctx->dim.status.p, sizeof(int) * ndim, st));
    }
  }
  ctx->r_dE3.resize(ntri);
  ctx->r_corr.resize(ntri);
  if (ntri) {
    CK(d2h(ctx->r_dE3.data(), ctx->d_dE3.p, sizeof(double) * ntri, st));
    CK(d2h(ctx->r_corr.data(), ctx->d_corr.p, sizeof(double) * ntri, st));
    CK(d2h(st_tri.data(), ctx->tri.status.p, sizeof(int) * ntri, st));
    CK(d2h(it_tri.data(), ctx->tri.iters.p, sizeof(int) * ntri, st));
  }
  cudaEventRecord(ev[6], st);
  sr.end();
  CK(sync_stream(st));
  ctx->stats.ms_setup = now_ms(ev[0], ev[1]);
  ctx->stats.ms_monomer = now_ms(ev[1], ev[2]);
  ctx->stats.ms_select = now_ms(ev[2], ev[3]);
  ctx->stats.ms_dimer = now_ms(ev[3], ev[4]);
  ctx->stats.ms_trimer = now_ms(ev[4], ev[5]);
  ctx->stats.ms_reduce = now_ms(ev[5], ev[6]);
  ctx->stats.kernel_launches = launch_count() - launches0;
  for (auto& e : ev) cudaEventDestroy(e);
  // per-pair host arrays in lexicographic order
  ctx->r_pair_scc.assign(npair, 0);
  ctx->r_e_dim_pair.assign(npair, std::nan(""));
  ctx->r_dEV_pair.assign(npair, 0.0);
  ctx->r_pair_iters.assign(npair, 0);
  int failed = 0;
  for (long long p = 0; p < npair && o.level >= 2; ++p) {
    const int k = pair_scc[p];
    if (k >= 0) {
      ctx->r_pair_scc[p] = 1;
      ctx->r_e_dim_pair[p] = e_dim[k];
      ctx->r_dEV_pair[p] = dev_dim[k];
      ctx->r_pair_iters[p] = it_dim[k];
      if (st_dim[k] != FMO_SCC_CONVERGED) ++failed;
    }
  }
  for (int f = 0; f < nf; ++f) if (ctx->r_mono_status[f] != FMO_SCC_CONVERGED) ++failed;
  for (size_t t = 0; t < ntri; ++t) if (st_tri[t] != FMO_SCC_CONVERGED) ++failed;
  ctx->r_tri = tri_flat;
  ctx->r_pair_k.assign(pair_scc.begin(), pair_scc.begin() + std::max<long long>(npair, 0));
  ctx->grad_ready = ((o.precision == FMO_PREC_FP64) || o.want_gradient) && world == 1;
  ctx->last_cuts_ok = true;
  for (auto& t : tri_tu) {
    const long long nf_ = nf;
    auto pix = [&](long long a, long long b) { return a * (2 * nf_ - a - 1) / 2 + (b - a - 1); };
    if (pair_scc[pix(t[0], t[1])] < 0 || pair_scc[pix(t[0], t[2])] < 0 || pair_scc[pix(t[1], t[2])] < 0)
      ctx->last_cuts_ok = false;
  }
  long long iters = 0;
  for (int p = 0; p < 3; ++p) iters += ctx->stats.iters_fp32[p] + ctx->stats.iters_fp64[p];
  ctx->stats.scc_iterations = iters;
  ctx->stats.n_failed = failed;
  ctx->stats.h2d_bytes = ctx->h2d_bytes;
  ctx->stats.d2h_bytes = ctx->d2h_bytes;
  ctx->h2d_bytes = 0;
  ctx->last_level = o.level;
  ctx->last_precision = o.precision;
  if (o.level < 2) ctx->totals[1] = std::nan("");
  if (o.level < 3) ctx->totals[2] = std::nan("");
  ctx->have_result = true;
  bool timeout = false;
  for (int s : ctx->r_mono_status) timeout |= (s == FMO_SCC_TIMEOUT);
  for (int s : st_dim) timeout |= (s == FMO_SCC_TIMEOUT);
  for (int s : st_tri) timeout |= (s == FMO_SCC_TIMEOUT);
  if (timeout) return fail(ctx, FMO_ERR_TIMEOUT, "deadline reached");
  for (int k = 0; k < o.level; ++k)
    if (!std::isfinite(ctx->totals[k])) return fail(ctx, FMO_ERR_NAN, "non-finite FMO total");
  if (failed > 0 || change >= o.outer_tol)
    return fail(ctx, FMO_ERR_NOT_CONVERGED, std::to_string(failed) + " n-mer solves did not converge");
  ctx->err.clear();
  return FMO_OK;
}

fmo_status fmo_set_exchange(fmo_ctx* ctx, fmo_exchange_fn fn, void* user) {
  if (!ctx) return FMO_ERR_ARG;
  ctx->ex_fn = fn;
  ctx->ex_user = user;
  return FMO_OK;
}

fmo_status fmo_lpt_partition(const double* cost, int64_t n, int32_t world, int32_t* owner) {
  if (n < 0 || world < 1 || (n > 0 && (!cost || !owner))) return FMO_ERR_ARG;
  std::vector<double> c(cost, cost + n);
  for (double x : c)
    if (!(x >= 0.0) || !std::isfinite(x)) return FMO_ERR_ARG;
  const std::vector<int> o = lpt_owner(c, world);
  for (int64_t i = 0; i < n; ++i) owner[i] = o[i];
  return FMO_OK;
}

fmo_status fmo_get_energy(fmo_ctx* ctx, double* e1, double* e2, double* e3) {
  if (!ctx) return FMO_ERR_ARG;
  if (!ctx->have_result) return fail(ctx, FMO_ERR_STATE, "no results: call fmo_run");
  if (e1) *e1 = ctx->totals[0];
  if (e2) *e2 = ctx->totals[1];
  if (e3) *e3 = ctx->totals[2];
  return FMO_OK;
}

fmo_status fmo_get_sizes(fmo_ctx* ctx, int32_t* n_shell, int32_t* n_ao) {
  if (!ctx) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  if (n_shell) *n_shell = ctx->n_sh;
  if (n_ao) *n_ao = ctx->n_ao;
  return FMO_OK;
}

fmo_status fmo_get_monomers(fmo_ctx* ctx, double* E_I, double* shell_dq, int32_t* iters, int32_t* status) {
  if (!ctx) return FMO_ERR_ARG;
  if (!ctx->have_result) return fail(ctx, FMO_ERR_STATE, "no results: call fmo_run");
  if (E_I) std::memcpy(E_I, ctx->r_e_mono.data(), sizeof(double) * ctx->n_frag);
  if (shell_dq) std::memcpy(shell_dq, ctx->r_dq_mono.data(), sizeof(double) * ctx->n_sh);
  if (iters) std::memcpy(iters, ctx->r_mono_iters.data(), sizeof(int) * ctx->n_frag);
  if (status) std::memcpy(status, ctx->r_mono_status.data(), sizeof(int) * ctx->n_frag);
  return FMO_OK;
}

fmo_status fmo_get_dimers(fmo_ctx* ctx, int64_t* n, int32_t* ij, double* dE, double* e_dimer, double* dEV,
                          uint8_t* scc, int32_t* iters) {
  if (!ctx || !n) return FMO_ERR_ARG;
  if (!ctx->have_result) return fail(ctx, FMO_ERR_STATE, "no results: call fmo_run");
  const long long np = ctx->last_level >= 2 ? (long long)ctx->n_frag * (ctx->n_frag - 1) / 2 : 0;
  *n = np;
  long long p = 0;
  if (ij)
    for (int I = 0; I < ctx->n_frag; ++I)
      for (int J = I + 1; J < ctx->n_frag && p < np; ++J, ++p) { ij[2 * p] = I; ij[2 * p + 1] = J; }
  if (np == 0) return FMO_OK;
  if (dE) std::memcpy(dE, ctx->r_dE_pair.data(), sizeof(double) * np);
  if (e_dimer) std::memcpy(e_dimer, ctx->r_e_dim_pair.data(), sizeof(double) * np);
  if (dEV) std::memcpy(dEV, ctx->r_dEV_pair.data(), sizeof(double) * np);
  if (scc) std::memcpy(scc, ctx->r_pair_scc.data(), np);
  if (iters) std::memcpy(iters, ctx->r_pair_iters.data(), sizeof(int) * np);
  return FMO_OK;
}

fmo_status fmo_get_gradient(fmo_ctx* ctx, double* grad) {
  if (!ctx || !grad) return FMO_ERR_ARG;
  if (!ctx->have_result) return fail(ctx, FMO_ERR_STATE, "no results: call fmo_run");
  if (ctx->n_cut > 0)
    return fail(ctx, FMO_ERR_UNSUPPORTED, "gradient: cut bonds (hybrid orbital projection) are not covered");
  if (!ctx->grad_ready)
    return fail(ctx, FMO_ERR_UNSUPPORTED,
                "gradient: the run's n-mer densities are not converged in FP64 (precision FP64, or mixed with "
                "want_gradient = 1)");
  if (!ctx->last_cuts_ok)
    return fail(ctx, FMO_ERR_UNSUPPORTED, "gradient: a trimer holds an ES-DIM pair (trimer_cut > dimer_cut)");
  g_ctx = ctx;
  cudaSetDevice(ctx->device);
  std::vector<double> g;
  const fmo_status fs = compute_gradient(ctx, g);
  if (fs != FMO_OK) return fs;
  for (int i = 0; i < ctx->n_atoms; ++i)   // internal atom order -> input order
    for (int c = 0; c < 3; ++c) grad[3 * ctx->perm[i] + c] = g[3 * (size_t)i + c];
  return FMO_OK;
}

fmo_status fmo_get_trimers(fmo_ctx* ctx, int64_t* n, int32_t* ijk, double* dE3, double* corr) {
  if (!ctx || !n) return FMO_ERR_ARG;
  if (!ctx->have_result) return fail(ctx, FMO_ERR_STATE, "no results: call fmo_run");
  const long long nt = (long long)ctx->r_dE3.size();
  *n = nt;
  if (ijk && nt) std::memcpy(ijk, ctx->r_tri.data(), sizeof(int) * 3 * nt);
  if (dE3 && nt) std::memcpy(dE3, ctx->r_dE3.data(), sizeof(double) * nt);
  if (corr && nt) std::memcpy(corr, ctx->r_corr.data(), sizeof(double) * nt);
  return FMO_OK;
}

fmo_status fmo_get_stats(fmo_ctx* ctx, fmo_stats* st) {
  if (!ctx || !st) return FMO_ERR_ARG;
  *st = ctx->stats;
  return FMO_OK;
}

static_assert(kMlpWeights == FMO_MLP_N_WEIGHTS, "weight layout of the header");
static_assert(kMlpTrained == FMO_MLP_N_TRAINED, "trained-weight count of the header");

fmo_status fmo_mlp_init(fmo_ctx* ctx, uint64_t seed) {
  g_ctx = ctx;
  if (!ctx) return FMO_ERR_ARG;
  cudaSetDevice(ctx->device);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<float> w(kMlpWeights, 0.0f);
  auto fill = [&](int off, int fo, int fi, double gain) {
    for (int k = 0; k < fo * fi; ++k) w[off + k] = float(nd(rng) * std::sqrt(1.0 / fi) * gain);
  };
  fill(kMlpOffW1, kMlpHidden, kMlpIn, 1.0);
  fill(kMlpOffW2, kMlpHidden, kMlpHidden, 1.0);
  fill(kMlpOffW3, 2, kMlpHidden, 0.1);
  for (int k = 0; k < kMlpIn; ++k) w[kMlpOffScale + k] = 1.0f;
  return fmo_mlp_set_weights(ctx, w.data(), kMlpWeights);
}

fmo_status fmo_mlp_set_weights(fmo_ctx* ctx, const float* w, int64_t n) {
  g_ctx = ctx;
  if (!ctx || !w) return FMO_ERR_ARG;
  if (n != kMlpWeights) return fail(ctx, FMO_ERR_ARG, "weight count must be " + std::to_string(kMlpWeights));
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->own_stream;
  CK(ctx->d_mlp_W.ensure(sizeof(float) * kMlpWeights));
  CK(ctx->d_mlp_W16.ensure(sizeof(__half) * kMlpTrained));
  CK(ctx->d_mlp_m.ensure(sizeof(float) * kMlpTrained));
  CK(ctx->d_mlp_v.ensure(sizeof(float) * kMlpTrained));
  CK(h2d(ctx->d_mlp_W.p, w, sizeof(float) * kMlpWeights, st));
  CK(cudaMemsetAsync(ctx->d_mlp_m.p, 0, sizeof(float) * kMlpTrained, st));
  CK(cudaMemsetAsync(ctx->d_mlp_v.p, 0, sizeof(float) * kMlpTrained, st));
  CK(mlp_to_half(st, kMlpTrained, ctx->d_mlp_W.as<float>(), ctx->d_mlp_W16.as<__half>()));
  CK(sync_stream(st));
  ctx->mlp_ready = true;
  return FMO_OK;
}

fmo_status fmo_mlp_get_weights(fmo_ctx* ctx, float* w, int64_t* n) {
  g_ctx = ctx;
  if (!ctx || !n) return FMO_ERR_ARG;
  *n = kMlpWeights;
  if (!w) return FMO_OK;
  if (!ctx->mlp_ready) return fail(ctx, FMO_ERR_STATE, "no model weights");
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->own_stream;
  CK(d2h(w, ctx->d_mlp_W.p, sizeof(float) * kMlpWeights, st));
  CK(sync_stream(st));
  return FMO_OK;
}

fmo_status fmo_mlp_predict(fmo_ctx* ctx, double* shell_dq) {
  g_ctx = ctx;
  if (!ctx || !shell_dq) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  if (!ctx->mlp_ready) return fail(ctx, FMO_ERR_STATE, "no model weights");
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->own_stream;
  DevBuf out;
  CK(out.ensure(sizeof(double) * ctx->n_sh));
  fmo_status fs = mlp_predict_device(ctx, st, out.as<double>());
  if (fs != FMO_OK) { out.release(); return fs; }
  int err = 0;
  CK(d2h(&err, ctx->d_mlp_err.p, sizeof(int), st));
  CK(d2h(shell_dq, out.p, sizeof(double) * ctx->n_sh, st));
  CK(sync_stream(st));
  out.release();
  if (err) return fail(ctx, FMO_ERR_UNSUPPORTED, "more than 256 neighbours within 6 A of an atom");
  return FMO_OK;
}

fmo_status fmo_mlp_loss_grad(fmo_ctx* ctx, int32_t n_frames, const double* xyz_frames, const double* shell_dq,
                             double* loss, float* grad) {
  g_ctx = ctx;
  if (!ctx || !xyz_frames || !shell_dq || !loss) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  if (!ctx->mlp_ready) return fail(ctx, FMO_ERR_STATE, "initialise or set the model weights first");
  if (n_frames < 1) return fail(ctx, FMO_ERR_ARG, "n_frames must be positive");
  cudaSetDevice(ctx->device);
  fmo_status fs = mlp_tables(ctx);
  if (fs != FMO_OK) return fs;
  cudaStream_t st = ctx->own_stream;
  const int N = ctx->n_int, B = n_frames, nsh = ctx->n_sh;
  const size_t rows = (size_t)N * B;
  const int chunk = 256, n_chunks = int((rows + chunk - 1) / chunk);
  DevBuf xyzb, tmp, Xb, y, q, gy, tb, x0, z1, h1, z2, h2, gz1, gz2, part, lpart, gbuf;
  CK(xyzb.ensure(sizeof(double) * 3 * rows));
  CK(tmp.ensure(sizeof(double) * 3 * (size_t)ctx->n_atoms));
  CK(tb.ensure(sizeof(float) * rows * 2));
  std::vector<float> tf(nsh);
  for (int f = 0; f < B; ++f) {
    CK(h2d(tmp.p, xyz_frames + (size_t)f * 3 * ctx->n_atoms, sizeof(double) * 3 * ctx->n_atoms, st));
    CK(launch_gather_xyz(st, N, ctx->d_perm.as<int>(), tmp.as<double>(), xyzb.as<double>() + (size_t)f * 3 * N));
    for (int k = 0; k < nsh; ++k) tf[k] = float(shell_dq[(size_t)f * nsh + k]);
    CK(h2d(tb.as<float>() + (size_t)f * nsh, tf.data(), sizeof(float) * nsh, st));
    CK(sync_stream(st));
  }
  CK(Xb.ensure(sizeof(float) * rows * kMlpStride));
  CK(y.ensure(sizeof(float) * rows * 2));
  CK(q.ensure(sizeof(float) * rows * 2));
  CK(gy.ensure(sizeof(float) * rows * 2));
  CK(x0.ensure(sizeof(float) * rows * kMlpStride));
  for (DevBuf* b : {&z1, &h1, &z2, &h2, &gz1, &gz2}) CK(b->ensure(sizeof(float) * rows * kMlpHidden));
  CK(part.ensure(sizeof(float) * (size_t)n_chunks * kMlpTrained));
  CK(lpart.ensure(sizeof(double) * (size_t)B * ctx->n_frag));
  CK(gbuf.ensure(sizeof(float) * kMlpTrained));
  CK(cudaMemsetAsync(ctx->d_mlp_err.p, 0, sizeof(int), st));
  CK(mlp_descriptors(st, B, N, xyzb.as<double>(), ctx->d_mlp_elem4.as<int>(), Xb.as<float>(), ctx->d_mlp_err.as<int>()));
  const float* W = ctx->d_mlp_W.as<float>();
  const __half* W16 = ctx->d_mlp_W16.as<__half>();
  const MlpCache none{nullptr, nullptr, nullptr, nullptr, nullptr};
  const MlpCache cache{x0.as<float>(), z1.as<float>(), h1.as<float>(), z2.as<float>(), h2.as<float>()};
  // the two passes of the training loss (pass-0 potential held fixed)
  CK(mlp_forward(st, int(rows), Xb.as<float>(), W16, W + kMlpOffMean, W + kMlpOffScale, y.as<float>(), none));
  CK(mlp_project(st, B, ctx->n_frag, N, ctx->d_f_atom0.as<int>(), ctx->d_f_nat.as<int>(), ctx->d_mlp_fcharge.as<int>(),
                 y.as<float>(), q.as<float>(), nullptr, 0.0, nullptr, nullptr));
  CK(mlp_esp(st, B, N, nsh, xyzb.as<double>(), ctx->d_mlp_atom_frag.as<int>(), ctx->d_mlp_atom_ie.as<float>(),
             ctx->d_sh_atom.as<int>(), ctx->d_mlp_sh_ie.as<float>(), q.as<float>(), Xb.as<float>()));
  CK(mlp_forward(st, int(rows), Xb.as<float>(), W16, W + kMlpOffMean, W + kMlpOffScale, y.as<float>(), cache));
  CK(mlp_project(st, B, ctx->n_frag, N, ctx->d_f_atom0.as<int>(), ctx->d_f_nat.as<int>(), ctx->d_mlp_fcharge.as<int>(),
                 y.as<float>(), q.as<float>(), tb.as<float>(), 1.0 / double(rows * 2), gy.as<float>(),
                 lpart.as<double>()));
  CK(mlp_gradient(st, int(rows), gy.as<float>(), W16, cache, gz2.as<float>(), gz1.as<float>(), part.as<float>(), chunk,
                  gbuf.as<float>()));
  std::vector<double> lp((size_t)B * ctx->n_frag);
  int err = 0;
  CK(d2h(lp.data(), lpart.p, sizeof(double) * lp.size(), st));
  if (grad) CK(d2h(grad, gbuf.p, sizeof(float) * kMlpTrained, st));
  CK(d2h(&err, ctx->d_mlp_err.p, sizeof(int), st));
  CK(sync_stream(st));
  double ls = 0.0;
  for (double v : lp) ls += v;
  *loss = ls / double(rows * 2);
  for (DevBuf* b : {&xyzb, &tmp, &Xb, &y, &q, &gy, &tb, &x0, &z1, &h1, &z2, &h2, &gz1, &gz2, &part, &lpart, &gbuf})
    b->release();
  if (err) return fail(ctx, FMO_ERR_UNSUPPORTED, "more than 256 neighbours within 6 A of an atom");
  return FMO_OK;
}

fmo_status fmo_mlp_train(fmo_ctx* ctx, int32_t n_frames, const double* xyz_frames, const double* shell_dq,
                         int32_t epochs, int32_t batch_frames, double lr, uint64_t seed, double* loss_per_epoch) {
  g_ctx = ctx;
  if (!ctx || !xyz_frames || !shell_dq) return FMO_ERR_ARG;
  if (!ctx->have_system) return fail(ctx, FMO_ERR_STATE, "fmo_set_system first");
  if (!ctx->mlp_ready) return fail(ctx, FMO_ERR_STATE, "initialise or set the model weights first");
  if (n_frames < 1 || epochs < 1 || batch_frames < 1 || !(lr > 0))
    return fail(ctx, FMO_ERR_ARG, "frames, epochs, batch size and learning rate must be positive");
  cudaSetDevice(ctx->device);
  fmo_status fs = mlp_tables(ctx);
  if (fs != FMO_OK) return fs;
  cudaStream_t st = ctx->own_stream;
  const int N = ctx->n_int, F = n_frames, B = std::min(batch_frames, n_frames), nsh = ctx->n_sh;
  // frames in internal atom order, their features and targets (float)
  DevBuf xyz_all, X_all, tgt_all, tmp;
  CK(xyz_all.ensure(sizeof(double) * 3 * (size_t)N * F));
  CK(X_all.ensure(sizeof(float) * (size_t)N * kMlpStride * F));
  CK(tgt_all.ensure(sizeof(float) * (size_t)nsh * F));
  CK(tmp.ensure(sizeof(double) * std::max((size_t)3 * ctx->n_atoms, (size_t)nsh)));
  std::vector<float> tf(nsh);
  for (int f = 0; f < F; ++f) {
    CK(h2d(tmp.p, xyz_frames + (size_t)f * 3 * ctx->n_atoms, sizeof(double) * 3 * ctx->n_atoms, st));
    CK(launch_gather_xyz(st, N, ctx->d_perm.as<int>(), tmp.as<double>(), xyz_all.as<double>() + (size_t)f * 3 * N));
    for (int k = 0; k < nsh; ++k) tf[k] = float(shell_dq[(size_t)f * nsh + k]);
    CK(h2d(tgt_all.as<float>() + (size_t)f * nsh, tf.data(), sizeof(float) * nsh, st));
    CK(sync_stream(st));
  }
  CK(cudaMemsetAsync(ctx->d_mlp_err.p, 0, sizeof(int), st));
  CK(mlp_descriptors(st, F, N, xyz_all.as<double>(), ctx->d_mlp_elem4.as<int>(), X_all.as<float>(),
                     ctx->d_mlp_err.as<int>()));
  float* W = ctx->d_mlp_W.as<float>();
  CK(mlp_feature_stats(st, (long long)N * F, X_all.as<float>(), W + kMlpOffMean, W + kMlpOffScale));
  {
    // ESP feature: fixed scale 10 (potentials of ~0.01-0.1 Eh/e); one-hot as is
    std::vector<float> ms = {0.0f, 10.0f, 0.0f, 1.0f, 0.0f, 1.0f, 0.0f, 1.0f, 0.0f, 1.0f};
    for (int k = 72; k < kMlpIn; ++k) {
      CK(h2d(W + kMlpOffMean + k, &ms[2 * (k - 72)], sizeof(float), st));
      CK(h2d(W + kMlpOffScale + k, &ms[2 * (k - 72) + 1], sizeof(float), st));
    }
  }
  CK(cudaMemsetAsync(ctx->d_mlp_m.p, 0, sizeof(float) * kMlpTrained, st));
  CK(cudaMemsetAsync(ctx->d_mlp_v.p, 0, sizeof(float) * kMlpTrained, st));
  CK(sync_stream(st));
  // batch buffers
  const size_t rows = (size_t)N * B;
  const int chunk = 256, n_chunks = int((rows + chunk - 1) / chunk);
  DevBuf Xb, xyzb, y, q, gy, tb, x0, z1, h1, z2, h2, gz1, gz2, part, lpart, idx;
  CK(Xb.ensure(sizeof(float) * rows * kMlpStride));
  CK(xyzb.ensure(sizeof(double) * rows * 3));
  CK(y.ensure(sizeof(float) * rows * 2));
  CK(q.ensure(sizeof(float) * rows * 2));
  CK(gy.ensure(sizeof(float) * rows * 2));
  CK(tb.ensure(sizeof(float) * rows * 2));
  CK(x0.ensure(sizeof(float) * rows * kMlpStride));
  for (DevBuf* b : {&z1, &h1, &z2, &h2, &gz1, &gz2}) CK(b->ensure(sizeof(float) * rows * kMlpHidden));
  CK(part.ensure(sizeof(float) * (size_t)n_chunks * kMlpTrained));
  CK(lpart.ensure(sizeof(double) * (size_t)B * ctx->n_frag));
  CK(idx.ensure(sizeof(int) * B));
  const MlpCache none{nullptr, nullptr, nullptr, nullptr, nullptr};
  const MlpCache cache{x0.as<float>(), z1.as<float>(), h1.as<float>(), z2.as<float>(), h2.as<float>()};
  std::mt19937_64 rng(seed);
  std::vector<int> order(F);
  for (int f = 0; f < F; ++f) order[f] = f;
  std::vector<double> lp((size_t)B * ctx->n_frag);
  int t = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    std::shuffle(order.begin(), order.end(), rng);
    double lsum = 0.0;
    long long lcount = 0;
    for (int b0 = 0; b0 + B <= F; b0 += B) {
      CK(h2d(idx.p, order.data() + b0, sizeof(int) * B, st));
      CK(mlp_gather(st, B, N, idx.as<int>(), X_all.as<float>(), xyz_all.as<double>(), Xb.as<float>(),
                    xyzb.as<double>()));
      for (int k = 0; k < B; ++k)
        CK(cudaMemcpyAsync(tb.as<float>() + (size_t)k * nsh, tgt_all.as<float>() + (size_t)order[b0 + k] * nsh,
                           sizeof(float) * nsh, cudaMemcpyDeviceToDevice, st));
      const __half* W16 = ctx->d_mlp_W16.as<__half>();
      // pass 0 (ESP = 0), then the ESP of its charges, then pass 1 with cache
      CK(mlp_forward(st, int(rows), Xb.as<float>(), W16, W + kMlpOffMean, W + kMlpOffScale, y.as<float>(), none));
      CK(mlp_project(st, B, ctx->n_frag, N, ctx->d_f_atom0.as<int>(), ctx->d_f_nat.as<int>(),
                     ctx->d_mlp_fcharge.as<int>(), y.as<float>(), q.as<float>(), nullptr, 0.0, nullptr, nullptr));
      CK(mlp_esp(st, B, N, nsh, xyzb.as<double>(), ctx->d_mlp_atom_frag.as<int>(), ctx->d_mlp_atom_ie.as<float>(),
                 ctx->d_sh_atom.as<int>(), ctx->d_mlp_sh_ie.as<float>(), q.as<float>(), Xb.as<float>()));
      CK(mlp_forward(st, int(rows), Xb.as<float>(), W16, W + kMlpOffMean, W + kMlpOffScale, y.as<float>(), cache));
      CK(mlp_project(st, B, ctx->n_frag, N, ctx->d_f_atom0.as<int>(), ctx->d_f_nat.as<int>(),
                     ctx->d_mlp_fcharge.as<int>(), y.as<float>(), q.as<float>(), tb.as<float>(),
                     1.0 / double(rows * 2), gy.as<float>(), lpart.as<double>()));
      ++t;
      CK(mlp_backward_step(st, int(rows), gy.as<float>(), W16, cache, gz2.as<float>(), gz1.as<float>(),
                           part.as<float>(), chunk, W, ctx->d_mlp_m.as<float>(), ctx->d_mlp_v.as<float>(),
                           ctx->d_mlp_W16.as<__half>(), float(lr), t));
      CK(d2h(lp.data(), lpart.p, sizeof(double) * lp.size(), st));
      CK(sync_stream(st));
      for (double v : lp) lsum += v;
      lcount += (long long)rows * 2;
    }
    if (loss_per_epoch) loss_per_epoch[ep] = lcount ? lsum / double(lcount) : 0.0;
  }
  int err = 0;
  CK(d2h(&err, ctx->d_mlp_err.p, sizeof(int), st));
  CK(sync_stream(st));
  for (DevBuf* b : {&xyz_all, &X_all, &tgt_all, &tmp, &Xb, &xyzb, &y, &q, &gy, &tb, &x0, &z1, &h1, &z2, &h2, &gz1,
                    &gz2, &part, &lpart, &idx})
    b->release();
  if (err) return fail(ctx, FMO_ERR_UNSUPPORTED, "more than 256 neighbours within 6 A of an atom");
  return FMO_OK;
}

}  // extern "C"
