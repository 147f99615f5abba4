// CUDA kernels of the batched FMO-xTB SCC path (sm_103a).
//
// Paper references (Einsele & Mitric, FMO-xTB):
//   Eq. 2        electronic energy        Eq. 3      Mulliken shell charges
//   Eqs. 4-5     gamma kernel, eta        Eq. 6      Fermi occupations
//   Eq. 7        Fock matrix              Eqs. 8-10  H0, Pi, CN-dependent levels
//   Eq. 11       repulsion                CN definition in the gradient section
//   Eqs. 12-15   FMO2, dE^V, ddq, ES-DIM  Eqs. 16-19 FMO3
//   Eqs. 20-21   embedding Fock matrix V^I from the other fragments' charges
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "fmo_device.cuh"
#include "kernels.h"
#include "tridiag.cuh"

namespace fmo {

// ---------------------------------------------------------------------------
// Coordination numbers of the whole system (CN definition; pairs beyond the
// cutoff are not counted).

__global__ void cn_kernel(int n_atoms, const double* __restrict__ xyz, const int* __restrict__ elem,
                          const DevElem* __restrict__ el, GParams g, const int* __restrict__ ghost_src,
                          double* __restrict__ cn) {
  // one warp per atom a, lanes over the partners b
  const int lane = threadIdx.x & 31;
  const int a = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (a >= n_atoms) return;
  const double xa = xyz[3 * a], ya = xyz[3 * a + 1], za = xyz[3 * a + 2];
  const double ra = el[elem[a]].rcov;
  const double cut2 = g.cn_cutoff * g.cn_cutoff * (1.0 + 1e-12);   // exact test on r below
  double s = 0.0;
  // a ghost (a copy of a bond-detachment atom at its position) gets that
  // atom's CN: ghosts are never partners, and its BDA is skipped like itself
  const int self2 = ghost_src ? ghost_src[a] : -1;
  for (int b = lane; b < n_atoms; b += 32) {
    if (b == a || b == self2 || (ghost_src && ghost_src[b] >= 0)) continue;
    const double dx = xyz[3 * b] - xa, dy = xyz[3 * b + 1] - ya, dz = xyz[3 * b + 2] - za;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= cut2) continue;
    const double r = sqrt(r2);
    if (r >= g.cn_cutoff) continue;
    const double arg = -g.cn_k1 * (g.cn_k2 * (ra + el[elem[b]].rcov) / r - 1.0);
    s += 1.0 / (1.0 + exp(arg));
  }
  s = warp_sum(s);
  if (lane == 0) cn[a] = s;
}

// ---------------------------------------------------------------------------
// n-mer index maps (built by thread 0 of a block into shared memory).

struct MapCounts {
  int nat, nsh, n;
};

__device__ void build_maps(const Nmer& nm, const FragTab ft, const int* __restrict__ elem,
                           const int* __restrict__ atom_sh0, const DevElem* __restrict__ el,
                           NmerMaps mp) {
  if (threadIdx.x == 0) {
    int la = 0, ls = 0, lao = 0;
    for (int k = 0; k < nm.nfrag; ++k) {
      const int f = nm.frag[k];
      const int a0 = ft.atom0[f], na = ft.nat[f];
      for (int i = 0; i < na; ++i) {
        const int ga = a0 + i;
        if (!atom_in_nmer(ft, nm.nfrag, nm.frag, ga)) continue;   // ghost of a healed bond
        mp.at_glob[la] = ga;
        const DevElem& e = el[elem[ga]];
        for (int s = 0; s < e.nsh; ++s) {
          mp.sh_at[ls] = (int16_t)la;
          mp.sh_glob[ls] = atom_sh0[ga] + s;
          mp.sh_ao0[ls] = (int16_t)lao;
          for (int m = 0; m < 2 * e.l[s] + 1; ++m) mp.ao_sh[lao++] = (int16_t)ls;
          ++ls;
        }
        ++la;
      }
    }
    mp.sh_ao0[ls] = (int16_t)lao;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Overlap and H0 of an n-mer (Eqs. 8-10), one thread per atom pair A <= B.
// Contracted s/p Gaussians: two primitives combine into one of exponent
// p = a + b at P = (aA + bB)/p; s-s overlap (pi/p)^{3/2} exp(-ab/p R^2); a p
// factor contributes (P - A)_i, a pair of p factors (P-A)_i (P-B)_j + d_ij/2p.

// Primitive pairs whose Gaussian factor exp(-ab/p R^2) is below e^-46 (about
// 1e-20) are skipped.  prim (optional) holds the geometry-free factors of
// every primitive pair (PrimPair); without it they are formed here.
constexpr double kPrimScreen = 46.0;

// With mono != nullptr the intra-fragment blocks are copied from the monomer
// pass (identical: the CN is that of the whole system) and only pairs of
// atoms in different fragments are evaluated.
__global__ void integrals_kernel(const Nmer* __restrict__ nmers, FragTab ft,
                                 const double* __restrict__ xyz, const int* __restrict__ elem,
                                 const int* __restrict__ atom_sh0, const double* __restrict__ cn,
                                 const DevElem* __restrict__ el, const double* __restrict__ kab,
                                 int ne, GParams g, double* __restrict__ S,
                                 double* __restrict__ H0, const Nmer* __restrict__ mono,
                                 const double* __restrict__ mono_S, const double* __restrict__ mono_H0,
                                 const PrimPair* __restrict__ prim) {
  const Nmer nm = nmers[blockIdx.y];
  __shared__ int s_glob[512];
  __shared__ int s_ao0[512];
  __shared__ unsigned char s_fk[512];
  __shared__ int s_foff[4];
  if (threadIdx.x == 0) {
    int la = 0, lao = 0;
    for (int k = 0; k < nm.nfrag; ++k) {
      const int f = nm.frag[k];
      s_foff[k] = lao;
      for (int i = 0; i < ft.nat[f]; ++i) {
        const int ga = ft.atom0[f] + i;
        if (!atom_in_nmer(ft, nm.nfrag, nm.frag, ga)) continue;   // ghost of a healed bond
        s_glob[la] = ga;
        s_ao0[la] = lao;
        s_fk[la] = (unsigned char)k;
        const DevElem& e = el[elem[ga]];
        for (int s = 0; s < e.nsh; ++s) lao += 2 * e.l[s] + 1;
        ++la;
      }
    }
    s_foff[nm.nfrag] = lao;
  }
  __syncthreads();
  if (mono) {
    // intra-fragment blocks from the monomer matrices
    const int n = nm.n;
    for (int k = 0; k < nm.nfrag; ++k) {
      const Nmer& m = mono[nm.frag[k]];
      const int o = s_foff[k], nk = m.n;
      for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nk * nk; e += gridDim.x * blockDim.x) {
        const int u = e / nk, v = e - u * nk;
        S[nm.mat + (long long)(o + u) * n + (o + v)] = mono_S[m.mat + e];
        H0[nm.mat + (long long)(o + u) * n + (o + v)] = mono_H0[m.mat + e];
      }
    }
  }
  const long long npairs = (long long)nm.nat * (nm.nat + 1) / 2;
  const int n = nm.n;
  double* Sm = S + nm.mat;
  double* Hm = H0 + nm.mat;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < npairs;
       e += (long long)gridDim.x * blockDim.x) {
    // triangular index -> (i, j), j <= i
    long long i = (long long)((sqrt(8.0 * double(e) + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > e) --i;
    while ((i + 1) * (i + 2) / 2 <= e) ++i;
    const int ai = int(i), bj = int(e - i * (i + 1) / 2);
    if (mono && s_fk[ai] == s_fk[bj]) continue;      // copied above
    const int ga = s_glob[ai], gb = s_glob[bj];
    const DevElem& EA = el[elem[ga]];
    const DevElem& EB = el[elem[gb]];
    const double Ax = xyz[3 * ga], Ay = xyz[3 * ga + 1], Az = xyz[3 * ga + 2];
    const double dx = xyz[3 * gb] - Ax, dy = xyz[3 * gb + 1] - Ay, dz = xyz[3 * gb + 2] - Az;
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double R = sqrt(r2);
    const bool same = (ai == bj);
    // pair prefactors of Eq. 8
    const double den = EA.en - EB.en;
    const double fen = 1.0 + g.k_en * den * den;
    const double kAB = kab[elem[ga] * ne + elem[gb]];
    const double rcov = EA.rcov + EB.rcov;
    const double ratio = same ? 0.0 : sqrt(R / rcov);
    int aoA = s_ao0[ai];
    for (int sa = 0; sa < EA.nsh; ++sa) {
      const int la = EA.l[sa];
      const double hA = EA.h[sa] * (1.0 + EA.kcn[sa] * cn[ga]);
      int aoB = s_ao0[bj];
      for (int sb = 0; sb < EB.nsh; ++sb) {
        const int lb = EB.l[sb];
        // PA = (b/p) d and PB = -(a/p) d are multiples of the bond vector d,
        // so each block is d-weighted sums of two scalars over the
        // primitive pairs: ss: sum s00; ps: d_u sum (b/p) s00; sp: -d_v sum
        // (a/p) s00; pp: -d_u d_v sum (a/p)(b/p) s00 + delta_uv sum 1/(2p) s00
        double t0 = 0.0, t1 = 0.0;
        for (int pa = 0; pa < EA.nprim[sa]; ++pa) {
          for (int pb = 0; pb < EB.nprim[sb]; ++pb) {
            PrimPair q;
            if (prim) {
              q = prim[prim_pair_index(ne, elem[ga], elem[gb], sa, sb, pa, pb)];
            } else {
              const double a = EA.alpha[sa][pa], b = EB.alpha[sb][pb];
              q.ip = 1.0 / (a + b);
              q.abp = a * b * q.ip;
              q.ap = a * q.ip;
              q.bp = b * q.ip;
              q.pref = EA.cn[sa][pa] * EB.cn[sb][pb] * (M_PI * q.ip) * sqrt(M_PI * q.ip);
            }
            const double xe = q.abp * r2;
            if (xe > kPrimScreen) continue;   // exp(-xe) < 1e-20
            const double s00 = q.pref * exp(-xe);
            if (la == 0 && lb == 0) {
              t0 += s00;
            } else if (la == 1 && lb == 0) {
              t0 = fma(q.bp, s00, t0);
            } else if (la == 0 && lb == 1) {
              t0 = fma(q.ap, s00, t0);
            } else {
              t0 = fma(q.ap * q.bp, s00, t0);
              t1 = fma(q.ip, s00, t1);
            }
          }
        }
        const double d[3] = {dx, dy, dz};
        double blk[3][3];
#pragma unroll
        for (int u = 0; u < 3; ++u)
#pragma unroll
          for (int v = 0; v < 3; ++v) {
            if (la == 0 && lb == 0) blk[u][v] = t0;
            else if (la == 1 && lb == 0) blk[u][v] = d[u] * t0;
            else if (la == 0 && lb == 1) blk[u][v] = -d[v] * t0;
            else blk[u][v] = -d[u] * d[v] * t0 + (u == v ? 0.5 * t1 : 0.0);
          }
        const int nu = 2 * la + 1, nv = 2 * lb + 1;
        double fac = 0.0;
        const double hB = EB.h[sb] * (1.0 + EB.kcn[sb] * cn[gb]);
        if (!same) {
          const double pi = (1.0 + EA.kpoly[sa] * ratio) * (1.0 + EB.kpoly[sb] * ratio);  // Eq. 9
          fac = kAB * 0.5 * (g.k_l[la] + g.k_l[lb]) * 0.5 * (hA + hB) * fen * pi;          // Eq. 8
        }
        for (int u = 0; u < nu; ++u) {
          for (int v = 0; v < nv; ++v) {
            const int mu = aoA + u, nu2 = aoB + v;
            const double sv = blk[u][v];
            double hv = fac * sv;
            if (same) hv = (mu == nu2) ? hA : 0.0;   // on-site: levels of Eq. 10
            Sm[(long long)mu * n + nu2] = sv;
            Sm[(long long)nu2 * n + mu] = sv;
            Hm[(long long)mu * n + nu2] = hv;
            Hm[(long long)nu2 * n + mu] = hv;
          }
        }
        aoB += nv;
      }
      aoA += 2 * la + 1;
    }
  }
}

// Hybrid orbital projection of an n-mer's cut-bond atoms (HOP section):
// V^HOP = sum over projected atoms A of S[:, A] D_A S[A, :] with
// D = V h h^T on a bond-detachment atom (BDA) whose attachment atom (BAA) is
// outside the n-mer, D = V (1_sp - h h^T) on a ghost, h = c_s s + c_p (b . p)
// (c_s = 1/2, c_p = sqrt(3)/2), b the unit vector from the BDA to the BAA.
// One block per n-mer; local AOs in the order of build_maps.
// With Qd non-null also the factors V = Q^T D Q of the n-mer (idx = its
// block index): Q rows = the S rows of the projected s/p functions
// (kHopCols x n per n-mer at offset kHopCols * nm.aov, FP64 in Qd and FP32 in
// Qf), D = the 4 x 4 blocks on the diagonal (kHopCols^2 per n-mer, FP64 in
// Dd, FP32 in Df), nq[idx] = the number of rows used (4 per projected atom).
__global__ void hop_projector_kernel(const Nmer* __restrict__ nmers, FragTab ft, const double* __restrict__ xyz,
                                     const int* __restrict__ elem, const DevElem* __restrict__ el, double v_hop,
                                     const double* __restrict__ S, double* __restrict__ V,
                                     double* __restrict__ Qd, float* __restrict__ Qf, double* __restrict__ Dd,
                                     float* __restrict__ Df, int* __restrict__ nq) {
  const Nmer nm = nmers[blockIdx.x];
  __shared__ int s_np;
  __shared__ int s_idx[kMaxProjected][4];
  __shared__ double s_D[kMaxProjected][16];
  if (threadIdx.x == 0) {
    int np = 0, lao = 0;
    for (int kf = 0; kf < nm.nfrag; ++kf) {
      const int f = nm.frag[kf];
      for (int i = 0; i < ft.nat[f]; ++i) {
        const int ga = ft.atom0[f] + i;
        if (!atom_in_nmer(ft, nm.nfrag, nm.frag, ga)) continue;
        const DevElem& e = el[elem[ga]];
        int kind = 0;   // 1: detached BDA, 2: ghost
        if (ft.ghost_frag[ga] >= 0) kind = 2;
        else if (ft.bda_baa_frag[ga] >= 0 && !frag_in_nmer(nm.nfrag, nm.frag, ft.bda_baa_frag[ga])) kind = 1;
        if (kind && np < kMaxProjected) {
          int ao = lao, is = -1, ip = -1;
          for (int k = 0; k < e.nsh; ++k) {
            if (e.l[k] == 0 && is < 0) is = ao;
            if (e.l[k] == 1 && ip < 0) ip = ao;
            ao += 2 * e.l[k] + 1;
          }
          const int baa = ft.hop_baa[ga];
          double b[3] = {xyz[3 * baa] - xyz[3 * ga], xyz[3 * baa + 1] - xyz[3 * ga + 1],
                         xyz[3 * baa + 2] - xyz[3 * ga + 2]};
          const double inv = 1.0 / sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
          const double cp = 0.5 * sqrt(3.0);
          const double h[4] = {0.5, cp * b[0] * inv, cp * b[1] * inv, cp * b[2] * inv};
          for (int a = 0; a < 4; ++a)
            for (int c = 0; c < 4; ++c)
              s_D[np][4 * a + c] = v_hop * (kind == 1 ? h[a] * h[c] : (a == c ? 1.0 : 0.0) - h[a] * h[c]);
          s_idx[np][0] = is;
          s_idx[np][1] = ip;
          s_idx[np][2] = ip + 1;
          s_idx[np][3] = ip + 2;
          ++np;
        }
        for (int k = 0; k < e.nsh; ++k) lao += 2 * e.l[k] + 1;
      }
    }
    s_np = np;
  }
  __syncthreads();
  const int n = nm.n, np = s_np;
  const double* Sm = S + nm.mat;
  double* Vm = V + nm.mat;
  if (Qd) {
    const long long qo = (long long)kHopCols * nm.aov, dof = (long long)blockIdx.x * kHopCols * kHopCols;
    for (int e = threadIdx.x; e < 4 * np * n; e += blockDim.x) {
      const int r = e / n, j = e - r * n;
      const double v = Sm[(long long)s_idx[r / 4][r % 4] * n + j];
      Qd[qo + e] = v;
      Qf[qo + e] = float(v);
    }
    for (int e = threadIdx.x; e < kHopCols * kHopCols; e += blockDim.x) {
      const int r = e / kHopCols, c = e - r * kHopCols;
      const double v = (r / 4 == c / 4 && r / 4 < np) ? s_D[r / 4][4 * (r % 4) + (c % 4)] : 0.0;
      Dd[dof + e] = v;
      Df[dof + e] = float(v);
    }
    if (threadIdx.x == 0) nq[blockIdx.x] = 4 * np;
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e - i * n;
    double v = 0.0;
    for (int k = 0; k < np; ++k) {
      for (int a = 0; a < 4; ++a) {
        const double si = Sm[(long long)i * n + s_idx[k][a]];
        double t = 0.0;
        for (int c = 0; c < 4; ++c) t += s_D[k][4 * a + c] * Sm[(long long)s_idx[k][c] * n + j];
        v += si * t;
      }
    }
    Vm[e] = v;
  }
}

// x^(-1/2) in FP64 from the FP32 hardware estimate y0 and one third-order
// correction: with r = 1 - x y0^2 (|r| ~ 1e-7; y0^2 is exact in FP64),
// y = y0 (1 + r/2 + 3r^2/8) has relative error O(r^3), below FP64 rounding.
// x must be a positive normal FP32 number.
__device__ __forceinline__ double rsqrt_fp64(double x) {
  const double y0 = (double)rsqrtf((float)x);
  const double r = fma(-x, y0 * y0, 1.0);
  return fma(y0 * r, fma(0.375, r, 0.5), y0);
}

// gamma of Eqs. 4-5 from the distance and the two shell hardnesses.
__device__ __forceinline__ double gamma_fn(double r2, double inv_eta_a, double inv_eta_b, double kg) {
  const double ie = 0.5 * (inv_eta_a + inv_eta_b);   // 1/eta, eta = harmonic mean
  if (kg == 2.0) return rsqrt_fp64(r2 + ie * ie);
  return pow(pow(sqrt(r2), kg) + pow(ie, kg), -1.0 / kg);
}

// Shell-resolved gamma block of an n-mer.
__global__ void gamma_kernel(const Nmer* __restrict__ nmers, FragTab ft, const double* __restrict__ xyz,
                             const int* __restrict__ elem, const int* __restrict__ sh_atom,
                             const double* __restrict__ sh_inv_eta, GParams g,
                             double* __restrict__ gam) {
  const Nmer nm = nmers[blockIdx.y];
  __shared__ int s_sh[1024];
  if (threadIdx.x == 0) {
    int ls = 0;
    for (int k = 0; k < nm.nfrag; ++k) {
      const int f = nm.frag[k];
      for (int i = 0; i < ft.nsh[f]; ++i)
        if (atom_in_nmer(ft, nm.nfrag, nm.frag, sh_atom[ft.sh0[f] + i])) s_sh[ls++] = ft.sh0[f] + i;
    }
  }
  __syncthreads();
  const long long tot = (long long)nm.nsh * nm.nsh;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = int(e / nm.nsh), j = int(e % nm.nsh);
    const int gi = s_sh[i], gj = s_sh[j];
    const int a = sh_atom[gi], b = sh_atom[gj];
    const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                 dz = xyz[3 * a + 2] - xyz[3 * b + 2];
    gam[nm.gam + e] = gamma_fn(dx * dx + dy * dy + dz * dz, sh_inv_eta[gi], sh_inv_eta[gj], g.k_g);
  }
}

// ---------------------------------------------------------------------------
// Loewdin orthogonaliser X = S^{-1/2} of each n-mer, written as the starting
// eigenvector rows CT = X (X is symmetric): coupled Newton-Schulz steps in
// FP32 when a spare n x n buffer W2 is given, else (FP64, or no convergence)
// from a Jacobi eigensolve of S.

template <typename T>
__device__ double max_dev_from_identity(const T* X, int m, int n, double* red, float* out = nullptr);

template <typename T>
__global__ void __launch_bounds__(kBlock) lowdin_kernel(const Nmer* __restrict__ nmers,
                                                        const double* __restrict__ S, T* __restrict__ CT,
                                                        T* __restrict__ W, T* __restrict__ Ag,
                                                        int a_in_smem, double tol, int* __restrict__ status,
                                                        T* __restrict__ W2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Nmer nm = nmers[blockIdx.x];
  const int n = nm.n, npad = nm.npad;
  unsigned char* sp = smem_raw;
  T* A;
  if (a_in_smem) { A = reinterpret_cast<T*>(sp); sp += sizeof(T) * (size_t)npad * npad; }
  else A = Ag + nm.apad;  // global scratch, npad*npad per n-mer
  T* gemm = reinterpret_cast<T*>(sp); sp += sizeof(double) * kGemmSmemElems;   // room for any GEMM variant
  double* red = reinterpret_cast<double*>(sp); sp += sizeof(double) * 32;
  double* scale = reinterpret_cast<double*>(sp); sp += sizeof(double) * npad;
  JacobiScratch<T> js;
  js.p = reinterpret_cast<int*>(sp); sp += sizeof(int) * npad;
  js.q = reinterpret_cast<int*>(sp); sp += sizeof(int) * npad;
  js.act = reinterpret_cast<int*>(sp); sp += sizeof(int) * npad;
  sp = (unsigned char*)(((uintptr_t)sp + 15) & ~uintptr_t(15));
  js.c = reinterpret_cast<T*>(sp); sp += sizeof(T) * npad;
  js.s = reinterpret_cast<T*>(sp); sp += sizeof(T) * npad;

  const double* Sm = S + nm.mat;
  T* CTm = CT + nm.mat;
  T* Wm = W + nm.mat;
  if (W2) {
    // S^-1/2 by the coupled Newton-Schulz iteration (Higham, Functions of
    // Matrices, Sec. 6.3): Y0 = S/c, Z0 = I, T = (3I - Z Y)/2, Y <- Y T,
    // Z <- T Z; Y -> (S/c)^1/2 and Z -> (S/c)^-1/2 while ||I - S/c|| < 1,
    // which c = max row sum of |S| (>= the largest eigenvalue) ensures.
    // Three GEMMs per step, ~10 steps for the condition numbers of these
    // bases, against a full Jacobi eigen-solve.  Ends at FP32 rounding (the
    // residual max |ZY - I| stops halving); the SCC's cold start restores
    // S-orthonormality of the rows to FP32 anyway.  Not converged: Jacobi.
    double rs = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double t = 0.0;
      for (int j = 0; j < n; ++j) t += fabs(Sm[(long long)i * n + j]);
      rs = fmax(rs, t);
    }
    const double c = block_max(rs, red);
    T* Y = Wm;
    T* Z = CTm;
    T* X = W2 + nm.mat;   // spare
    T* P = A;             // n x n, leading dimension n
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      Y[e] = T(Sm[e] / c);
      Z[e] = T((e / n) == (e % n) ? 1.0 : 0.0);
    }
    __syncthreads();
    double prev = 1e30, err = 1e30;
    for (int it = 0; it < 60; ++it) {
      block_gemm<T>(n, n, n, Z, n, 1, Y, 1, n, P, n, nullptr, nullptr, nullptr, gemm);   // Z Y
      err = max_dev_from_identity(P, n, n, red);
      if (err < 1e-6 || (err < 1e-3 && err > 0.5 * prev)) break;
      prev = err;
      for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        P[e] = T((e / n) == (e % n) ? 1.5 : 0.0) - T(0.5) * P[e];
      __syncthreads();
      block_gemm<T>(n, n, n, Y, n, 1, P, 1, n, X, n, nullptr, nullptr, nullptr, gemm);   // Y T
      T* t = Y; Y = X; X = t;
      block_gemm<T>(n, n, n, P, n, 1, Z, 1, n, X, n, nullptr, nullptr, nullptr, gemm);   // T Z
      t = Z; Z = X; X = t;
    }
    if (err < 1e-3) {
      const T f = T(1.0 / sqrt(c));
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) CTm[e] = Z[e] * f;   // Z may be CTm itself
      __syncthreads();
      return;
    }
  }
  for (int e = threadIdx.x; e < npad * npad; e += blockDim.x) {
    const int i = e / npad, j = e % npad;
    A[e] = (i < n && j < n) ? T(Sm[(long long)i * n + j]) : T(0);
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) CTm[e] = T((e / n) == (e % n) ? 1.0 : 0.0);
  __syncthreads();
  const int sw = block_jacobi<T>(A, npad, n, CTm, n, n, tol, 60, js, red);
  if (sw < 0 && threadIdx.x == 0) status[blockIdx.x] = FMO_SCC_JACOBI_CODE;
  for (int i = threadIdx.x; i < n; i += blockDim.x) scale[i] = 1.0 / sqrt(double(A[i * npad + i]));
  __syncthreads();
  // X = V diag(s^-1/2) V^T with V^T = CT rows
  block_gemm<T>(n, n, n, CTm, 1, n, CTm, 1, n, Wm, n, nullptr, nullptr, scale, gemm);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) CTm[e] = Wm[e];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Warm start of an n-mer from its monomers' final eigenvector rows: the
// block-diagonal C_I (+) C_J (+) C_K in the n-mer's AO order (fragments in
// the n-mer's order).  These rows are S-orthonormal within each fragment but
// not across fragments; the SCC kernel restores that by Newton-Schulz
// steps before its first iteration.

__global__ void warm_start_kernel(const Nmer* __restrict__ nmers, const Nmer* __restrict__ mono,
                                  const float* __restrict__ mono_ct, float* __restrict__ ct) {
  const Nmer nm = nmers[blockIdx.x];
  const int n = nm.n;
  int off[4] = {0, n, n, n};
  for (int k = 0; k < nm.nfrag; ++k) off[k + 1] = off[k] + mono[nm.frag[k]].n;
  float* C = ct + nm.mat;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = wid; r < n; r += nw) {
    const int kr = (r >= off[1]) + (r >= off[2]);
    const Nmer& m = mono[nm.frag[kr]];
    const long long row0 = m.mat + (long long)(r - off[kr]) * m.n;
    for (int c = lane; c < n; c += 32) {
      const int kc = (c >= off[1]) + (c >= off[2]);
      C[(long long)r * n + c] = (kr == kc) ? mono_ct[row0 + (c - off[kr])] : 0.f;
    }
  }
}

// ---------------------------------------------------------------------------
// Persistent batched SCC kernel: one block per n-mer iterates the SCC loop of
// Eqs. 2-7 to self-consistency in its embedding potential (Eqs. 20-21).

struct SccArgs {
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
  const double* phi;       // supersystem potential sum_lambda gamma dq_mono (or null)
  const double* vhop;      // per-n-mer hybrid orbital projector V^HOP (n x n, or null)
  // its factors V = Q^T D Q (hop_projector_kernel; null: not used): mixed
  // precision keeps the 1e6 Eh projector out of the low-precision products
  const double* hop_Qd;
  const float* hop_Qf;
  const double* hop_Dd;
  const float* hop_Df;
  const int* hop_nq;
  const double* dq_mono;   // monomer charges, global shell order
  double* esp;             // out: the n-mer's embedding potential
  double* dq;              // in: guess (if !guess_from_mono), out: charges
  double* eps;             // out: orbital energies
  double* hist;            // Broyden history scratch
  double* energy;          // out per n-mer (index = n-mer index)
  double* e_el;
  double* e_rep;
  double* dEV;
  int* iters;
  int* iters32;
  int* status;
  int guess_from_mono;
  int precision;
  int max_iter;
  int fp32_cap;
  int single_step;   // 1: exactly one SCC iteration, no mixing (global monomer loop)
  int step_phase;    // single step: 0 FP32, 1 FP64
  int reortho;       // single step: carry the FP32 vectors over to FP64 first
  int cold_refine;   // the vectors are the Loewdin start: restore S-orthonormality in FP64 first
  int reortho32;     // single step: one FP32 Newton-Schulz step before the iteration
  const int* step_dev;   // if set: reortho32 from the device step count (graph-launched FP32 steps)
  double jac_hint;   // SCC residual before this launch (sets the first Jacobi threshold)
  const double* jac_hint_dev;   // if set: read jac_hint from the device (graph-launched steps)
  const float* S32;  // mixed precision: S and H0 rounded to FP32 (the FP32 iterations read these)
  const float* H32;
  int fp64_finish;   // mixed: stop after this many FP64 iterations (0: converge in FP64)
  int energy_finish; // mixed n-mers: end with the FP64 energy of the FP32-converged density
  int cold_steps;    // Newton-Schulz steps allowed for the cold start (far from orthonormal: more)
  int first_rot;     // the first iteration may use the rotation update (warm rows)
  double first_jac_tol;  // > 0: Jacobi threshold of the first FP32 iteration (warm rows)
  double* trace;     // optional: residual per iteration of the first n-mer in the order
  double tol, etol, switch_tol;
  double jacobi_tol_d, jacobi_tol_f;
  const unsigned long long* t0;
  unsigned long long budget_ns;
  int a_smem_d, a_smem_f;
  int max_n, max_nsh, max_nat;
  // > 0: shared-memory floats for packed rows of the tridiagonal eigen-solver
  // (FP32 iterations of n-mers whose matrix is in global memory)
  int tri_cap;
};

// Shared-memory layout of the SCC kernel (sizes from the launch maxima).
struct SccSmem {
  void* A;
  void* gemm;
  double* red;
  double* sig;
  float* sig32;  // FP32 copy of sig for the FP32 Fock build
  double* dqin;
  double* dqout;
  double* esp;
  double* q0;
  double* dqat;
  double* g3;
  double* eps;
  double* focc;
  int* occ;
  int* virt;     // rows with zero occupation (orbital-rotation updates)
  int* misc;     // [0] number of virt rows, [1] rotation update allowed, [2] rows to rotate, [3] trace
  double* bro;   // Broyden small matrix (kHist*kHist + 2*kHist)
  NmerMaps mp;
  int* jsp;
  int* jsq;
  int* jsact;
  void* jsc;
  void* jss;
  float* tri;    // tridiagonal eigen-solver work (after the regular layout; null if none)
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t scc_smem_bytes(int max_n, int max_nsh, int max_nat, int a_bytes) {
  const int npad = max_n + (max_n & 1);
  size_t b = 0;
  b += align16((size_t)a_bytes);
  b += align16(sizeof(double) * kGemmSmemElems);
  b += align16(sizeof(double) * 32);
  b += 7 * align16(sizeof(double) * max_nsh);          // sig dqin dqout esp q0 + spare
  b += 2 * align16(sizeof(double) * max_nat);          // dqat g3
  b += 2 * align16(sizeof(double) * npad);             // eps focc
  b += align16(sizeof(int) * npad);                    // occ
  b += align16(sizeof(int) * npad);                    // virt
  b += align16(sizeof(int) * 4);                       // misc
  b += align16(sizeof(double) * (kHist * kHist + 4 * kHist + 8));
  b += align16(sizeof(int16_t) * npad);                // ao_sh
  b += align16(sizeof(int16_t) * max_nsh);             // sh_at
  b += align16(sizeof(int) * max_nat);                 // at_glob
  b += align16(sizeof(int) * max_nsh);                 // sh_glob
  b += align16(sizeof(int16_t) * (max_nsh + 1));       // sh_ao0
  b += 3 * align16(sizeof(int) * npad);                // js p q act
  b += 2 * align16(sizeof(double) * npad);             // js c s
  return b;
}

// gamma between shell k_b of atom b and a shell (1/eta = ie_a) of atom a
__device__ __forceinline__ double shell_gamma(const SccArgs& ar, int a, double ie_a, int b, int k_b) {
  const double dx = ar.xyz[3 * a] - ar.xyz[3 * b], dy = ar.xyz[3 * a + 1] - ar.xyz[3 * b + 1],
               dz = ar.xyz[3 * a + 2] - ar.xyz[3 * b + 2];
  return gamma_fn(dx * dx + dy * dy + dz * dz, ie_a, 1.0 / ar.el[ar.elem[b]].eta_sh[k_b], ar.g.k_g);
}

__device__ SccSmem carve_scc_smem(unsigned char* base, int max_n, int max_nsh, int max_nat, int a_bytes) {
  const int npad = max_n + (max_n & 1);
  SccSmem s;
  unsigned char* p = base;
  auto take = [&](size_t bytes) { unsigned char* r = p; p += align16(bytes); return (void*)r; };
  s.A = take(a_bytes);
  s.gemm = take(sizeof(double) * kGemmSmemElems);
  s.red = (double*)take(sizeof(double) * 32);
  s.sig = (double*)take(sizeof(double) * max_nsh);
  s.dqin = (double*)take(sizeof(double) * max_nsh);
  s.dqout = (double*)take(sizeof(double) * max_nsh);
  s.esp = (double*)take(sizeof(double) * max_nsh);
  s.q0 = (double*)take(sizeof(double) * max_nsh);
  s.sig32 = (float*)take(sizeof(double) * max_nsh);
  take(sizeof(double) * max_nsh);
  s.dqat = (double*)take(sizeof(double) * max_nat);
  s.g3 = (double*)take(sizeof(double) * max_nat);
  s.eps = (double*)take(sizeof(double) * npad);
  s.focc = (double*)take(sizeof(double) * npad);
  s.occ = (int*)take(sizeof(int) * npad);
  s.virt = (int*)take(sizeof(int) * npad);
  s.misc = (int*)take(sizeof(int) * 4);
  s.bro = (double*)take(sizeof(double) * (kHist * kHist + 4 * kHist + 8));
  s.mp.ao_sh = (int16_t*)take(sizeof(int16_t) * npad);
  s.mp.sh_at = (int16_t*)take(sizeof(int16_t) * max_nsh);
  s.mp.at_glob = (int*)take(sizeof(int) * max_nat);
  s.mp.sh_glob = (int*)take(sizeof(int) * max_nsh);
  s.mp.sh_ao0 = (int16_t*)take(sizeof(int16_t) * (max_nsh + 1));
  s.jsp = (int*)take(sizeof(int) * npad);
  s.jsq = (int*)take(sizeof(int) * npad);
  s.jsact = (int*)take(sizeof(int) * npad);
  s.jsc = take(sizeof(double) * npad);
  s.jss = take(sizeof(double) * npad);
  return s;
}

// Fermi occupations of Eq. 6 (closed shell: f_i = 2 / (exp((eps_i - eF)/kT)
// + 1)) for the orbital energies sm.eps, eF by bisection on sum_i f_i = N
// (warp 0), and -TS of Eq. 2.  T is the working precision of the SCC
// iteration: the FP32 phase needs its occupations only to FP32 accuracy
// (the bisection stops at |sum f - N| < 1e-6 there, 1e-13 in FP64); with a
// gap wider than 40 kT eF is then set from the balance of the Boltzmann tails.
// Lists (ascending orbital index, built with warp ballots): occ = rows that
// enter the density (f > 1e-30), the occupied ones (f > 1) first; virt =
// rows with f <= 1.  misc[0] = |virt|, misc[2] = number of rows with f > 1,
// misc[1] = 1 iff every occupation is 2 or 0 to within 1e-6 (FP32) or 1e-10
// (FP64) (the orbital-rotation update is allowed).  Returns -TS; *n_occ_out = |occ|.
template <typename T>
__device__ double fermi_step(int n, double nel, double kT, SccSmem& sm, int* n_occ_out) {
  __shared__ double s_mts;
  __shared__ int s_nocc;
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double lo = 1e300, hi = -1e300;
    for (int i = lane; i < n; i += 32) { lo = fmin(lo, sm.eps[i]); hi = fmax(hi, sm.eps[i]); }
    lo = -warp_max(-lo);
    hi = warp_max(hi);
    lo -= 50.0 * kT + 1.0;
    hi += 50.0 * kT + 1.0;
    const T ikT = T(1.0 / kT);
    const T xmax = T(sizeof(T) == 8 ? 700.0 : 80.0);
    const double ntol = sizeof(T) == 8 ? 1e-13 : 1e-6;
    double ef = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
      ef = 0.5 * (lo + hi);
      T tot = T(0);
      for (int i = lane; i < n; i += 32) {
        const T x = fmin(fmax(T(sm.eps[i] - ef) * ikT, -xmax), xmax);
        tot += T(2) / (exp(x) + T(1));
      }
      const double tsum = warp_sum(double(tot));
      if (fabs(tsum - nel) < ntol || hi - lo < 1e-15) break;
      if (tsum > nel) hi = ef; else lo = ef;
    }
    {
      // a gap much wider than kT with exactly N/2 levels below eF: the
      // bisection stops anywhere in the gap once |sum f - N| is small
      // enough.  There the root of sum f = N balances the Boltzmann tails
      // (holes 2 exp((e_i - eF)/kT) below, electrons 2 exp((eF - e_a)/kT)
      // above): eF = (elo + ehi)/2 + kT/2 ln(S_h / S_e) with
      // S_h = sum_i exp((e_i - elo)/kT), S_e = sum_a exp((ehi - e_a)/kT),
      // exact to a relative exp(-gap/2kT) in each tail.
      double elo = -1e300, ehi = 1e300;
      int cnt = 0;
      for (int i = lane; i < n; i += 32) {
        const double e = sm.eps[i];
        if (e <= ef) { elo = fmax(elo, e); ++cnt; } else { ehi = fmin(ehi, e); }
      }
      elo = warp_max(elo);
      ehi = -warp_max(-ehi);
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      if (fabs(2.0 * cnt - nel) < 1e-9 && ehi - elo > 40.0 * kT) {
        T sh = T(0), se = T(0);
        for (int i = lane; i < n; i += 32) {
          const double e = sm.eps[i];
          if (e <= elo) sh += exp(fmax(T((e - elo) / kT), -xmax));
          else se += exp(fmax(T((ehi - e) / kT), -xmax));
        }
        const double shs = warp_sum(double(sh)), ses = warp_sum(double(se));
        ef = 0.5 * (elo + ehi) + 0.5 * kT * (log(shs) - log(ses));
      }
    }
    T mts = T(0);
    double fo_min = 2.0, fv_max = 0.0;
    for (int i = lane; i < n; i += 32) {
      const T x = fmin(fmax(T(sm.eps[i] - ef) * ikT, -xmax), xmax);
      const T f = T(2) / (exp(x) + T(1));
      sm.focc[i] = double(f);
      const T h = T(0.5) * f;
      T t = T(0);
      if (h > T(1e-30)) t += h * log(h);
      if (T(1) - h > T(1e-30)) t += (T(1) - h) * log(T(1) - h);
      mts += t;
      if (f > T(1)) fo_min = fmin(fo_min, double(f)); else fv_max = fmax(fv_max, double(f));
    }
    const double mts_sum = warp_sum(double(mts));
    fo_min = -warp_max(-fo_min);
    fv_max = warp_max(fv_max);
    __syncwarp();
    int k = 0, v = 0;
    const unsigned below = (1u << lane) - 1u;
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      const double f = (i < n) ? sm.focc[i] : 0.0;
      const bool po = (i < n) && f > 1.0;
      const bool pv = (i < n) && !(f > 1.0);
      const unsigned bo = __ballot_sync(0xffffffffu, po), bv = __ballot_sync(0xffffffffu, pv);
      if (po) sm.occ[k + __popc(bo & below)] = i;
      if (pv) sm.virt[v + __popc(bv & below)] = i;
      k += __popc(bo);
      v += __popc(bv);
    }
    const int nro = k;
    for (int base = 0; base < n; base += 32) {
      const int i = base + lane;
      const double f = (i < n) ? sm.focc[i] : 0.0;
      const bool pt = (i < n) && f <= 1.0 && f > 1e-30;
      const unsigned bt = __ballot_sync(0xffffffffu, pt);
      if (pt) sm.occ[k + __popc(bt & below)] = i;
      k += __popc(bt);
    }
    if (lane == 0) {
      s_mts = 2.0 * kT * mts_sum;
      s_nocc = k;
      sm.misc[0] = v;
      // tails below ftol (1e-6 in FP32, 1e-10 in FP64) count as integer:
      // the virtual block is not re-diagonalised by the rotation update, so
      // a tail occupation f enters the density only through f times the
      // small residual virtual-virtual rotation
      const double ftol = sizeof(T) == 8 ? 1e-10 : 1e-6;
      sm.misc[1] = (nro > 0 && v > 0 && fo_min > 2.0 - ftol && fv_max < ftol) ? 1 : 0;
      sm.misc[2] = nro;
    }
  }
  __syncthreads();
  *n_occ_out = s_nocc;
  return s_mts;
}

// Modified Broyden mixing (Johnson 1988) of the shell-charge vector, FP64.
// x_new = x_in + a F - sum_n g_n u_n, F = x_out - x_in, dF/dx normalised
// differences, u = a dF + dx, (w0^2 I + dF dF^T) g = dF F.
// With secant = false the step uses the stored history but adds no new pair:
// the first step after the FP32 -> FP64 hand-over, whose residual difference
// would mix the two precisions' slightly different fixed points.
__device__ void broyden_step(int nsh, int it, double* hist, SccSmem& sm, int& hcount, int& hhead,
                             double alpha, double w0, bool secant = true) {
  double* dF = hist;                          // [kHist][nsh]
  double* U = hist + (size_t)kHist * nsh;     // [kHist][nsh]
  double* px = hist + (size_t)2 * kHist * nsh;
  double* pF = px + nsh;
  double* red = sm.red;
  __shared__ double s_norm;
  if (it > 1 && secant) {
    double nn = 0.0;
    for (int i = threadIdx.x; i < nsh; i += blockDim.x) {
      const double F = sm.dqout[i] - sm.dqin[i];
      const double d = F - pF[i];
      nn += d * d;
    }
    nn = block_sum(nn, red);
    if (threadIdx.x == 0) s_norm = sqrt(nn);
    __syncthreads();
    const double norm = s_norm;
    if (norm > 0.0) {
      const int slot = (hhead + hcount) % kHist;
      for (int i = threadIdx.x; i < nsh; i += blockDim.x) {
        const double F = sm.dqout[i] - sm.dqin[i];
        const double d = (F - pF[i]) / norm;
        const double dx = (sm.dqin[i] - px[i]) / norm;
        dF[(size_t)slot * nsh + i] = d;
        U[(size_t)slot * nsh + i] = alpha * d + dx;
      }
      if (hcount < kHist) ++hcount; else hhead = (hhead + 1) % kHist;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nsh; i += blockDim.x) {
    px[i] = sm.dqin[i];
    pF[i] = sm.dqout[i] - sm.dqin[i];
  }
  __syncthreads();
  const int m = hcount;
  double* a = sm.bro;                 // m x m
  double* c = sm.bro + kHist * kHist; // m
  double* gv = c + kHist;             // m
  if (m > 0) {
    // a_kn = dF_k . dF_n, c_k = dF_k . F  (one warp per entry)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int e = wid; e < m * m + m; e += nw) {
      double s = 0.0;
      if (e < m * m) {
        const int k = (hhead + e / m) % kHist, l = (hhead + e % m) % kHist;
        for (int i = lane; i < nsh; i += 32) s += dF[(size_t)k * nsh + i] * dF[(size_t)l * nsh + i];
      } else {
        const int k = (hhead + (e - m * m)) % kHist;
        for (int i = lane; i < nsh; i += 32) s += dF[(size_t)k * nsh + i] * pF[i];
      }
      s = warp_sum(s);
      if (lane == 0) { if (e < m * m) a[e] = s; else c[e - m * m] = s; }
    }
    __syncthreads();
    // solve (w0^2 I + a) g = c, Gaussian elimination with partial pivoting
    if (threadIdx.x < 32) warp_gj_solve(m, a, c, w0 * w0, gv);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < nsh; i += blockDim.x) {
    const double F = sm.dqout[i] - sm.dqin[i];
    double x = sm.dqin[i] + alpha * F;
    for (int k = 0; k < m; ++k) x -= gv[k] * U[(size_t)((hhead + k) % kHist) * nsh + i];
    sm.dqin[i] = x;
  }
  __syncthreads();
}

// Energy of Eq. 2 without the -TS term from the output shell charges
// sm.dqout and the per-shell band energies sm.sig (sum_mu in shell P_mu,nu
// H0_nu,mu); also max |dq_out - dq_in| (into *diff_out).
__device__ double energy_of_output(const Nmer& nm, const SccArgs& ar, SccSmem& sm, double* diff_out) {
  const int nsh = nm.nsh, nat = nm.nat;
  const double* G = ar.gam + nm.gam;
  for (int a = threadIdx.x; a < nat; a += blockDim.x) sm.dqat[a] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < nsh; ++s) sm.dqat[sm.mp.sh_at[s]] += sm.dqout[s];
  }
  __syncthreads();
  double part = 0.0, dmax = 0.0;
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double v = 0.0;
      for (int t = lane; t < nsh; t += 32) v += G[(size_t)s * nsh + t] * sm.dqout[t];
      v = warp_sum(v);
      if (lane == 0) {
        part += sm.sig[s] + 0.5 * sm.dqout[s] * v;
        dmax = nan_max(dmax, fabs(sm.dqout[s] - sm.dqin[s]));
      }
    }
  }
  for (int a = threadIdx.x; a < nat; a += blockDim.x)
    part -= sm.g3[a] * sm.dqat[a] * sm.dqat[a] * sm.dqat[a] / 3.0;
  const double e_sum = block_sum(part, sm.red);
  *diff_out = block_max(dmax, sm.red);
  return e_sum;
}

template <typename T>
struct PrecPtrs {
  T* CT;
  T* W1;
  T* W2;
  T* A;
  int lda;
};

// 1/d in precision T: FP32 division, or for FP64 the FP32 reciprocal
// refined by one Newton step r <- r (2 - d r) (relative error ~1e-7 -> ~1e-14).
template <typename T>
__device__ __forceinline__ T recip(double d);
template <>
__device__ __forceinline__ float recip<float>(double d) { return 1.0f / float(d); }
template <>
__device__ __forceinline__ double recip<double>(double d) {
  const double r = double(1.0f / float(d));
  return r * (2.0 - d * r);
}

// max |X - I| over an m x n row-major matrix (a warp per row); optionally
// stores X - I in FP32 into out.  Block-uniform result.
template <typename T>
__device__ double max_dev_from_identity(const T* X, int m, int n, double* red, float* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double err = 0.0;
  for (int i = wid; i < m; i += nw) {
    const T* row = X + (long long)i * n;
    for (int j = lane; j < n; j += 32) {
      const double d = double(row[j]) - (i == j ? 1.0 : 0.0);
      if (out) out[(long long)i * n + j] = float(d);
      err = fmax(err, fabs(d));
    }
  }
  return block_max(err, red);
}

// One SCC iteration in precision T.  Returns E_el; writes dq_out, eps.
// Rotation of the rows CT (type T) by the generator K (n_o x n_v, type TG,
// stored at Kg): C_o += K C_v - 1/2 K K^T C_o, C_v += -K^T C_o - 1/2 K^T K C_v
// with the products formed in precision TG on the TG copy src of the rows.
// w1: n x n, w2 after K: n_o x n, yv: n_v x n (all TG).
template <typename T, typename TG>
__device__ void rotate_rows(int n, int no, int nv, const int* occ, const int* virt, T* CT, const TG* src,
                            const TG* Kg, TG* w1, TG* w2, TG* yv, TG* gemm) {
  TG* dCo = w1;                               // no x n : K C_v
  TG* Dv = w1 + (long long)no * n;            // nv x n : K^T C_o
  TG* Yo = w2;                                // no x n : K Dv
  block_gemm<TG>(no, n, nv, Kg, nv, 1, src, 1, n, dCo, n, nullptr, virt, nullptr, gemm);
  block_gemm<TG>(nv, n, no, Kg, 1, nv, src, 1, n, Dv, n, nullptr, occ, nullptr, gemm);
  block_gemm<TG>(no, n, nv, Kg, nv, 1, Dv, 1, n, Yo, n, nullptr, nullptr, nullptr, gemm);
  block_gemm<TG>(nv, n, no, Kg, 1, nv, dCo, 1, n, yv, n, nullptr, nullptr, nullptr, gemm);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = wid; i < no; i += nw) {
    T* row = CT + (long long)occ[i] * n;
    const TG* d = dCo + (long long)i * n;
    const TG* y = Yo + (long long)i * n;
    for (int j = lane; j < n; j += 32) row[j] = row[j] + T(d[j] - TG(0.5) * y[j]);
  }
  for (int a = wid; a < nv; a += nw) {
    T* row = CT + (long long)virt[a] * n;
    const TG* d = Dv + (long long)a * n;
    const TG* y = yv + (long long)a * n;
    for (int j = lane; j < n; j += 32) row[j] = row[j] - T(d[j] + TG(0.5) * y[j]);
  }
  __syncthreads();
}

template <typename T>
__device__ double scc_iteration(const Nmer& nm, const SccArgs& ar, SccSmem& sm, PrecPtrs<T> pp,
                                double jac_tol, int* jac_fail, double* diff_out, bool allow_rot,
                                float* f_ct = nullptr, float* f_w1 = nullptr, float* f_w2 = nullptr) {
  const int n = nm.n, nsh = nm.nsh, nat = nm.nat, npad = nm.npad;
  const double* Sm = ar.S + nm.mat;
  const double* Hm = ar.H0 + nm.mat;
  const double* G = ar.gam + nm.gam;
  // diagnostic trace: SM cycles per part of the iteration, summed over the
  // iterations of the first block (thread 0 reads the clock after a barrier)
  const bool tr = ar.trace && blockIdx.x == 0 && threadIdx.x == 0;
  long long tmark = tr ? clock64() : 0;
  auto mark = [&](int j) {
    if (tr) { const long long t = clock64(); ar.trace[kTraceParts + j] += double(t - tmark); tmark = t; }
  };
  // atomic charges and shell shifts (Eq. 7 and the ESP of Eq. 21)
  for (int a = threadIdx.x; a < nat; a += blockDim.x) sm.dqat[a] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int s = 0; s < nsh; ++s) sm.dqat[sm.mp.sh_at[s]] += sm.dqin[s];
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double v = 0.0;
      for (int t = lane; t < nsh; t += 32) v += G[(size_t)s * nsh + t] * sm.dqin[t];
      v = warp_sum(v);
      if (lane == 0) {
        const int a = sm.mp.sh_at[s];
        const double sg = v - sm.g3[a] * sm.dqat[a] * sm.dqat[a] + sm.esp[s];
        sm.sig[s] = sg;
        if constexpr (sizeof(T) == 4) sm.sig32[s] = float(sg);
      }
    }
  }
  __syncthreads();
  // Fock matrix F = H0 + 1/2 S (sig_mu + sig_nu), into W1 (a warp per row)
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // hybrid orbital projectors, if any (with their factors given they are
    // added in the MO basis after the transform instead)
    const double* Vm = (ar.vhop && !ar.hop_Qd) ? ar.vhop + nm.mat : nullptr;
    if constexpr (sizeof(T) == 4) {
      // FP32 iteration: built in FP32 from the FP32 copies of H0 and S (the
      // result is rounded to FP32 anyway; no FP64 work per element)
      const float* H32 = ar.H32 + nm.mat;
      const float* S32 = ar.S32 + nm.mat;
      for (int i = wid; i < n; i += nw) {
        const float si = sm.sig32[sm.mp.ao_sh[i]];
        const float* hr = H32 + (long long)i * n;
        const float* sr = S32 + (long long)i * n;
        T* fr = pp.W1 + (long long)i * n;
        for (int j = lane; j < n; j += 32) fr[j] = fmaf(0.5f * sr[j], si + sm.sig32[sm.mp.ao_sh[j]], hr[j]);
      }
    } else for (int i = wid; i < n; i += nw) {
      const double si = sm.sig[sm.mp.ao_sh[i]];
      const double* hr = Hm + (long long)i * n;
      const double* sr = Sm + (long long)i * n;
      T* fr = pp.W1 + (long long)i * n;
      if (Vm) {
        const double* vr = Vm + (long long)i * n;
        for (int j = lane; j < n; j += 32) fr[j] = T(hr[j] + 0.5 * sr[j] * (si + sm.sig[sm.mp.ao_sh[j]]) + vr[j]);
      } else {
        for (int j = lane; j < n; j += 32) fr[j] = T(hr[j] + 0.5 * sr[j] * (si + sm.sig[sm.mp.ao_sh[j]]));
      }
    }
  }
  // zero the padding row/column of A
  if (n != npad) {
    for (int i = threadIdx.x; i < npad; i += blockDim.x) {
      pp.A[(long long)i * pp.lda + n] = T(0);
      pp.A[(long long)n * pp.lda + i] = T(0);
    }
  }
  __syncthreads();
  T* gemm = reinterpret_cast<T*>(sm.gemm);
  mark(0);
  // U = CT F  (W2), then A = U CT^T: the Fock matrix in the current MO basis
  if constexpr (sizeof(T) == 8) {
    if (f_ct) {
      // FP64 iteration of a mixed-precision solve: double-float products
      // (FP64-grade, on the FP32 pipe); F is symmetric, so its rows serve as B
      float* gdf = reinterpret_cast<float*>(sm.gemm);
      block_gemm_df<double>(n, n, n, pp.CT, nullptr, n, pp.W1, n, pp.W2, n, gdf);
      block_gemm_df<double>(n, n, n, pp.W2, nullptr, n, pp.CT, n, pp.A, pp.lda, gdf);
    } else {
      block_gemm<T>(n, n, n, pp.CT, n, 1, pp.W1, n, 1, pp.W2, n, nullptr, nullptr, nullptr, gemm);
      block_gemm<T>(n, n, n, pp.W2, n, 1, pp.CT, n, 1, pp.A, pp.lda, nullptr, nullptr, nullptr, gemm);
    }
  } else {
    block_gemm<T>(n, n, n, pp.CT, n, 1, pp.W1, n, 1, pp.W2, n, nullptr, nullptr, nullptr, gemm);
    block_gemm<T>(n, n, n, pp.W2, n, 1, pp.CT, n, 1, pp.A, pp.lda, nullptr, nullptr, nullptr, gemm);
  }
  if (ar.hop_Qd) {
    // A += (CT Q^T) D (CT Q^T)^T: the projector in the MO basis from its
    // factors, Y = CT Q^T (n x nq, in W1), T = Y D (in W2).  FP32 iterations:
    // FP32 products (the projected levels, ~1e6 Eh, sit far above the Fermi
    // level, and the occupied rows have small Y); FP64 iterations: FP64
    // products.  The Fock matrix above was built without the projector.
    const int nb = ar.order[blockIdx.x];
    const int nq = ar.hop_nq[nb];
    if (nq > 0) {
      const long long qo = (long long)kHopCols * nm.aov, dof = (long long)nb * kHopCols * kHopCols;
      T* Y = pp.W1;
      T* Tq = pp.W2;
      if constexpr (sizeof(T) == 4) {
        block_gemm<T>(n, nq, n, pp.CT, n, 1, ar.hop_Qf + qo, n, 1, Y, nq, nullptr, nullptr, nullptr, gemm);
        block_gemm<T>(n, nq, nq, Y, nq, 1, ar.hop_Df + dof, 1, kHopCols, Tq, nq, nullptr, nullptr, nullptr, gemm);
      } else {
        block_gemm<T, double>(n, nq, n, pp.CT, n, 1, ar.hop_Qd + qo, n, 1, Y, nq, nullptr, nullptr, nullptr, gemm);
        block_gemm<T, double>(n, nq, nq, Y, nq, 1, ar.hop_Dd + dof, 1, kHopCols, Tq, nq, nullptr, nullptr, nullptr,
                              gemm);
      }
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int i = wid; i < n; i += nw) {
        for (int j = lane; j < n; j += 32) {
          T acc = T(0);
          for (int c = 0; c < nq; ++c) acc = fma(Tq[(long long)i * nq + c], Y[(long long)j * nq + c], acc);
          pp.A[(long long)i * pp.lda + j] += acc;
        }
      }
      __syncthreads();
    }
  }
  mark(1);
  int nocc = 0;
  double mts = 0.0;
  bool rotated = false;
  if (threadIdx.x == 0) sm.misc[3] = -1;   // -1: rotation step, else Jacobi sweeps
  if (allow_rot) {
    // Warm start: the rows of CT are eigenvectors of the previous Fock
    // matrix, so A is nearly diagonal.  With integer occupations only the
    // occupied-virtual block matters for the density: one second-order
    // rotation C <- (1 + k + k^2/2) C with k_ia = A_ia / (A_ii - A_aa) (i
    // occupied, a empty; first-order perturbation theory) removes it to
    // second order in |A_ia|.  At the SCC
    // fixed point A_ia = 0, so the fixed point is unchanged.
    for (int i = threadIdx.x; i < n; i += blockDim.x) sm.eps[i] = double(pp.A[(long long)i * pp.lda + i]);
    __syncthreads();
    mts = fermi_step<T>(n, nm.nel, ar.g.kT, sm, &nocc);
    if (sm.misc[1]) {
      const int no = sm.misc[2], nv = sm.misc[0];
      T* K = pp.W2;                                 // no x nv
      T kmax_t = T(0);
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int r = wid; r < no; r += nw) {
        const int i = sm.occ[r];
        const double ei = sm.eps[i];
        const T* arow = pp.A + (long long)i * pp.lda;
        T* krow = K + (long long)r * nv;
        for (int c = lane; c < nv; c += 32) {
          const int a = sm.virt[c];
          const T k = arow[a] * recip<T>(ei - sm.eps[a]);
          krow[c] = k;
          kmax_t = fmax(kmax_t, fabs(k));
        }
      }
      const double kmax = block_max(double(kmax_t), sm.red);
      // (1 + k + k^2/2) keeps orthonormality up to k^4/4: rotate only while
      // that stays below the working precision, otherwise diagonalise
      rotated = kmax <= (sizeof(T) == 8 ? 1e-4 : 2e-2);
    }
    mark(2);
    if (rotated) {
      const int no = sm.misc[2], nv = sm.misc[0];
      if (sizeof(T) == 8 && f_ct) {
        // mixed-precision FP64 iteration: the rotation is a small correction
        // (|k| ~ FP32 rounding), so its products run in FP32 on FP32 copies
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) f_ct[e] = float(pp.CT[e]);
        for (long long e = threadIdx.x; e < (long long)no * nv; e += blockDim.x) f_w2[e] = float(pp.W2[e]);
        __syncthreads();
        rotate_rows<T, float>(n, no, nv, sm.occ, sm.virt, pp.CT, f_ct, f_w2, f_w1, f_w2 + (long long)no * nv,
                              reinterpret_cast<float*>(pp.A), reinterpret_cast<float*>(sm.gemm));
      } else {
        rotate_rows<T, T>(n, no, nv, sm.occ, sm.virt, pp.CT, pp.CT, pp.W2, pp.W1, pp.W2 + (long long)no * nv, pp.A,
                          gemm);
      }
    }
  }
  if (!rotated) {
    bool solved = false;
    if constexpr (sizeof(T) == 4) {
      // n-mers of 64 to 512 basis functions: Householder tridiagonalisation
      // with bisection and twisted-factorisation eigenvectors (Jacobi if it
      // reports a failure)
      if (sm.tri && n >= kTriMinN && n <= 512) {
        TriWork tw{sm.tri, ar.tri_cap, reinterpret_cast<float*>(ar.W1d + nm.mat),
                   reinterpret_cast<float*>(ar.W2d + nm.mat)};
        // columns per lane: the smallest multiple of 32 lanes covering n
        if (n <= 128) solved = tri_eigh<4>(pp.A, pp.lda, n, pp.CT, pp.W1, pp.W2, tw, gemm, sm.red, sm.eps);
        else if (n <= 256) solved = tri_eigh<8>(pp.A, pp.lda, n, pp.CT, pp.W1, pp.W2, tw, gemm, sm.red, sm.eps);
        else if (n <= 384) solved = tri_eigh<12>(pp.A, pp.lda, n, pp.CT, pp.W1, pp.W2, tw, gemm, sm.red, sm.eps);
        else solved = tri_eigh<16>(pp.A, pp.lda, n, pp.CT, pp.W1, pp.W2, tw, gemm, sm.red, sm.eps);
        if (solved && threadIdx.x == 0) sm.misc[3] = -2;   // trace: tridiagonal solve
      }
    }
    if (!solved) {
      JacobiScratch<T> js{sm.jsp, sm.jsq, reinterpret_cast<T*>(sm.jsc), reinterpret_cast<T*>(sm.jss), sm.jsact};
      const int sw = block_jacobi<T>(pp.A, pp.lda, n, pp.CT, n, n, jac_tol, 40, js, sm.red);
      if (sw < 0 && sizeof(T) == 8) *jac_fail = 1;
      if (threadIdx.x == 0) sm.misc[3] = sw;   // sweeps (diagnostic trace)
      for (int i = threadIdx.x; i < n; i += blockDim.x) sm.eps[i] = double(pp.A[(long long)i * pp.lda + i]);
    }
    if (ar.trace && threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(ar.trace + kTraceJacobi), 1ULL);
    __syncthreads();
    mts = fermi_step<T>(n, nm.nel, ar.g.kT, sm, &nocc);
  }
  mark(3);
  // compacted occupations
  T* fc = reinterpret_cast<T*>(sm.jsc);   // js scratch is free here (npad doubles)
  for (int k = threadIdx.x; k < nocc; k += blockDim.x) fc[k] = T(sm.focc[sm.occ[k]]);
  __syncthreads();
  // density P = sum_occ f_i c_i c_i^T  (W1)
  block_gemm<T, T, T>(n, n, nocc, pp.CT, 1, n, pp.CT, 1, n, pp.W1, n, sm.occ, sm.occ, fc, gemm);
  mark(4);
  // Mulliken shell populations (Eq. 3) and the band energy sum P H0, one warp per shell
  double eb_local = 0.0;
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double pop = 0.0, eb = 0.0;
      if constexpr (sizeof(T) == 4) {
        // FP32 iteration: per-lane FP32 partial sums (a few rows of n/32
        // terms each) of the FP32 density with the FP32 copies, lanes summed
        // in FP64
        const float* S32 = ar.S32 + nm.mat;
        const float* H32 = ar.H32 + nm.mat;
        float popf = 0.f, ebf = 0.f;
        for (int k = sm.mp.sh_ao0[s]; k < sm.mp.sh_ao0[s + 1]; ++k) {
          for (int j = lane; j < n; j += 32) {
            const float pv = pp.W1[(long long)k * n + j];
            popf = fmaf(pv, S32[(long long)k * n + j], popf);
            ebf = fmaf(pv, H32[(long long)k * n + j], ebf);
          }
        }
        pop = double(popf);
        eb = double(ebf);
      } else {
        for (int k = sm.mp.sh_ao0[s]; k < sm.mp.sh_ao0[s + 1]; ++k) {
          for (int j = lane; j < n; j += 32) {
            const double pv = double(pp.W1[(long long)k * n + j]);
            pop += pv * Sm[(long long)k * n + j];
            eb += pv * Hm[(long long)k * n + j];
          }
        }
      }
      pop = warp_sum(pop);
      eb = warp_sum(eb);
      if (lane == 0) {
        sm.dqout[s] = pop - sm.q0[s];
        sm.sig[s] = eb;   // per-shell band energy (sig is free now)
      }
    }
  }
  __syncthreads();
  (void)eb_local;
  mark(5);
  const double e_out = energy_of_output(nm, ar, sm, diff_out) + mts;
  mark(6);
  return e_out;
}

constexpr bool kCholStart = true;   // Cholesky pass in the warm start of large n-mers

// Dot products of the two passes below: sum_{k < len} x[k] (y0[k sy], y1[k sy])
// with x in shared memory (staged once for the block: every thread uses the
// same x) and y0/y1 per thread in global memory.  Those live in L2 (an
// n-mer's matrices do not fit in L1 beside the kernel's shared memory), so 32
// terms of each are loaded before any is added: one L2 round trip per 32.
__device__ __forceinline__ void chol_dot2(int len, const float* x, const float* y0, const float* y1, long long sy,
                                          float& r0, float& r1) {
  constexpr int kU = 32;
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
  int k = 0;
  for (; k + kU <= len; k += kU) {
    float v0[kU], v1[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      v0[u] = y0[(long long)(k + u) * sy];
      v1[u] = y1[(long long)(k + u) * sy];
    }
#pragma unroll
    for (int u = 0; u < kU; u += 2) {
      a0 = fmaf(x[k + u], v0[u], a0);
      a1 = fmaf(x[k + u + 1], v0[u + 1], a1);
      b0 = fmaf(x[k + u], v1[u], b0);
      b1 = fmaf(x[k + u + 1], v1[u + 1], b1);
    }
  }
  for (; k < len; ++k) {
    a0 = fmaf(x[k], y0[(long long)k * sy], a0);
    b0 = fmaf(x[k], y1[(long long)k * sy], b0);
  }
  r0 = a0 + a1;
  r1 = b0 + b1;
}

// Cholesky orthonormalisation of rows far from S-orthonormal (the warm start
// of an n-mer from its monomers' rows).  With M = CT S CT^T = U^T U (U upper
// triangular), the rows U^-T CT are S-orthonormal: a Gram-Schmidt pass over
// the rows in order, which keeps the first fragment's rows and makes every
// later row orthogonal to the rows before it.  These rows span the same space
// as the Loewdin rows M^-1/2 CT and differ from them by an orthogonal
// transformation, so they serve n-mers whose first iteration diagonalises
// exactly.  It replaces the Newton-Schulz steps that bring |M - I| from order
// 0.1 to 1e-2 (about ten n^3 products) by O(n^3 / 3) scalar work that needs no
// tensor-core tiles.
//   E: n x n, row-major, M - I on entry; its upper triangle becomes U.
//   Lt: n x n scratch (U^T, row-major); xs: n floats of shared memory.
// Returns false, with CT untouched, if a pivot is not positive (M not
// numerically positive definite); the caller then keeps Newton-Schulz.
__device__ __noinline__ bool chol_orthonormalise(int n, float* CT, float* E, float* Lt, float* xs) {
  __shared__ float s_piv;
  __shared__ int s_bad;
  // n <= 2 * kBlock: every thread owns up to two rows i (two columns c below),
  // taken in one loop so that their loads overlap
  for (int j = 0; j < n; ++j) {
    // left-looking column j: d_i = M_ji - sum_{k<j} U_kj U_ki for i >= j
    for (int k = threadIdx.x; k < j; k += blockDim.x) xs[k] = E[(long long)k * n + j];
    __syncthreads();
    const int i0 = j + threadIdx.x, i1 = i0 + blockDim.x;
    const bool h0 = i0 < n, h1 = i1 < n;
    float s0 = 0.f, s1 = 0.f;
    if (h0) chol_dot2(j, xs, E + i0, E + (h1 ? i1 : i0), n, s0, s1);
    const float d0 = h0 ? (i0 == j ? 1.f : 0.f) + E[(long long)j * n + i0] - s0 : 0.f;
    const float d1 = h1 ? E[(long long)j * n + i1] - s1 : 0.f;
    if (threadIdx.x == 0) {
      s_bad = !(d0 > 1e-6f);
      s_piv = s_bad ? 1.f : sqrtf(d0);
    }
    __syncthreads();
    if (s_bad) return false;          // CT not yet touched; E is rebuilt by the caller
    const float inv = 1.f / s_piv;
    if (h0) E[(long long)j * n + i0] = (i0 == j) ? s_piv : d0 * inv;
    if (h1) E[(long long)j * n + i1] = d1 * inv;
    __syncthreads();
  }
  // Lt = U^T (row i of Lt: column i of U, lower triangle)
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = int(e / n), k = int(e - (long long)i * n);
    if (k <= i) Lt[e] = E[(long long)k * n + i];
  }
  __syncthreads();
  // CT <- U^-T CT by forward substitution, columns c0 and c1 of CT per thread
  // (every thread takes part in staging row i of Lt)
  const int c0 = threadIdx.x, c1 = c0 + blockDim.x;
  const bool h0 = c0 < n, h1 = c1 < n;
  float* y0 = CT + (h0 ? c0 : 0);
  float* y1 = CT + (h1 ? c1 : (h0 ? c0 : 0));
  for (int i = 0; i < n; ++i) {
    for (int k = threadIdx.x; k <= i; k += blockDim.x) xs[k] = Lt[(long long)i * n + k];
    __syncthreads();
    if (h0) {
      float s0, s1;
      chol_dot2(i, xs, y0, y1, n, s0, s1);
      const float inv = 1.f / xs[i];
      const float r0 = (y0[(long long)i * n] - s0) * inv;
      const float r1 = (y1[(long long)i * n] - s1) * inv;
      y0[(long long)i * n] = r0;
      if (h1) y1[(long long)i * n] = r1;
    }
    __syncthreads();
  }
  return true;
}

// CT <- (M^{-1/2}) CT with M = CT S CT^T, by Newton-Schulz steps
// CT <- 1.5 CT - 0.5 M CT (each squares the error of M - I), until
// max |M - I| < tol or max_steps: restores the S-orthonormality of the
// eigenvector rows (the FP32 Loewdin start, FP32 rotations and the hand-over
// from FP32 to FP64 all leave it slightly off).
template <typename T>
__device__ void reorthonormalise(const Nmer& nm, const SccArgs& ar, SccSmem& sm, PrecPtrs<T> pp, int max_steps,
                                 double tol) {
  const int n = nm.n;
  T* gemm = reinterpret_cast<T*>(sm.gemm);
  const double* Sm = ar.S + nm.mat;
  bool chol_tried = !kCholStart;
  for (int step = 0; step < max_steps; ++step) {
    if constexpr (sizeof(T) == 4)   // S rounded to FP32 either way; the FP32 copy skips the conversions
      block_gemm<T>(n, n, n, pp.CT, n, 1, ar.S32 + nm.mat, n, 1, pp.W2, n, nullptr, nullptr, nullptr, gemm);
    else
      block_gemm<T, double>(n, n, n, pp.CT, n, 1, Sm, n, 1, pp.W2, n, nullptr, nullptr, nullptr, gemm);   // V = CT S
    block_gemm<T>(n, n, n, pp.W2, n, 1, pp.CT, n, 1, pp.W1, n, nullptr, nullptr, nullptr, gemm);       // M = V CT^T
    if constexpr (sizeof(T) == 4) {
      // far from orthonormal (a warm start from monomer rows): third-order
      // steps CT <- (I - E/2 + 3/8 E^2) CT with E = M - I, the series of
      // M^-1/2 to second order: the error goes as ~|E|^3 per step for 4
      // GEMMs instead of ~|E|^2 for 3 (A is free scratch here)
      const double err = max_dev_from_identity(pp.W1, n, n, sm.red, pp.W1);   // W1 <- E
      if (err < tol) break;
      // n-mers whose first iteration is a tridiagonal solve: one Cholesky pass
      // instead of the third-order steps (once; Newton-Schulz polishes after)
      if (err > 1e-2 && !chol_tried && sm.tri && n >= kTriMinN && n <= 2 * kBlock) {
        chol_tried = true;
        if (chol_orthonormalise(n, pp.CT, pp.W1, pp.W2, reinterpret_cast<float*>(gemm))) continue;
        // not positive definite: E was partly overwritten, rebuild it
        block_gemm<T>(n, n, n, pp.CT, n, 1, ar.S32 + nm.mat, n, 1, pp.W2, n, nullptr, nullptr, nullptr, gemm);
        block_gemm<T>(n, n, n, pp.W2, n, 1, pp.CT, 1, n, pp.W1, n, nullptr, nullptr, nullptr, gemm);
        max_dev_from_identity(pp.W1, n, n, sm.red, pp.W1);
      }
      if (err > 1e-2) {
        block_gemm<T>(n, n, n, pp.W1, n, 1, pp.CT, 1, n, pp.W2, n, nullptr, nullptr, nullptr, gemm);     // Y = E CT
        block_gemm<T>(n, n, n, pp.W1, n, 1, pp.W2, 1, n, pp.A, pp.lda, nullptr, nullptr, nullptr, gemm); // E Y
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
          const long long i = e / n, j = e - i * n;
          pp.CT[e] = pp.CT[e] - T(0.5) * pp.W2[e] + T(0.375) * pp.A[i * pp.lda + j];
        }
      } else {
        block_gemm<T>(n, n, n, pp.W1, n, 1, pp.CT, 1, n, pp.W2, n, nullptr, nullptr, nullptr, gemm);     // E CT
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x)
          pp.CT[e] = pp.CT[e] - T(0.5) * pp.W2[e];
        __syncthreads();
        // from |E| < 3e-4 this step leaves (3/4)|E|^2 < 1e-7 plus FP32
        // rounding, below any tolerance used here: no product to confirm it
        if (err < 3e-4 && tol >= 1e-6) break;
        continue;
      }
      __syncthreads();
      continue;
    }
    const double err = max_dev_from_identity(pp.W1, n, n, sm.red);
    if (err < tol) break;
    block_gemm<T>(n, n, n, pp.W1, n, 1, pp.CT, 1, n, pp.W2, n, nullptr, nullptr, nullptr, gemm);       // M CT
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x)
      pp.CT[e] = T(1.5) * pp.CT[e] - T(0.5) * pp.W2[e];
    __syncthreads();
  }
}

// FP32 -> FP64 hand-over: the FP64 rows (converted from FP32) are
// S-orthonormal to about 1e-7.  M = CT S CT^T is formed in FP64; the
// Newton-Schulz correction CT <- CT - 1/2 (M - I) CT only needs the small
// (M - I) to relative FP32 accuracy, so that product runs in FP32 (on the
// FP32 rows, equal to CT to 1e-7).  One step leaves ~1e-14; a second,
// all-FP64 step follows only if the start was worse than 1e-6.
__device__ void reortho_handover(const Nmer& nm, const SccArgs& ar, SccSmem& sm, PrecPtrs<double> pd,
                                 const float* ct32, float* wf1, float* wf2) {
  const int n = nm.n;
  const double* Sm = ar.S + nm.mat;
  float* gdf = reinterpret_cast<float*>(sm.gemm);
  // double-float products (FP64-grade); the rows are exact FP32 values
  block_gemm_df<float>(n, n, n, ct32, nullptr, n, Sm, n, pd.W2, n, gdf);     // V = CT S (S symmetric)
  block_gemm_df<double>(n, n, n, pd.W2, nullptr, n, pd.CT, n, pd.W1, n, gdf);  // M = V CT^T
  const double err = max_dev_from_identity(pd.W1, n, n, sm.red, wf1);
  float* gf = reinterpret_cast<float*>(sm.gemm);
  block_gemm<float>(n, n, n, wf1, n, 1, ct32, 1, n, wf2, n, nullptr, nullptr, nullptr, gf);   // (M - I) CT
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) pd.CT[e] -= 0.5 * double(wf2[e]);
  __syncthreads();
  if (err > 1e-6) reorthonormalise<double>(nm, ar, sm, pd, 3, 1e-13);
}

// FP64 energy of the density held by FP32 eigenvector rows (mixed
// precision, dimers and trimers).  The FP32 phase has converged the n-mer to
// a charge residual near FP32 rounding.  Only the occupied rows c_k enter
// P = sum_k f_k c_k c_k^T, so only they are made S-orthonormal in FP64:
// W = C_o S and Y = C_o H0 are formed in FP64 once, M = W C_o^T (no x no),
// and each Newton-Schulz step X <- X - 1/2 (M - I) X is applied to C_o, W and
// Y together (the small (M - I) X products in FP32).  Then the Mulliken
// populations (P S)_mu,mu = sum_k f_k C_k,mu W_k,mu (Eq. 3) and the band
// energy sum_k f_k C_k . Y_k give E_el of Eq. 2 from sm.dqout.  Rounding of
// the FP32 rows is a rotation of the occupied space by ~1e-7 once the rows
// are orthonormal, and the n-mer energy in its fixed ESP is stationary under
// such rotations, so it enters the energy at second order.
// ct32: the FP32 rows in global memory; wf1, wf2: n x n FP32 scratch.
__device__ double fp64_energy_of_rows(const Nmer& nm, const SccArgs& ar, SccSmem& sm, PrecPtrs<double> pd,
                                      const float* ct32, float* wf1, float* wf2) {
  const int n = nm.n, nsh = nm.nsh;
  const double* Sm = ar.S + nm.mat;
  const double* Hm = ar.H0 + nm.mat;
  int no = 0;
  const double mts = fermi_step<double>(n, nm.nel, ar.g.kT, sm, &no);   // occupations of the last FP32 iteration
  double* Co = pd.CT;   // no x n
  double* W = pd.W1;    // no x n
  double* Y = pd.W2;    // no x n
  double* M = pd.A;     // no x no
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = wid; k < no; k += nw) {
      const float* src = ct32 + (long long)sm.occ[k] * n;
      double* dst = Co + (long long)k * n;
      for (int j = lane; j < n; j += 32) dst[j] = double(src[j]);
    }
  }
  __syncthreads();
  double* gemm = reinterpret_cast<double*>(sm.gemm);
  float* gf = reinterpret_cast<float*>(sm.gemm);
  // the rows are exact FP32 values: the three products with them run in
  // double-float arithmetic (FP64-grade results from FP32 instructions)
  block_gemm_df<float>(no, n, n, ct32, sm.occ, n, Sm, n, W, n, gf);   // W = C_o S (S symmetric)
  block_gemm_df<float>(no, n, n, ct32, sm.occ, n, Hm, n, Y, n, gf);   // Y = C_o H0 (H0 symmetric)
  double err0 = 0.0;
  for (int step = 0; step < 2; ++step) {
    if (step == 0) block_gemm_df<float>(no, no, n, ct32, sm.occ, n, W, n, M, no, gf);   // M = C_o W^T = C_o S C_o^T
    else block_gemm<double>(no, no, n, W, n, 1, Co, n, 1, M, no, nullptr, nullptr, nullptr, gemm);
    const double err = max_dev_from_identity(M, no, no, sm.red, wf1);
    if (step == 0) err0 = err;
    if (step == 0 && err0 <= 1e-6) {
      // one Newton-Schulz step leaves ~err0^2 plus the FP32 rounding of the
      // correction (~1e-7 err0): below 1e-12, nothing for a second step
      step = 1;
    }
    double* X[3] = {Co, W, Y};
    for (int x = 0; x < 3; ++x) {
      block_gemm<float, double>(no, n, no, wf1, no, 1, X[x], 1, n, wf2, n, nullptr, nullptr, nullptr, gf);
      for (long long e = threadIdx.x; e < (long long)no * n; e += blockDim.x) X[x][e] -= 0.5 * double(wf2[e]);
      __syncthreads();
    }
  }
  // per-AO population and band energy, one thread per AO (coalesced rows)
  double* pop = reinterpret_cast<double*>(sm.jsc);
  double* band = reinterpret_cast<double*>(sm.jss);
  for (int mu = threadIdx.x; mu < n; mu += blockDim.x) {
    double p = 0.0, b = 0.0;
    for (int k = 0; k < no; ++k) {
      const double fc = sm.focc[sm.occ[k]] * Co[(long long)k * n + mu];
      p += fc * W[(long long)k * n + mu];
      b += fc * Y[(long long)k * n + mu];
    }
    pop[mu] = p;
    band[mu] = b;
  }
  __syncthreads();
  for (int s = threadIdx.x; s < nsh; s += blockDim.x) {
    double p = 0.0, b = 0.0;
    for (int k = sm.mp.sh_ao0[s]; k < sm.mp.sh_ao0[s + 1]; ++k) { p += pop[k]; b += band[k]; }
    sm.dqout[s] = p - sm.q0[s];
    sm.sig[s] = b;
  }
  __syncthreads();
  double diff = 0.0;
  return energy_of_output(nm, ar, sm, &diff) + mts;
}

// Jacobi threshold (relative to max |A_ii|) for an SCC iteration whose
// previous residual was `last`: rotations far below the SCC error change
// nothing the loop needs, so early iterations rotate only the large elements.
__device__ __forceinline__ double jacobi_threshold(double last, double floor_tol) {
  return fmax(floor_tol, fmin(1e-4, 1e-3 * last));
}

// FP32 iterations without a 10% improvement of the best residual before the
// FP32 phase gives up and hands over to FP64
constexpr int kStall32 = 8;
// iterations without a 10% improvement of the best residual before an n-mer
// SCC switches to full-precision eigen-solves
constexpr int kStallTight = 6;

// kMinBlocks = 2: at most 128 registers per thread, so that two CTAs share an
// SM (more warps to hide latency) when the pass's matrices live in global
// memory; kMinBlocks = 1: all 255 registers (n-mers whose matrices fill the
// shared memory run one CTA per SM anyway).
template <int kMinBlocks>
__global__ void __launch_bounds__(kBlock, kMinBlocks) scc_kernel(SccArgs ar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (ar.jac_hint_dev) ar.jac_hint = *ar.jac_hint_dev;
  const int idx = ar.order[blockIdx.x];
  const Nmer nm = ar.nmers[idx];
  const int n = nm.n, nsh = nm.nsh, nat = nm.nat, npad = nm.npad;
  const int a_bytes = (ar.a_smem_d ? int(sizeof(double)) : (ar.a_smem_f ? int(sizeof(float)) : 0)) *
                      ((ar.max_n + (ar.max_n & 1)) * (ar.max_n + (ar.max_n & 1)));
  SccSmem sm = carve_scc_smem(smem_raw, ar.max_n, ar.max_nsh, ar.max_nat, a_bytes);
  sm.tri = ar.tri_cap > 0 ? reinterpret_cast<float*>(smem_raw + scc_smem_bytes(ar.max_n, ar.max_nsh, ar.max_nat, a_bytes))
                          : nullptr;
  const long long t_start = clock64();
  build_maps(nm, ar.ft, ar.elem, ar.atom_sh0, ar.el, sm.mp);
  // ghosts of cut bonds healed in this n-mer (hybrid orbital projection):
  // not in its basis, but their monomer charges leave its embedding potential
  // and enter dE^V as the charge transfer -dq_mono
  __shared__ int s_hg_sh[kMaxHealedShells], s_hg_at[kMaxHealedShells], s_hg_k[kMaxHealedShells];
  __shared__ int s_nhg;
  if (threadIdx.x == 0) {
    int c = 0;
    if (ar.ft.ghost_frag) {
      for (int kf = 0; kf < nm.nfrag; ++kf) {
        const int f = nm.frag[kf];
        for (int i = 0; i < ar.ft.nat[f]; ++i) {
          const int ga = ar.ft.atom0[f] + i;
          if (atom_in_nmer(ar.ft, nm.nfrag, nm.frag, ga)) continue;
          const DevElem& e = ar.el[ar.elem[ga]];
          for (int k = 0; k < e.nsh && c < kMaxHealedShells; ++k, ++c) {
            s_hg_sh[c] = ar.atom_sh0[ga] + k;
            s_hg_at[c] = ga;
            s_hg_k[c] = k;
          }
        }
      }
    }
    s_nhg = c;
  }
  // per-shell / per-atom constants
  for (int s = threadIdx.x; s < nsh; s += blockDim.x) {
    const int ga = sm.mp.at_glob[sm.mp.sh_at[s]];
    const DevElem& e = ar.el[ar.elem[ga]];
    const int k = sm.mp.sh_glob[s] - ar.atom_sh0[ga];
    double q = e.q0[k];
    if (ar.ft.ghost_frag && ar.ft.ghost_frag[ga] >= 0) {
      q = (e.l[k] == 0) ? 0.25 : 0.75;          // ghost: one electron, c_s^2 and c_p^2 of the hybrid
    } else if (ar.ft.bda_baa_frag && ar.ft.bda_baa_frag[ga] >= 0 &&
               !frag_in_nmer(nm.nfrag, nm.frag, ar.ft.bda_baa_frag[ga])) {
      double tot = 0.0;                         // detached BDA: one electron less, shared
      for (int kk = 0; kk < e.nsh; ++kk) tot += e.q0[kk];   // in proportion to q0
      q *= (tot - 1.0) / tot;
    }
    sm.q0[s] = q;
  }
  for (int a = threadIdx.x; a < nat; a += blockDim.x) sm.g3[a] = ar.el[ar.elem[sm.mp.at_glob[a]]].gamma3;
  __syncthreads();
  // repulsion energy inside the n-mer (Eq. 11), unordered atom pairs
  double er = 0.0;
  for (int e = threadIdx.x; e < nat * nat; e += blockDim.x) {
    const int i = e / nat, j = e % nat;
    if (j >= i) continue;
    const int ga = sm.mp.at_glob[i], gb = sm.mp.at_glob[j];
    if (ar.ft.ghost_frag && (ar.ft.ghost_frag[ga] >= 0 || ar.ft.ghost_frag[gb] >= 0)) continue;   // ghosts: none
    const DevElem& EA = ar.el[ar.elem[ga]];
    const DevElem& EB = ar.el[ar.elem[gb]];
    const double dx = ar.xyz[3 * ga] - ar.xyz[3 * gb], dy = ar.xyz[3 * ga + 1] - ar.xyz[3 * gb + 1],
                 dz = ar.xyz[3 * ga + 2] - ar.xyz[3 * gb + 2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    er += EA.zeff * EB.zeff / r * exp(-sqrt(EA.arep * EB.arep) * pow(r, ar.g.k_f));
  }
  const double e_rep = block_sum(er, sm.red);
  // embedding potential of this n-mer: ESP_mu = phi_mu - sum_{lambda in X} gamma dq_mono
  const double* G = ar.gam + nm.gam;
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double v = 0.0;
      if (ar.phi) {
        for (int t = lane; t < nsh; t += 32) v += G[(size_t)s * nsh + t] * ar.dq_mono[sm.mp.sh_glob[t]];
        if (s_nhg > 0) {
          const int ga = sm.mp.at_glob[sm.mp.sh_at[s]];
          const double ie = 1.0 / ar.el[ar.elem[ga]].eta_sh[sm.mp.sh_glob[s] - ar.atom_sh0[ga]];
          for (int t = lane; t < s_nhg; t += 32)
            v += shell_gamma(ar, ga, ie, s_hg_at[t], s_hg_k[t]) * ar.dq_mono[s_hg_sh[t]];
        }
        v = warp_sum(v);
        v = ar.phi[sm.mp.sh_glob[s]] - v;
      }
      if (lane == 0) {
        sm.esp[s] = v;
        ar.esp[nm.shv + s] = v;
        sm.dqin[s] = ar.guess_from_mono ? ar.dq_mono[sm.mp.sh_glob[s]] : ar.dq[nm.shv + s];
      }
    }
  }
  __syncthreads();

  // non-finite start charges or potential (a NaN guess): no iterations, NaN
  // results and status
  bool bad_in = false;
  {
    int b = 0;
    for (int s = threadIdx.x; s < nsh; s += blockDim.x) b |= !isfinite(sm.dqin[s]) || !isfinite(sm.esp[s]);
    bad_in = __syncthreads_or(b);
  }
  const int lda_d = npad;
  PrecPtrs<double> pd{ar.CTd + nm.mat, ar.W1d + nm.mat, ar.W2d + nm.mat,
                      ar.a_smem_d ? reinterpret_cast<double*>(sm.A) : ar.Agd + nm.apad,
                      lda_d};
  PrecPtrs<float> pf{nullptr, nullptr, nullptr, nullptr, npad};
  if (ar.precision == 1) {
    pf.CT = ar.CTf + nm.mat;
    pf.W1 = ar.W1f + nm.mat;
    pf.W2 = ar.W2f + nm.mat;
    pf.A = ar.a_smem_f ? reinterpret_cast<float*>(sm.A) : ar.Agf + nm.apad;
  }
  // Mixed precision with the FP64 eigen-solve matrix in shared memory: that
  // region (8 npad^2 bytes) also holds the FP32 matrix (4 npad^2) and the FP32
  // eigenvector rows (4 n^2) during the FP32 phase, so the rotations of every
  // Jacobi round stay on chip.  The FP64 matrix takes the region over after
  // the hand-over, when the FP32 rows are no longer needed.
  float* const ctf_g = (ar.precision == 1) ? ar.CTf + nm.mat : nullptr;
  const bool ct_smem = ar.a_smem_d && ar.precision == 1;
  float* const ctf_s = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sm.A) +
                                                align16(sizeof(float) * (size_t)npad * npad));
  auto load_ct_smem = [&]() {
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) ctf_s[e] = ctf_g[e];
    __syncthreads();
    pf.CT = ctf_s;
  };
  double* hist = ar.hist + nm.hist;
  int hcount = 0, hhead = 0;
  int phase = (ar.precision == 1) ? 0 : 1;   // 0: FP32 loose, 1: FP64
  double e_prev = 0.0;
  bool have_prev = false;
  int status = FMO_SCC_MAX_ITER_CODE;
  int it = 0, it32 = 0, jac_fail = 0;
  double e_el = 0.0;
  if (ar.single_step && !bad_in) {
    // one iteration from the given charges in the given precision; the
    // caller mixes the charges of all monomers together
    phase = ar.step_phase;
    if (phase == 1 && ar.precision == 1 && ar.reortho) {
      for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) pd.CT[e] = double(pf.CT[e]);
      __syncthreads();
      reortho_handover(nm, ar, sm, pd, pf.CT, pf.W1, pf.W2);
    } else if (ar.cold_refine && phase == 1) {
      reorthonormalise<double>(nm, ar, sm, pd, 4, 1e-14);
    } else if (ar.cold_refine) {
      reorthonormalise<float>(nm, ar, sm, pf, 2, 1e-6);
    }
    if (phase == 0 && ct_smem) load_ct_smem();
    // every fourth FP32 step (1-based, after the first) restores orthonormality
    const int step = ar.step_dev ? *ar.step_dev + 1 : 0;
    const bool r32 = ar.step_dev ? (step > 1 && step % 4 == 0) : (ar.reortho32 != 0);
    if (phase == 0 && r32 && !ar.cold_refine) reorthonormalise<float>(nm, ar, sm, pf, 1, 0.0);
    double diff = 0.0;
    // every step diagonalises to the working precision (no threshold loosened
    // by the residual): the global mixer then iterates one fixed map.  A
    // threshold that followed the residual changed the map from step to step
    // and left the monomer loop of distorted frames oscillating.
    if (phase == 0) {
      e_el = scc_iteration<float>(nm, ar, sm, pf, ar.jacobi_tol_f, &jac_fail, &diff, !ar.cold_refine);
      it32 = 1;
    } else {
      e_el = scc_iteration<double>(nm, ar, sm, pd, ar.jacobi_tol_d, &jac_fail, &diff, !ar.cold_refine,
                                   ar.precision == 1 ? ctf_g : nullptr, pf.W1, pf.W2);
    }
    it = 1;
    status = (phase == 1 && jac_fail) ? FMO_SCC_JACOBI_CODE
             : (__syncthreads_or(!isfinite(e_el)) ? FMO_SCC_NAN_CODE : FMO_SCC_CONVERGED_CODE);
  }
  double last = ar.jac_hint;
  bool fresh64 = false;
  int n64 = 0;
  bool fp32_converged = false;
  bool energy_done = false;
  bool full64 = false;
  double min32 = 1e300;
  int stall32 = 0;
  // Jacobi thresholds follow the residual (early iterations rotate only the
  // large elements) until the FP64 iterations stall: kStallTight iterations
  // without a 10% improvement of their best residual.  From then on every
  // eigen-solve is to working precision and the Broyden history restarts, so
  // the mixer iterates one fixed map (a map that changed from step to step
  // left dimers of distorted geometries oscillating).  A stalled FP32 phase
  // hands over to FP64 instead (kStall32).
  bool tight = false;
  double min_all = 1e300;
  int stall_all = 0;
  if (!ar.single_step && ar.cold_refine) {
    // the starting rows made S-orthonormal to the working precision
    if (phase == 0) reorthonormalise<float>(nm, ar, sm, pf, ar.cold_steps, 1e-6);
    else reorthonormalise<double>(nm, ar, sm, pd, 4, 1e-14);
  }
  if (!ar.single_step && phase == 0 && ct_smem) load_ct_smem();
  long long t_it = clock64();
  if (ar.trace && blockIdx.x == 0 && threadIdx.x == 0) ar.trace[1024] = double(t_it - t_start);
  for (it = (ar.single_step || bad_in ? ar.max_iter + 2 : 1); it <= ar.max_iter; ++it) {
    double diff = 0.0;
    if (phase == 0) {
      if (it32 > 0 && it32 % 4 == 0) reorthonormalise<float>(nm, ar, sm, pf, 1, 0.0);
      // a warm start only needs near-canonical rows before the rotation
      // updates take over: its first eigen-solve may be loose
      const double thr = tight ? ar.jacobi_tol_f
                               : ((it == 1 && ar.first_jac_tol > 0) ? ar.first_jac_tol
                                                                    : jacobi_threshold(last, ar.jacobi_tol_f));
      e_el = scc_iteration<float>(nm, ar, sm, pf, thr, &jac_fail, &diff, it > 1 || !ar.cold_refine || ar.first_rot);
      ++it32;
    } else {
      e_el = scc_iteration<double>(nm, ar, sm, pd, tight ? ar.jacobi_tol_d : jacobi_threshold(last, ar.jacobi_tol_d),
                                   &jac_fail, &diff, it > 1 || !ar.cold_refine, ar.precision == 1 ? ctf_g : nullptr,
                                   pf.W1, pf.W2);
    }
    last = diff;
    if (phase == 1 && !tight) {
      if (diff < 0.9 * min_all) { min_all = diff; stall_all = 0; }
      else if (++stall_all >= kStallTight) {
        tight = true;
        hcount = 0;
        hhead = 0;
        have_prev = false;
        fresh64 = true;   // no secant pair across the switch
      }
    }
    if (ar.trace && blockIdx.x == 0 && threadIdx.x == 0 && it < 512) {
      // per iteration: residual (negative in FP32), Jacobi sweeps (-1 =
      // rotation step) and SM cycles
      const long long t1 = clock64();
      ar.trace[it] = phase ? diff : -diff;
      ar.trace[512 + it] = sm.misc[3];
      ar.trace[1024 + it] = double(t1 - t_it);
      t_it = t1;
    }
    // FP32 phase: converged, or no longer improving (FP32 rounding floor, e.g.
    // the 1e6 Eh hybrid-orbital projector) or at its cap -> FP64
    if (phase == 0) {
      if (diff < 0.9 * min32) { min32 = diff; stall32 = 0; } else { ++stall32; }
    }
    const bool fp32_done = phase == 0 && diff < ar.switch_tol;
    const bool fp32_give_up = phase == 0 && !fp32_done && (it32 >= ar.fp32_cap || stall32 >= kStall32);
    if (phase == 1 && ar.precision == 1 && ar.fp64_finish > 0 && !full64 && ++n64 >= ar.fp64_finish) {
      // FP64 energy of the FP32-converged charges (variational for n-mers
      // in a fixed ESP); the loop ends here
      status = fp32_converged ? FMO_SCC_CONVERGED_CODE : FMO_SCC_MAX_ITER_CODE;
      if (__syncthreads_or(!isfinite(e_el))) status = FMO_SCC_NAN_CODE;
      break;
    }
    // loop decisions are made block-uniform with barrier votes (thread 0's
    // timer read decides the deadline)
    if (__syncthreads_or(!isfinite(e_el) || !isfinite(diff))) { status = FMO_SCC_NAN_CODE; break; }
    if (ar.energy_finish && __syncthreads_and(fp32_done)) {
      // n-mer in mixed precision: FP64 energy of the FP32-converged density
      const long long tf = clock64();
      if (ct_smem) {
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) ctf_g[e] = pf.CT[e];
        __syncthreads();
      }
      e_el = fp64_energy_of_rows(nm, ar, sm, pd, ctf_g, pf.W1, pf.W2);
      status = FMO_SCC_CONVERGED_CODE;
      if (__syncthreads_or(!isfinite(e_el))) status = FMO_SCC_NAN_CODE;
      if (ar.trace && blockIdx.x == 0 && threadIdx.x == 0) ar.trace[1535] = double(clock64() - tf);
      energy_done = true;
      break;
    }
    if (__syncthreads_and(phase == 1 && have_prev && diff < ar.tol && fabs(e_el - e_prev) < ar.etol)) {
      status = FMO_SCC_CONVERGED_CODE;
      break;
    }
    e_prev = e_el;
    have_prev = true;
    if (__syncthreads_or(threadIdx.x == 0 && ar.budget_ns && globaltimer_ns() > *ar.t0 + ar.budget_ns)) {
      status = FMO_SCC_TIMEOUT_CODE;
      break;
    }
    broyden_step(nsh, it, hist, sm, hcount, hhead, 0.4, 0.01, !fresh64);
    fresh64 = false;
    if (__syncthreads_and(fp32_done || fp32_give_up)) {
      // an FP32 phase that gave up converges fully in FP64
      full64 = fp32_give_up;
      for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) pd.CT[e] = double(pf.CT[e]);
      __syncthreads();
      if (ct_smem) {
        // the FP32 rows leave shared memory (the FP64 matrix takes it over)
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) ctf_g[e] = pf.CT[e];
        __syncthreads();
      }
      reortho_handover(nm, ar, sm, pd, ct_smem ? ctf_g : pf.CT, pf.W1, pf.W2);
      phase = 1;
      have_prev = false;
      fresh64 = true;
      fp32_converged = diff < ar.switch_tol;
    }
  }
  if (ar.single_step) it = 1;
  else if (it > ar.max_iter) it = ar.max_iter;
  if (bad_in) {
    it = 0;
    status = FMO_SCC_NAN_CODE;
    e_el = __longlong_as_double(0x7ff8000000000000LL);
    for (int s = threadIdx.x; s < nsh; s += blockDim.x) sm.dqout[s] = sm.dqin[s];
    for (int i = threadIdx.x; i < n; i += blockDim.x) sm.eps[i] = e_el;
    __syncthreads();
  }
  if (jac_fail && status == FMO_SCC_CONVERGED_CODE) status = FMO_SCC_JACOBI_CODE;
  // keep a float copy of the final eigenvectors in global memory for a later
  // warm start
  if (ar.precision == 1 && phase == 1) {
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) ctf_g[e] = float(pd.CT[e]);
  } else if (ar.precision == 1 && ct_smem && !energy_done) {
    for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) ctf_g[e] = pf.CT[e];
  }
  // results
  double dev = 0.0;
  for (int s = threadIdx.x; s < nsh; s += blockDim.x) {
    ar.dq[nm.shv + s] = sm.dqout[s];
    if (ar.phi) dev += (sm.dqout[s] - ar.dq_mono[sm.mp.sh_glob[s]]) * sm.esp[s];   // Eq. 13
  }
  if (ar.phi && s_nhg > 0) {
    // healed ghost shells: charge transfer -dq_mono in the ESP of the n-mer's
    // environment, phi_g - sum over all monomer shells of the n-mer's fragments
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int h = wid; h < s_nhg; h += nw) {
      const int gat = s_hg_at[h];
      const double ie = 1.0 / ar.el[ar.elem[gat]].eta_sh[s_hg_k[h]];
      double v = 0.0;
      for (int t = lane; t < nsh; t += 32) {
        const int tat = sm.mp.at_glob[sm.mp.sh_at[t]];
        v += shell_gamma(ar, gat, ie, tat, sm.mp.sh_glob[t] - ar.atom_sh0[tat]) * ar.dq_mono[sm.mp.sh_glob[t]];
      }
      for (int t = lane; t < s_nhg; t += 32)
        v += shell_gamma(ar, gat, ie, s_hg_at[t], s_hg_k[t]) * ar.dq_mono[s_hg_sh[t]];
      v = warp_sum(v);
      if (lane == 0) dev += -ar.dq_mono[s_hg_sh[h]] * (ar.phi[s_hg_sh[h]] - v);
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) ar.eps[nm.aov + i] = sm.eps[i];
  dev = block_sum(dev, sm.red);
  if (ar.trace && threadIdx.x == 0) {
    const unsigned long long cyc = (unsigned long long)(clock64() - t_start);
    atomicMax(reinterpret_cast<unsigned long long*>(ar.trace + kTraceSlowest), (cyc << 20) | blockIdx.x);
  }
  if (threadIdx.x == 0) {
    ar.energy[idx] = e_el + e_rep;
    ar.e_el[idx] = e_el;
    ar.e_rep[idx] = e_rep;
    ar.dEV[idx] = dev;
    ar.iters[idx] = it;
    ar.iters32[idx] = it32;
    ar.status[idx] = status;
  }
}

// ---------------------------------------------------------------------------
// Supersystem potential phi_mu = sum_lambda gamma_mu,lambda dq_lambda over all
// shells (the ESP of Eq. 21 before the fragment's own shells are removed).
// Grid: blockIdx.x selects 256 target shells mu, blockIdx.y a chunk of source
// shells lambda staged through shared memory; each chunk writes its partial
// sums, which phi_reduce_kernel adds in chunk order (deterministic).

// T = double: the potential in FP64.  T = float: an FP32 estimate (pair terms
// and the sum over one chunk in FP32) for the FP32 phase of the mixed-
// precision monomer loop, whose charges are only FP32-accurate anyway.
template <typename T>
__global__ void __launch_bounds__(256) phi_kernel(int n_sh, int chunk, const double* __restrict__ xyz,
                                                  const int* __restrict__ sh_atom,
                                                  const double* __restrict__ sh_inv_eta,
                                                  const double* __restrict__ dq, GParams g,
                                                  double* __restrict__ part) {
  __shared__ T tx[256], ty[256], tz[256], te[256], tq[256];
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  T x = 0, y = 0, z = 0, ie = 1;
  if (mu < n_sh) {
    const int a = sh_atom[mu];
    x = T(xyz[3 * a]); y = T(xyz[3 * a + 1]); z = T(xyz[3 * a + 2]);
    ie = T(sh_inv_eta[mu]);
  }
  const int l0 = blockIdx.y * chunk, l1 = min(n_sh, l0 + chunk);
  T acc = 0;
  for (int t0 = l0; t0 < l1; t0 += 256) {
    const int l = t0 + threadIdx.x;
    if (l < l1) {
      const int b = sh_atom[l];
      tx[threadIdx.x] = T(xyz[3 * b]); ty[threadIdx.x] = T(xyz[3 * b + 1]); tz[threadIdx.x] = T(xyz[3 * b + 2]);
      te[threadIdx.x] = T(sh_inv_eta[l]);
      tq[threadIdx.x] = T(dq[l]);
    }
    __syncthreads();
    const int m = min(256, l1 - t0);
    if (g.k_g == 2.0) {
      for (int k = 0; k < m; ++k) {
        const T dx = x - tx[k], dy = y - ty[k], dz = z - tz[k];
        const T e = T(0.5) * (ie + te[k]);
        const T r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, e * e)));
        if constexpr (sizeof(T) == 8) acc = fma(rsqrt_fp64(r2), tq[k], acc);
        else acc = fma(rsqrtf(r2), tq[k], acc);
      }
    } else {
      for (int k = 0; k < m; ++k) {
        const double dx = double(x) - double(tx[k]), dy = double(y) - double(ty[k]), dz = double(z) - double(tz[k]);
        acc += T(gamma_fn(dx * dx + dy * dy + dz * dz, double(ie), double(te[k]), g.k_g) * double(tq[k]));
      }
    }
    __syncthreads();
  }
  if (mu < n_sh) part[(size_t)blockIdx.y * n_sh + mu] = double(acc);
}

// gamma of Eqs. 4-5 between every pair of shells of the system, row-major
// n_sh x n_sh.  With it held in HBM the supersystem potential of each
// monomer-loop step is a matrix-vector product (HBM-bound) instead of n_sh^2
// FP64 kernel evaluations.  Block (x: 256 columns lambda, y: every gridDim.y-th
// row mu).
__global__ void __launch_bounds__(256) gamma_full_kernel(int n_sh, const double* __restrict__ xyz,
                                                         const int* __restrict__ sh_atom,
                                                         const double* __restrict__ sh_inv_eta, GParams g,
                                                         double* __restrict__ gam) {
  const int lam = blockIdx.x * blockDim.x + threadIdx.x;
  if (lam >= n_sh) return;
  const int b = sh_atom[lam];
  const double xb = xyz[3 * b], yb = xyz[3 * b + 1], zb = xyz[3 * b + 2], ieb = sh_inv_eta[lam];
  for (int mu = blockIdx.y; mu < n_sh; mu += gridDim.y) {
    const int a = sh_atom[mu];
    const double dx = xyz[3 * a] - xb, dy = xyz[3 * a + 1] - yb, dz = xyz[3 * a + 2] - zb;
    gam[(size_t)mu * n_sh + lam] = gamma_fn(dx * dx + dy * dy + dz * dz, sh_inv_eta[mu], ieb, g.k_g);
  }
}

// phi_mu = sum_lambda gamma_mu,lambda dq_lambda from the stored matrix, one
// warp per row (fixed summation order).
__global__ void __launch_bounds__(256) phi_gemv_kernel(int n_sh, const double* __restrict__ gam,
                                                       const double* __restrict__ dq, double* __restrict__ phi) {
  const int lane = threadIdx.x & 31;
  const int mu = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (mu >= n_sh) return;
  const double* row = gam + (size_t)mu * n_sh;
  // four independent loads in flight per lane: the row stream needs the
  // memory-level parallelism to approach HBM bandwidth
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int l = lane;
  for (; l + 96 < n_sh; l += 128) {
    const double a0 = __ldcs(row + l), a1 = __ldcs(row + l + 32), a2 = __ldcs(row + l + 64),
                 a3 = __ldcs(row + l + 96);
    s0 = fma(a0, dq[l], s0);
    s1 = fma(a1, dq[l + 32], s1);
    s2 = fma(a2, dq[l + 64], s2);
    s3 = fma(a3, dq[l + 96], s3);
  }
  for (; l < n_sh; l += 32) s0 = fma(row[l], dq[l], s0);
  const double v = warp_sum((s0 + s1) + (s2 + s3));
  if (lane == 0) phi[mu] = v;
}

__global__ void phi_reduce_kernel(int n_sh, int n_chunk, const double* __restrict__ part,
                                  double* __restrict__ phi) {
  const int mu = blockIdx.x * blockDim.x + threadIdx.x;
  if (mu >= n_sh) return;
  double s = 0.0;
  for (int c = 0; c < n_chunk; ++c) s += part[(size_t)c * n_sh + mu];
  phi[mu] = s;
}

// Fragment centroids and bounding radii (for pruning the pair search).
__global__ void frag_bounds_kernel(int n_frag, FragTab ft, const double* __restrict__ xyz,
                                   double* __restrict__ bounds) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_frag) return;
  const int a0 = ft.atom0[f], na = ft.nat[f];
  double cx = 0, cy = 0, cz = 0;
  for (int i = 0; i < na; ++i) { cx += xyz[3 * (a0 + i)]; cy += xyz[3 * (a0 + i) + 1]; cz += xyz[3 * (a0 + i) + 2]; }
  cx /= na; cy /= na; cz /= na;
  double r = 0;
  for (int i = 0; i < na; ++i) {
    const double dx = xyz[3 * (a0 + i)] - cx, dy = xyz[3 * (a0 + i) + 1] - cy, dz = xyz[3 * (a0 + i) + 2] - cz;
    r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
  }
  bounds[4 * f] = cx; bounds[4 * f + 1] = cy; bounds[4 * f + 2] = cz; bounds[4 * f + 3] = r;
}

// Closest inter-fragment atom distance of every pair I<J (lexicographic pair
// index); pairs whose bounding spheres are farther apart than `cut` get the
// sphere gap, a lower bound that already decides the (strict <) test.
__global__ void pair_distance_kernel(int n_frag, FragTab ft, const double* __restrict__ xyz,
                                     const double* __restrict__ bounds, double cut,
                                     double* __restrict__ rmin) {
  const long long npair = (long long)n_frag * (n_frag - 1) / 2;
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long e = warp; e < npair; e += nwarps) {
    // pair index -> (I, J): rows I hold n-1-I entries
    long long I = 0, base = 0;
    {
      // solve base(I) = I*(2n - I - 1)/2 <= e
      double nn = double(n_frag);
      double disc = (2 * nn - 1) * (2 * nn - 1) - 8.0 * double(e);
      I = (long long)((2 * nn - 1 - sqrt(fmax(disc, 0.0))) * 0.5);
      if (I < 0) I = 0;
      while (I > 0 && I * (2 * n_frag - I - 1) / 2 > e) --I;
      while ((I + 1) * (2 * n_frag - I - 2) / 2 <= e) ++I;
      base = I * (2 * n_frag - I - 1) / 2;
    }
    const int J = int(I + 1 + (e - base));
    const double cdx = bounds[4 * I] - bounds[4 * J], cdy = bounds[4 * I + 1] - bounds[4 * J + 1],
                 cdz = bounds[4 * I + 2] - bounds[4 * J + 2];
    const double gap = sqrt(cdx * cdx + cdy * cdy + cdz * cdz) - bounds[4 * I + 3] - bounds[4 * J + 3];
    if (gap >= cut) {
      if (lane == 0) rmin[e] = gap;
      continue;
    }
    const int a0 = ft.atom0[I], na = ft.nat[I], b0 = ft.atom0[J], nb = ft.nat[J];
    double best = 1e300;
    for (int k = lane; k < na * nb; k += 32) {
      const int a = a0 + k / nb, b = b0 + k % nb;
      if (ft.ghost_frag && (ft.ghost_frag[a] >= 0 || ft.ghost_frag[b] >= 0)) continue;   // ghosts are not atoms
      const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                   dz = xyz[3 * a + 2] - xyz[3 * b + 2];
      best = fmin(best, dx * dx + dy * dy + dz * dz);
    }
    best = -warp_max(-best);
    if (lane == 0) rmin[e] = sqrt(best);
  }
}

// ES-DIM pair energies (Eq. 15): sum_{mu in I, nu in J} gamma dq_I dq_J.
__global__ void esdim_kernel(int n_pairs, const int2* __restrict__ pairs, const long long* __restrict__ out_idx,
                             FragTab ft, const double* __restrict__ xyz, const int* __restrict__ sh_atom,
                             const double* __restrict__ sh_inv_eta, const double* __restrict__ dq,
                             GParams g, double* __restrict__ out, const double* __restrict__ gam_full,
                             int n_sh) {
  __shared__ double red[32];
  for (int p = blockIdx.x; p < n_pairs; p += gridDim.x) {
    const int I = pairs[p].x, J = pairs[p].y;
    const int s0 = ft.sh0[I], ns = ft.nsh[I], t0 = ft.sh0[J], nt = ft.nsh[J];
    double acc = 0.0;
    for (int k = threadIdx.x; k < ns * nt; k += blockDim.x) {
      const int mu = s0 + k / nt, nu = t0 + k % nt;
      if (gam_full) {   // the stored gamma of all shell pairs: the same values
        acc += gam_full[(size_t)mu * n_sh + nu] * dq[mu] * dq[nu];
        continue;
      }
      const int a = sh_atom[mu], b = sh_atom[nu];
      const double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                   dz = xyz[3 * a + 2] - xyz[3 * b + 2];
      acc += gamma_fn(dx * dx + dy * dy + dz * dz, sh_inv_eta[mu], sh_inv_eta[nu], g.k_g) * dq[mu] * dq[nu];
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) out[out_idx[p]] = acc;
    __syncthreads();
  }
}

// Neumaier-compensated sum of one thread's strided subset, then a fixed tree.
__device__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}

// Global monomer loop: one modified-Broyden step (Johnson 1988) on the
// concatenated shell charges of all monomers.  x = current input (updated in
// place), xo = the monomers' output charges, e = monomer energies.  Decides
// convergence on the device: max |xo - x| < tol and |E1 - E1_prev| < etol
// (E1 = sum of monomer energies, fixed order); then x <- xo.  One block.
struct MixState {
  double e_prev, diff, e1;
  int have_prev, hcount, hhead, converged, count;
  double gram[kHist * kHist];   // dF_k . dF_l by history slot (each pair formed once)
};

__global__ void __launch_bounds__(1024) global_mix_kernel(int n, double* __restrict__ x, const double* __restrict__ xo, int nf,
                                  const double* __restrict__ e, double* __restrict__ hist, MixState* st,
                                  double alpha, double w0, double tol, double etol, int allow_converge) {
  __shared__ double red[32];
  __shared__ double sa[kHist * kHist + 2 * kHist];
  double* dF = hist;
  double* U = hist + (size_t)kHist * n;
  double* px = hist + (size_t)2 * kHist * n;
  double* pF = px + n;
  double dm = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dm = nan_max(dm, fabs(xo[i] - x[i]));
  dm = block_max(dm, red);
  double es = 0.0, ec = 0.0;
  for (int i = threadIdx.x; i < nf; i += blockDim.x) neumaier_add(es, ec, e[i]);
  const double e1 = block_sum(es + ec, red);
  const int conv = allow_converge && st->have_prev && dm < tol && fabs(e1 - st->e_prev) < etol;
  __syncthreads();
  if (threadIdx.x == 0) { st->diff = dm; st->e1 = e1; st->converged = conv; st->e_prev = e1; st->have_prev = 1; }
  if (conv) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = xo[i];
    return;
  }
  int hcount = st->hcount, hhead = st->hhead;
  const int step = st->count;
  int new_slot = -1;   // history slot written in this step
  if (step > 0) {
    double nn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double d = (xo[i] - x[i]) - pF[i];
      nn += d * d;
    }
    const double norm = sqrt(block_sum(nn, red));
    if (norm > 0.0) {
      const int slot = (hhead + hcount) % kHist;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = ((xo[i] - x[i]) - pF[i]) / norm;
        dF[(size_t)slot * n + i] = d;
        U[(size_t)slot * n + i] = alpha * d + (x[i] - px[i]) / norm;
      }
      if (hcount < kHist) ++hcount; else hhead = (hhead + 1) % kHist;
      new_slot = slot;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) { px[i] = x[i]; pF[i] = xo[i] - x[i]; }
  __syncthreads();
  const int m = hcount;
  double* a = sa;
  double* c = sa + kHist * kHist;
  double* gv = c + kHist;
  {
    // dot products, one warp each (fixed order: deterministic): c_k = dF_k . F
    // for every history vector, and dF_new . dF_k for the vector written in this
    // step; the other Gram entries are kept in the state from earlier steps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nd = m + (new_slot >= 0 ? m : 0);
    for (int q = wid; q < nd; q += nw) {
      const int k = (hhead + (q % m)) % kHist;
      const double* va = dF + (size_t)k * n;
      const double* vb = (q < m) ? pF : dF + (size_t)new_slot * n;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      int i = lane;
      for (; i + 96 < n; i += 128) {
        s0 = fma(va[i], vb[i], s0);
        s1 = fma(va[i + 32], vb[i + 32], s1);
        s2 = fma(va[i + 64], vb[i + 64], s2);
        s3 = fma(va[i + 96], vb[i + 96], s3);
      }
      for (; i < n; i += 32) s0 = fma(va[i], vb[i], s0);
      const double v = warp_sum((s0 + s1) + (s2 + s3));
      if (lane == 0) {
        if (q < m) {
          c[q] = v;
        } else {
          st->gram[new_slot * kHist + k] = v;
          st->gram[k * kHist + new_slot] = v;
        }
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
      const int k = (hhead + q / m) % kHist, l = (hhead + q % m) % kHist;
      a[q] = st->gram[k * kHist + l];
    }
  }
  __syncthreads();
  if (threadIdx.x < 32 && m > 0) warp_gj_solve(m, a, c, w0 * w0, gv);   // (w0^2 I + a) g = c
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double v = x[i] + alpha * (xo[i] - x[i]);
    for (int k = 0; k < m; ++k) v -= gv[k] * U[(size_t)((hhead + k) % kHist) * n + i];
    x[i] = v;
  }
  if (threadIdx.x == 0) { st->hcount = hcount; st->hhead = hhead; st->count = step + 1; }
}

// max |a - b| over a vector (single block).
__global__ void maxdiff_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                               double* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = nan_max(m, fabs(a[i] - b[i]));
  m = block_max(m, red);
  if (threadIdx.x == 0) *out = m;
}


__device__ double block_sum_compensated(double s, double c, double* red) {
  // combine (s + c) pairs with a fixed-shape tree
  const double v = s + c;
  return block_sum(v, red);
}

// FMO sums (Eqs. 12-19).  One block; fixed summation order.
//   dE_pair[p]      in: ES-DIM values for ES-DIM pairs; out: dE_IJ for all pairs
//   pair_scc[p]     index of the pair in the SCC-dimer pass or -1
__global__ void fmo_sum_kernel(int n_frag, const double* __restrict__ e_mono, long long n_pair,
                               const int* __restrict__ pair_scc, const double* __restrict__ e_dim,
                               const double* __restrict__ dEV_dim, double* __restrict__ dE_pair,
                               int n_tri, const int* __restrict__ tri_frag, const double* __restrict__ e_tri,
                               const double* __restrict__ dEV_tri, double* __restrict__ dE3,
                               double* __restrict__ corr, double* __restrict__ totals) {
  __shared__ double red[32];
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < n_frag; i += blockDim.x) neumaier_add(s, c, e_mono[i]);
  const double e1 = block_sum_compensated(s, c, red);
  s = 0.0; c = 0.0;
  for (long long p = threadIdx.x; p < n_pair; p += blockDim.x) {
    // (I, J) of the lexicographic pair index
    double nn = double(n_frag);
    long long I = (long long)((2 * nn - 1 - sqrt(fmax((2 * nn - 1) * (2 * nn - 1) - 8.0 * double(p), 0.0))) * 0.5);
    if (I < 0) I = 0;
    while (I > 0 && I * (2 * n_frag - I - 1) / 2 > p) --I;
    while ((I + 1) * (2 * n_frag - I - 2) / 2 <= p) ++I;
    const long long J = I + 1 + (p - I * (2 * n_frag - I - 1) / 2);
    const int k = pair_scc[p];
    double d;
    if (k >= 0) d = e_dim[k] - e_mono[I] - e_mono[J] + dEV_dim[k];   // Eq. 12
    else d = dE_pair[p];                                             // Eq. 15
    dE_pair[p] = d;
    neumaier_add(s, c, d);
  }
  const double e2 = e1 + block_sum_compensated(s, c, red);
  __syncthreads();
  s = 0.0; c = 0.0;
  for (int t = threadIdx.x; t < n_tri; t += blockDim.x) {
    const int I = tri_frag[3 * t], J = tri_frag[3 * t + 1], K = tri_frag[3 * t + 2];
    const double d3 = e_tri[t] - e_mono[I] - e_mono[J] - e_mono[K] + dEV_tri[t];   // Eq. 17
    auto pidx = [&](long long a, long long b) { return a * (2 * n_frag - a - 1) / 2 + (b - a - 1); };
    const double cr = d3 - dE_pair[pidx(I, J)] - dE_pair[pidx(I, K)] - dE_pair[pidx(J, K)];  // Eq. 16
    dE3[t] = d3;
    corr[t] = cr;
    neumaier_add(s, c, cr);
  }
  const double e3c = block_sum_compensated(s, c, red);
  if (threadIdx.x == 0) {
    totals[0] = e1;
    totals[1] = e2;
    totals[2] = e2 + e3c;
  }
}

// Reorder coordinates from input atom order to the internal order.
__global__ void gather_xyz_kernel(int n_atoms, const int* __restrict__ perm, const double* __restrict__ in,
                                  double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_atoms) return;
  const int s = perm[i];
  out[3 * i] = in[3 * s];
  out[3 * i + 1] = in[3 * s + 1];
  out[3 * i + 2] = in[3 * s + 2];
}

// ---------------------------------------------------------------------------
// launch wrappers

// every kernel launch of the library goes through a launch_* wrapper and is
// followed by exactly one LAUNCH_CHECK, which also counts it
static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

#define LAUNCH_CHECK()                                   \
  do {                                                   \
    g_launches.fetch_add(1, std::memory_order_relaxed);  \
    cudaError_t e_ = cudaGetLastError();                 \
    if (e_ != cudaSuccess) return e_;                    \
  } while (0)

cudaError_t launch_cn(cudaStream_t st, int n_atoms, const double* xyz, const int* elem, const DevElem* el,
                      GParams g, double* cn, const int* ghost_src) {
  cn_kernel<<<(int)(((long long)n_atoms * 32 + 255) / 256), 256, 0, st>>>(n_atoms, xyz, elem, el, g, ghost_src, cn);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_integrals(cudaStream_t st, int n_nmer, int max_pairs, const Nmer* nmers, FragTab ft,
                             const double* xyz, const int* elem, const int* atom_sh0, const double* cn,
                             const DevElem* el, const double* kab, int ne, GParams g, double* S, double* H0,
                             const Nmer* mono, const double* mono_S, const double* mono_H0, const PrimPair* prim) {
  if (n_nmer == 0) return cudaSuccess;
  const int chunks = max(1, min(64, (max_pairs + 127) / 128));
  for (int b0 = 0; b0 < n_nmer; b0 += 65535) {
    dim3 grid(chunks, min(65535, n_nmer - b0));
    integrals_kernel<<<grid, 128, 0, st>>>(nmers + b0, ft, xyz, elem, atom_sh0, cn, el, kab, ne, g, S, H0, mono,
                                           mono_S, mono_H0, prim);
    LAUNCH_CHECK();
  }
  return cudaSuccess;
}

cudaError_t launch_gamma(cudaStream_t st, int n_nmer, int max_nsh, const Nmer* nmers, FragTab ft,
                         const double* xyz, const int* elem, const int* sh_atom, const double* sh_inv_eta,
                         GParams g, double* gam) {
  if (n_nmer == 0) return cudaSuccess;
  const int chunks = max(1, min(64, (max_nsh * max_nsh + 255) / 256));
  for (int b0 = 0; b0 < n_nmer; b0 += 65535) {
    dim3 grid(chunks, min(65535, n_nmer - b0));
    gamma_kernel<<<grid, 256, 0, st>>>(nmers + b0, ft, xyz, elem, sh_atom, sh_inv_eta, g, gam);
    LAUNCH_CHECK();
  }
  return cudaSuccess;
}

static size_t lowdin_smem(int max_n, int elem_bytes, int a_in_smem) {
  const int npad = max_n + (max_n & 1);
  size_t b = 0;
  if (a_in_smem) b += (size_t)elem_bytes * npad * npad;
  b += sizeof(double) * kGemmSmemElems + sizeof(double) * 32 + sizeof(double) * npad + 3 * sizeof(int) * npad;
  b = (b + 15) & ~size_t(15);
  b += 2 * (size_t)elem_bytes * npad + 16;
  return b;
}

cudaError_t launch_lowdin(cudaStream_t st, int n_nmer, int max_n, const Nmer* nmers, const double* S,
                          void* CT, void* W, void* Ag, int use_float, int a_in_smem, int* status, void* W2) {
  if (n_nmer == 0) return cudaSuccess;
  if (use_float) {
    const size_t sb = lowdin_smem(max_n, 4, a_in_smem);
    cudaFuncSetAttribute(lowdin_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    lowdin_kernel<float><<<n_nmer, kBlock, sb, st>>>(nmers, S, (float*)CT, (float*)W, (float*)Ag, a_in_smem,
                                                     1e-7, status, (float*)W2);
  } else {
    const size_t sb = lowdin_smem(max_n, 8, a_in_smem);
    cudaFuncSetAttribute(lowdin_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    lowdin_kernel<double><<<n_nmer, kBlock, sb, st>>>(nmers, S, (double*)CT, (double*)W, (double*)Ag,
                                                      a_in_smem, 1e-14, status, nullptr);
  }
  LAUNCH_CHECK();
  return cudaSuccess;
}

size_t scc_smem_size(int max_n, int max_nsh, int max_nat, int a_bytes) {
  return scc_smem_bytes(max_n, max_nsh, max_nat, a_bytes);
}

cudaError_t launch_scc(cudaStream_t st, int n_nmer, const SccLaunch& L) {
  if (n_nmer == 0) return cudaSuccess;
  SccArgs ar;
  ar.nmers = L.nmers; ar.order = L.order; ar.ft = L.ft; ar.xyz = L.xyz; ar.elem = L.elem;
  ar.atom_sh0 = L.atom_sh0; ar.el = L.el; ar.g = L.g; ar.S = L.S; ar.H0 = L.H0; ar.gam = L.gam;
  ar.CTd = L.CTd; ar.W1d = L.W1d; ar.W2d = L.W2d; ar.Agd = L.Agd;
  ar.CTf = L.CTf; ar.W1f = L.W1f; ar.W2f = L.W2f; ar.Agf = L.Agf;
  ar.phi = L.phi; ar.vhop = L.vhop; ar.dq_mono = L.dq_mono;
  ar.hop_Qd = L.hop_Qd; ar.hop_Qf = L.hop_Qf; ar.hop_Dd = L.hop_Dd; ar.hop_Df = L.hop_Df; ar.hop_nq = L.hop_nq; ar.esp = L.esp; ar.dq = L.dq; ar.eps = L.eps; ar.hist = L.hist;
  ar.energy = L.energy; ar.e_el = L.e_el; ar.e_rep = L.e_rep; ar.dEV = L.dEV; ar.iters = L.iters; ar.iters32 = L.iters32;
  ar.status = L.status; ar.guess_from_mono = L.guess_from_mono; ar.precision = L.precision;
  ar.max_iter = L.max_iter; ar.fp32_cap = L.fp32_cap;
  ar.single_step = L.single_step; ar.step_phase = L.step_phase; ar.reortho = L.reortho;
  ar.cold_refine = L.cold_refine; ar.reortho32 = L.reortho32; ar.step_dev = L.step_dev; ar.jac_hint = L.jac_hint; ar.jac_hint_dev = L.jac_hint_dev; ar.S32 = L.S32; ar.H32 = L.H32; ar.trace = L.trace;
  ar.fp64_finish = L.fp64_finish; ar.energy_finish = L.energy_finish; ar.first_jac_tol = L.first_jac_tol; ar.cold_steps = L.cold_steps; ar.first_rot = L.first_rot; ar.tol = L.tol; ar.etol = L.etol;
  ar.switch_tol = L.switch_tol; ar.jacobi_tol_d = L.jacobi_tol_d; ar.jacobi_tol_f = L.jacobi_tol_f;
  ar.t0 = L.t0; ar.budget_ns = L.budget_ns; ar.a_smem_d = L.a_smem_d; ar.a_smem_f = L.a_smem_f;
  ar.max_n = L.max_n; ar.max_nsh = L.max_nsh; ar.max_nat = L.max_nat;
  const int npad = L.max_n + (L.max_n & 1);
  const int a_bytes = (L.a_smem_d ? 8 : (L.a_smem_f ? 4 : 0)) * npad * npad;
  size_t sb = scc_smem_bytes(L.max_n, L.max_nsh, L.max_nat, a_bytes);
  // FP32 iterations of n-mers (no FP64 matrix in shared memory): the rest of
  // the shared memory holds the tridiagonal eigen-solver's vectors and as
  // many packed rows of its trailing matrix as fit.  With the eigen-solve
  // matrix in global memory two CTAs share an SM (each gets half of the SM's
  // shared memory).
  ar.tri_cap = 0;
  const bool two = L.ctas_per_sm == 2 ||
                   (L.ctas_per_sm == 0 && L.precision == 1 && a_bytes == 0 && L.max_n >= kTriMinN);
  if (L.precision == 1 && !L.a_smem_d && L.max_n >= kTriMinN && L.max_n <= 512) {
    int dev = 0, optin = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaFuncAttributes fa{};
    if (two) cudaFuncGetAttributes(&fa, scc_kernel<2>);
    else cudaFuncGetAttributes(&fa, scc_kernel<1>);
    // per CTA: dynamic + static + 1 KB reserved by the runtime
    const long long budget = two ? std::min<long long>(optin, per_sm / 2 - 1024) : optin;
    const long long room = budget - (long long)fa.sharedSizeBytes - (long long)sb - 1024;
    const long long want = (long long)npad * (npad + 1) / 2;
    const long long cap = std::min(want, room / 4 - tri_vec_floats(npad));
    if (cap > 0) {
      ar.tri_cap = int(cap);
      sb += sizeof(float) * ((size_t)tri_vec_floats(npad) + (size_t)cap);
    }
  }
  if (two) {
    cudaError_t e = cudaFuncSetAttribute(scc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e != cudaSuccess) return e;
    scc_kernel<2><<<n_nmer, kBlock, sb, st>>>(ar);
  } else {
    cudaError_t e = cudaFuncSetAttribute(scc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e != cudaSuccess) return e;
    scc_kernel<1><<<n_nmer, kBlock, sb, st>>>(ar);
  }
  LAUNCH_CHECK();
  return cudaSuccess;
}

// Source-shell chunking of the phi kernel: enough blocks for 4 per SM.
int phi_chunks(int n_sh) {
  const int mu_blocks = (n_sh + 255) / 256;
  const int want = (4 * 148 + mu_blocks - 1) / mu_blocks;
  return std::max(1, std::min(want, (n_sh + 255) / 256));
}

cudaError_t launch_warm_start(cudaStream_t st, int n_nmer, const Nmer* nmers, const Nmer* mono, const float* mono_ct,
                              float* ct) {
  if (n_nmer == 0) return cudaSuccess;
  warm_start_kernel<<<n_nmer, 256, 0, st>>>(nmers, mono, mono_ct, ct);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_phi(cudaStream_t st, int n_sh, const double* xyz, const int* sh_atom, const double* sh_inv_eta,
                       const double* dq, GParams g, double* phi, double* part, int use_float) {
  const int nc = phi_chunks(n_sh);
  const int chunk = (((n_sh + nc - 1) / nc) + 255) / 256 * 256;
  const int ncu = (n_sh + chunk - 1) / chunk;
  const dim3 grid((n_sh + 255) / 256, ncu);
  if (use_float) phi_kernel<float><<<grid, 256, 0, st>>>(n_sh, chunk, xyz, sh_atom, sh_inv_eta, dq, g, part);
  else phi_kernel<double><<<grid, 256, 0, st>>>(n_sh, chunk, xyz, sh_atom, sh_inv_eta, dq, g, part);
  LAUNCH_CHECK();
  phi_reduce_kernel<<<(n_sh + 255) / 256, 256, 0, st>>>(n_sh, ncu, part, phi);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_gamma_full(cudaStream_t st, int n_sh, const double* xyz, const int* sh_atom,
                              const double* sh_inv_eta, GParams g, double* gam) {
  if (n_sh == 0) return cudaSuccess;
  const dim3 grid((n_sh + 255) / 256, std::min(n_sh, 4096));
  gamma_full_kernel<<<grid, 256, 0, st>>>(n_sh, xyz, sh_atom, sh_inv_eta, g, gam);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_phi_gemv(cudaStream_t st, int n_sh, const double* gam, const double* dq, double* phi) {
  if (n_sh == 0) return cudaSuccess;
  phi_gemv_kernel<<<(int)(((long long)n_sh * 32 + 255) / 256), 256, 0, st>>>(n_sh, gam, dq, phi);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_hop_projector(cudaStream_t st, int n_nmer, const Nmer* nmers, FragTab ft, const double* xyz,
                                 const int* elem, const DevElem* el, double v_hop, const double* S, double* V,
                                 double* Qd, float* Qf, double* Dd, float* Df, int* nq) {
  if (n_nmer == 0) return cudaSuccess;
  hop_projector_kernel<<<n_nmer, 256, 0, st>>>(nmers, ft, xyz, elem, el, v_hop, S, V, Qd, Qf, Dd, Df, nq);
  LAUNCH_CHECK();
  return cudaSuccess;
}

// Device-side control of the monomer loop inside a CUDA graph: counts the
// step and keeps the graph's while node running until the global mixer
// reports convergence, a NaN residual or the step limit.
__global__ void loop_control_kernel(cudaGraphConditionalHandle handle, const MixState* st, int* outer,
                                    int max_outer) {
  const int o = ++*outer;
  const bool more = !st->converged && st->diff == st->diff && o < max_outer;
  cudaGraphSetConditional(handle, more ? 1u : 0u);
}

// The FP32 steps' bookkeeping of the host-driven loop, in the same order: stop
// on convergence or NaN; otherwise track the best residual and end the FP32
// phase at the switch tolerance, the step cap or kStall32 steps without a
// 10% improvement; continue while none of these and steps remain.
__global__ void loop_control32_kernel(cudaGraphConditionalHandle handle, const MixState* st, Phase32State* p,
                                      int* outer, int max_outer, double switch_tol, int cap32, int stall_limit) {
  const int o = ++*outer;
  const double d = st->diff;
  const bool stop = st->converged || !(d == d);
  bool hand = false;
  if (!stop) {
    if (d < 0.9 * p->min32) { p->min32 = d; p->stall32 = 0; } else { ++p->stall32; }
    hand = d < switch_tol || ++p->n32 >= cap32 || p->stall32 >= stall_limit;
  }
  p->hand_over = hand ? 1 : 0;
  cudaGraphSetConditional(handle, (!stop && !hand && o < max_outer) ? 1u : 0u);
}

cudaError_t launch_loop_control32(cudaStream_t st, unsigned long long handle, const void* mix_state,
                                  Phase32State* p32, int* outer, int max_outer, double switch_tol, int cap32,
                                  int stall_limit) {
  loop_control32_kernel<<<1, 1, 0, st>>>((cudaGraphConditionalHandle)handle, (const MixState*)mix_state, p32, outer,
                                         max_outer, switch_tol, cap32, stall_limit);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_loop_control(cudaStream_t st, unsigned long long handle, const void* mix_state, int* outer,
                                int max_outer) {
  loop_control_kernel<<<1, 1, 0, st>>>((cudaGraphConditionalHandle)handle, (const MixState*)mix_state, outer,
                                       max_outer);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_frag_bounds(cudaStream_t st, int n_frag, FragTab ft, const double* xyz, double* bounds) {
  frag_bounds_kernel<<<(n_frag + 127) / 128, 128, 0, st>>>(n_frag, ft, xyz, bounds);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_pair_distance(cudaStream_t st, int n_frag, FragTab ft, const double* xyz, const double* bounds,
                                 double cut, double* rmin) {
  const long long npair = (long long)n_frag * (n_frag - 1) / 2;
  if (npair == 0) return cudaSuccess;
  const long long warps = npair;
  const int blocks = (int)std::min<long long>((warps * 32 + 255) / 256, 148LL * 64);
  pair_distance_kernel<<<blocks, 256, 0, st>>>(n_frag, ft, xyz, bounds, cut, rmin);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_esdim(cudaStream_t st, int n_pairs, const int2* pairs, const long long* out_idx, FragTab ft,
                         const double* xyz, const int* sh_atom, const double* sh_inv_eta, const double* dq,
                         GParams g, double* out, const double* gam_full, int n_sh) {
  if (n_pairs == 0) return cudaSuccess;
  const int blocks = std::min(n_pairs, 148 * 16);
  esdim_kernel<<<blocks, 256, 0, st>>>(n_pairs, pairs, out_idx, ft, xyz, sh_atom, sh_inv_eta, dq, g, out, gam_full,
                                       n_sh);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_global_mix(cudaStream_t st, int n, double* x, const double* xo, int nf, const double* e,
                              double* hist, void* state, double tol, double etol, int allow_converge) {
  global_mix_kernel<<<1, 1024, 0, st>>>(n, x, xo, nf, e, hist, (MixState*)state, 0.4, 0.01, tol, etol,
                                         allow_converge);
  LAUNCH_CHECK();
  return cudaSuccess;
}

size_t mix_state_bytes() { return sizeof(MixState); }

cudaError_t launch_maxdiff(cudaStream_t st, int n, const double* a, const double* b, double* out) {
  maxdiff_kernel<<<1, 1024, 0, st>>>(n, a, b, out);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_fmo_sum(cudaStream_t st, int n_frag, const double* e_mono, long long n_pair, const int* pair_scc,
                           const double* e_dim, const double* dEV_dim, double* dE_pair, int n_tri,
                           const int* tri_frag, const double* e_tri, const double* dEV_tri, double* dE3,
                           double* corr, double* totals) {
  fmo_sum_kernel<<<1, 1024, 0, st>>>(n_frag, e_mono, n_pair, pair_scc, e_dim, dEV_dim, dE_pair, n_tri, tri_frag,
                                      e_tri, dEV_tri, dE3, corr, totals);
  LAUNCH_CHECK();
  return cudaSuccess;
}

__global__ void stamp_kernel(unsigned long long* t) { *t = globaltimer_ns(); }

// out[i] = in[i] rounded to FP32 (grid-stride)
__global__ void __launch_bounds__(256) to_float_kernel(long long n, const double* __restrict__ in,
                                                       float* __restrict__ out) {
  for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
    out[i] = float(in[i]);
}

cudaError_t launch_to_float(cudaStream_t st, long long n, const double* in, float* out) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((n + 255) / 256, 148LL * 16);
  to_float_kernel<<<int(blocks), 256, 0, st>>>(n, in, out);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_stamp(cudaStream_t st, unsigned long long* t) {
  stamp_kernel<<<1, 1, 0, st>>>(t);
  LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_gather_xyz(cudaStream_t st, int n_atoms, const int* perm, const double* in, double* out) {
  gather_xyz_kernel<<<(n_atoms + 255) / 256, 256, 0, st>>>(n_atoms, perm, in, out);
  LAUNCH_CHECK();
  return cudaSuccess;
}

}  // namespace fmo
