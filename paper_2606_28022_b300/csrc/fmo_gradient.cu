// Analytic nuclear gradient of the FMO1/FMO2/FMO3 energy on the GPU (Sec. 2.4
// of the paper: the GFN1-xTB energy gradient of Eqs. 23-28 as the building
// block, the explicit FMO terms, and the response of the monomer charges).
//
// With L_X = E'_X + esp_X . dq_X stationary in the density of n-mer X (its
// ESP fixed), the FMO energy is
//   sum_I c_I E'_I + sum_X m_X [L_X - esp_X . (monomer charges of X)]
//   + sum over ES-DIM pairs dq_I Gamma_IJ dq_J,
// c_I and m_X counting the FMO2/FMO3 subtractions (Eqs. 12, 16).  Its
// gradient is
//   (1) per term: the explicit single-system gradient of its converged
//       density with the ESP inside the shell shifts and the energy-weighted
//       density, times its coefficient (kernel grad_explicit_kernel);
//   (2) the charge-transfer part of dE^V (Eq. 13): ddq^X . dGamma . dq_K over
//       fragments K outside X, and the ES-DIM pairs (Eq. 15);
//   (3) every term linear in the derivatives of the monomer charges collects
//       into one charge-space vector w; the Z-vector z = (1 - Gamma chi)^-1 w
//       (chi: the monomers' coupled-perturbed susceptibilities) gives the
//       response z . dQ/dxi|_esp + (chi z)^T dGamma dq, the first part being
//       the explicit gradient along the first-order density of each monomer
//       in the potential z_I.
// The supersystem coordination numbers couple all terms through
// sum_A F_A dCN_A (Eqs. 26-28), applied once to the summed F_A.
//
// The paper writes its self-consistent Z-vector equations in orbital space
// (one n_vir x n_occ block per fragment); fragments interact only through
// their shell charges, so each orbital Hessian folds into the n_sh x n_sh
// susceptibility chi_I and the Z-vector has one entry per shell.
//
// Deterministic: every per-term result goes to its own slots and is summed in
// a fixed order per fragment; every reduction has a fixed order.
#include <cstdio>

#include "fmo_device.cuh"
#include "kernels.h"

namespace fmo {

namespace {

__host__ __device__ inline size_t a16(size_t b) { return (b + 15) & ~size_t(15); }

// local index maps of a term (no cut bonds: its fragments' atoms in order)
struct GradMaps {
  int* at_glob;    // [nat] global atom
  int* at_fk;      // [nat] fragment slot (0..nfrag-1) within the n-mer
  int* sh_at;      // [nsh] local atom
  int* sh_k;       // [nsh] shell index within the element
  int* sh_glob;    // [nsh] global shell
  int* sh_ao0;     // [nsh + 1] first local AO
  int* ao_sh;      // [n] local shell
};

__host__ __device__ inline size_t maps_bytes(int n, int nsh, int nat) {
  return 2 * a16(sizeof(int) * nat) + 3 * a16(sizeof(int) * nsh) + a16(sizeof(int) * (nsh + 1)) +
         a16(sizeof(int) * n);
}

__device__ GradMaps carve_maps(unsigned char*& p, int n, int nsh, int nat) {
  GradMaps m;
  auto take = [&](size_t b) { unsigned char* r = p; p += a16(b); return reinterpret_cast<int*>(r); };
  m.at_glob = take(sizeof(int) * nat);
  m.at_fk = take(sizeof(int) * nat);
  m.sh_at = take(sizeof(int) * nsh);
  m.sh_k = take(sizeof(int) * nsh);
  m.sh_glob = take(sizeof(int) * nsh);
  m.sh_ao0 = take(sizeof(int) * (nsh + 1));
  m.ao_sh = take(sizeof(int) * n);
  return m;
}

__device__ void build_grad_maps(const Nmer& nm, const GradLaunch& L, GradMaps mp) {
  if (threadIdx.x == 0) {
    int la = 0, ls = 0, lao = 0;
    for (int k = 0; k < nm.nfrag; ++k) {
      const int f = nm.frag[k];
      for (int i = 0; i < L.ft.nat[f]; ++i) {
        const int ga = L.ft.atom0[f] + i;
        mp.at_glob[la] = ga;
        mp.at_fk[la] = k;
        const DevElem& e = L.el[L.elem[ga]];
        for (int s = 0; s < e.nsh; ++s) {
          mp.sh_at[ls] = la;
          mp.sh_k[ls] = s;
          mp.sh_glob[ls] = L.atom_sh0[ga] + s;
          mp.sh_ao0[ls] = lao;
          for (int q = 0; q < 2 * e.l[s] + 1; ++q) mp.ao_sh[lao++] = ls;
          ++ls;
        }
        ++la;
      }
    }
    mp.sh_ao0[ls] = lao;
  }
  __syncthreads();
}

// Fermi level of Eq. 6 by bisection on sum f = N over the orbital energies
// eps[0..n) (warp 0; result in *ef_out, visible after the caller's barrier).
__device__ void fermi_level(int n, const double* eps, double nel, double kT, double* ef_out) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  double lo = 1e300, hi = -1e300;
  for (int i = lane; i < n; i += 32) { lo = fmin(lo, eps[i]); hi = fmax(hi, eps[i]); }
  lo = -warp_max(-lo) - 50.0 * kT - 1.0;
  hi = warp_max(hi) + 50.0 * kT + 1.0;
  double ef = 0.5 * (lo + hi);
  for (int it = 0; it < 400; ++it) {
    ef = 0.5 * (lo + hi);
    double t = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double x = fmin(fmax((eps[i] - ef) / kT, -700.0), 700.0);
      t += 2.0 / (exp(x) + 1.0);
    }
    t = warp_sum(t);
    if (fabs(t - nel) < 1e-13 || hi - lo < 1e-15) break;
    if (t > nel) hi = ef; else lo = ef;
  }
  if (lane == 0) *ef_out = ef;
}

// x^(-1/2) in FP64 from the FP32 estimate and one third-order correction
// (relative error O(r^3), r = 1 - x y0^2 ~ 1e-7).
__device__ __forceinline__ double rsqrt_d(double x) {
  const double y0 = (double)rsqrtf((float)x);
  const double r = fma(-x, y0 * y0, 1.0);
  return fma(y0 * r, fma(0.375, r, 0.5), y0);
}

// d gamma / dR of Eq. 4 (gamma = (R^kg + (1/eta)^kg)^(-1/kg), 1/eta the mean
// of the two shells' 1/eta), divided by R: dgamma/dR = R * dgr.
__device__ __forceinline__ double dgamma_over_r(double r2, double ie, double kg) {
  if (kg == 2.0) {
    const double gm = rsqrt_d(r2 + ie * ie);
    return -gm * gm * gm;
  }
  const double r = sqrt(r2);
  const double gm = pow(pow(r, kg) + pow(ie, kg), -1.0 / kg);
  return -pow(r, kg - 2.0) * pow(gm, kg + 1.0);
}

}  // namespace

// ---------------------------------------------------------------------------
// Energy terms: occupations f from the stored orbital energies (Eq. 6), shell
// shifts sigma = gamma dq - Gamma_A dq_A^2 + ESP (Eq. 7 with Eq. 21), density
// P = sum_k f_k c_k c_k^T and energy-weighted density W~ = sum_k f_k e_k c_k
// c_k^T (Eq. 24).  With every occupation 2 or 0 (to 1e-10) the SCC's rotation
// updates leave the occupied and the empty orbitals unresolved among
// themselves; there W~ = 1/2 P F P = 2 C_o^T (C_o F C_o^T) C_o, invariant to
// those rotations, with F = H0 + 1/2 S (sigma_mu + sigma_nu).  With
// fractional occupations the SCC diagonalises every iteration, so the rows
// are canonical and the sums are taken as they stand.

__global__ void __launch_bounds__(kBlock) grad_prep_kernel(const GradTerm* __restrict__ terms, GradLaunch L,
                                                           int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTerm t = terms[blockIdx.x];
  const Nmer& nm = t.nm;
  const int n = nm.n, nsh = nm.nsh, nat = nm.nat;
  unsigned char* sp = smem_raw;
  GradMaps mp = carve_maps(sp, L.max_n, L.max_nsh, L.max_nat);
  auto takeD = [&](size_t k) { double* r = reinterpret_cast<double*>(sp); sp += a16(sizeof(double) * k); return r; };
  double* gemm = takeD(kGemmSmemElems);
  double* red = takeD(32);
  double* focc = takeD(L.max_n);
  double* fs = takeD(L.max_n);     // scale of each listed row: 2, or f (P) / f e (W~)
  double* dqat = takeD(L.max_nat);
  double* sig = takeD(L.max_nsh);
  int* occ = reinterpret_cast<int*>(sp);
  __shared__ double s_ef;
  __shared__ int s_no;
  (void)red;
  (void)flag;
  build_grad_maps(nm, L, mp);
  fermi_level(n, t.eps, nm.nel, L.g.kT, &s_ef);
  __syncthreads();
  int frac = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = fmin(fmax((t.eps[i] - s_ef) / L.g.kT, -700.0), 700.0);
    focc[i] = 2.0 / (exp(x) + 1.0);
    frac |= (focc[i] > 1e-10 && focc[i] < 2.0 - 1e-10);
  }
  const bool integer = !__syncthreads_or(frac);
  if (threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < n; ++i)
      if (integer ? focc[i] > 1.0 : focc[i] > 1e-30) occ[k++] = i;
    s_no = k;
    for (int a = 0; a < nat; ++a) dqat[a] = 0.0;
    for (int s = 0; s < nsh; ++s) dqat[mp.sh_at[s]] += t.dq[s];
  }
  __syncthreads();
  const int no = s_no;
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double v = 0.0;
      for (int u = lane; u < nsh; u += 32) v += t.gam[(size_t)s * nsh + u] * t.dq[u];
      v = warp_sum(v);
      if (lane == 0) {
        const int a = mp.sh_at[s];
        const double g3 = L.el[L.elem[mp.at_glob[a]]].gamma3;
        sig[s] = v - g3 * dqat[a] * dqat[a] + (t.esp ? t.esp[s] : 0.0);
        t.sa[s] = sig[s];
      }
    }
  }
  for (int k = threadIdx.x; k < no; k += blockDim.x) fs[k] = integer ? 2.0 : focc[occ[k]];
  __syncthreads();
  if (!integer) {
    // canonical rows: P = sum f c c^T, W~ = sum f e c c^T
    block_gemm<double>(n, n, no, t.CT, 1, n, t.CT, 1, n, t.Pa, n, occ, occ, fs, gemm);
    for (int k = threadIdx.x; k < no; k += blockDim.x) fs[k] = focc[occ[k]] * t.eps[occ[k]];
    __syncthreads();
    block_gemm<double>(n, n, no, t.CT, 1, n, t.CT, 1, n, t.W, n, occ, occ, fs, gemm);
    return;
  }
  double* Co = t.work;                       // no x n
  double* F = t.work + (size_t)n * n;        // n x n
  double* E = t.work + 2 * (size_t)n * n;    // no x n: C_o F, then G = A_oo C_o
  double* Aoo = t.work + 3 * (size_t)n * n;  // no x no
  for (long long e = threadIdx.x; e < (long long)no * n; e += blockDim.x) {
    const int i = int(e / n), j = int(e - (long long)i * n);
    Co[e] = t.CT[(long long)occ[i] * n + j];
  }
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = int(e / n), j = int(e - (long long)i * n);
    F[e] = t.H0[e] + 0.5 * t.S[e] * (sig[mp.ao_sh[i]] + sig[mp.ao_sh[j]]);
  }
  __syncthreads();
  block_gemm<double>(n, n, no, Co, 1, n, Co, 1, n, t.Pa, n, nullptr, nullptr, fs, gemm);       // P = 2 C_o^T C_o
  block_gemm<double>(no, n, n, Co, n, 1, F, n, 1, E, n, nullptr, nullptr, nullptr, gemm);      // C_o F
  block_gemm<double>(no, no, n, E, n, 1, Co, n, 1, Aoo, no, nullptr, nullptr, nullptr, gemm);  // C_o F C_o^T
  block_gemm<double>(no, n, no, Aoo, no, 1, Co, 1, n, E, n, nullptr, nullptr, nullptr, gemm);  // A_oo C_o
  block_gemm<double>(n, n, no, Co, 1, n, E, 1, n, t.W, n, nullptr, nullptr, fs, gemm);         // 2 C_o^T G
}

// ---------------------------------------------------------------------------
// Explicit gradient of one term (Eqs. 23-28 at fixed density), one CTA per
// term, one warp per atom A over its partners B in the n-mer:
//   sum dS_mu,nu M_mu,nu with M = Pa (Hp + 1/2 (sa_mu + sa_nu))
//       + Pb 1/2 (sb_mu + sb_nu) - W   (H0 = Hp S off the atom blocks),
//   Pa S dHp/dR through the distance polynomial Pi (Eq. 9),
//   1/2 sum Q_st dgamma_st with Q = qa qb^T + qb qa^T (qa = dq; qb = dq/2 for
//       energy terms, the first-order charges for response terms),
//   the repulsion (Eq. 11) for energy terms,
//   F_A = dE/dCN_A (Eq. 28, applied later with the supersystem CN gradient);
// for n-mer terms also the charge-transfer part of dE^V inside the n-mer,
// -sum over shell pairs of different fragments (ddq_s q_t + q_s ddq_t) dgamma,
// and for SCC dimers at level >= 2 (coefficient es) the removal of their pair
// from the all-pairs ES-DIM sum, -q_I dGamma_IJ q_J.  Shell slots (energy
// terms): the term's part of the Z-vector right-hand side w and of the
// charge-transfer vector d (see the file head).

__global__ void __launch_bounds__(kBlock) grad_explicit_kernel(const GradTerm* __restrict__ terms, GradLaunch L,
                                                               double* __restrict__ aslots,
                                                               double* __restrict__ sslots) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTerm t = terms[blockIdx.x];
  const Nmer& nm = t.nm;
  const int n = nm.n, nsh = nm.nsh, nat = nm.nat;
  unsigned char* sp = smem_raw;
  GradMaps mp = carve_maps(sp, L.max_n, L.max_nsh, L.max_nat);
  auto takeD = [&](size_t k) { double* r = reinterpret_cast<double*>(sp); sp += a16(sizeof(double) * k); return r; };
  double* qa = takeD(L.max_nsh);
  double* qb = takeD(L.max_nsh);
  double* qm = takeD(L.max_nsh);
  double* ddq = takeD(L.max_nsh);
  double* sa = takeD(L.max_nsh);
  double* sb = takeD(L.max_nsh);
  build_grad_maps(nm, L, mp);
  const bool nmer = (t.kind == kGradNmer);
  for (int s = threadIdx.x; s < nsh; s += blockDim.x) {
    const double d = t.dq[s];
    qa[s] = d;
    qb[s] = t.qb ? t.qb[s] : 0.5 * d;
    qm[s] = L.dq_mono[mp.sh_glob[s]];
    ddq[s] = nmer ? d - qm[s] : 0.0;
    sa[s] = t.sa[s];
    sb[s] = t.sb ? t.sb[s] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // shell slots: w = -m esp - m gamma ddq - es (gamma q_mono over the other
  // fragment), d = m ddq
  if (t.kind != kGradResponse) {
    for (int s = wid; s < nsh; s += nw) {
      double v1 = 0.0, v2 = 0.0;
      const int fs = mp.at_fk[mp.sh_at[s]];
      for (int u = lane; u < nsh; u += 32) {
        const double gsu = t.gam[(size_t)s * nsh + u];
        v1 += gsu * ddq[u];
        if (mp.at_fk[mp.sh_at[u]] != fs) v2 += gsu * qm[u];
      }
      v1 = warp_sum(v1);
      v2 = warp_sum(v2);
      if (lane == 0) {
        const double w = -t.m * (t.esp ? t.esp[s] : 0.0) - t.m * v1 - t.es * v2;
        sslots[t.sslot + 2 * s] = w;
        sslots[t.sslot + 2 * s + 1] = t.m * ddq[s];
      }
    }
  }
  const double* Pa = t.Pa;
  const double* W = t.W;
  const double* Pb = t.Pb;
  const double* Sm = t.S;
  // per atom A: a warp, lanes over the partners B
  for (int A = wid; A < nat; A += nw) {
    const int ga = mp.at_glob[A];
    const int ea = L.elem[ga];
    const DevElem& EA = L.el[ea];
    const int fA = mp.at_fk[A];
    int sA0 = 0;
    while (sA0 < nsh && mp.sh_at[sA0] != A) ++sA0;
    double g0 = 0.0, g1 = 0.0, g2 = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0, fcn = 0.0;
    for (int B = lane; B < nat; B += 32) {
      if (B == A) continue;
      const int gb = mp.at_glob[B];
      const int eb = L.elem[gb];
      const DevElem& EB = L.el[eb];
      const bool cross = mp.at_fk[B] != fA;
      int sB0 = 0;
      while (sB0 < nsh && mp.sh_at[sB0] != B) ++sB0;
      const double R[3] = {L.xyz[3 * ga] - L.xyz[3 * gb], L.xyz[3 * ga + 1] - L.xyz[3 * gb + 1],
                           L.xyz[3 * ga + 2] - L.xyz[3 * gb + 2]};
      const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
      const double rr = sqrt(r2);
      const double u[3] = {R[0] / rr, R[1] / rr, R[2] / rr};
      if (t.with_rep) {   // repulsion (Eq. 11)
        const double al = sqrt(EA.arep * EB.arep);
        const double ex = exp(-al * pow(rr, L.g.k_f));
        const double de = EA.zeff * EB.zeff * ex * (-1.0 / r2 - al * L.g.k_f * pow(rr, L.g.k_f - 2.0));
        g0 += de * u[0]; g1 += de * u[1]; g2 += de * u[2];
      }
      // Coulomb kernel at fixed charges
      for (int ka = 0; ka < EA.nsh; ++ka) {
        for (int kb = 0; kb < EB.nsh; ++kb) {
          const int s = sA0 + ka, v = sB0 + kb;
          const double ie = 0.5 * (1.0 / EA.eta_sh[ka] + 1.0 / EB.eta_sh[kb]);
          const double dgr = dgamma_over_r(r2, ie, L.g.k_g);
          double wm = qa[s] * qb[v] + qb[s] * qa[v];
          double we = 0.0;
          if (cross) {
            wm -= ddq[s] * qm[v] + ddq[v] * qm[s];
            we = -qm[s] * qm[v];
          }
          g0 += wm * dgr * R[0]; g1 += wm * dgr * R[1]; g2 += wm * dgr * R[2];
          e0 += we * dgr * R[0]; e1 += we * dgr * R[1]; e2 += we * dgr * R[2];
        }
      }
      // H0 prefactors (Eq. 8) and the distance polynomial Pi (Eq. 9)
      const double den = EA.en - EB.en;
      const double fen = 1.0 + L.g.k_en * den * den;
      const double kAB = L.kab[ea * L.ne + eb];
      const double rcov = EA.rcov + EB.rcov;
      const double x = sqrt(rr / rcov);
      const double dxdR = x / (2.0 * rr);
      for (int s_a = 0; s_a < EA.nsh; ++s_a) {
        const int la = EA.l[s_a];
        const int shA = sA0 + s_a;
        const double hA = EA.h[s_a] * (1.0 + EA.kcn[s_a] * L.cn[ga]);
        for (int s_b = 0; s_b < EB.nsh; ++s_b) {
          const int lb = EB.l[s_b];
          const int shB = sB0 + s_b;
          const double hB = EB.h[s_b] * (1.0 + EB.kcn[s_b] * L.cn[gb]);
          const double kll = 0.5 * (L.g.k_l[la] + L.g.k_l[lb]);
          const double Pi = (1.0 + EA.kpoly[s_a] * x) * (1.0 + EB.kpoly[s_b] * x);
          const double dPi = EA.kpoly[s_a] * (1.0 + EB.kpoly[s_b] * x) + EB.kpoly[s_b] * (1.0 + EA.kpoly[s_a] * x);
          const double Hp = kAB * kll * 0.5 * (hA + hB) * fen * Pi;
          const double cPi = kAB * kll * 0.5 * (hA + hB) * fen * dPi * dxdR;
          const double cCN = kAB * kll * fen * Pi * EA.h[s_a] * EA.kcn[s_a];
          const double shift_a = 0.5 * (sa[shA] + sa[shB]);
          const double shift_b = 0.5 * (sb[shA] + sb[shB]);
          // primitive sums of the overlap derivative (closed form of the s/p
          // Gaussian overlap, R = A - B)
          double T1 = 0, B0 = 0, B1 = 0, A0 = 0, A1 = 0, Q0 = 0, Q1 = 0, H1 = 0;
          for (int pa = 0; pa < EA.nprim[s_a]; ++pa) {
            for (int pb = 0; pb < EB.nprim[s_b]; ++pb) {
              const PrimPair q = L.prim[prim_pair_index(L.ne, ea, eb, s_a, s_b, pa, pb)];
              const double xe = q.abp * r2;
              if (xe > 46.0) continue;   // exp(-xe) < 1e-20
              const double s00 = q.pref * exp(-xe);
              const double ms = q.abp * s00;
              T1 += ms;
              B0 += q.bp * s00; B1 += q.bp * ms;
              A0 += q.ap * s00; A1 += q.ap * ms;
              const double qq = q.ap * q.bp;
              Q0 += qq * s00; Q1 += qq * ms;
              H1 += 0.5 * q.ip * ms;
            }
          }
          const int nu_ = 2 * la + 1, nv_ = 2 * lb + 1;
          for (int uu = 0; uu < nu_; ++uu) {
            for (int vv = 0; vv < nv_; ++vv) {
              const long long mu = mp.sh_ao0[shA] + uu, nu = mp.sh_ao0[shB] + vv;
              const long long e = mu * n + nu;
              const double p = Pa[e];
              const double sv = Sm[e];
              double M = p * (Hp + shift_a) - W[e];
              if (Pb) M += Pb[e] * shift_b;
              double d[3];
              for (int c = 0; c < 3; ++c) {
                if (la == 0 && lb == 0) d[c] = -2.0 * R[c] * T1;
                else if (la == 1 && lb == 0) d[c] = -(uu == c ? B0 : 0.0) + 2.0 * R[uu] * R[c] * B1;
                else if (la == 0 && lb == 1) d[c] = (vv == c ? A0 : 0.0) - 2.0 * R[vv] * R[c] * A1;
                else
                  d[c] = -((uu == c ? R[vv] : 0.0) + (vv == c ? R[uu] : 0.0)) * Q0 + 2.0 * R[c] * R[uu] * R[vv] * Q1 -
                         (uu == vv ? 2.0 * R[c] * H1 : 0.0);
              }
              const double pp = 2.0 * p * sv * cPi;
              g0 += 2.0 * M * d[0] + pp * u[0];
              g1 += 2.0 * M * d[1] + pp * u[1];
              g2 += 2.0 * M * d[2] + pp * u[2];
              fcn += p * sv * cCN;
            }
          }
        }
      }
    }
    g0 = warp_sum(g0); g1 = warp_sum(g1); g2 = warp_sum(g2);
    e0 = warp_sum(e0); e1 = warp_sum(e1); e2 = warp_sum(e2);
    fcn = warp_sum(fcn);
    if (lane == 0) {
      // on-site levels: d h_A^l / d CN_A (Eq. 10)
      for (int k = 0; k < EA.nsh; ++k)
        for (int mu = mp.sh_ao0[sA0 + k]; mu < mp.sh_ao0[sA0 + k + 1]; ++mu)
          fcn += Pa[(long long)mu * n + mu] * EA.h[k] * EA.kcn[k];
      double* o = aslots + t.aslot + 4 * (long long)A;
      o[0] = t.m * g0 + t.es * e0;
      o[1] = t.m * g1 + t.es * e1;
      o[2] = t.m * g2 + t.es * e2;
      o[3] = t.m * fcn;
    }
  }
}

// Per global atom and shell, the slots of every term holding its fragment,
// summed in term order: g_atom[a][0..3] (+)= (g, F), w[s] (+)= w, d[s] (+)= d.
__global__ void grad_gather_kernel(int n_frag, FragTab ft, int n_atoms, int n_sh, const int* __restrict__ atom_frag,
                                   const int* __restrict__ sh_frag, const int* __restrict__ frag_ptr,
                                   const long long* __restrict__ ent_aoff, const long long* __restrict__ ent_soff,
                                   const double* __restrict__ aslots, const double* __restrict__ sslots,
                                   double* __restrict__ g_atom, double* __restrict__ w, double* __restrict__ d,
                                   int accumulate) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_atoms) {
    const int f = atom_frag[i];
    const int li = i - ft.atom0[f];
    double acc[4] = {0, 0, 0, 0};
    for (int e = frag_ptr[f]; e < frag_ptr[f + 1]; ++e) {
      const double* s = aslots + ent_aoff[e] + 4 * (long long)li;
      for (int c = 0; c < 4; ++c) acc[c] += s[c];
    }
    for (int c = 0; c < 4; ++c) g_atom[4 * (long long)i + c] = (accumulate ? g_atom[4 * (long long)i + c] : 0.0) + acc[c];
  }
  if (sslots && i < n_sh) {
    const int f = sh_frag[i];
    const int ls = i - ft.sh0[f];
    double aw = 0.0, ad = 0.0;
    for (int e = frag_ptr[f]; e < frag_ptr[f + 1]; ++e) {
      if (ent_soff[e] < 0) continue;
      aw += sslots[ent_soff[e] + 2 * (long long)ls];
      ad += sslots[ent_soff[e] + 2 * (long long)ls + 1];
    }
    w[i] = (accumulate ? w[i] : 0.0) + aw;
    d[i] = (accumulate ? d[i] : 0.0) + ad;
  }
}

// ---------------------------------------------------------------------------
// Monomer response data.  Per monomer at its converged charges q and ESP:
//   1. shifts sigma and Fock matrix F; canonical orbitals by Jacobi on
//      C F C^T from the run's rows (the SCC's rotation updates leave the
//      occupied and empty blocks undiagonalised) and Fermi occupations f;
//   2. bare response at fixed shifts (first-order perturbation theory with
//      Fermi occupations): for a unit potential on shell s,
//      dF = 1/2 S (delta_s(mu) + delta_s(nu)), and with
//      B^t_ij = sum_{mu in t} (c_i,mu (S c_j)_mu + c_j,mu (S c_i)_mu),
//      chi0[t][s] = 1/4 sum_{i,j} M_ij B^t_ij B^s_ij
//                   - u_t u_s / sum_k f'_k,  u_t = 1/2 sum_k f'_k B^t_kk,
//      M_ij = (f_i - f_j) / (e_i - e_j) (f'_i = df/de for equal energies),
//      the last term the shift of the Fermi level that keeps the electron
//      count; pairs of two full or two empty orbitals have M = 0 and are
//      skipped;
//   3. chi = (1 - chi0 K)^-1 chi0 with the charge kernel of the shifts
//      K = gamma - 2 Gamma_A dq_A on the shells of atom A (Eq. 7), by
//      Gauss-Jordan elimination with partial pivoting.

__device__ __forceinline__ double charge_kernel(const double* gam, int nsh, int s, int u, const GradMaps& mp,
                                                const double* g3dq) {
  double k = gam[(size_t)s * nsh + u];
  if (mp.sh_at[s] == mp.sh_at[u]) k -= 2.0 * g3dq[mp.sh_at[s]];
  return k;
}

// M_ij of the first-order density response, for i != j
__device__ __forceinline__ double resp_m(double fi, double fj, double ei, double ej, double fpi, double fpj) {
  const double de = ei - ej;
  return fabs(de) > 1e-12 ? (fi - fj) / de : 0.5 * (fpi + fpj);
}

constexpr int kChiChunk = 32;
constexpr double kFullTol = 1e-13;   // occupations within this of 2 (0) count as full (empty)

__global__ void __launch_bounds__(kBlock) grad_mono_response_kernel(const GradTerm* __restrict__ terms,
                                                                    MonoResp* __restrict__ mr, GradLaunch L,
                                                                    int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTerm t = terms[blockIdx.x];
  const MonoResp R = mr[blockIdx.x];
  const Nmer& nm = t.nm;
  const int n = nm.n, nsh = nm.nsh, nat = nm.nat, npad = nm.npad;
  unsigned char* sp = smem_raw;
  GradMaps mp = carve_maps(sp, L.max_n, L.max_nsh, L.max_nat);
  auto takeD = [&](size_t k) { double* r = reinterpret_cast<double*>(sp); sp += a16(sizeof(double) * k); return r; };
  auto takeI = [&](size_t k) { int* r = reinterpret_cast<int*>(sp); sp += a16(sizeof(int) * k); return r; };
  double* gemm = takeD(kGemmSmemElems);
  double* red = takeD(32);
  double* dqat = takeD(L.max_nat);
  double* g3dq = takeD(L.max_nat);
  double* sig = takeD(L.max_nsh);
  double* eps = takeD(L.max_n + 1);
  double* focc = takeD(L.max_n + 1);
  double* hm = takeD(kChiChunk);
  double* Bc = takeD((size_t)L.max_nsh * kChiChunk);
  double* fac = takeD(2 * L.max_nsh);
  int* order = takeI(L.max_n + 1);
  JacobiScratch<double> js;
  js.p = takeI(L.max_n + 2);
  js.q = takeI(L.max_n + 2);
  js.act = takeI(L.max_n + 2);
  js.c = takeD(L.max_n + 2);
  js.s = takeD(L.max_n + 2);
  __shared__ double s_ef, s_sfp;
  __shared__ int s_nf, s_np, s_piv;
  build_grad_maps(nm, L, mp);
  double* F = R.work;                                // n x n
  double* U = F + (size_t)n * n;                     // n x n (C F, then S C)
  double* Cw = U + (size_t)n * n;                    // n x n working rows
  double* A = Cw + (size_t)n * n;                    // npad x npad
  double* chi0 = A + (size_t)npad * npad;            // nsh x nsh
  double* aug = chi0 + (size_t)nsh * nsh;            // nsh x 2 nsh
  // 1. shifts and Fock matrix at the converged charges
  if (threadIdx.x == 0) {
    for (int a = 0; a < nat; ++a) dqat[a] = 0.0;
    for (int s = 0; s < nsh; ++s) dqat[mp.sh_at[s]] += t.dq[s];
    for (int a = 0; a < nat; ++a) g3dq[a] = L.el[L.elem[mp.at_glob[a]]].gamma3 * dqat[a];
  }
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double v = 0.0;
      for (int u = lane; u < nsh; u += 32) v += t.gam[(size_t)s * nsh + u] * t.dq[u];
      v = warp_sum(v);
      if (lane == 0) {
        const int a = mp.sh_at[s];
        sig[s] = v - g3dq[a] * dqat[a] + t.esp[s];
        R.sig[s] = sig[s];
      }
    }
  }
  __syncthreads();
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = int(e / n), j = int(e - (long long)i * n);
    F[e] = t.H0[e] + 0.5 * t.S[e] * (sig[mp.ao_sh[i]] + sig[mp.ao_sh[j]]);
    Cw[e] = t.CT[e];
  }
  __syncthreads();
  block_gemm<double>(n, n, n, Cw, n, 1, F, n, 1, U, n, nullptr, nullptr, nullptr, gemm);      // C F
  block_gemm<double>(n, n, n, U, n, 1, Cw, n, 1, A, npad, nullptr, nullptr, nullptr, gemm);   // C F C^T
  if (n != npad) {
    for (int i = threadIdx.x; i < npad; i += blockDim.x) { A[(long long)i * npad + n] = 0.0; A[(long long)n * npad + i] = 0.0; }
  }
  __syncthreads();
  const int sw = block_jacobi<double>(A, npad, n, Cw, n, n, 1e-14, 80, js, red);
  if (sw < 0 && threadIdx.x == 0) atomicOr(flag, 2);
  for (int i = threadIdx.x; i < n; i += blockDim.x) eps[i] = A[(long long)i * npad + i];
  __syncthreads();
  fermi_level(n, eps, nm.nel, L.g.kT, &s_ef);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = fmin(fmax((eps[i] - s_ef) / L.g.kT, -700.0), 700.0);
    focc[i] = 2.0 / (exp(x) + 1.0);
    R.eps[i] = eps[i];
    R.focc[i] = focc[i];
  }
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) R.C[e] = Cw[e];
  __syncthreads();
  if (threadIdx.x == 0) {   // rows by class: full, partial, empty (each in index order)
    int k = 0;
    for (int i = 0; i < n; ++i) if (focc[i] > 2.0 - kFullTol) order[k++] = i;
    const int nf = k;
    for (int i = 0; i < n; ++i) if (focc[i] <= 2.0 - kFullTol && focc[i] >= kFullTol) order[k++] = i;
    s_np = k - nf;
    s_nf = nf;
    for (int i = 0; i < n; ++i) if (focc[i] < kFullTol) order[k++] = i;
    double sfp = 0.0;
    for (int i = 0; i < n; ++i) sfp += -2.0 * (0.5 * focc[i]) * (1.0 - 0.5 * focc[i]) / L.g.kT;
    s_sfp = sfp;
  }
  __syncthreads();
  const double* C = R.C;
  const int nF = s_nf, nP = s_np;
  const int nlo = nF + nP, nhi = n - nF;     // rows i: full or partial; rows j: partial or empty
  const double kT = L.g.kT;
  // 2. bare response chi0 over the pairs (i, j) with M_ij != 0
  block_gemm<double>(n, n, n, C, n, 1, t.S, n, 1, U, n, nullptr, nullptr, nullptr, gemm);   // rows (S c_i)^T
  for (int e = threadIdx.x; e < nsh * nsh; e += blockDim.x) chi0[e] = 0.0;
  __syncthreads();
  const long long n_pair = (long long)nlo * nhi;
  for (long long p0 = 0; p0 < n_pair; p0 += kChiChunk) {
    for (int c = threadIdx.x; c < kChiChunk; c += blockDim.x) {
      const long long p = p0 + c;
      double h = 0.0;
      if (p < n_pair) {
        const int x = int(p / nhi), y = int(p - (long long)(p / nhi) * nhi);
        const int i = order[x], j = order[nF + y];
        const double fpi = -2.0 * (0.5 * focc[i]) * (1.0 - 0.5 * focc[i]) / kT;
        const double fpj = -2.0 * (0.5 * focc[j]) * (1.0 - 0.5 * focc[j]) / kT;
        if (x >= nF && y < nP) {             // two partial orbitals: each pair once
          const int xp = x - nF;
          if (xp == y) h = 0.25 * fpi;       // 1/4 M_ii, with B_ii counted once
          else if (xp < y) h = 0.5 * resp_m(focc[i], focc[j], eps[i], eps[j], fpi, fpj);
        } else {
          h = 0.5 * resp_m(focc[i], focc[j], eps[i], eps[j], fpi, fpj);
        }
      }
      hm[c] = h;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nsh * kChiChunk; e += blockDim.x) {
      const int s = e / kChiChunk, c = e - s * kChiChunk;
      const long long p = p0 + c;
      double b = 0.0;
      if (p < n_pair && hm[c] != 0.0) {
        const int x = int(p / nhi), y = int(p - (long long)(p / nhi) * nhi);
        const int i = order[x], j = order[nF + y];
        for (int mu = mp.sh_ao0[s]; mu < mp.sh_ao0[s + 1]; ++mu)
          b += C[(long long)i * n + mu] * U[(long long)j * n + mu] + C[(long long)j * n + mu] * U[(long long)i * n + mu];
      }
      Bc[s * kChiChunk + c] = b;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nsh * nsh; e += blockDim.x) {
      const int a_ = e / nsh, b_ = e - a_ * nsh;
      double acc = 0.0;
#pragma unroll 8
      for (int c = 0; c < kChiChunk; ++c) acc += hm[c] * Bc[a_ * kChiChunk + c] * Bc[b_ * kChiChunk + c];
      chi0[e] += acc;
    }
    __syncthreads();
  }
  // Fermi-level shift: chi0 -= u u^T / sum f', u_t = sum_k f'_k (c_k S c_k on t)
  if (nP > 0 && s_sfp != 0.0) {
    for (int s = threadIdx.x; s < nsh; s += blockDim.x) {
      double u = 0.0;
      for (int x = nF; x < nF + nP; ++x) {
        const int k = order[x];
        const double fpk = -2.0 * (0.5 * focc[k]) * (1.0 - 0.5 * focc[k]) / kT;
        double bkk = 0.0;
        for (int mu = mp.sh_ao0[s]; mu < mp.sh_ao0[s + 1]; ++mu) bkk += C[(long long)k * n + mu] * U[(long long)k * n + mu];
        u += fpk * bkk;
      }
      fac[s] = u;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nsh * nsh; e += blockDim.x) {
      const int a_ = e / nsh, b_ = e - a_ * nsh;
      chi0[e] -= fac[a_] * fac[b_] / s_sfp;
    }
    __syncthreads();
  }
  // 3. [1 - chi0 K | chi0] -> [1 | chi]
  for (int e = threadIdx.x; e < nsh * nsh; e += blockDim.x) {
    const int r = e / nsh, c = e - r * nsh;
    double v = 0.0;
    for (int u = 0; u < nsh; ++u) v += chi0[(size_t)r * nsh + u] * charge_kernel(t.gam, nsh, u, c, mp, g3dq);
    aug[(size_t)r * 2 * nsh + c] = (r == c ? 1.0 : 0.0) - v;
    aug[(size_t)r * 2 * nsh + nsh + c] = chi0[e];
  }
  __syncthreads();
  const int w2 = 2 * nsh;
  for (int col = 0; col < nsh; ++col) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = col;
      for (int r = col + threadIdx.x; r < nsh; r += 32) {
        const double v = fabs(aug[(size_t)r * w2 + col]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) s_piv = bi;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != col) {
      for (int j = threadIdx.x; j < w2; j += blockDim.x) {
        const double a = aug[(size_t)col * w2 + j];
        aug[(size_t)col * w2 + j] = aug[(size_t)piv * w2 + j];
        aug[(size_t)piv * w2 + j] = a;
      }
      __syncthreads();
    }
    const double pv = aug[(size_t)col * w2 + col];
    __syncthreads();
    for (int j = threadIdx.x; j < w2; j += blockDim.x) aug[(size_t)col * w2 + j] /= pv;
    for (int r = threadIdx.x; r < nsh; r += blockDim.x) fac[r] = aug[(size_t)r * w2 + col];
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)nsh * w2; e += blockDim.x) {
      const int r = int(e / w2), j = int(e - (long long)r * w2);
      if (r == col) continue;
      aug[e] -= fac[r] * aug[(size_t)col * w2 + j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nsh * nsh; e += blockDim.x) {
    const int r = e / nsh, c = e - r * nsh;
    R.chi[e] = aug[(size_t)r * w2 + nsh + c];
  }
}

// y = chi z, block by block (one block per monomer, one warp per row).
__global__ void chi_apply_kernel(const GradTerm* __restrict__ terms, const MonoResp* __restrict__ mr,
                                 const double* __restrict__ z, double* __restrict__ y, const int* __restrict__ sh0) {
  const int I = blockIdx.x;
  const int nsh = terms[I].nm.nsh, s0 = sh0[I];
  const double* chi = mr[I].chi;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = wid; r < nsh; r += nw) {
    double v = 0.0;
    for (int c = lane; c < nsh; c += 32) v += chi[(size_t)r * nsh + c] * z[s0 + c];
    v = warp_sum(v);
    if (lane == 0) y[s0 + r] = v;
  }
}

// out = intra-fragment part of gamma v (the monomers' own gamma blocks).
__global__ void intra_gamma_kernel(const GradTerm* __restrict__ terms, const double* __restrict__ v,
                                   double* __restrict__ out, const int* __restrict__ sh0) {
  const int I = blockIdx.x;
  const int nsh = terms[I].nm.nsh, s0 = sh0[I];
  const double* gam = terms[I].gam;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = wid; r < nsh; r += nw) {
    double a = 0.0;
    for (int c = lane; c < nsh; c += 32) a += gam[(size_t)r * nsh + c] * v[s0 + c];
    a = warp_sum(a);
    if (lane == 0) out[s0 + r] = a;
  }
}

// out[j] = V_j . u for j < k (one block per j, fixed-order reduction).
__global__ void vec_dots_kernel(int n, const double* __restrict__ V, long long ldv, const double* __restrict__ u,
                                double* __restrict__ out) {
  __shared__ double red[32];
  const double* v = V + (long long)blockIdx.x * ldv;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * u[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// u -= sum_j h_j V_j (fixed order in j).
__global__ void vec_update_kernel(int n, int k, const double* __restrict__ V, long long ldv,
                                  const double* __restrict__ h, double* __restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = u[i];
  for (int j = 0; j < k; ++j) v -= h[j] * V[(long long)j * ldv + i];
  u[i] = v;
}

__global__ void vec_lincomb_kernel(int n, double a, const double* __restrict__ x, double b,
                                   const double* __restrict__ y, double c, const double* __restrict__ z,
                                   double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = a * x[i];
  if (y) v += b * y[i];
  if (z) v += c * z[i];
  out[i] = v;
}

// ---------------------------------------------------------------------------
// First-order change of each monomer under the potential z_I (coupled-
// perturbed SCC with Fermi occupations): dq1 = (chi z)_I (given), shifts
// dsigma = K dq1 + z_I, dF = 1/2 S (dsigma_mu + dsigma_nu), and in the
// canonical orbitals C (rows), D = C dF C^T,
//   dP  = C^T X C,  X_ij = M_ij D_ij - delta_ij f'_i de_F,
//   dW~ = C^T Y C,  Y_ij = N_ij D_ij - delta_ij f'_i e_i de_F,
// M_ij = (f_i - f_j)/(e_i - e_j), N_ij = (f_i e_i - f_j e_j)/(e_i - e_j)
// (their derivative limits for equal energies), de_F = sum f'_k D_kk /
// sum f'_k the Fermi-level shift.  Fills the response term: Pa = dP,
// W = dW~, Pb = P = C^T diag(f) C, sb = dsigma.

__global__ void __launch_bounds__(kBlock) grad_first_order_kernel(const GradTerm* __restrict__ terms,
                                                                  const MonoResp* __restrict__ mr, GradLaunch L,
                                                                  const double* __restrict__ z,
                                                                  const double* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GradTerm t = terms[blockIdx.x];
  const MonoResp R = mr[blockIdx.x];
  const Nmer& nm = t.nm;
  const int n = nm.n, nsh = nm.nsh, nat = nm.nat;
  unsigned char* sp = smem_raw;
  GradMaps mp = carve_maps(sp, L.max_n, L.max_nsh, L.max_nat);
  auto takeD = [&](size_t k) { double* r = reinterpret_cast<double*>(sp); sp += a16(sizeof(double) * k); return r; };
  double* gemm = takeD(kGemmSmemElems);
  double* red = takeD(32);
  double* dqat = takeD(L.max_nat);
  double* g3dq = takeD(L.max_nat);
  double* ds = takeD(L.max_nsh);
  double* fp = takeD(L.max_n);
  build_grad_maps(nm, L, mp);
  const int s0 = mp.sh_glob[0];
  const double kT = L.g.kT;
  if (threadIdx.x == 0) {
    for (int a = 0; a < nat; ++a) dqat[a] = 0.0;
    for (int s = 0; s < nsh; ++s) dqat[mp.sh_at[s]] += t.dq[s];
    for (int a = 0; a < nat; ++a) g3dq[a] = L.el[L.elem[mp.at_glob[a]]].gamma3 * dqat[a];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) fp[i] = -2.0 * (0.5 * R.focc[i]) * (1.0 - 0.5 * R.focc[i]) / kT;
  __syncthreads();
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double v = 0.0;
      for (int u = lane; u < nsh; u += 32) v += charge_kernel(t.gam, nsh, s, u, mp, g3dq) * y[s0 + u];
      v = warp_sum(v);
      if (lane == 0) {
        ds[s] = v + z[s0 + s];
        const_cast<double*>(t.sb)[s] = ds[s];
      }
    }
  }
  __syncthreads();
  const double* C = R.C;
  const double* E = R.eps;
  const double* f = R.focc;
  double* dF = R.work;                 // n x n
  double* T = dF + (size_t)n * n;      // C dF, then Y
  double* D = T + (size_t)n * n;       // D, then X
  double* U = D + (size_t)n * n;       // X C, then Y C
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = int(e / n), j = int(e - (long long)i * n);
    dF[e] = 0.5 * t.S[e] * (ds[mp.ao_sh[i]] + ds[mp.ao_sh[j]]);
  }
  __syncthreads();
  block_gemm<double>(n, n, n, C, n, 1, dF, n, 1, T, n, nullptr, nullptr, nullptr, gemm);   // C dF
  block_gemm<double>(n, n, n, T, n, 1, C, n, 1, D, n, nullptr, nullptr, nullptr, gemm);    // C dF C^T
  double sfp = 0.0, sfd = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { sfp += fp[i]; sfd += fp[i] * D[(long long)i * n + i]; }
  sfp = block_sum(sfp, red);
  sfd = block_sum(sfd, red);
  const double def = sfp != 0.0 ? sfd / sfp : 0.0;
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = int(e / n), j = int(e - (long long)i * n);
    const double d = D[e];
    double x, yv;
    if (i == j) {
      x = fp[i] * d - fp[i] * def;
      yv = (fp[i] * E[i] + f[i]) * d - fp[i] * E[i] * def;
    } else if (fabs(E[i] - E[j]) > 1e-12) {
      x = (f[i] - f[j]) / (E[i] - E[j]) * d;
      yv = (f[i] * E[i] - f[j] * E[j]) / (E[i] - E[j]) * d;
    } else {
      x = 0.5 * (fp[i] + fp[j]) * d;
      yv = 0.5 * (fp[i] * E[i] + f[i] + fp[j] * E[j] + f[j]) * d;
    }
    T[e] = yv;
    D[e] = x;
  }
  __syncthreads();
  block_gemm<double>(n, n, n, D, n, 1, C, 1, n, U, n, nullptr, nullptr, nullptr, gemm);    // X C
  block_gemm<double>(n, n, n, C, 1, n, U, 1, n, t.Pa, n, nullptr, nullptr, nullptr, gemm);  // C^T X C
  block_gemm<double>(n, n, n, T, n, 1, C, 1, n, U, n, nullptr, nullptr, nullptr, gemm);    // Y C
  block_gemm<double>(n, n, n, C, 1, n, U, 1, n, t.W, n, nullptr, nullptr, nullptr, gemm);   // C^T Y C
  block_gemm<double>(n, n, n, C, 1, n, C, 1, n, const_cast<double*>(t.Pb), n, nullptr, nullptr, f, gemm);
}

// ---------------------------------------------------------------------------
// Per atom A (one warp): the coordination-number chain rule over every
// partner of the whole system, sum_B (F_A + F_B) df(R_AB)/dR_A (Eqs. 26-28;
// pairs beyond the CN cutoff are not counted), and the inter-fragment Coulomb
// sum over every shell t outside A's fragment,
// sum_{s in A} (a_s q_t + q_s a_t) dgamma_st/dR_A; plus the gathered per-term
// gradient.  grad[3 n_atoms] in the internal atom order.
__global__ void __launch_bounds__(256) grad_cn_coulomb_kernel(int n_atoms, int n_sh, GradLaunch L,
                                                              const int* __restrict__ atom_frag,
                                                              const int* __restrict__ sh_atom,
                                                              const double* __restrict__ sh_inv_eta,
                                                              const double* __restrict__ a,
                                                              const double* __restrict__ g_atom,
                                                              double* __restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int A = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (A >= n_atoms) return;
  const double xa = L.xyz[3 * A], ya = L.xyz[3 * A + 1], za = L.xyz[3 * A + 2];
  const double ra = L.el[L.elem[A]].rcov;
  const double fA = g_atom[4 * (long long)A + 3];
  const int frA = atom_frag[A];
  double g0 = 0.0, g1 = 0.0, g2 = 0.0;
  // CN chain rule
  for (int B = lane; B < n_atoms; B += 32) {
    if (B == A) continue;
    const double R0 = xa - L.xyz[3 * B], R1 = ya - L.xyz[3 * B + 1], R2 = za - L.xyz[3 * B + 2];
    const double rr = sqrt(R0 * R0 + R1 * R1 + R2 * R2);
    if (rr >= L.g.cn_cutoff) continue;
    const double rc = ra + L.el[L.elem[B]].rcov;
    const double f = 1.0 / (1.0 + exp(-L.g.cn_k1 * (L.g.cn_k2 * rc / rr - 1.0)));
    const double df = -f * (1.0 - f) * L.g.cn_k1 * L.g.cn_k2 * rc / (rr * rr);
    const double c = (fA + g_atom[4 * (long long)B + 3]) * df / rr;
    g0 += c * R0; g1 += c * R1; g2 += c * R2;
  }
  // inter-fragment Coulomb
  const int s0 = L.atom_sh0[A], ns = L.el[L.elem[A]].nsh;
  for (int k = 0; k < ns; ++k) {
    const int s = s0 + k;
    const double as = a[s], qs = L.dq_mono[s], ies = sh_inv_eta[s];
    double h0 = 0.0, h1 = 0.0, h2 = 0.0;
    for (int t = lane; t < n_sh; t += 32) {
      const int B = sh_atom[t];
      if (atom_frag[B] == frA) continue;
      const double R0 = xa - L.xyz[3 * B], R1 = ya - L.xyz[3 * B + 1], R2 = za - L.xyz[3 * B + 2];
      const double r2 = R0 * R0 + R1 * R1 + R2 * R2;
      const double ie = 0.5 * (ies + sh_inv_eta[t]);
      const double c = (as * L.dq_mono[t] + qs * a[t]) * dgamma_over_r(r2, ie, L.g.k_g);
      h0 += c * R0; h1 += c * R1; h2 += c * R2;
    }
    g0 += h0; g1 += h1; g2 += h2;
  }
  g0 = warp_sum(g0); g1 = warp_sum(g1); g2 = warp_sum(g2);
  if (lane == 0) {
    grad[3 * (long long)A] = g_atom[4 * (long long)A] + g0;
    grad[3 * (long long)A + 1] = g_atom[4 * (long long)A + 1] + g1;
    grad[3 * (long long)A + 2] = g_atom[4 * (long long)A + 2] + g2;
  }
}

// ---------------------------------------------------------------------------
// launch wrappers (every launch counted)

static size_t prep_smem(const GradLaunch& L) {
  return maps_bytes(L.max_n, L.max_nsh, L.max_nat) + a16(sizeof(double) * kGemmSmemElems) + a16(sizeof(double) * 32) +
         2 * a16(sizeof(double) * L.max_n) + a16(sizeof(double) * L.max_nat) + a16(sizeof(double) * L.max_nsh) +
         a16(sizeof(int) * L.max_n);
}

static size_t explicit_smem(const GradLaunch& L) {
  return maps_bytes(L.max_n, L.max_nsh, L.max_nat) + 6 * a16(sizeof(double) * L.max_nsh);
}

static size_t response_smem(const GradLaunch& L) {
  return maps_bytes(L.max_n, L.max_nsh, L.max_nat) + a16(sizeof(double) * kGemmSmemElems) +
         a16(sizeof(double) * 32) + 2 * a16(sizeof(double) * L.max_nat) + a16(sizeof(double) * L.max_nsh) +
         2 * a16(sizeof(double) * (L.max_n + 1)) + a16(sizeof(double) * kChiChunk) +
         a16(sizeof(double) * (size_t)L.max_nsh * kChiChunk) + a16(sizeof(double) * 2 * L.max_nsh) +
         a16(sizeof(int) * (L.max_n + 1)) + 3 * a16(sizeof(int) * (L.max_n + 2)) +
         2 * a16(sizeof(double) * (L.max_n + 2));
}

static size_t first_order_smem(const GradLaunch& L) {
  return maps_bytes(L.max_n, L.max_nsh, L.max_nat) + a16(sizeof(double) * kGemmSmemElems) +
         a16(sizeof(double) * 32) + 2 * a16(sizeof(double) * L.max_nat) + a16(sizeof(double) * L.max_nsh) +
         a16(sizeof(double) * L.max_n);
}

#define GRAD_LAUNCH_CHECK()                   \
  do {                                        \
    note_launch();                            \
    cudaError_t e_ = cudaGetLastError();      \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_grad_prep(cudaStream_t st, int n_terms, const GradTerm* terms, const GradLaunch& L, int* flag) {
  if (n_terms == 0) return cudaSuccess;
  const size_t sb = prep_smem(L);
  cudaError_t e = set_smem(grad_prep_kernel, sb);
  if (e != cudaSuccess) return e;
  grad_prep_kernel<<<n_terms, kBlock, sb, st>>>(terms, L, flag);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_grad_explicit(cudaStream_t st, int n_terms, const GradTerm* terms, const GradLaunch& L,
                                 double* aslots, double* sslots) {
  if (n_terms == 0) return cudaSuccess;
  const size_t sb = explicit_smem(L);
  cudaError_t e = set_smem(grad_explicit_kernel, sb);
  if (e != cudaSuccess) return e;
  grad_explicit_kernel<<<n_terms, kBlock, sb, st>>>(terms, L, aslots, sslots);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_grad_gather(cudaStream_t st, int n_atoms, int n_sh, const GradLaunch& L, const int* atom_frag,
                               const int* sh_frag, const int* frag_ptr, const long long* ent_aoff,
                               const long long* ent_soff, const double* aslots, const double* sslots,
                               double* g_atom, double* w, double* d, int accumulate) {
  const int nmax = n_atoms > n_sh ? n_atoms : n_sh;
  if (nmax == 0) return cudaSuccess;
  grad_gather_kernel<<<(nmax + 255) / 256, 256, 0, st>>>(0, L.ft, n_atoms, n_sh, atom_frag, sh_frag, frag_ptr,
                                                         ent_aoff, ent_soff, aslots, sslots, g_atom, w, d,
                                                         accumulate);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_grad_mono_response(cudaStream_t st, int n_mono, const GradTerm* mono_terms, MonoResp* mr,
                                      const GradLaunch& L, int* flag) {
  if (n_mono == 0) return cudaSuccess;
  const size_t sb = response_smem(L);
  cudaError_t e = set_smem(grad_mono_response_kernel, sb);
  if (e != cudaSuccess) return e;
  grad_mono_response_kernel<<<n_mono, kBlock, sb, st>>>(mono_terms, mr, L, flag);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_chi_apply(cudaStream_t st, int n_mono, const GradTerm* mono_terms, const MonoResp* mr,
                             const int* sh0, const double* z, double* y) {
  chi_apply_kernel<<<n_mono, 256, 0, st>>>(mono_terms, mr, z, y, sh0);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_intra_gamma(cudaStream_t st, int n_mono, const GradTerm* mono_terms, const int* sh0,
                               const double* v, double* out) {
  intra_gamma_kernel<<<n_mono, 256, 0, st>>>(mono_terms, v, out, sh0);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_vec_dots(cudaStream_t st, int n, int k, const double* V, long long ldv, const double* u,
                            double* out) {
  if (k <= 0) return cudaSuccess;
  vec_dots_kernel<<<k, 512, 0, st>>>(n, V, ldv, u, out);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_vec_update(cudaStream_t st, int n, int k, const double* V, long long ldv, const double* h,
                              double* u) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  vec_update_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, k, V, ldv, h, u);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_vec_lincomb3(cudaStream_t st, int n, double a, const double* x, double b, const double* y,
                                double c, const double* z, double* out) {
  if (n <= 0) return cudaSuccess;
  vec_lincomb_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, a, x, b, y, c, z, out);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_grad_first_order(cudaStream_t st, int n_mono, const GradTerm* resp_terms, const MonoResp* mr,
                                    const GradLaunch& L, const double* z, const double* y) {
  if (n_mono == 0) return cudaSuccess;
  const size_t sb = first_order_smem(L);
  cudaError_t e = set_smem(grad_first_order_kernel, sb);
  if (e != cudaSuccess) return e;
  grad_first_order_kernel<<<n_mono, kBlock, sb, st>>>(resp_terms, mr, L, z, y);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

cudaError_t launch_grad_cn_coulomb(cudaStream_t st, int n_atoms, int n_sh, const GradLaunch& L,
                                   const int* atom_frag, const int* sh_atom, const double* sh_inv_eta,
                                   const double* a, const double* g_atom, double* grad) {
  if (n_atoms == 0) return cudaSuccess;
  grad_cn_coulomb_kernel<<<(int)(((long long)n_atoms * 32 + 255) / 256), 256, 0, st>>>(
      n_atoms, n_sh, L, atom_frag, sh_atom, sh_inv_eta, a, g_atom, grad);
  GRAD_LAUNCH_CHECK();
  return cudaSuccess;
}

size_t grad_smem_max(const GradLaunch& L) {
  size_t m = prep_smem(L);
  if (explicit_smem(L) > m) m = explicit_smem(L);
  if (response_smem(L) > m) m = response_smem(L);
  if (first_order_smem(L) > m) m = first_order_smem(L);
  return m;
}

}  // namespace fmo
