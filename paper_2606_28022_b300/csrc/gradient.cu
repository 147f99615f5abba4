// Analytic nuclear gradient of the GFN1-xTB energy of one SCC system (the
// single-system building block of the gradient section, Eqs. 23-28):
//   dE = sum P dH0 + sum W dS + 1/2 sum dq dq dgamma + dE_rep
// with dH0 = H dS + S dH (Eq. 25): the S part of dH0 and the shell-shift
// and third-order parts of W (Eq. 24) contract with dS; the rest is the
// derivative of the distance polynomial Pi (Eq. 9) and of the CN-dependent
// levels (Eq. 10) through the CN gradient F_A dCN_A (Eqs. 26-28).
//
// One CTA per n-mer (here: a system that is one fragment, no hybrid-orbital
// projection), FP64 throughout:
//   1. occupations from the stored orbital energies (Fermi, Eq. 6);
//   2. P = sum_i f_i c_i c_i^T from the stored FP64 rows;
//   3. Mulliken charges of P (Eq. 3), shell shifts sigma = gamma dq -
//      Gamma_A dq_A^2, Fock matrix F = H0 + 1/2 S (sigma_mu + sigma_nu);
//   4. energy-weighted density W~ = sum_i f_i e_i c_i c_i^T = 1/2 P F P for
//      occupations of exactly 2 or 0 (P = 2 C_o^T C_o with C_o S C_o^T = 1,
//      so P F P = 4 C_o^T (C_o F C_o^T) C_o; a gap of many kT puts the
//      Fermi tails below FP64 rounding);
//   5. one thread per atom A over all partners B: the derivative of every
//      overlap block (closed form of the s/p Gaussian overlap: with R = A - B,
//      mu = ab/p, s00 = c_a c_b (pi/p)^1.5 exp(-mu R^2), PA = -(b/p) R,
//      PB = (a/p) R, each block is a few scalar sums over the primitive pairs
//      times components of R), the Pi and gamma derivatives, the repulsion,
//      and F_A = dE/dCN_A;
//   6. after a barrier, the CN gradient (F_A + F_B) f'(R_AB) R_AB/|R_AB|.
// Each atom's gradient is summed by its own thread in a fixed order.

#include "fmo_device.cuh"
#include "kernels.h"

namespace fmo {

struct GradArgs {
  const Nmer* nm;
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
  const double* S;
  const double* H0;
  const double* CT;      // FP64 rows (orbitals) of the converged solve
  const double* eps;     // their orbital energies
  const double* gam;     // nsh x nsh gamma block
  double* P;             // n x n scratch
  double* F;
  double* T;
  double* W;
  double* grad;          // [nat][3], local atom order
  int* frac;             // set to 1 if an occupation is not 2 or 0 to 1e-10
};

__global__ void __launch_bounds__(kBlock) xtb_gradient_kernel(GradArgs ar) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Nmer nm = ar.nm[0];
  const int n = nm.n, nsh = nm.nsh, nat = nm.nat;
  const int f0 = nm.frag[0];
  const int a0 = ar.ft.atom0[f0];
  unsigned char* sp = smem_raw;
  auto take = [&](size_t bytes) { unsigned char* r = sp; sp += (bytes + 15) & ~size_t(15); return (void*)r; };
  double* gemm = (double*)take(sizeof(double) * kGemmSmemElems);
  double* red = (double*)take(sizeof(double) * 32);
  double* focc = (double*)take(sizeof(double) * n);
  double* dq = (double*)take(sizeof(double) * nsh);
  double* sig = (double*)take(sizeof(double) * nsh);
  double* dqat = (double*)take(sizeof(double) * nat);
  double* fcn = (double*)take(sizeof(double) * nat);
  int* ao_sh = (int*)take(sizeof(int) * n);
  int* sh_at = (int*)take(sizeof(int) * nsh);
  int* sh_k = (int*)take(sizeof(int) * nsh);
  int* sh_ao0 = (int*)take(sizeof(int) * (nsh + 1));
  __shared__ double s_ef;

  // 0. local maps: atoms of the fragment in order, their shells, their AOs
  if (threadIdx.x == 0) {
    int s = 0, ao = 0;
    for (int i = 0; i < nat; ++i) {
      const DevElem& e = ar.el[ar.elem[a0 + i]];
      for (int k = 0; k < e.nsh; ++k, ++s) {
        sh_at[s] = i;
        sh_k[s] = k;
        sh_ao0[s] = ao;
        for (int m = 0; m < 2 * e.l[k] + 1; ++m) ao_sh[ao++] = s;
      }
    }
    sh_ao0[s] = ao;
  }
  // 1. occupations: bisection on sum f = N (Eq. 6)
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double lo = 1e300, hi = -1e300;
    for (int i = lane; i < n; i += 32) { lo = fmin(lo, ar.eps[nm.aov + i]); hi = fmax(hi, ar.eps[nm.aov + i]); }
    lo = -warp_max(-lo) - 50.0 * ar.g.kT - 1.0;
    hi = warp_max(hi) + 50.0 * ar.g.kT + 1.0;
    double ef = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
      ef = 0.5 * (lo + hi);
      double t = 0.0;
      for (int i = lane; i < n; i += 32) {
        const double x = fmin(fmax((ar.eps[nm.aov + i] - ef) / ar.g.kT, -700.0), 700.0);
        t += 2.0 / (exp(x) + 1.0);
      }
      t = warp_sum(t);
      if (fabs(t - nm.nel) < 1e-13 || hi - lo < 1e-15) break;
      if (t > nm.nel) hi = ef; else lo = ef;
    }
    if (lane == 0) s_ef = ef;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = fmin(fmax((ar.eps[nm.aov + i] - s_ef) / ar.g.kT, -700.0), 700.0);
    focc[i] = 2.0 / (exp(x) + 1.0);
    if (focc[i] > 1e-10 && focc[i] < 2.0 - 1e-10) *ar.frac = 1;   // W~ = 1/2 PFP needs 2 or 0
  }
  __syncthreads();
  // 2. density (rows of CT are the orbitals)
  const double* Sm = ar.S + nm.mat;
  const double* Hm = ar.H0 + nm.mat;
  const double* CT = ar.CT + nm.mat;
  block_gemm<double>(n, n, n, CT, 1, n, CT, 1, n, ar.P, n, nullptr, nullptr, focc, gemm);
  // 3. Mulliken charges, atomic charges, shell shifts, Fock matrix
  {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double pop = 0.0;
      for (int k = sh_ao0[s]; k < sh_ao0[s + 1]; ++k)
        for (int j = lane; j < n; j += 32) pop += ar.P[(long long)k * n + j] * Sm[(long long)k * n + j];
      pop = warp_sum(pop);
      if (lane == 0) dq[s] = pop - ar.el[ar.elem[a0 + sh_at[s]]].q0[sh_k[s]];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int a = 0; a < nat; ++a) dqat[a] = 0.0;
    for (int s = 0; s < nsh; ++s) dqat[sh_at[s]] += dq[s];
  }
  __syncthreads();
  {
    const double* G = ar.gam + nm.gam;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = wid; s < nsh; s += nw) {
      double v = 0.0;
      for (int t = lane; t < nsh; t += 32) v += G[(size_t)s * nsh + t] * dq[t];
      v = warp_sum(v);
      if (lane == 0) {
        const int a = sh_at[s];
        sig[s] = v - ar.el[ar.elem[a0 + a]].gamma3 * dqat[a] * dqat[a];
      }
    }
  }
  __syncthreads();
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int i = int(e / n), j = int(e - (long long)i * n);
    ar.F[e] = Hm[e] + 0.5 * Sm[e] * (sig[ao_sh[i]] + sig[ao_sh[j]]);
  }
  __syncthreads();
  // 4. W~ = 1/2 P F P (the factor is applied below)
  block_gemm<double>(n, n, n, ar.F, n, 1, ar.P, 1, n, ar.T, n, nullptr, nullptr, nullptr, gemm);   // F P
  block_gemm<double>(n, n, n, ar.P, n, 1, ar.T, 1, n, ar.W, n, nullptr, nullptr, nullptr, gemm);   // P F P
  // 5. per atom A: every pair term on A's side
  double gacc[8][3];   // up to 8 atoms per thread (nat <= 2048)
  for (int r = 0; r < 8; ++r) gacc[r][0] = gacc[r][1] = gacc[r][2] = 0.0;
  int r = 0;
  for (int A = threadIdx.x; A < nat; A += blockDim.x, ++r) {
    const int ga = a0 + A;
    const int ea = ar.elem[ga];
    const DevElem& EA = ar.el[ea];
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    double fA = 0.0;
    int sA0 = 0;
    while (sA0 < nsh && sh_at[sA0] != A) ++sA0;
    for (int k = 0; k < EA.nsh; ++k) {   // on-site levels: d h_A^l / d CN_A
      const int s = sA0 + k;
      for (int mu = sh_ao0[s]; mu < sh_ao0[s + 1]; ++mu) fA += ar.P[(long long)mu * n + mu] * EA.h[k] * EA.kcn[k];
    }
    int sB0 = 0;
    for (int B = 0; B < nat; ++B) {
      const int gb = a0 + B;
      const int eb = ar.elem[gb];
      const DevElem& EB = ar.el[eb];
      if (B == A) { sB0 += EB.nsh; continue; }
      const double R[3] = {ar.xyz[3 * ga] - ar.xyz[3 * gb], ar.xyz[3 * ga + 1] - ar.xyz[3 * gb + 1],
                           ar.xyz[3 * ga + 2] - ar.xyz[3 * gb + 2]};
      const double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
      const double rr = sqrt(r2);
      const double u[3] = {R[0] / rr, R[1] / rr, R[2] / rr};
      // repulsion (Eq. 11)
      {
        const double al = sqrt(EA.arep * EB.arep);
        const double ex = exp(-al * pow(rr, ar.g.k_f));
        const double de = EA.zeff * EB.zeff * ex * (-1.0 / r2 - al * ar.g.k_f * pow(rr, ar.g.k_f - 2.0));
        g0 += de * u[0]; g1 += de * u[1]; g2 += de * u[2];
      }
      // Coulomb kernel at fixed charges: dq_s dq_t dgamma_st / dR_A
      for (int ka = 0; ka < EA.nsh; ++ka) {
        for (int kb = 0; kb < EB.nsh; ++kb) {
          const double ie = 0.5 * (1.0 / EA.eta_sh[ka] + 1.0 / EB.eta_sh[kb]);
          const double gm = pow(pow(rr, ar.g.k_g) + pow(ie, ar.g.k_g), -1.0 / ar.g.k_g);
          const double dg = -pow(rr, ar.g.k_g - 1.0) * pow(gm, ar.g.k_g + 1.0);
          const double c = dq[sA0 + ka] * dq[sB0 + kb] * dg;
          g0 += c * u[0]; g1 += c * u[1]; g2 += c * u[2];
        }
      }
      // H0 prefactors of the pair (Eq. 8) and the polynomial Pi (Eq. 9)
      const double den = EA.en - EB.en;
      const double fen = 1.0 + ar.g.k_en * den * den;
      const double kAB = ar.kab[ea * ar.ne + eb];
      const double rcov = EA.rcov + EB.rcov;
      const double x = sqrt(rr / rcov);
      const double dxdR = x / (2.0 * rr);
      for (int sa = 0; sa < EA.nsh; ++sa) {
        const int la = EA.l[sa];
        const int shA = sA0 + sa;
        const double hA = EA.h[sa] * (1.0 + EA.kcn[sa] * ar.cn[ga]);
        for (int sb = 0; sb < EB.nsh; ++sb) {
          const int lb = EB.l[sb];
          const int shB = sB0 + sb;
          const double hB = EB.h[sb] * (1.0 + EB.kcn[sb] * ar.cn[gb]);
          const double kll = 0.5 * (ar.g.k_l[la] + ar.g.k_l[lb]);
          const double Pi = (1.0 + EA.kpoly[sa] * x) * (1.0 + EB.kpoly[sb] * x);
          const double dPi = EA.kpoly[sa] * (1.0 + EB.kpoly[sb] * x) + EB.kpoly[sb] * (1.0 + EA.kpoly[sa] * x);
          const double Hp = kAB * kll * 0.5 * (hA + hB) * fen * Pi;           // H0 = Hp S
          const double cPi = kAB * kll * 0.5 * (hA + hB) * fen * dPi * dxdR;  // dHp/dR
          const double cCN = kAB * kll * fen * Pi * EA.h[sa] * EA.kcn[sa];    // 2 x 1/2 d hbar / dCN_A
          const double shift = 0.5 * (sig[shA] + sig[shB]);
          // primitive sums of the overlap derivative
          double T1 = 0, B0 = 0, B1 = 0, A0 = 0, A1 = 0, Q0 = 0, Q1 = 0, H1 = 0;
          for (int pa = 0; pa < EA.nprim[sa]; ++pa) {
            for (int pb = 0; pb < EB.nprim[sb]; ++pb) {
              const PrimPair q = ar.prim[prim_pair_index(ar.ne, ea, eb, sa, sb, pa, pb)];
              const double s00 = q.pref * exp(-q.abp * r2);
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
              const long long mu = sh_ao0[shA] + uu, nu = sh_ao0[shB] + vv;
              const double p = ar.P[mu * n + nu];
              const double sv = Sm[mu * n + nu];
              const double M = p * (Hp + shift) - 0.5 * ar.W[mu * n + nu];
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
              fA += p * sv * cCN;
            }
          }
        }
      }
      sB0 += EB.nsh;
    }
    fcn[A] = fA;
    if (r < 8) { gacc[r][0] = g0; gacc[r][1] = g1; gacc[r][2] = g2; }
  }
  __syncthreads();
  // 6. CN gradient (Eqs. 26-28): sum over partners of (F_A + F_B) f'(R_AB)
  r = 0;
  for (int A = threadIdx.x; A < nat; A += blockDim.x, ++r) {
    const int ga = a0 + A;
    const double ra = ar.el[ar.elem[ga]].rcov;
    double g0 = gacc[r][0], g1 = gacc[r][1], g2 = gacc[r][2];
    for (int B = 0; B < nat; ++B) {
      if (B == A) continue;
      const int gb = a0 + B;
      const double R0 = ar.xyz[3 * ga] - ar.xyz[3 * gb], R1 = ar.xyz[3 * ga + 1] - ar.xyz[3 * gb + 1],
                   R2 = ar.xyz[3 * ga + 2] - ar.xyz[3 * gb + 2];
      const double rr = sqrt(R0 * R0 + R1 * R1 + R2 * R2);
      if (rr >= ar.g.cn_cutoff) continue;
      const double rc = ra + ar.el[ar.elem[gb]].rcov;
      const double f = 1.0 / (1.0 + exp(-ar.g.cn_k1 * (ar.g.cn_k2 * rc / rr - 1.0)));
      const double df = -f * (1.0 - f) * ar.g.cn_k1 * ar.g.cn_k2 * rc / (rr * rr);
      const double c = (fcn[A] + fcn[B]) * df / rr;
      g0 += c * R0; g1 += c * R1; g2 += c * R2;
    }
    ar.grad[3 * A] = g0;
    ar.grad[3 * A + 1] = g1;
    ar.grad[3 * A + 2] = g2;
  }
}

size_t gradient_smem(int n, int nsh, int nat) {
  auto a16 = [](size_t b) { return (b + 15) & ~size_t(15); };
  return a16(sizeof(double) * kGemmSmemElems) + a16(sizeof(double) * 32) + a16(sizeof(double) * n) +
         2 * a16(sizeof(double) * nsh) + 2 * a16(sizeof(double) * nat) + a16(sizeof(int) * n) +
         2 * a16(sizeof(int) * nsh) + a16(sizeof(int) * (nsh + 1));
}

cudaError_t launch_xtb_gradient(cudaStream_t st, const Nmer* nm, int n, int nsh, int nat, FragTab ft,
                                const double* xyz, const int* elem, const int* atom_sh0, const DevElem* el,
                                const double* kab, int ne, const PrimPair* prim, const double* cn, GParams g,
                                const double* S, const double* H0, const double* CT, const double* eps,
                                const double* gam, double* work, double* grad, int* frac) {
  if (nat > 8 * kBlock) return cudaErrorInvalidValue;
  GradArgs ar;
  ar.nm = nm; ar.ft = ft; ar.xyz = xyz; ar.elem = elem; ar.atom_sh0 = atom_sh0; ar.el = el; ar.kab = kab;
  ar.ne = ne; ar.prim = prim; ar.cn = cn; ar.g = g; ar.S = S; ar.H0 = H0; ar.CT = CT; ar.eps = eps; ar.gam = gam;
  const size_t nn = (size_t)n * n;
  ar.P = work; ar.F = work + nn; ar.T = work + 2 * nn; ar.W = work + 3 * nn;
  ar.grad = grad; ar.frac = frac;
  const size_t sb = gradient_smem(n, nsh, nat);
  cudaError_t e = cudaFuncSetAttribute(xtb_gradient_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
  if (e != cudaSuccess) return e;
  xtb_gradient_kernel<<<1, kBlock, sb, st>>>(ar);
  note_launch();
  return cudaGetLastError();
}

}  // namespace fmo
