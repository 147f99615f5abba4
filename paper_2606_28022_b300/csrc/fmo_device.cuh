// Device-side data layouts and block-level building blocks of the batched
// FMO-xTB SCC path (sm_103a).  Included by every .cu file of the library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fmo {

constexpr int kMaxShell = 3;
constexpr int kMaxPrim = 12;
constexpr int kMaxElem = 16;      // distinct elements in one system
#ifndef FMO_HIST
#define FMO_HIST 8
#endif
constexpr int kHist = FMO_HIST;   // Broyden history length
constexpr int kBlock = 256;       // threads of the SCC kernels

// One element of the table, compacted to the elements present.  cn[][] holds
// the contraction coefficient times the primitive normalisation.
struct DevElem {
  int nsh;
  int l[kMaxShell];
  int nprim[kMaxShell];
  int pad_;
  double alpha[kMaxShell][kMaxPrim];
  double cn[kMaxShell][kMaxPrim];
  double h[kMaxShell];       // H_A^l
  double kcn[kMaxShell];     // k_CN,l
  double kpoly[kMaxShell];   // k^poly_l
  double eta_sh[kMaxShell];  // (1 + kappa_A^l) eta_A
  double q0[kMaxShell];
  double gamma3, en, rcov, zeff, arep;
};

struct GParams {
  double k_l[3];
  double k_en, k_g, k_f;
  double cn_k1, cn_k2, cn_cutoff;
  double kT;                 // k_B * T_el (Eh)
};

// Fragment table (atoms are stored fragment by fragment).
struct FragTab {
  const int* atom0;   // first atom
  const int* nat;
  const int* sh0;     // first global shell
  const int* nsh;
  const int* ao0;     // first global AO
  const int* nao;
  // hybrid orbital projection at cut bonds (all null without cut bonds); per
  // internal atom:
  const int* ghost_frag;     // ghost: fragment of its detachment atom (BDA); else -1
  const int* ghost_src;      // ghost: internal index of its BDA; else -1
  const int* bda_baa_frag;   // BDA: fragment of its attachment atom (BAA); else -1
  const int* hop_baa;        // BDA or ghost: internal index of the BAA; else -1
};

constexpr int kMaxHealedShells = 32;   // ghost shells of bonds healed in one n-mer
constexpr int kMaxProjected = 16;      // hybrid-orbital-projected atoms in one n-mer
constexpr int kHopCols = 4 * kMaxProjected;   // s and p functions of the projected atoms

__device__ __forceinline__ bool frag_in_nmer(int nfrag, const int* frags, int f) {
  for (int k = 0; k < nfrag; ++k)
    if (frags[k] == f) return true;
  return false;
}

// a ghost belongs to an n-mer unless its bond is healed there (the BDA's
// fragment is part of the n-mer too); real atoms always do
__device__ __forceinline__ bool atom_in_nmer(const FragTab& ft, int nfrag, const int* frags, int ga) {
  return !ft.ghost_frag || ft.ghost_frag[ga] < 0 || !frag_in_nmer(nfrag, frags, ft.ghost_frag[ga]);
}

// One n-mer (monomer, dimer or trimer) of a pass.
struct Nmer {
  int nfrag;
  int frag[3];
  int n, nsh, nat;     // AOs, shells, atoms
  int npad;            // n rounded up to even
  double nel;          // electrons
  long long mat;       // offset of its n x n matrices (elements) in the pools
  long long shv;       // offset of its shell vectors
  long long gam;       // offset of its nsh x nsh gamma block
  long long aov;       // offset of its AO vectors
  long long hist;      // offset of its Broyden history
  long long apad;      // offset of its npad x npad scratch (eigen-solve matrix)
};

// Geometry-free factors of one pair of contracted Gaussian primitives (a on
// shell sa of element ea, b on shell sb of element eb): with p = a + b,
// pref = c_a c_b (pi/p)^{3/2}, abp = a b / p, ip = 1/p, ap = a/p, bp = b/p.
// The s-s overlap of the pair at distance R is pref exp(-abp R^2).
struct PrimPair {
  double pref, abp, ip, ap, bp;
};

__host__ __device__ inline long long prim_pair_index(int ne, int ea, int eb, int sa, int sb, int pa, int pb) {
  return (((((long long)ea * ne + eb) * kMaxShell + sa) * kMaxShell + sb) * kMaxPrim + pa) * kMaxPrim + pb;
}

// Local -> global index maps of an n-mer, held in shared memory.
struct NmerMaps {
  int16_t* ao_sh;      // [n]   local shell of each AO
  int16_t* sh_at;      // [nsh] local atom of each shell
  int* at_glob;        // [nat] global atom of each local atom
  int* sh_glob;        // [nsh] global shell of each local shell
  int16_t* sh_ao0;     // [nsh+1] first local AO of each shell
};

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Block-level reductions (fixed order: deterministic).
//
// Every thread must see the bit-identical result: convergence tests branch on
// these values, and threads that disagree in the last bit would leave a loop
// at different iterations and deadlock at the next barrier.  A sum is
// therefore reduced onto lane 0 and broadcast from there (an XOR butterfly
// leaves each lane with a differently rounded total).  Max is exact, so its
// butterfly gives identical values everywhere; it propagates NaN.

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}
// max that propagates NaN (fmax would drop it: a NaN residual must not read
// as converged)
template <typename T>
__device__ __forceinline__ T nan_max(T a, T b) {
  return (a != a || b != b) ? (a != a ? a : b) : fmax(a, b);
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the block; every thread gets the result.  red: >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (lane < nw) ? red[lane] : 0.0;
  t = warp_sum(t);
  return t;
}
__device__ __forceinline__ double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (lane < nw) ? red[lane] : -1e300;
  t = warp_max(t);
  return t;
}

// ---------------------------------------------------------------------------
// Block-level GEMM: C[m][n] = sum_k a(m,k) * b(n,k) with
//   a(m,k) = A[m*sam + ka*sak] * (kscale ? kscale[k] : 1),  ka = kidx ? kidx[k] : k,
//   b(n,k) = B[n*sbn + kb*sbk],                             kb = kidx_b ? kidx_b[k] : k
// (B may be stored in a wider type TB; it is rounded to T on load; kscale is
// of type TS: double scales multiply in FP64, scales of type T in T).
// 256 threads as a 16 x 16 grid, each computing TM x TN outputs of a
// (16 TM) x (16 TN) tile; BK = 16.  The tile edge (64 or 80) is chosen per
// dimension to waste the least padding (an n = 76 monomer fits one 80-row
// tile instead of two 64-row tiles).  The next k-slice is fetched into
// registers while the current one is multiplied from shared memory (smem:
// kGemmSmemElems elements of T).  Ends with __syncthreads().

constexpr int kGemmSmemElems = 2 * 16 * (80 + 1);

template <typename T, typename TB, typename TS, int TM, int TN>
__device__ __forceinline__ void block_gemm_tile(int M, int N, int K, const T* __restrict__ A, long long sam,
                                                long long sak, const TB* __restrict__ B, long long sbn,
                                                long long sbk, T* __restrict__ C, long long ldc,
                                                const int* __restrict__ kidx, const int* __restrict__ kidx_b,
                                                const TS* __restrict__ kscale, T* smem) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  // rows of the staged slices padded by one element: the k-contiguous
  // stores (16 k values per warp) then fall into distinct banks
  constexpr int LDA = BM + 1, LDB = BN + 1;
  T* As = smem;              // [BK][LDA]
  T* Bs = smem + BK * LDA;   // [BK][LDB]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const bool a_k_contig = (sak == 1);
  const bool b_k_contig = (sbk == 1);
  // per-thread slice elements: k offset, shared-memory slot, row offset in
  // global memory (-1: outside the matrix)
  int ka[TM], kb[TN], sa[TM], sb[TN];
  long long oa[TM], ob[TN];
  T ra[TM], rb[TN];
  for (int m0 = 0; m0 < M; m0 += BM) {
    for (int n0 = 0; n0 < N; n0 += BN) {
#pragma unroll
      for (int r = 0; r < TM; ++r) {
        const int e = tid + r * kBlock;
        int kk, mm;
        if (a_k_contig) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
        ka[r] = kk;
        sa[r] = kk * LDA + mm;
        oa[r] = (m0 + mm < M) ? (long long)(m0 + mm) * sam : -1;
      }
#pragma unroll
      for (int r = 0; r < TN; ++r) {
        const int e = tid + r * kBlock;
        int kk, nn;
        if (b_k_contig) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
        kb[r] = kk;
        sb[r] = kk * LDB + nn;
        ob[r] = (n0 + nn < N) ? (long long)(n0 + nn) * sbn : -1;
      }
      T acc[TM][TN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
      // global -> registers for the k-slice at k0
      auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < TM; ++r) {
          const int gk = k0 + ka[r];
          T v = T(0);
          if (oa[r] >= 0 && gk < K) {
            v = A[oa[r] + (long long)(kidx ? kidx[gk] : gk) * sak];
            if (kscale) {
              if constexpr (sizeof(TS) == sizeof(T)) v = v * T(kscale[gk]);
              else v = T(double(v) * kscale[gk]);
            }
          }
          ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < TN; ++r) {
          const int gk = k0 + kb[r];
          rb[r] = (ob[r] >= 0 && gk < K) ? T(B[ob[r] + (long long)(kidx_b ? kidx_b[gk] : gk) * sbk]) : T(0);
        }
      };
      fetch(0);
      for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int r = 0; r < TM; ++r) As[sa[r]] = ra[r];
#pragma unroll
        for (int r = 0; r < TN; ++r) Bs[sb[r]] = rb[r];
        __syncthreads();
        if (k0 + BK < K) fetch(k0 + BK);   // in flight during the multiply
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
          T a[TM], b[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[kk * LDA + ty * TM + i];
#pragma unroll
          for (int j = 0; j < TN; ++j) b[j] = Bs[kk * LDB + tx * TN + j];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty * TM + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int gn = n0 + tx * TN + j;
          if (gn < N) C[gm * ldc + gn] = acc[i][j];
        }
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Block-level FP32 GEMM on the tensor cores, same interface and result
// definition as block_gemm_tile (A, B float; kscale of type TS; kidx / kidx_b
// index lists over k): C[m][n] = sum_k a(m,k) b(n,k).
//
// mma.sync m16n8k8 TF32 with FP32 accumulation, each operand split as
// x = hi + lo (hi = x rounded to TF32, lo = x - hi rounded to TF32) and
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs): the dropped a_lo b_lo
// is ~2^-22 of |a b|, so the products keep FP32-grade accuracy (the SCC's
// FP32 phase converges its charges to 1e-5 through them).  The tensor cores'
// accumulation does not round to nearest, so over K terms its error would
// grow like K: the three MMAs of each k-step go into a zeroed register and
// are added to the running sum by an ordinary round-to-nearest addition.
// CTA tile 64 x 64, k-slices of 32 staged in shared memory (rows padded to 36
// floats: the fragment reads of a warp hit 32 distinct banks); 8 warps as
// 2 (m) x 4 (n), each 32 x 16 = two m16 x two n8 MMA tiles.  The next k-slice
// is fetched into registers while the current one is multiplied.
// smem: 2 * 64 * 36 floats (<= kGemmSmemElems doubles).  Ends with __syncthreads().

constexpr int kTcBM = 64, kTcBN = 64, kTcBK = 32, kTcLD = kTcBK + 4;
static_assert(2 * 64 * (32 + 4) * 4 <= kGemmSmemElems * 8, "tensor-core GEMM staging exceeds the GEMM smem region");

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <typename TS>
__device__ __forceinline__ void block_gemm_tc(int M, int N, int K, const float* __restrict__ A, long long sam,
                                           long long sak, const float* __restrict__ B, long long sbn,
                                           long long sbk, float* __restrict__ C, long long ldc,
                                           const int* __restrict__ kidx, const int* __restrict__ kidx_b,
                                           const TS* __restrict__ kscale, float* smem) {
  float* As = smem;                      // [64][36]
  float* Bs = smem + kTcBM * kTcLD;      // [64][36]
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int g = lane >> 2, tg = lane & 3;
  const int wm = wid >> 2, wn = wid & 3;   // warp tile: rows wm*32 + [0,32), cols wn*16 + [0,16)
  // staging map: 8 elements of each operand per thread along its contiguous
  // dimension (k if the k stride is 1, else m / n)
  const bool a_kc = (sak == 1), b_kc = (sbk == 1);
  for (int m0 = 0; m0 < M; m0 += kTcBM) {
    for (int n0 = 0; n0 < N; n0 += kTcBN) {
      float acc[2][2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
      float ra[8], rb[8];
      auto fetch = [&](int k0) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int e = tid + r * kBlock;
          int mm, kk;
          if (a_kc) { kk = e % kTcBK; mm = e / kTcBK; } else { mm = e % kTcBM; kk = e / kTcBM; }
          const int gm = m0 + mm, gk = k0 + kk;
          float v = 0.f;
          if (gm < M && gk < K) {
            v = A[(long long)gm * sam + (long long)(kidx ? kidx[gk] : gk) * sak];
            if (kscale) {
              if constexpr (sizeof(TS) == 4) v *= float(kscale[gk]);
              else v = float(double(v) * kscale[gk]);
            }
          }
          ra[r] = v;
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int e = tid + r * kBlock;
          int nn, kk;
          if (b_kc) { kk = e % kTcBK; nn = e / kTcBK; } else { nn = e % kTcBN; kk = e / kTcBN; }
          const int gn = n0 + nn, gk = k0 + kk;
          rb[r] = (gn < N && gk < K) ? B[(long long)gn * sbn + (long long)(kidx_b ? kidx_b[gk] : gk) * sbk] : 0.f;
        }
      };
      fetch(0);
      for (int k0 = 0; k0 < K; k0 += kTcBK) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const int e = tid + r * kBlock;
          int mm, kk;
          if (a_kc) { kk = e % kTcBK; mm = e / kTcBK; } else { mm = e % kTcBM; kk = e / kTcBM; }
          As[mm * kTcLD + kk] = ra[r];
          int nn, kb;
          if (b_kc) { kb = e % kTcBK; nn = e / kTcBK; } else { nn = e % kTcBN; kb = e / kTcBN; }
          Bs[nn * kTcLD + kb] = rb[r];
        }
        __syncthreads();
        if (k0 + kTcBK < K) fetch(k0 + kTcBK);   // in flight during the MMAs
#pragma unroll
        for (int ks = 0; ks < kTcBK; ks += 8) {
          uint32_t ah[2][4], al[2][4], bh[2][2], bl[2][2];
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const float* ap = As + (wm * 32 + i * 16 + g) * kTcLD + ks + tg;
            const float x[4] = {ap[0], ap[8 * kTcLD], ap[4], ap[8 * kTcLD + 4]};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              ah[i][c] = to_tf32(x[c]);
              al[i][c] = to_tf32(x[c] - __uint_as_float(ah[i][c]));
            }
          }
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const float* bp = Bs + (wn * 16 + j * 8 + g) * kTcLD + ks + tg;
            const float x[2] = {bp[0], bp[4]};
#pragma unroll
            for (int c = 0; c < 2; ++c) {
              bh[j][c] = to_tf32(x[c]);
              bl[j][c] = to_tf32(x[c] - __uint_as_float(bh[j][c]));
            }
          }
#pragma unroll
          for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              float t[4] = {0.f, 0.f, 0.f, 0.f};
              mma_tf32(t, al[i], bh[j]);
              mma_tf32(t, ah[i], bl[j]);
              mma_tf32(t, ah[i], bh[j]);
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[i][j][c] = __fadd_rn(acc[i][j][c], t[c]);
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int r0 = m0 + wm * 32 + i * 16 + g, c0 = n0 + wn * 16 + j * 8 + 2 * tg;
          if (r0 < M) {
            if (c0 < N) C[(long long)r0 * ldc + c0] = acc[i][j][0];
            if (c0 + 1 < N) C[(long long)r0 * ldc + c0 + 1] = acc[i][j][1];
          }
          if (r0 + 8 < M) {
            if (c0 < N) C[(long long)(r0 + 8) * ldc + c0] = acc[i][j][2];
            if (c0 + 1 < N) C[(long long)(r0 + 8) * ldc + c0 + 1] = acc[i][j][3];
          }
        }
    }
  }
  __syncthreads();
}

// micro-tile (4 or 5 per thread: tile edge 64 or 80) with the least padding
// of a dimension d, the smaller on ties
__device__ __forceinline__ int gemm_micro(int d) {
  const int p4 = (d + 63) / 64 * 64, p5 = (d + 79) / 80 * 80;
  return p5 < p4 ? 5 : 4;
}

template <typename X>
struct NoDeduce { using type = X; };   // keeps kscale out of template deduction (nullptr -> TS = double)

template <typename T, typename TB = T, typename TS = double>
__device__ void block_gemm(int M, int N, int K, const T* __restrict__ A, long long sam, long long sak,
                           const TB* __restrict__ B, long long sbn, long long sbk, T* __restrict__ C,
                           long long ldc, const int* __restrict__ kidx, const int* __restrict__ kidx_b,
                           const typename NoDeduce<TS>::type* __restrict__ kscale, T* smem) {
  if constexpr (sizeof(T) == 4 && sizeof(TB) == 4) {
    // tensor cores where the 64 x 64 tiles waste little (n = 116, 174, 232,
    // 348: ~10%); the SIMT tiles (64 or 80 wide) fit the rest better
    const float pad = float((M + 63) / 64 * 64) / float(M) * (float((N + 63) / 64 * 64) / float(N));
    if (M >= 96 && N >= 96 && pad <= 1.25f) {
      block_gemm_tc<TS>(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, kidx, kidx_b, kscale, smem);
      return;
    }
  }
  const int tm = gemm_micro(M), tn = gemm_micro(N);
#define FMO_GEMM_CASE(a, b)                                                                              \
  if (tm == a && tn == b) {                                                                              \
    block_gemm_tile<T, TB, TS, a, b>(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, kidx, kidx_b, kscale, smem); \
    return;                                                                                              \
  }
  FMO_GEMM_CASE(4, 4) FMO_GEMM_CASE(4, 5) FMO_GEMM_CASE(5, 4) FMO_GEMM_CASE(5, 5)
#undef FMO_GEMM_CASE
}

// ---------------------------------------------------------------------------
// Block-level GEMM in double-float arithmetic, for products whose result is
// needed to FP64 accuracy: C[m][n] = sum_k A[arow(m)][k] * B[n][k], with A
// float (exact FP32 values) or double (row arow(m) = arow ? arow[m] : m,
// leading dimension lda), B double (leading dimension ldb) and C double.
// A double A is split like b below and a_lo*b_hi joins the small terms.  Each b is split on staging into b_hi = fl32(b) and
// b_lo = fl32(b - b_hi) (b to ~2^-48 relative); a*b_hi is formed exactly as
// p + e (p = fl32(a b_hi), e = fma(a, b_hi, -p)), a*b_lo is added to e, and
// the running sum is kept as an unevaluated pair (hi, lo) by Knuth's
// TwoSum on hi with the small parts accumulated in lo (renormalised after
// every 16 terms).  The error is ~1e-14 relative to sum |a b| per output: FP64-grade accuracy from
// ~10 FP32 instructions per term, where B300 issues FP64 FMAs at 1/64 of the
// FP32 rate.  Same thread/tile layout as block_gemm_tile (TM x TN per thread,
// BK = 16); smem: 4 * 16 * (16*max(TM,TN) + 1) floats (kGemmSmemElems doubles).  Ends with __syncthreads().

template <int TM, int TN, typename TA>
__device__ __noinline__ void block_gemm_df_tile(int M, int N, int K, const TA* __restrict__ A,
                                                   const int* __restrict__ arow, long long lda,
                                                   const double* __restrict__ B, long long ldb,
                                                   double* __restrict__ C, long long ldc, float* smem) {
  constexpr int BM = 16 * TM, BN = 16 * TN, BK = 16;
  constexpr int LDA = BM + 1, LDB = BN + 1;
  constexpr bool kSplitA = sizeof(TA) == 8;   // A in FP64: split like B
  float* As = smem;                 // [BK][LDA]
  float* Bh = As + BK * LDA;        // [BK][LDB]
  float* Bl = Bh + BK * LDB;        // [BK][LDB]
  float* Al = Bl + BK * LDB;        // [BK][LDA] (kSplitA only)
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < M; m0 += BM) {
    for (int n0 = 0; n0 < N; n0 += BN) {
      float hi[TM][TN], lo[TM][TN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) { hi[i][j] = 0.f; lo[i][j] = 0.f; }
      for (int k0 = 0; k0 < K; k0 += BK) {
        // stage: 16 consecutive k of a row per 16 threads (coalesced)
        for (int e = tid; e < BM * BK; e += kBlock) {
          const int kk = e % BK, mm = e / BK, gm = m0 + mm, gk = k0 + kk;
          float v = 0.f, vl = 0.f;
          if (gm < M && gk < K) {
            const TA a = A[(long long)(arow ? arow[gm] : gm) * lda + gk];
            v = float(a);
            if constexpr (kSplitA) vl = float(double(a) - double(v));
          }
          As[kk * LDA + mm] = v;
          if constexpr (kSplitA) Al[kk * LDA + mm] = vl;
        }
        for (int e = tid; e < BN * BK; e += kBlock) {
          const int kk = e % BK, nn = e / BK, gn = n0 + nn, gk = k0 + kk;
          float h = 0.f, l = 0.f;
          if (gn < N && gk < K) {
            const double b = B[(long long)gn * ldb + gk];
            h = float(b);
            l = float(b - double(h));
          }
          Bh[kk * LDB + nn] = h;
          Bl[kk * LDB + nn] = l;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
          float a[TM], al[TM], bh[TN], bl[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) {
            a[i] = As[kk * LDA + ty * TM + i];
            if constexpr (kSplitA) al[i] = Al[kk * LDA + ty * TM + i];
          }
#pragma unroll
          for (int j = 0; j < TN; ++j) { bh[j] = Bh[kk * LDB + tx * TN + j]; bl[j] = Bl[kk * LDB + tx * TN + j]; }
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) {
              // _rn intrinsics: never contracted into FMAs, so the
              // error-free transformations stay exact
              const float p = __fmul_rn(a[i], bh[j]);
              float e = fmaf(a[i], bh[j], -p);
              e = fmaf(a[i], bl[j], e);
              if constexpr (kSplitA) e = fmaf(al[i], bh[j], e);
              const float s = __fadd_rn(hi[i][j], p);
              const float bb = __fsub_rn(s, hi[i][j]);
              const float err = __fadd_rn(__fsub_rn(hi[i][j], __fsub_rn(s, bb)), __fsub_rn(p, bb));
              hi[i][j] = s;
              lo[i][j] = __fadd_rn(lo[i][j], __fadd_rn(err, e));
            }
        }
        // renormalise once per slice (Fast2Sum, |lo| << |hi|): keeps lo, and
        // so its own rounding, small
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) {
            const float s = __fadd_rn(hi[i][j], lo[i][j]);
            lo[i][j] = __fsub_rn(lo[i][j], __fsub_rn(s, hi[i][j]));
            hi[i][j] = s;
          }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int gm = m0 + ty * TM + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int gn = n0 + tx * TN + j;
          if (gn < N) C[gm * ldc + gn] = double(hi[i][j]) + double(lo[i][j]);
        }
      }
    }
  }
  __syncthreads();
}

template <typename TA>
__device__ inline void block_gemm_df(int M, int N, int K, const TA* __restrict__ A, const int* __restrict__ arow,
                                     long long lda, const double* __restrict__ B, long long ldb, double* __restrict__ C,
                                     long long ldc, float* smem) {
  const int tm = gemm_micro(M), tn = gemm_micro(N);
  if (tm == 4 && tn == 4) block_gemm_df_tile<4, 4, TA>(M, N, K, A, arow, lda, B, ldb, C, ldc, smem);
  else if (tm == 4) block_gemm_df_tile<4, 5, TA>(M, N, K, A, arow, lda, B, ldb, C, ldc, smem);
  else if (tn == 4) block_gemm_df_tile<5, 4, TA>(M, N, K, A, arow, lda, B, ldb, C, ldc, smem);
  else block_gemm_df_tile<5, 5, TA>(M, N, K, A, arow, lda, B, ldb, C, ldc, smem);
}

// ---------------------------------------------------------------------------
// Solve (a + w0sq I) g = c for the Broyden coefficients (m x m, m <= kHist,
// a row-major) by Gauss-Jordan elimination with partial pivoting on one
// warp: lane r holds row r (the right-hand side in column kHist, columns
// m..kHist-1 zero), the rows are updated in parallel.  Pivot choice (the
// first row of largest |M[r][col]|), factors, updates and the final division
// are those of the serial textbook loop, element by element, so the result is
// the same; one thread doing it alone waits ~60 cycles on every dependent
// FP64 instruction, on B300's FP64 pipe.  All 32 lanes of the warp call it.
static __device__ __noinline__ void warp_gj_solve(int m, const double* a, const double* c, double w0sq, double* g) {
  const int lane = threadIdx.x & 31;
  double row[kHist + 1];
#pragma unroll
  for (int j = 0; j < kHist; ++j) row[j] = (lane < m && j < m) ? a[lane * m + j] + (lane == j ? w0sq : 0.0) : 0.0;
  row[kHist] = (lane < m) ? c[lane] : 0.0;
#pragma unroll
  for (int col = 0; col < kHist; ++col) {
    if (col >= m) break;
    double v = (lane >= col && lane < m) ? fabs(row[col]) : -1.0;
    int idx = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, off);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
      if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    const int piv = idx;
    if (piv != col) {
      const int src = (lane == col) ? piv : (lane == piv ? col : lane);
#pragma unroll
      for (int j = 0; j <= kHist; ++j) row[j] = __shfl_sync(0xffffffffu, row[j], src);
    }
    double prow[kHist + 1];
#pragma unroll
    for (int j = 0; j <= kHist; ++j) prow[j] = __shfl_sync(0xffffffffu, row[j], col);
    if (lane < m && lane != col) {
      const double f = row[col] / prow[col];
#pragma unroll
      for (int j = col; j <= kHist; ++j) row[j] -= f * prow[j];
    }
  }
  double diag = 1.0;
#pragma unroll
  for (int j = 0; j < kHist; ++j)
    if (j == lane) diag = row[j];
  if (lane < m) g[lane] = row[kHist] / diag;
}

// ---------------------------------------------------------------------------
// Block-level cyclic Jacobi eigensolver for a symmetric n x n matrix A
// (row-major, leading dimension lda >= npad, padding row/column zero).
// Parallel (round-robin) ordering: each round rotates npad/2 disjoint index
// pairs, applied as independent 2x2 block updates A <- J^T A J.  Pairs with
// |A_pq| <= thr are skipped; the solve ends after a sweep with no rotation.
// The rows of CT (ncol entries each, leading dimension ldc) are rotated along
// (CT <- J^T CT), so rows of CT become the eigenvectors in the basis CT
// started from.  Rotation angle: Golub & Van Loan, symmetric Schur 2x2.
// Returns the number of sweeps, or -1 if max_sweeps was reached.

template <typename T>
struct JacobiScratch {
  int* p;
  int* q;
  T* c;
  T* s;
  int* act;
};

template <typename T, int kUnroll>
__device__ int block_jacobi_u(T* A, int lda, int n, T* CT, long long ldc, int ncol, double tol,
                              int max_sweeps, JacobiScratch<T> js, double* red) {
  const int npad = n + (n & 1);
  const int half = npad / 2;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  int* list = js.act + half;   // act holds npad ints: [0, half) flags, [half, npad) active pairs
  // active-pair counters, one per round modulo 3: a counter is cleared two
  // rounds after it was read, so no thread can still be using it
  __shared__ int s_cnt[3];
  if (tid == 0) { s_cnt[0] = 0; s_cnt[1] = 0; s_cnt[2] = 0; }
  __syncthreads();
  int round = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double dmax = 0.0;
    // scale of the threshold: the largest |A_ii| below 1e3 Eh (levels shifted
    // by a hybrid-orbital projector, ~1e6 Eh, would make it meaningless)
    for (int i = tid; i < n; i += blockDim.x) {
      const double d = fabs(double(A[i * lda + i]));
      if (d < 1e3) dmax = fmax(dmax, d);
    }
    dmax = block_max(dmax, red);
    const double thr = tol * fmax(dmax, 1e-30);
    int rotations = 0;
    for (int r = 0; r < npad - 1; ++r, ++round) {
      const int slot = round % 3;
      for (int k = tid; k < half; k += blockDim.x) {
        const int m = npad - 1;
        int p, q;
        if (k == 0) { p = 0; q = ((0 + r) % m) + 1; }
        else { p = ((k + r) % m) + 1; q = ((m - k + r) % m) + 1; }
        if (p > q) { int t = p; p = q; q = t; }
        T c = T(1), s = T(0);
        int a = 0;
        if (q < n) {
          const T apq = A[p * lda + q];
          if (fabs(double(apq)) > thr) {
            const T app = A[p * lda + p], aqq = A[q * lda + q];
            const T tau = (aqq - app) / (T(2) * apq);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            s = t * c;
            a = 1;
          }
        }
        js.p[k] = p; js.q[k] = q; js.c[k] = c; js.s[k] = s; js.act[k] = a;
        if (a) list[atomicAdd(&s_cnt[slot], 1)] = k;
      }
      __syncthreads();
      const int na = s_cnt[slot];
      if (tid == 0) s_cnt[(round + 2) % 3] = 0;
      if (na == 0) continue;
      ++rotations;
      // 2x2 block updates A <- J^T A J: one warp per active pair k, lanes over
      // the partner pairs k2 (a block of two active pairs is done once, by
      // the warp of the smaller k).  Every block is read and written by one
      // lane only, so each lane first loads kUnroll partner blocks and then
      // updates them: the loads are in flight together (A in global memory,
      // large n-mers: one load's latency is ~1 us).
      for (int i = wid; i < na; i += nw) {
        const int k = list[i];
        const int p = js.p[k], q = js.q[k];
        const T c = js.c[k], s = js.s[k];
        for (int k2b = lane; k2b < half; k2b += 32 * kUnroll) {
          int p2[kUnroll], q2[kUnroll];
          bool ok[kUnroll];
          T c2[kUnroll], s2[kUnroll], b00[kUnroll], b01[kUnroll], b10[kUnroll], b11[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const int k2 = k2b + 32 * u;
            ok[u] = k2 < half && !(js.act[k2] && k2 < k);
            if (ok[u]) {
              p2[u] = js.p[k2]; q2[u] = js.q[k2];
              c2[u] = js.c[k2]; s2[u] = js.s[k2];
              b00[u] = A[p * lda + p2[u]]; b01[u] = A[p * lda + q2[u]];
              b10[u] = A[q * lda + p2[u]]; b11[u] = A[q * lda + q2[u]];
            }
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            if (!ok[u]) continue;
            const T t00 = b00[u] * c2[u] - b01[u] * s2[u], t01 = b00[u] * s2[u] + b01[u] * c2[u];
            const T t10 = b10[u] * c2[u] - b11[u] * s2[u], t11 = b10[u] * s2[u] + b11[u] * c2[u];
            const T x00 = c * t00 - s * t10, x01 = c * t01 - s * t11;
            const T x10 = s * t00 + c * t10, x11 = s * t01 + c * t11;
            if (k == k2b + 32 * u) {
              A[p * lda + p] = x00;
              A[q * lda + q] = x11;
              A[p * lda + q] = T(0);
              A[q * lda + p] = T(0);
            } else {
              A[p * lda + p2[u]] = x00; A[p * lda + q2[u]] = x01;
              A[q * lda + p2[u]] = x10; A[q * lda + q2[u]] = x11;
              A[p2[u] * lda + p] = x00; A[q2[u] * lda + p] = x01;
              A[p2[u] * lda + q] = x10; A[q2[u] * lda + q] = x11;
            }
          }
        }
      }
      // rotate the rows p, q of CT: one warp per active pair, lanes over
      // columns, kUnroll loads of each row in flight
      for (int i = wid; i < na; i += nw) {
        const int k = list[i];
        const int p = js.p[k], q = js.q[k];
        const T c = js.c[k], s = js.s[k];
        T* rp = CT + p * ldc;
        T* rq = CT + q * ldc;
        for (int jb = lane; jb < ncol; jb += 32 * kUnroll) {
          T vp[kUnroll], vq[kUnroll];
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const int j = jb + 32 * u;
            if (j < ncol) { vp[u] = rp[j]; vq[u] = rq[j]; }
          }
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            const int j = jb + 32 * u;
            if (j < ncol) {
              rp[j] = c * vp[u] - s * vq[u];
              rq[j] = s * vp[u] + c * vq[u];
            }
          }
        }
      }
      __syncthreads();
    }
    if (rotations == 0) return sweep;
  }
  return -1;
}

// A in shared memory (every n-mer that fits): one partner block per lane at a
// time (fewer live registers); A in global memory: four blocks in flight per
// lane.
template <typename T>
__device__ int block_jacobi(T* A, int lda, int n, T* CT, long long ldc, int ncol, double tol, int max_sweeps,
                            JacobiScratch<T> js, double* red) {
  if (__isShared(A)) return block_jacobi_u<T, 1>(A, lda, n, CT, ldc, ncol, tol, max_sweeps, js, red);
  return block_jacobi_u<T, 4>(A, lda, n, CT, ldc, ncol, tol, max_sweeps, js, red);
}

}  // namespace fmo
