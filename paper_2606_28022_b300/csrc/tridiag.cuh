// FP32 symmetric eigen-solver for one thread block, for the FP32 iterations
// of n-mers whose matrix A = C F C^T lives in global memory (Eq. 5 solved in
// the current orbital basis).
//
//   1. Householder reduction A = Q T Q^T to tridiagonal T (d, e).  Each step
//      updates the trailing matrix A22 <- A22 - v w^T - w v^T and, in the same
//      pass, forms A22' v' for the next reflector (the next row is updated
//      first), so the trailing upper triangle is read and written once per
//      step.  Rows from ks on sit in shared memory (packed upper triangle),
//      rows above ks in global memory; the global rows are used up first.
//   2. Eigenvalues of T by Sturm-sequence bisection, two per thread.
//   3. Eigenvectors of T from twisted factorisations T - lambda I =
//      N_r Delta_r N_r^T (forward L D L^T and backward U D U^T pivots, the
//      twist r at the smallest |gamma_r|; Dhillon's thesis, 1997), one per
//      thread; modified Gram-Schmidt within clusters of close eigenvalues.
//   4. Back-transformation: the rows of Zt become eigenvectors of A,
//      Zt <- Zt H_{n-3} ... H_0, then CT <- Zt CT.
//
// Its memory traffic is ~n^3/3 elements for step 1 (mostly on chip), against
// ~sweeps x n^3 for a cyclic Jacobi solve on a matrix in global memory.
// Failure (non-finite values, a Gram-Schmidt remainder that vanishes) is
// reported before CT is touched; the caller then restores A and
// diagonalises by Jacobi.
#pragma once
#include "fmo_device.cuh"

namespace fmo {

constexpr int kTriVecs = 20;        // npad-float vectors in shared memory (d e tau v vn w p pd lam inv cl part[8])
constexpr int kTriMinN = 64;

// shared-memory floats needed besides the packed triangle
__host__ __device__ inline int tri_vec_floats(int npad) { return kTriVecs * npad; }

struct TriWork {
  float* sh;       // shared memory: tri_vec_floats(npad) floats, then the packed rows
  int cap;         // floats available for packed rows
  float* glu;      // global scratch, >= 2 n min(n, blockDim.x) floats
  float* abak;     // global scratch, >= n * lda floats (copy of A for the fallback)
};

// element (i, j), i <= j, of the trailing matrix: rows < ks in global memory
// (row-major, leading dimension lda), rows >= ks packed in shared memory
struct TriAcc {
  float* A;
  int lda;
  float* t;
  int ks, m0;
  __device__ __forceinline__ float* at(int i, int j) const {
    if (i < ks) return A + (long long)i * lda + j;
    const int a = i - ks;
    return t + (a * m0 - (a * (a - 1)) / 2 + (j - i));
  }
};

// Rows i in [r0, n) of the upper triangle: with upd, b <- b - v_i w_j - w_i v_j
// (stored); always p += B u (B symmetric): the direct part of row i in
// pdir[i], the mirrored part per warp in part[warp][j].  Lane l owns columns
// j = 32 c + l (c < kC): their v, w, u and mirrored sums stay in registers;
// chunks left of the diagonal or past n are skipped by warp-uniform branches.
template <int kC>
__device__ __forceinline__ void tri_pass(const TriAcc& acc, int r0, int n, int npad, bool upd, const float* v,
                                         const float* w, const float* u, float* pdir, float* part) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  float pc[kC], vr[kC], wr[kC], ur[kC];
#pragma unroll
  for (int c = 0; c < kC; ++c) {
    const int j = 32 * c + lane;
    const bool in = j >= r0 && j < n;
    pc[c] = 0.f;
    vr[c] = (upd && in) ? v[j] : 0.f;
    wr[c] = (upd && in) ? w[j] : 0.f;
    ur[c] = in ? u[j] : 0.f;
  }
  // two rows per warp at a time (i and i + nw): their loads and their
  // reductions overlap
  for (int i = r0 + wid; i < n; i += 2 * nw) {
    const int i2 = i + nw;
    const bool has2 = i2 < n;
    const float vi = upd ? v[i] : 0.f, wi = upd ? w[i] : 0.f, ui = u[i];
    const float vi2 = (upd && has2) ? v[i2] : 0.f, wi2 = (upd && has2) ? w[i2] : 0.f, ui2 = has2 ? u[i2] : 0.f;
    float* ra = acc.at(i, i);                    // element (i, j) at ra[j - i]
    float* rb = has2 ? acc.at(i2, i2) : ra;
    const int c0 = i >> 5;
    float b[kC], b2[kC];
    // every load of both rows first (rows in global memory: all in flight)
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      b[c] = 0.f;
      b2[c] = 0.f;
      if (c < c0) continue;
      if (32 * c >= n) break;
      const int j = 32 * c + lane;
      if (j >= i && j < n) b[c] = ra[j - i];
      if (has2 && j >= i2 && j < n) b2[c] = rb[j - i2];
    }
    float di = 0.f, di2 = 0.f;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      if (c < c0) continue;
      if (32 * c >= n) break;
      const int j = 32 * c + lane;
      const bool live = j >= i && j < n, live2 = has2 && j >= i2 && j < n;
      float x = b[c], x2 = b2[c];
      if (upd) {
        x = live ? fmaf(-vi, wr[c], fmaf(-wi, vr[c], x)) : 0.f;
        x2 = live2 ? fmaf(-vi2, wr[c], fmaf(-wi2, vr[c], x2)) : 0.f;
        if (live) ra[j - i] = x;
        if (live2) rb[j - i2] = x2;
      }
      // outside the rows x, x2 are 0
      di = fmaf(x, ur[c], di);
      di2 = fmaf(x2, ur[c], di2);
      pc[c] = fmaf(x, j > i ? ui : 0.f, pc[c]);
      pc[c] = fmaf(x2, j > i2 ? ui2 : 0.f, pc[c]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      di += __shfl_down_sync(0xffffffffu, di, o);
      di2 += __shfl_down_sync(0xffffffffu, di2, o);
    }
    if (lane == 0) {
      pdir[i] = di;
      if (has2) pdir[i2] = di2;
    }
  }
#pragma unroll
  for (int c = 0; c < kC; ++c) {
    const int j = 32 * c + lane;
    if (j < npad) part[wid * npad + j] = pc[c];
  }
}

// Sum over the block in FP32 (every thread gets the result; red >= 32 floats)
__device__ __forceinline__ float block_sum_f(float x, float* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) red[wid] = x;
  __syncthreads();
  float t = lane < nw ? red[lane] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  return __shfl_sync(0xffffffffu, t, 0);
}

// Sturm counts (eigenvalues of T below x0 and below x1), two chains
// interleaved; pivots below pivmin in magnitude are replaced by -pivmin.
__device__ __forceinline__ void tri_sturm2(const float* d, const float* e2, int n, float x0, float x1, float pivmin,
                                           int& c0, int& c1) {
  float q0 = d[0] - x0, q1 = d[0] - x1;
  if (fabsf(q0) < pivmin) q0 = -pivmin;
  if (fabsf(q1) < pivmin) q1 = -pivmin;
  int a0 = q0 < 0.f, a1 = q1 < 0.f;
  for (int i = 1; i < n; ++i) {
    const float di = d[i], ei = e2[i - 1];
    q0 = (di - x0) - __fdividef(ei, q0);
    q1 = (di - x1) - __fdividef(ei, q1);
    if (fabsf(q0) < pivmin) q0 = -pivmin;
    if (fabsf(q1) < pivmin) q1 = -pivmin;
    a0 += q0 < 0.f;
    a1 += q1 < 0.f;
  }
  c0 = a0;
  c1 = a1;
}

// Eigen-decomposition of the symmetric n x n matrix A (FP32, global memory,
// leading dimension lda; destroyed).  On success the rows of CT are replaced
// by CT_new = V^T CT (V: eigenvectors of A, ascending eigenvalues written to
// eps) and true is returned; on failure A is restored from the copy and CT is
// untouched.  Zt, W: n x n FP32 scratch in global memory.  Ends with
// __syncthreads().
// prof (optional, thread 0): SM cycles at the end of each step, prof[0..6];
// prof[8..11]: parts of step 1 summed over its iterations
template <int kC>
__device__ __noinline__ bool tri_eigh(float* A, int lda, int n, float* CT, float* Zt, float* W, TriWork tw,
                                      float* gemm, double* red, double* eps, long long* prof = nullptr) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5, nt = blockDim.x;
  const bool pr = prof && tid == 0;
  if (pr) prof[0] = clock64();
  const int npad = n + (n & 1);
  float* d = tw.sh;
  float* e = d + npad;
  float* tau = e + npad;
  float* v = tau + npad;
  float* vn = v + npad;
  float* w = vn + npad;
  float* p = w + npad;
  float* pdir = p + npad;
  float* lam = pdir + npad;
  float* inv = lam + npad;
  int* cl = reinterpret_cast<int*>(inv + npad);
  float* part = reinterpret_cast<float*>(cl + npad);   // nw * npad
  float* tri = part + 8 * npad;
  __shared__ int s_fail;
  __shared__ int s_ncl;
  if (tid == 0) s_fail = 0;

  // copy of A for the fallback
  for (long long x = tid; x < (long long)n * lda; x += nt) tw.abak[x] = A[x];
  // rows from ks on in shared memory: the largest tail that fits
  int ks = 0;
  while ((long long)(n - ks) * (n - ks + 1) / 2 > tw.cap) ++ks;
  TriAcc acc{A, lda, tri, ks, n - ks};
  for (int i = ks + wid; i < n; i += nw)
    for (int j = i + lane; j < n; j += 32) *acc.at(i, j) = A[(long long)i * lda + j];
  __syncthreads();

  // reflector from x = row[k+1 .. n-1] held in vec at those positions:
  // H = I - tau u u^T with u[k+1] = 1, H x = beta e_{k+1} (LAPACK's slarfg
  // convention); u overwrites vec, written to A's row k for step 4.  The
  // scalars are formed by one thread (FP64 is slow on every thread).
  __shared__ float s_par[2];
  float* redf = reinterpret_cast<float*>(red);
  auto reflector = [&](int k, float* vec) {
    float s = 0.f;
    for (int j = k + 2 + tid; j < n; j += nt) s = fmaf(vec[j], vec[j], s);
    s = block_sum_f(s, redf);
    if (tid == 0) {
      const float alpha = vec[k + 1];
      float beta = alpha, tk = 0.f, scale = 0.f;
      if (s > 0.f) {
        const double bd = -copysign(sqrt(double(alpha) * alpha + double(s)), double(alpha));
        beta = float(bd);
        tk = float((bd - alpha) / bd);
        scale = float(1.0 / (double(alpha) - bd));
      }
      s_par[0] = scale;
      vec[k + 1] = 1.f;
      A[(long long)k * lda + k + 1] = 1.f;
      e[k] = beta;
      tau[k] = tk;
    }
    __syncthreads();
    const float scale = s_par[0];
    for (int j = k + 2 + tid; j < n; j += nt) {
      const float u = vec[j] * scale;
      vec[j] = u;
      A[(long long)k * lda + j] = u;
    }
    __syncthreads();
  };
  // p[j] = t * (pdir[j] + sum_w part[w][j]) for j >= r0; returns sum_j p_j v_j
  auto reduce_p = [&](int r0, float t, const float* vv) {
    float pv = 0.f;
    for (int j = r0 + tid; j < n; j += nt) {
      float x = pdir[j];
      for (int q = 0; q < nw; ++q) x += part[q * npad + j];
      x *= t;
      p[j] = x;
      pv = fmaf(x, vv[j], pv);
    }
    return block_sum_f(pv, redf);
  };

  // step 1: tridiagonalisation
  if (tid == 0) d[0] = *acc.at(0, 0);
  for (int j = 1 + tid; j < n; j += nt) v[j] = *acc.at(0, j);
  __syncthreads();
  reflector(0, v);
  tri_pass<kC>(acc, 1, n, npad, false, v, w, v, pdir, part);
  __syncthreads();
  float pv = reduce_p(1, tau[0], v);
  long long tacc[4] = {0, 0, 0, 0};
  for (int k = 0; k <= n - 3; ++k) {
    long long tq = pr ? clock64() : 0;
    auto tick = [&](int s) { if (pr) { const long long t = clock64(); tacc[s] += t - tq; tq = t; } };
    // w = p - (tau/2)(p.v) v, and row k+1 after this step's update
    const float K = 0.5f * tau[k] * pv;
    const float vk1 = v[k + 1], wk1 = fmaf(-K, v[k + 1], p[k + 1]);
    for (int j = k + 1 + tid; j < n; j += nt) {
      const float wj = fmaf(-K, v[j], p[j]);
      w[j] = wj;
      vn[j] = fmaf(-vk1, wj, fmaf(-wk1, v[j], *acc.at(k + 1, j)));
    }
    __syncthreads();
    if (tid == 0) d[k + 1] = vn[k + 1];
    tick(0);
    if (k + 1 <= n - 3) {
      reflector(k + 1, vn);
      tick(1);
      tri_pass<kC>(acc, k + 2, n, npad, true, v, w, vn, pdir, part);
      __syncthreads();
      tick(2);
      pv = reduce_p(k + 2, tau[k + 1], vn);
      tick(3);
      float* t = v; v = vn; vn = t;
    } else {
      // last step: rows n-2 and n-1 remain
      if (tid == 0) {
        e[n - 2] = vn[n - 1];
        d[n - 1] = fmaf(-2.f * v[n - 1], w[n - 1], *acc.at(n - 1, n - 1));
        tau[n - 2] = 0.f;
      }
      __syncthreads();
    }
  }

  if (pr) {
    prof[1] = clock64();
    for (int q = 0; q < 4; ++q) prof[8 + q] = tacc[q];
  }
  // step 2: eigenvalues by bisection
  float* e2 = w;
  double lo_l = 1e300, hi_l = -1e300, em_l = 0.0;
  for (int i = tid; i < n; i += nt) {
    const float ea = i > 0 ? fabsf(e[i - 1]) : 0.f, eb = i < n - 1 ? fabsf(e[i]) : 0.f;
    lo_l = fmin(lo_l, double(d[i]) - ea - eb);
    hi_l = fmax(hi_l, double(d[i]) + ea + eb);
    if (i < n - 1) {
      e2[i] = e[i] * e[i];
      em_l = fmax(em_l, double(e2[i]));
    }
  }
  const double gl0 = -block_max(-lo_l, red);
  const double gu0 = block_max(hi_l, red);
  const double emax2 = block_max(em_l, red);
  const double tnorm = fmax(fabs(gl0), fabs(gu0));
  const float pivmin = float(1e-30 * fmax(1.0, emax2));
  const float tolb = float(4.0 * 1.2e-7 * tnorm) + 2.f * pivmin;
  const float gl = float(gl0 - tolb - 2.0 * 1.2e-7 * tnorm), gu = float(gu0 + tolb + 2.0 * 1.2e-7 * tnorm);
  {
    const int half = (n + 1) / 2;
    if (tid < half) {
      const int j0 = tid, j1 = tid + half < n ? tid + half : tid;
      float lo0 = gl, hi0 = gu, lo1 = gl, hi1 = gu;
      for (int it = 0; it < 80; ++it) {
        const float m0 = 0.5f * (lo0 + hi0), m1 = 0.5f * (lo1 + hi1);
        const bool done0 = hi0 - lo0 <= tolb || m0 <= lo0 || m0 >= hi0;
        const bool done1 = hi1 - lo1 <= tolb || m1 <= lo1 || m1 >= hi1;
        if (done0 && done1) break;
        int c0, c1;
        tri_sturm2(d, e2, n, m0, m1, pivmin, c0, c1);
        if (!done0) { if (c0 > j0) hi0 = m0; else lo0 = m0; }
        if (!done1) { if (c1 > j1) hi1 = m1; else lo1 = m1; }
      }
      lam[j0] = 0.5f * (lo0 + hi0);
      if (j1 != j0) lam[j1] = 0.5f * (lo1 + hi1);
    }
  }
  __syncthreads();

  if (pr) prof[2] = clock64();
  // step 3: eigenvectors of T, rows of Zt
  {
    const int S = n < nt ? n : nt;   // scratch stride
    if (tid < S) {
      float* Lp = tw.glu;
      float* Um = tw.glu + (long long)n * S;
      for (int j = tid; j < n; j += S) {
        const float lm = lam[j];
        int bad = 0;
        float Dp = d[0] - lm;
        if (fabsf(Dp) < pivmin) Dp = -pivmin;
#pragma unroll 4
        for (int i = 0; i < n - 1; ++i) {
          const float L = e[i] / Dp;
          Lp[(long long)i * S + tid] = L;
          Dp = (d[i + 1] - lm) - L * e[i];
          if (fabsf(Dp) < pivmin) Dp = -pivmin;
        }
        float gmin = fabsf(Dp);   // gamma_{n-1} = D+_{n-1}
        int r = n - 1;
        float Dm = d[n - 1] - lm;
        if (fabsf(Dm) < pivmin) Dm = -pivmin;
#pragma unroll 4
        for (int i = n - 2; i >= 0; --i) {
          const float U = e[i] / Dm;
          Um[(long long)i * S + tid] = U;
          const float dl = d[i] - lm;
          Dm = dl - U * e[i];
          if (fabsf(Dm) < pivmin) Dm = -pivmin;
          const float up = i > 0 ? Lp[(long long)(i - 1) * S + tid] * e[i - 1] : 0.f;
          const float g = dl - up - U * e[i];
          if (fabsf(g) < gmin) { gmin = fabsf(g); r = i; }
        }
        float* zr = Zt + (long long)j * n;
        float z = 1.f, nrm = 1.f;
        zr[r] = 1.f;
#pragma unroll 4
        for (int i = r - 1; i >= 0; --i) {
          z = -Lp[(long long)i * S + tid] * z;
          zr[i] = z;
          nrm = fmaf(z, z, nrm);
        }
        z = 1.f;
#pragma unroll 4
        for (int i = r + 1; i < n; ++i) {
          z = -Um[(long long)(i - 1) * S + tid] * z;
          zr[i] = z;
          nrm = fmaf(z, z, nrm);
        }
        if (!(nrm < 1e30f)) bad = 1;   // overflow or NaN
        inv[j] = rsqrtf(nrm);
        if (bad) s_fail = 1;
      }
    }
    if (pr) prof[3] = clock64();
    // clusters: eigenvalues closer than 1e-3 |T| to their predecessor
    if (tid == 0) {
      const float tc = float(1e-3 * tnorm);
      int c = 0;
      for (int j = 0; j < n; ++j)
        if (j == 0 || lam[j] - lam[j - 1] > tc) cl[c++] = j;
      cl[c] = n;
      s_ncl = c;
    }
    __syncthreads();
    const int ncl = s_ncl;
    for (int c = wid; c < ncl; c += nw) {
      const int j0 = cl[c], j1 = cl[c + 1];
      for (int m = j0; m < j1; ++m) {
        float z[kC];
        float* zr = Zt + (long long)m * n;
        const float s0 = inv[m];
#pragma unroll
        for (int q = 0; q < kC; ++q) {
          const int i = 32 * q + lane;
          z[q] = i < n ? zr[i] * s0 : 0.f;
        }
        if (m > j0) {
          for (int pidx = j0; pidx < m; ++pidx) {
            const float* zp = Zt + (long long)pidx * n;
            float dot = 0.f;
#pragma unroll
            for (int q = 0; q < kC; ++q) {
              const int i = 32 * q + lane;
              if (i < n) dot = fmaf(z[q], zp[i], dot);
            }
            dot = warp_sum(dot);
#pragma unroll
            for (int q = 0; q < kC; ++q) {
              const int i = 32 * q + lane;
              if (i < n) z[q] = fmaf(-dot, zp[i], z[q]);
            }
          }
          float nr = 0.f;
#pragma unroll
          for (int q = 0; q < kC; ++q) nr = fmaf(z[q], z[q], nr);
          nr = warp_sum(nr);
          if (!(nr > 1e-4f)) {
            if (lane == 0) s_fail = 1;
            nr = 1.f;
          }
          const float sc = rsqrtf(nr);
#pragma unroll
          for (int q = 0; q < kC; ++q) z[q] *= sc;
        }
#pragma unroll
        for (int q = 0; q < kC; ++q) {
          const int i = 32 * q + lane;
          if (i < n) zr[i] = z[q];
        }
      }
    }
  }
  __syncthreads();
  if (s_fail) {
    for (long long x = tid; x < (long long)n * lda; x += nt) A[x] = tw.abak[x];
    __syncthreads();
    return false;
  }

  if (pr) prof[4] = clock64();
  // step 4: Zt <- Zt H_{n-3} ... H_0 (kR rows per warp in registers), then
  // CT <- Zt CT
  constexpr int kR = 8;
  for (int r0 = kR * wid; r0 < n; r0 += kR * nw) {
    float z[kR][kC];
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      const float* a = Zt + (long long)(r0 + r < n ? r0 + r : r0) * n;
#pragma unroll
      for (int q = 0; q < kC; ++q) {
        const int i = 32 * q + lane;
        z[r][q] = i < n ? a[i] : 0.f;
      }
    }
    for (int k = n - 3; k >= 0; --k) {
      const float tk = tau[k];
      if (tk == 0.f) continue;
      const float* uk = A + (long long)k * lda;
      float uu[kC];
#pragma unroll
      for (int q = 0; q < kC; ++q) {
        const int i = 32 * q + lane;
        uu[q] = (i > k && i < n) ? uk[i] : 0.f;
      }
      float sr[kR];
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < kC; ++q) t = fmaf(z[r][q], uu[q], t);
        sr[r] = t;
      }
      // kR sums over the warp: butterfly, every lane ends with every sum
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int r = 0; r < kR; ++r) sr[r] += __shfl_xor_sync(0xffffffffu, sr[r], o);
      }
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const float g = sr[r] * tk;
#pragma unroll
        for (int q = 0; q < kC; ++q) z[r][q] = fmaf(-g, uu[q], z[r][q]);
      }
    }
#pragma unroll
    for (int r = 0; r < kR; ++r) {
      if (r0 + r < n) {
        float* b = Zt + (long long)(r0 + r) * n;
#pragma unroll
        for (int q = 0; q < kC; ++q) {
          const int i = 32 * q + lane;
          if (i < n) b[i] = z[r][q];
        }
      }
    }
  }
  for (int j = tid; j < n; j += nt) eps[j] = double(lam[j]);
  __syncthreads();
  if (pr) prof[5] = clock64();
  block_gemm<float>(n, n, n, Zt, n, 1, CT, 1, n, W, n, nullptr, nullptr, nullptr, gemm);
  for (long long x = tid; x < (long long)n * n; x += nt) CT[x] = W[x];
  __syncthreads();
  if (pr) prof[6] = clock64();
  return true;
}

}  // namespace fmo
