// Density-matrix purification: the occupied-subspace projector of a batch of
// orthogonalised Fock matrices from matrix products alone, in place of the
// diagonalisation that makes each SCC iteration cubic (Introduction; the
// GFN1-xTB SCC step of the Methodology).  Second-order spectral projection
// (SP2, Niklasson, Phys. Rev. B 66, 155115 (2002)):
//   X0 = (e_max I - F) / (e_max - e_min)      (Gershgorin bounds, spectrum in [0,1],
//                                              lowest orbital energies near 1)
//   X <- X^2        if |tr(X^2) - n_occ| < |2 tr(X) - tr(X^2) - n_occ|
//   X <- 2X - X^2   otherwise
// until the idempotency error tr(X) - tr(X^2) stops falling (parameter-free
// stop: no decrease over two steps once it is below a gate, 1e-6 in FP64).
//
// One CTA per matrix; X lives in the output buffer and X^2 in the caller's
// work buffer (both n x n row-major, L2-resident for n-mer sizes); products
// through 32 x 32 shared-memory tiles in FP64 or, for the loose iterations of
// a mixed-precision SCC, in FP32.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "../../include/fmo_xtb.h"

namespace {

constexpr int kThreads = 256;
constexpr int kTile = 32;

__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < kThreads / 32; ++i) s += red[i];   // same order in every thread
  return s;
}

__device__ double block_min(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = red[0];
  for (int i = 1; i < kThreads / 32; ++i) s = fmin(s, red[i]);
  return s;
}

// Y = X X for one symmetric n x n matrix; every thread of the CTA takes part.
// Y is symmetric too: only the tiles on and above the diagonal are computed,
// each off-diagonal one also stored transposed (through shared memory, so
// both stores are row-contiguous).
template <typename T>
__device__ void square(const T *X, T *Y, int n, T (*As)[kTile + 1], T (*Bs)[kTile + 1]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // ty in 0..7
  const int nt = (n + kTile - 1) / kTile;
  for (int t = 0; t < nt * nt; ++t) {
    const int ti = t / nt, tj = t % nt;
    if (tj < ti) continue;                 // uniform over the CTA
    const int i0 = ti * kTile, j0 = tj * kTile;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int k0 = 0; k0 < n; k0 += kTile) {
      for (int r = ty; r < kTile; r += kThreads / 32) {
        const int ia = i0 + r, ka = k0 + tx, kb = k0 + r, jb = j0 + tx;
        As[r][tx] = (ia < n && ka < n) ? X[(size_t)ia * n + ka] : T(0);
        Bs[r][tx] = (kb < n && jb < n) ? X[(size_t)kb * n + jb] : T(0);
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < kTile; ++kk) {
        const T b = Bs[kk][tx];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(As[ty + 8 * q][kk], b, acc[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty + 8 * q, j = j0 + tx;
      if (i < n && j < n) Y[(size_t)i * n + j] = acc[q];
    }
    if (tj > ti) {
      // the k-loop ended on a barrier, so As is free
#pragma unroll
      for (int q = 0; q < 4; ++q) As[ty + 8 * q][tx] = acc[q];
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = ty + 8 * q;          // row of the transposed tile
        const int i = j0 + r, j = i0 + tx;
        if (i < n && j < n) Y[(size_t)i * n + j] = As[tx][r];
      }
      __syncthreads();
    }
  }
}

// Stop gate on the idempotency error: FP64 reaches ~1e-13; FP32 stalls near
// n * 1e-7, so its parameter-free stop is opened at 1e-2 (all eigenvalues of X
// within ~1e-2 of 0 or 1, where the error falls quadratically until rounding).
template <typename T> struct Sp2Gate;
template <> struct Sp2Gate<double> { static constexpr double value = 1e-6; };
template <> struct Sp2Gate<float> { static constexpr double value = 1e-2; };

// Traces and the branch decision are taken in FP64 in both precisions.
template <typename T>
__global__ void __launch_bounds__(kThreads) sp2_kernel(const T *__restrict__ F,
                                                       const int32_t *__restrict__ n_occ, int n,
                                                       int max_iter, T *D, T *W, int32_t *iters) {
  __shared__ T As[kTile][kTile + 1];
  __shared__ T Bs[kTile][kTile + 1];
  __shared__ double red[kThreads / 32];
  const size_t nn = (size_t)n * n;
  const T *f = F + blockIdx.x * nn;
  T *X = D + blockIdx.x * nn;
  T *Y = W + blockIdx.x * nn;
  const int occ = n_occ[blockIdx.x];
  if (occ < 0 || occ > n) {
    if (threadIdx.x == 0) iters[blockIdx.x] = -2;
    return;
  }

  // Gershgorin interval [lo, hi] holding the spectrum of F
  double lo = CUDART_INF, nhi = CUDART_INF;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    double r = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) r += fabs(f[(size_t)i * n + j]);
    lo = fmin(lo, f[(size_t)i * n + i] - r);
    nhi = fmin(nhi, -(f[(size_t)i * n + i] + r));
  }
  lo = block_min(lo, red);
  const double hi = -block_min(nhi, red);
  const double scale = hi > lo ? 1.0 / (hi - lo) : 0.0;
  for (size_t idx = threadIdx.x; idx < nn; idx += kThreads) {
    const size_t i = idx / n, j = idx % n;
    X[idx] = (T)(((i == j ? hi : 0.0) - (double)f[idx]) * scale);
  }
  __syncthreads();

  double e1 = CUDART_INF, e2 = CUDART_INF;
  int done = -1;
  for (int it = 1; it <= max_iter; ++it) {
    square(X, Y, n, As, Bs);
    __syncthreads();
    double tx = 0.0, ty = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
      tx += (double)X[(size_t)i * n + i];
      ty += (double)Y[(size_t)i * n + i];
    }
    tx = block_sum(tx, red);
    ty = block_sum(ty, red);
    const double e = fabs(tx - ty);
    const bool sq = fabs(ty - occ) < fabs(2.0 * tx - ty - occ);
    for (size_t idx = threadIdx.x; idx < nn; idx += kThreads)
      X[idx] = sq ? Y[idx] : T(2) * X[idx] - Y[idx];
    __syncthreads();
    if (e < Sp2Gate<T>::value && e >= e2) {
      // a gapless F (e.g. a multiple of I) can stall at a non-projector
      // whose trace is not n_occ: reported as not converged
      const double tr_new = sq ? ty : 2.0 * tx - ty;
      done = fabs(tr_new - occ) < 0.5 ? it : -1;
      break;
    }
    e2 = e1;
    e1 = e;
  }
  if (threadIdx.x == 0) iters[blockIdx.x] = done;
}

}  // namespace

extern "C" fmo_status fmo_sp2_projector(const double *F_dev, const int32_t *n_occ_dev, int32_t n,
                                        int32_t batch, int32_t max_iter, double *D_dev,
                                        double *work_dev, int32_t *iters_dev, void *cuda_stream) {
  if (n < 1 || n > FMO_SP2_MAX_N || batch < 0 || max_iter < 1) return FMO_ERR_ARG;
  if (batch == 0) return FMO_OK;
  if (!F_dev || !n_occ_dev || !D_dev || !work_dev || !iters_dev) return FMO_ERR_ARG;
  sp2_kernel<double><<<batch, kThreads, 0, (cudaStream_t)cuda_stream>>>(
      F_dev, n_occ_dev, n, max_iter, D_dev, work_dev, iters_dev);
  return cudaGetLastError() == cudaSuccess ? FMO_OK : FMO_ERR_CUDA;
}

extern "C" fmo_status fmo_sp2_projector_f32(const float *F_dev, const int32_t *n_occ_dev,
                                            int32_t n, int32_t batch, int32_t max_iter,
                                            float *D_dev, float *work_dev, int32_t *iters_dev,
                                            void *cuda_stream) {
  if (n < 1 || n > FMO_SP2_MAX_N || batch < 0 || max_iter < 1) return FMO_ERR_ARG;
  if (batch == 0) return FMO_OK;
  if (!F_dev || !n_occ_dev || !D_dev || !work_dev || !iters_dev) return FMO_ERR_ARG;
  sp2_kernel<float><<<batch, kThreads, 0, (cudaStream_t)cuda_stream>>>(
      F_dev, n_occ_dev, n, max_iter, D_dev, work_dev, iters_dev);
  return cudaGetLastError() == cudaSuccess ? FMO_OK : FMO_ERR_CUDA;
}
