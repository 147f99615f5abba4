// Learned initial shell charges (the guess of the monomer loop): descriptors,
// the embedding-ESP feature, a 77-128-128-2 SiLU MLP with FP16 weights and
// FP32 accumulation, the per-fragment neutrality projection, the MSE loss,
// backward and Adam.  The paper has no learned guess; the model is the one the
// oracle (oracle/mlp.py) defines:
//   radial   G_{e,k} = sum_{j of element e} exp(-ETA_R (r_ij - RS_k)^2) fc(r_ij)
//   angular  G_{p,t} = 2^(1-zeta) sum_{j<k, {e_j,e_k}=p} (1 + lambda cos theta)^zeta
//                      exp(-ETA_A (r_ij^2 + r_ik^2)) fc(r_ij) fc(r_ik)
//   fc(r) = (cos(pi r / RC) + 1) / 2 for r < RC = 6 A
// Feature layout (stride kMlpStride floats per atom): 0..31 radial (element
// major), 32..71 angular (pair major), 72 ESP, 73..76 element one-hot.
#include <cuda_fp16.h>

#include <cmath>

#include "mlp.h"

namespace fmo {

namespace {

constexpr float kRc = 6.0f;
constexpr float kEtaR = 2.0f;          // 1 / (2 * 0.5^2) A^-2
constexpr float kEtaA = 0.02f;         // A^-2
constexpr float kBohrToA = 0.529177210903f;
constexpr int kMaxNb = 256;            // neighbours within RC per atom
constexpr int kWarpsPerBlock = 4;

__device__ __forceinline__ float fcut(float r) { return r < kRc ? 0.5f * (cosf(3.14159265358979f * r / kRc) + 1.0f) : 0.0f; }

__device__ __forceinline__ float wsum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ int pair_index(int a, int b) {   // unordered element pair, a <= b
  // (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3)
  return a * 4 - a * (a - 1) / 2 + (b - a);
}

__device__ __forceinline__ float silu(float x) { return x / (1.0f + expf(-x)); }
__device__ __forceinline__ float dsilu(float x) {
  const float s = 1.0f / (1.0f + expf(-x));
  return s * (1.0f + x * (1.0f - s));
}

}  // namespace

// Geometric descriptors of every atom of n_frames frames (one warp per atom;
// frames stacked, n_atoms each).  xyz in bohr; elem4: element index 0..3
// (H, C, N, O).  Writes features 0..71 and 73..76, zero at 72.
__global__ void __launch_bounds__(32 * kWarpsPerBlock) mlp_descriptor_kernel(
    int n_frames, int n_atoms, const double* __restrict__ xyz, const int* __restrict__ elem4,
    float* __restrict__ X, int* __restrict__ err) {
  __shared__ int s_nb[kWarpsPerBlock][kMaxNb];
  __shared__ int s_cnt[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kWarpsPerBlock + w;
  if (gw >= (long long)n_frames * n_atoms) return;
  const int frame = int(gw / n_atoms), i = int(gw - (long long)frame * n_atoms);
  const double* fx = xyz + (size_t)frame * n_atoms * 3;
  const float xi = float(fx[3 * i]) * kBohrToA, yi = float(fx[3 * i + 1]) * kBohrToA,
              zi = float(fx[3 * i + 2]) * kBohrToA;
  // neighbour list (ascending index: ballots)
  int cnt = 0;
  for (int base = 0; base < n_atoms; base += 32) {
    const int j = base + lane;
    bool in = false;
    if (j < n_atoms && j != i) {
      const float dx = float(fx[3 * j]) * kBohrToA - xi, dy = float(fx[3 * j + 1]) * kBohrToA - yi,
                  dz = float(fx[3 * j + 2]) * kBohrToA - zi;
      in = dx * dx + dy * dy + dz * dz < kRc * kRc;
    }
    const unsigned b = __ballot_sync(0xffffffffu, in);
    const int pos = cnt + __popc(b & ((1u << lane) - 1u));
    if (in && pos < kMaxNb) s_nb[w][pos] = j;
    cnt += __popc(b);
  }
  if (cnt > kMaxNb) {
    if (lane == 0) atomicExch(err, 1);
    cnt = kMaxNb;
  }
  __syncwarp();
  float rad[32], ang[40];
#pragma unroll
  for (int k = 0; k < 32; ++k) rad[k] = 0.0f;
#pragma unroll
  for (int k = 0; k < 40; ++k) ang[k] = 0.0f;
  for (int a = lane; a < cnt; a += 32) {
    const int j = s_nb[w][a];
    const float dx = float(fx[3 * j]) * kBohrToA - xi, dy = float(fx[3 * j + 1]) * kBohrToA - yi,
                dz = float(fx[3 * j + 2]) * kBohrToA - zi;
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    const float fc = fcut(r);
    const int e = elem4[j];
#pragma unroll
    for (int ee = 0; ee < 4; ++ee) {
      if (ee != e) continue;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float rs = 0.8f + k * (kRc - 0.8f) / 7.0f;
        rad[ee * 8 + k] += expf(-kEtaR * (r - rs) * (r - rs)) * fc;
      }
    }
  }
  // angular terms: lanes over the neighbour pairs (a < b)
  const int npair = cnt * (cnt - 1) / 2;
  for (int q = lane; q < npair; q += 32) {
    // q -> (a, b) with a < b, rows a hold cnt-1-a entries
    int a = 0, rem = q;
    while (rem >= cnt - 1 - a) { rem -= cnt - 1 - a; ++a; }
    const int b = a + 1 + rem;
    const int j = s_nb[w][a], k = s_nb[w][b];
    const float ax = float(fx[3 * j]) * kBohrToA - xi, ay = float(fx[3 * j + 1]) * kBohrToA - yi,
                az = float(fx[3 * j + 2]) * kBohrToA - zi;
    const float bx = float(fx[3 * k]) * kBohrToA - xi, by = float(fx[3 * k + 1]) * kBohrToA - yi,
                bz = float(fx[3 * k + 2]) * kBohrToA - zi;
    const float r1s = ax * ax + ay * ay + az * az, r2s = bx * bx + by * by + bz * bz;
    const float r1 = sqrtf(r1s), r2 = sqrtf(r2s);
    const float c = (ax * bx + ay * by + az * bz) / (r1 * r2);
    const float wgt = expf(-kEtaA * (r1s + r2s)) * fcut(r1) * fcut(r2);
    const int e1 = elem4[j], e2 = elem4[k];
    const int p = pair_index(min(e1, e2), max(e1, e2));
    const float t0 = (1.0f + c) * wgt, t1 = (1.0f - c) * wgt;
    const float u0 = (1.0f + c) * (1.0f + c), u1 = (1.0f - c) * (1.0f - c);
    const float t2 = 0.125f * u0 * u0 * wgt, t3 = 0.125f * u1 * u1 * wgt;
#pragma unroll
    for (int pp = 0; pp < 10; ++pp) {
      if (pp != p) continue;
      ang[4 * pp] += t0;
      ang[4 * pp + 1] += t1;
      ang[4 * pp + 2] += t2;
      ang[4 * pp + 3] += t3;
    }
  }
  float* out = X + (size_t)gw * kMlpStride;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const float v = wsum(rad[k]);
    if (lane == 0) out[k] = v;
  }
#pragma unroll
  for (int k = 0; k < 40; ++k) {
    const float v = wsum(ang[k]);
    if (lane == 0) out[32 + k] = v;
  }
  if (lane < kMlpStride - 72) {
    const int f = 72 + lane;
    out[f] = (f >= 73 && f < 77) ? (elem4[i] == f - 73 ? 1.0f : 0.0f) : 0.0f;
  }
}

// ESP feature: phi at every atom (its first shell's 1/eta) from the shell
// charges of all other fragments of the same frame, gamma with k_g = 2
// (Eqs. 4-5).  One warp per atom.
__global__ void mlp_esp_kernel(int n_frames, int n_atoms, int n_sh, const double* __restrict__ xyz,
                               const int* __restrict__ atom_frag, const float* __restrict__ atom_ie,
                               const int* __restrict__ sh_atom, const float* __restrict__ sh_ie,
                               const float* __restrict__ dq, float* __restrict__ X) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (long long)n_frames * n_atoms) return;
  const int frame = int(gw / n_atoms), i = int(gw - (long long)frame * n_atoms);
  const double* fx = xyz + (size_t)frame * n_atoms * 3;
  const float* fq = dq + (size_t)frame * n_sh;
  const double xi = fx[3 * i], yi = fx[3 * i + 1], zi = fx[3 * i + 2];
  const float iei = atom_ie[i];
  const int fi = atom_frag[i];
  float v = 0.0f;
  for (int s = lane; s < n_sh; s += 32) {
    const int b = sh_atom[s];
    if (atom_frag[b] == fi) continue;
    const float dx = float(fx[3 * b] - xi), dy = float(fx[3 * b + 1] - yi), dz = float(fx[3 * b + 2] - zi);
    const float e = 0.5f * (iei + sh_ie[s]);
    v += fq[s] * rsqrtf(dx * dx + dy * dy + dz * dz + e * e);
  }
  v = wsum(v);
  if (lane == 0) X[(size_t)gw * kMlpStride + 72] = v;
}

// Forward pass of n rows of X; 128 threads per block (one per hidden unit),
// 32 rows per tile.  Optional cache of x0 (standardised input), z1, h1, z2,
// h2 for the backward pass.
__global__ void __launch_bounds__(128) mlp_forward_kernel(int n, const float* __restrict__ X,
                                                         const __half* __restrict__ W16,
                                                         const float* __restrict__ mean,
                                                         const float* __restrict__ scale, float* __restrict__ y,
                                                         MlpCache cache) {
  __shared__ float s_x[32][kMlpIn + 1];
  __shared__ float s_h[32][kMlpHidden + 1];
  const int t = threadIdx.x;
  const __half* W1 = W16 + kMlpOffW1;
  const __half* W2 = W16 + kMlpOffW2;
  const __half* W3 = W16 + kMlpOffW3;
  const float b1 = __half2float(W16[kMlpOffB1 + t]), b2 = __half2float(W16[kMlpOffB2 + t]);
  for (int r0 = blockIdx.x * 32; r0 < n; r0 += gridDim.x * 32) {
    const int nr = min(32, n - r0);
    for (int e = t; e < 32 * kMlpIn; e += 128) {
      const int r = e / kMlpIn, k = e - r * kMlpIn;
      const float v = (r < nr) ? (X[(size_t)(r0 + r) * kMlpStride + k] - mean[k]) * scale[k] : 0.0f;
      s_x[r][k] = v;
      if (cache.x0 && r < nr) cache.x0[(size_t)(r0 + r) * kMlpStride + k] = v;
    }
    __syncthreads();
    float acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = b1;
    for (int k = 0; k < kMlpIn; ++k) {
      const float wv = __half2float(W1[t * kMlpIn + k]);
#pragma unroll
      for (int r = 0; r < 32; ++r) acc[r] = fmaf(wv, s_x[r][k], acc[r]);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const float h = silu(acc[r]);
      s_h[r][t] = h;
      if (cache.z1 && r < nr) {
        cache.z1[(size_t)(r0 + r) * kMlpHidden + t] = acc[r];
        cache.h1[(size_t)(r0 + r) * kMlpHidden + t] = h;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = b2;
    for (int k = 0; k < kMlpHidden; ++k) {
      const float wv = __half2float(W2[t * kMlpHidden + k]);
#pragma unroll
      for (int r = 0; r < 32; ++r) acc[r] = fmaf(wv, s_h[r][k], acc[r]);
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const float h = silu(acc[r]);
      s_h[r][t] = h;
      if (cache.z2 && r < nr) {
        cache.z2[(size_t)(r0 + r) * kMlpHidden + t] = acc[r];
        cache.h2[(size_t)(r0 + r) * kMlpHidden + t] = h;
      }
    }
    __syncthreads();
    if (t < 64) {
      const int r = t >> 1, o = t & 1;
      if (r < nr) {
        float v = __half2float(W16[kMlpOffB3 + o]);
        for (int k = 0; k < kMlpHidden; ++k) v = fmaf(__half2float(W3[o * kMlpHidden + k]), s_h[r][k], v);
        y[(size_t)(r0 + r) * 2 + o] = v;
      }
    }
    __syncthreads();
  }
}

// Per (frame, fragment) block: shell charges q = y shifted so the fragment
// sums to minus its charge; with a target also the residual's squared sum
// (loss_part[block]) and the gradient of mean((q - target)^2) projected back
// onto y (the projection is linear and self-adjoint).  Atoms of a fragment
// are contiguous (2 shells each).
__global__ void mlp_project_kernel(int n_frag, int n_atoms, const int* __restrict__ f_atom0,
                                   const int* __restrict__ f_nat, const int* __restrict__ f_charge,
                                   const float* __restrict__ y, float* __restrict__ q,
                                   const float* __restrict__ target, double inv_count,
                                   float* __restrict__ gy, double* __restrict__ loss_part) {
  __shared__ float red[32];
  const int frame = blockIdx.x / n_frag, f = blockIdx.x - frame * n_frag;
  const size_t base = (size_t)frame * n_atoms * 2 + (size_t)f_atom0[f] * 2;
  const int m = 2 * f_nat[f];
  auto bsum = [&](float v) {
    v = wsum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.0f;
    if (threadIdx.x < 32) {
      s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0f;
      s = wsum(s);
    }
    __syncthreads();
    if (threadIdx.x == 0) red[0] = s;
    __syncthreads();
    const float r = red[0];
    __syncthreads();
    return r;
  };
  float s = 0.0f;
  for (int k = threadIdx.x; k < m; k += blockDim.x) s += y[base + k];
  const float shift = (bsum(s) + float(f_charge[f])) / float(m);
  float rs = 0.0f, gs = 0.0f;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const float v = y[base + k] - shift;
    q[base + k] = v;
    if (target) {
      const float r = v - target[base + k];
      rs += r * r;
      gs += r;
    }
  }
  if (!target) return;
  const float rsum = bsum(rs), gsum = bsum(gs);
  const float gmean = gsum / float(m);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const float r = q[base + k] - target[base + k];
    gy[base + k] = float(2.0 * inv_count) * (r - gmean);
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = double(rsum);
}

// Backward through the hidden layers, per row: gz2 = (gy W3) * silu'(z2),
// gz1 = (gz2 W2) * silu'(z1).  128 threads, 32 rows per tile.
__global__ void __launch_bounds__(128) mlp_backprop_kernel(int n, const float* __restrict__ gy,
                                                          const __half* __restrict__ W16, MlpCache cache,
                                                          float* __restrict__ gz2, float* __restrict__ gz1) {
  __shared__ float s_g[32][kMlpHidden + 1];
  const int t = threadIdx.x;
  const __half* W2 = W16 + kMlpOffW2;
  const __half* W3 = W16 + kMlpOffW3;
  const float w30 = __half2float(W3[t]), w31 = __half2float(W3[kMlpHidden + t]);
  for (int r0 = blockIdx.x * 32; r0 < n; r0 += gridDim.x * 32) {
    const int nr = min(32, n - r0);
    for (int r = 0; r < 32; ++r) {
      float v = 0.0f;
      if (r < nr) {
        v = (gy[(size_t)(r0 + r) * 2] * w30 + gy[(size_t)(r0 + r) * 2 + 1] * w31) *
            dsilu(cache.z2[(size_t)(r0 + r) * kMlpHidden + t]);
        gz2[(size_t)(r0 + r) * kMlpHidden + t] = v;
      }
      s_g[r][t] = v;
    }
    __syncthreads();
    float acc[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) acc[r] = 0.0f;
    for (int k = 0; k < kMlpHidden; ++k) {
      const float wv = __half2float(W2[k * kMlpHidden + t]);   // (W2^T)_{t,k}
#pragma unroll
      for (int r = 0; r < 32; ++r) acc[r] = fmaf(wv, s_g[r][k], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (r < nr) gz1[(size_t)(r0 + r) * kMlpHidden + t] = acc[r] * dsilu(cache.z1[(size_t)(r0 + r) * kMlpHidden + t]);
    __syncthreads();
  }
}

// Weight gradients summed over one chunk of rows (partial[blockIdx.x] over
// the trained weights, kMlpTrained floats): every thread owns a fixed set of
// weight entries and loops over the chunk's rows in order.
__global__ void __launch_bounds__(256) mlp_wgrad_kernel(int n, int chunk, const float* __restrict__ gy,
                                                       const float* __restrict__ gz2, const float* __restrict__ gz1,
                                                       MlpCache cache, float* __restrict__ partial) {
  const int r0 = blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  float* out = partial + (size_t)blockIdx.x * kMlpTrained;
  for (int w = threadIdx.x; w < kMlpTrained; w += blockDim.x) {
    float acc = 0.0f;
    if (w < kMlpOffB1) {                                  // W1 (hidden x in)
      const int o = w / kMlpIn, i = w - o * kMlpIn;
      for (int r = r0; r < r1; ++r) acc = fmaf(gz1[(size_t)r * kMlpHidden + o], cache.x0[(size_t)r * kMlpStride + i], acc);
    } else if (w < kMlpOffW2) {                           // b1
      const int o = w - kMlpOffB1;
      for (int r = r0; r < r1; ++r) acc += gz1[(size_t)r * kMlpHidden + o];
    } else if (w < kMlpOffB2) {                           // W2
      const int o = (w - kMlpOffW2) / kMlpHidden, i = (w - kMlpOffW2) - o * kMlpHidden;
      for (int r = r0; r < r1; ++r) acc = fmaf(gz2[(size_t)r * kMlpHidden + o], cache.h1[(size_t)r * kMlpHidden + i], acc);
    } else if (w < kMlpOffW3) {                           // b2
      const int o = w - kMlpOffB2;
      for (int r = r0; r < r1; ++r) acc += gz2[(size_t)r * kMlpHidden + o];
    } else if (w < kMlpOffB3) {                           // W3
      const int o = (w - kMlpOffW3) / kMlpHidden, i = (w - kMlpOffW3) - o * kMlpHidden;
      for (int r = r0; r < r1; ++r) acc = fmaf(gy[(size_t)r * 2 + o], cache.h2[(size_t)r * kMlpHidden + i], acc);
    } else {                                              // b3
      const int o = w - kMlpOffB3;
      for (int r = r0; r < r1; ++r) acc += gy[(size_t)r * 2 + o];
    }
    out[w] = acc;
  }
}

// Sum of the chunk partials in chunk order, then one Adam step (Kingma & Ba,
// beta1 0.9, beta2 0.999, eps 1e-8) of the FP32 master weights and their FP16
// copy.
__global__ void mlp_adam_kernel(int n_chunks, const float* __restrict__ partial, float* __restrict__ W,
                                float* __restrict__ m, float* __restrict__ v, __half* __restrict__ W16, float lr,
                                float bc1, float bc2) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= kMlpTrained) return;
  float g = 0.0f;
  for (int c = 0; c < n_chunks; ++c) g += partial[(size_t)c * kMlpTrained + w];
  const float mm = 0.9f * m[w] + 0.1f * g;
  const float vv = 0.999f * v[w] + 0.001f * g * g;
  m[w] = mm;
  v[w] = vv;
  const float nw = W[w] - lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
  W[w] = nw;
  W16[w] = __float2half_rn(nw);
}

// Sum of the chunk partials in chunk order: the gradient of the batch loss.
__global__ void mlp_grad_sum_kernel(int n_chunks, const float* __restrict__ partial, float* __restrict__ grad) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= kMlpTrained) return;
  float g = 0.0f;
  for (int c = 0; c < n_chunks; ++c) g += partial[(size_t)c * kMlpTrained + w];
  grad[w] = g;
}

__global__ void mlp_to_half_kernel(int n, const float* __restrict__ W, __half* __restrict__ W16) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < n) W16[w] = __float2half_rn(W[w]);
}

// Mean and 1/(std + 1) of the first 72 feature columns over all rows (fixed
// order: one block per column).
__global__ void mlp_feature_stats_kernel(long long n, const float* __restrict__ X, float* __restrict__ mean,
                                         float* __restrict__ scale) {
  __shared__ double red[2][256];
  const int k = blockIdx.x;
  double s = 0.0, s2 = 0.0;
  for (long long r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = X[(size_t)r * kMlpStride + k];
    s += v;
    s2 += v * v;
  }
  red[0][threadIdx.x] = s;
  red[1][threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double mu = red[0][0] / double(n);
    const double var = fmax(red[1][0] / double(n) - mu * mu, 0.0);
    mean[k] = float(mu);
    scale[k] = float(1.0 / (sqrt(var) + 1.0));
  }
}

// shell charges (float, frames stacked) -> double copy of one frame
__global__ void mlp_to_double_kernel(int n, const float* __restrict__ q, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = double(q[i]);
}

// rows of the frames listed in idx (batch order) gathered from the stored
// features and coordinates
__global__ void mlp_gather_kernel(int n_batch, int n_atoms, const int* __restrict__ idx,
                                  const float* __restrict__ Xall, const double* __restrict__ xyz_all,
                                  float* __restrict__ Xb, double* __restrict__ xyz_b) {
  const long long per = (long long)n_atoms * kMlpStride;
  const long long tot = per * n_batch;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int b = int(e / per);
    Xb[e] = Xall[(size_t)idx[b] * per + (e - (long long)b * per)];
  }
  const long long pc = (long long)n_atoms * 3;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < pc * n_batch; e += (long long)gridDim.x * blockDim.x) {
    const int b = int(e / pc);
    xyz_b[e] = xyz_all[(size_t)idx[b] * pc + (e - (long long)b * pc)];
  }
}

#define MLP_CHECK()                                  \
  do {                                               \
    note_launch();                                   \
    cudaError_t e_ = cudaGetLastError();             \
    if (e_ != cudaSuccess) return e_;                \
  } while (0)

cudaError_t mlp_descriptors(cudaStream_t st, int n_frames, int n_atoms, const double* xyz, const int* elem4,
                            float* X, int* err) {
  const long long warps = (long long)n_frames * n_atoms;
  mlp_descriptor_kernel<<<(int)((warps + kWarpsPerBlock - 1) / kWarpsPerBlock), 32 * kWarpsPerBlock, 0, st>>>(
      n_frames, n_atoms, xyz, elem4, X, err);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_esp(cudaStream_t st, int n_frames, int n_atoms, int n_sh, const double* xyz, const int* atom_frag,
                    const float* atom_ie, const int* sh_atom, const float* sh_ie, const float* dq, float* X) {
  const long long warps = (long long)n_frames * n_atoms;
  mlp_esp_kernel<<<(int)((warps * 32 + 255) / 256), 256, 0, st>>>(n_frames, n_atoms, n_sh, xyz, atom_frag, atom_ie,
                                                                   sh_atom, sh_ie, dq, X);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_forward(cudaStream_t st, int n, const float* X, const __half* W16, const float* mean,
                        const float* scale, float* y, const MlpCache& cache) {
  const int blocks = std::min((n + 31) / 32, 148 * 8);
  mlp_forward_kernel<<<blocks, 128, 0, st>>>(n, X, W16, mean, scale, y, cache);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_project(cudaStream_t st, int n_frames, int n_frag, int n_atoms, const int* f_atom0, const int* f_nat,
                        const int* f_charge, const float* y, float* q, const float* target, double inv_count,
                        float* gy, double* loss_part) {
  mlp_project_kernel<<<n_frames * n_frag, 64, 0, st>>>(n_frag, n_atoms, f_atom0, f_nat, f_charge, y, q, target,
                                                       inv_count, gy, loss_part);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_backward_step(cudaStream_t st, int n, const float* gy, const __half* W16, const MlpCache& cache,
                              float* gz2, float* gz1, float* partial, int chunk, float* W, float* m, float* v,
                              __half* W16out, float lr, int t) {
  const int blocks = std::min((n + 31) / 32, 148 * 8);
  mlp_backprop_kernel<<<blocks, 128, 0, st>>>(n, gy, W16, cache, gz2, gz1);
  MLP_CHECK();
  const int n_chunks = (n + chunk - 1) / chunk;
  mlp_wgrad_kernel<<<n_chunks, 256, 0, st>>>(n, chunk, gy, gz2, gz1, cache, partial);
  MLP_CHECK();
  const float bc1 = 1.0f - powf(0.9f, float(t)), bc2 = 1.0f - powf(0.999f, float(t));
  mlp_adam_kernel<<<(kMlpTrained + 255) / 256, 256, 0, st>>>(n_chunks, partial, W, m, v, W16out, lr, bc1, bc2);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_gradient(cudaStream_t st, int n, const float* gy, const __half* W16, const MlpCache& cache,
                         float* gz2, float* gz1, float* partial, int chunk, float* grad) {
  const int blocks = std::min((n + 31) / 32, 148 * 8);
  mlp_backprop_kernel<<<blocks, 128, 0, st>>>(n, gy, W16, cache, gz2, gz1);
  MLP_CHECK();
  const int n_chunks = (n + chunk - 1) / chunk;
  mlp_wgrad_kernel<<<n_chunks, 256, 0, st>>>(n, chunk, gy, gz2, gz1, cache, partial);
  MLP_CHECK();
  mlp_grad_sum_kernel<<<(kMlpTrained + 255) / 256, 256, 0, st>>>(n_chunks, partial, grad);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_to_half(cudaStream_t st, int n, const float* W, __half* W16) {
  mlp_to_half_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, W, W16);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_feature_stats(cudaStream_t st, long long n, const float* X, float* mean, float* scale) {
  mlp_feature_stats_kernel<<<72, 256, 0, st>>>(n, X, mean, scale);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_to_double(cudaStream_t st, int n, const float* q, double* out) {
  mlp_to_double_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, q, out);
  MLP_CHECK();
  return cudaSuccess;
}

cudaError_t mlp_gather(cudaStream_t st, int n_batch, int n_atoms, const int* idx, const float* Xall,
                       const double* xyz_all, float* Xb, double* xyz_b) {
  mlp_gather_kernel<<<148 * 8, 256, 0, st>>>(n_batch, n_atoms, idx, Xall, xyz_all, Xb, xyz_b);
  MLP_CHECK();
  return cudaSuccess;
}

}  // namespace fmo
