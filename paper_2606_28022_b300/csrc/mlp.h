// Learned initial shell charges: launch interface between the host library
// (capi.cu) and the kernels of mlp.cu.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

namespace fmo {

constexpr int kMlpIn = 77;          // 32 radial + 40 angular + ESP + 4 element one-hot
constexpr int kMlpStride = 80;      // floats per feature row
constexpr int kMlpHidden = 128;
// flat weight layout: W1 (hidden x in), b1, W2 (hidden x hidden), b2,
// W3 (2 x hidden), b3, then the feature mean and scale (not trained)
constexpr int kMlpOffW1 = 0;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpHidden * kMlpIn;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpHidden;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpHidden * kMlpHidden;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpHidden;
constexpr int kMlpOffB3 = kMlpOffW3 + 2 * kMlpHidden;
constexpr int kMlpTrained = kMlpOffB3 + 2;
constexpr int kMlpOffMean = kMlpTrained;
constexpr int kMlpOffScale = kMlpOffMean + kMlpIn;
constexpr int kMlpWeights = kMlpOffScale + kMlpIn;

// activations kept by the forward pass for the backward pass (all null:
// inference)
struct MlpCache {
  float* x0;   // [n][kMlpStride] standardised input
  float* z1;   // [n][hidden]
  float* h1;
  float* z2;
  float* h2;
};

void note_launch();   // counts a kernel launch of the library

cudaError_t mlp_descriptors(cudaStream_t st, int n_frames, int n_atoms, const double* xyz, const int* elem4,
                            float* X, int* err);
cudaError_t mlp_esp(cudaStream_t st, int n_frames, int n_atoms, int n_sh, const double* xyz, const int* atom_frag,
                    const float* atom_ie, const int* sh_atom, const float* sh_ie, const float* dq, float* X);
cudaError_t mlp_forward(cudaStream_t st, int n, const float* X, const __half* W16, const float* mean,
                        const float* scale, float* y, const MlpCache& cache);
cudaError_t mlp_project(cudaStream_t st, int n_frames, int n_frag, int n_atoms, const int* f_atom0, const int* f_nat,
                        const int* f_charge, const float* y, float* q, const float* target, double inv_count,
                        float* gy, double* loss_part);
cudaError_t mlp_backward_step(cudaStream_t st, int n, const float* gy, const __half* W16, const MlpCache& cache,
                              float* gz2, float* gz1, float* partial, int chunk, float* W, float* m, float* v,
                              __half* W16out, float lr, int t);
// backward pass and the weight gradient of the batch loss (no update):
// grad[kMlpTrained] in the flat weight layout
cudaError_t mlp_gradient(cudaStream_t st, int n, const float* gy, const __half* W16, const MlpCache& cache,
                         float* gz2, float* gz1, float* partial, int chunk, float* grad);
cudaError_t mlp_to_half(cudaStream_t st, int n, const float* W, __half* W16);
cudaError_t mlp_feature_stats(cudaStream_t st, long long n, const float* X, float* mean, float* scale);
cudaError_t mlp_to_double(cudaStream_t st, int n, const float* q, double* out);
cudaError_t mlp_gather(cudaStream_t st, int n_batch, int n_atoms, const int* idx, const float* Xall,
                       const double* xyz_all, float* Xb, double* xyz_b);

}  // namespace fmo
