// Learned initial guess (per-subdomain MLP): device buffers and launchers (mlp.cu).
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace bd {

struct MlpDev {
  int n_in = 0, n_hidden = 256, n_out = 0, maxq = 0, batch = 0;
  long long off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_W3 = 0, off_b3 = 0, n_params = 0;
  float *w = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;  // packed FP32 parameters, grads, Adam moments
  float *b1 = nullptr, *b2 = nullptr, *b3 = nullptr;               // views into w
  __nv_bfloat16 *Wb1 = nullptr, *Wb2 = nullptr, *Wb3 = nullptr;    // bfloat16 weights of the forward pass
  float *X = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Y = nullptr;
  float *T = nullptr, *mask = nullptr, *dY = nullptr, *dZ1 = nullptr, *dZ2 = nullptr;
  int t = 0;  // Adam step count
};

void mlp_forward(const MlpDev &m, int B, cudaStream_t s);
// loss partials (kRedBlocks doubles, already divided by the count) and packed gradients in m.g
void mlp_backward(const MlpDev &m, int B, float inv_cnt, double *partial, cudaStream_t s);
void mlp_adam(MlpDev &m, float lr, cudaStream_t s);
void mlp_refresh_bf16(const MlpDev &m, cudaStream_t s);
void mlp_features(const MlpDev &m, int nq, const int *q_sub, const int *q_loc, const int *q_node, const double *ui0,
                  const double *ue0, const double *ui1, const double *ue1, const double *ui2, const double *ue2,
                  const double *ti, const double *te, cudaStream_t s);
void mlp_guess(const MlpDev &m, int n, const int *ptr, const int *ent, const double *ui, const double *ue, double *gi,
               double *ge, cudaStream_t s);

}  // namespace bd
