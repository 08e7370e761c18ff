// Learned initial guess (per-subdomain MLP): device buffers and launchers (mlp.cu,
// gemm_tc.cu).
#pragma once
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace bd {

// Epilogue of one tensor-core GEMM C = A B^T (gemm_tc.cu):
//   mode 0 (forward layer): z = acc + bias[n]; Z = z; Hb = bf16(relu ? max(z, 0) : z), HbT its transpose
//   mode 1 (hidden gradient): d = acc * (Zprev > 0); Z = d; Hb = bf16(d), HbT its transpose
//   mode 2 (weight gradient): Z = acc
// Every output pointer may be null.
struct GemmEpi {
  int mode = 0, relu = 0;
  const float *bias = nullptr;
  float *Z = nullptr;
  int ldz = 0;
  __nv_bfloat16 *Hb = nullptr;
  int ldh = 0;
  __nv_bfloat16 *HbT = nullptr;
  int ldht = 0;
  const float *Zprev = nullptr;
  int ldzp = 0;
};
bool gemm_tc_configure();
// M x N output, K a multiple of 64 (zero-padded operands), lda / ldb multiples of 8
void launch_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb,
                      const GemmEpi &ep, int *err, cudaStream_t s);

// The network n_in -> 256 -> 256 -> n_out over a batch of B subdomains.  Parameters are
// packed FP32 masters (W1, b1, W2, b2, W3, b3, row-major W[out][in]); every GEMM
// operand is a bf16 buffer padded to a multiple of 64 along its K dimension (zeros in
// the padding), in the row-major form and, where a backward product needs it, the
// transposed one.
struct MlpDev {
  int n_tr = 0;                    // trace nodes per subdomain (padded to the largest)
  int n_in = 0, n_hidden = 256, n_out = 0, batch = 0;
  int ld_in = 0, ld_out = 0, ld_b = 0;  // padded K extents: n_in, n_out, batch
  long long off_W1 = 0, off_b1 = 0, off_W2 = 0, off_b2 = 0, off_W3 = 0, off_b3 = 0, n_params = 0;
  float *w = nullptr, *g = nullptr, *am = nullptr, *av = nullptr;  // packed FP32 parameters, grads, Adam moments
  float *b1 = nullptr, *b2 = nullptr, *b3 = nullptr;               // views into w
  // bf16 weights of the products: W1b [H][ld_in], W2b [H][H], W2bT [H][H], W3b [n_out][H], W3bT [H][ld_out]
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2bT = nullptr, *W3b = nullptr, *W3bT = nullptr;
  // activations: inputs Xb [B][ld_in] and XbT [n_in][ld_b]; hidden H1b/H2b [B][H] and their transposes [H][ld_b]
  __nv_bfloat16 *Xb = nullptr, *XbT = nullptr, *H1b = nullptr, *H1bT = nullptr, *H2b = nullptr, *H2bT = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Y = nullptr;  // FP32 pre-activations and outputs
  float *T = nullptr, *mask = nullptr;               // targets and mask [B][n_out]
  float *Xf = nullptr;                               // FP32 staging of host inputs [B][n_in]
  // gradients: dY [B][n_out] (FP32), dYb [B][ld_out], dYbT [n_out][ld_b]; dZ2 [B][H], dZ2b, dZ2bT; dZ1, dZ1bT
  float *dY = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  __nv_bfloat16 *dYb = nullptr, *dYbT = nullptr, *dZ2b = nullptr, *dZ2bT = nullptr, *dZ1bT = nullptr;
  int t = 0;  // Adam step count
};

void mlp_forward(const MlpDev &m, int *err, cudaStream_t s);
// loss partials (kRedBlocks doubles, already divided by the count) and packed gradients in m.g
void mlp_backward(const MlpDev &m, float inv_cnt, double *partial, int *err, cudaStream_t s);
void mlp_adam(MlpDev &m, float lr, cudaStream_t s);
void mlp_refresh_bf16(const MlpDev &m, cudaStream_t s);
// FP32 inputs in m.Xf (B x n_in) -> the bf16 operand buffers Xb and XbT
void mlp_inputs_from_f32(const MlpDev &m, cudaStream_t s);
// Features of the trace nodes: entry t (subdomain t_sub[t], trace position t_pos[t], global
// node t_node[t]) -> Xb / XbT; with ti given also targets T = u^{n+1} - u^n and mask
void mlp_features(const MlpDev &m, int nt, const int *t_sub, const int *t_pos, const int *t_node, const double *ui0,
                  const double *ue0, const double *ui1, const double *ue1, const double *ui2, const double *ue2,
                  const double *ti, const double *te, cudaStream_t s);
// Predicted interface increment: for every global interface node g (iface order), the mean
// of the predictions of the subdomains holding it, into dG[2g + field]
void mlp_trace_increment(const MlpDev &m, int n_if_nodes, const int *ptr, const int *ent, double *dG,
                         cudaStream_t s);

}  // namespace bd
