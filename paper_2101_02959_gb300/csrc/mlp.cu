// Learned initial guess: a per-subdomain MLP (interface traces -> 256 -> 256 ->
// interface increments, ReLU) with bf16 operands on the tensor cores (gemm_tc.cu),
// float32 accumulation, MSE loss and Adam.  Not in the paper (it only requires some
// Newton starting value, Section 3c).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "mlp.cuh"

namespace bd {

// dY = 2 mask (Y - T) / count (FP32, its bf16 copy and the transposed bf16 copy) and
// per-block partial sums of mask (Y - T)^2.
__global__ void k_mlp_loss(int B, int n_out, int ld_out, int ld_b, const float *__restrict__ Y,
                           const float *__restrict__ T, const float *__restrict__ mask, float inv_cnt,
                           float *__restrict__ dY, __nv_bfloat16 *__restrict__ dYb, __nv_bfloat16 *__restrict__ dYbT,
                           double *__restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  const long long total = (long long)B * n_out;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(i / n_out), o = (int)(i % n_out);
    const float r = (Y[i] - T[i]) * mask[i];
    const float d = 2.f * r * inv_cnt;
    dY[i] = d;
    const __nv_bfloat16 db = __float2bfloat16(d);
    dYb[(long long)m * ld_out + o] = db;
    dYbT[(long long)o * ld_b + m] = db;
    acc += (double)r * r;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc * inv_cnt;
}

// db[n] = sum_m dZ[m][n] (fixed order: deterministic)
__global__ void k_colsum(int M, int N, const float *__restrict__ dZ, float *__restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int m = 0; m < M; ++m) acc += dZ[(long long)m * N + n];
  db[n] = acc;
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t).
__global__ void k_mlp_adam(long long n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, float lr, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// bf16 copies of a row-major FP32 matrix W [rows][cols]: dst [rows][ld] and, when dstT is
// given, dstT [cols][ldT] (padding columns are never written: they stay zero)
__global__ void k_to_bf16(int rows, int cols, const float *__restrict__ w, __nv_bfloat16 *__restrict__ dst, int ld,
                          __nv_bfloat16 *__restrict__ dstT, int ldT) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  const __nv_bfloat16 b = __float2bfloat16(w[i]);
  dst[(long long)r * ld + c] = b;
  if (dstT) dstT[(long long)c * ldT + r] = b;
}

// Features of trace entry t = (subdomain j, trace position a, node x):
// [V^n, V^n - V^{n-1}, V^{n-1} - V^{n-2}, u_e^n, u_e^n - u_e^{n-1}, u_e^{n-1} - u_e^{n-2}] / 100,
// V = u_i - u_e, as bf16 into Xb[j][6a + f] and XbT[6a + f][j]; targets (u^{n+1} - u^n per field)
// and mask when ti is given.
__global__ void k_mlp_features(int nt, int ld_in, int ld_b, int n_out, const int *__restrict__ t_sub,
                               const int *__restrict__ t_pos, const int *__restrict__ t_node,
                               const double *__restrict__ ui0, const double *__restrict__ ue0,
                               const double *__restrict__ ui1, const double *__restrict__ ue1,
                               const double *__restrict__ ui2, const double *__restrict__ ue2,
                               __nv_bfloat16 *__restrict__ Xb, __nv_bfloat16 *__restrict__ XbT,
                               const double *__restrict__ ti, const double *__restrict__ te, float *__restrict__ T,
                               float *__restrict__ mask) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int j = t_sub[t], a = t_pos[t], x = t_node[t];
  const double v0 = ui0[x] - ue0[x], v1 = ui1[x] - ue1[x], v2 = ui2[x] - ue2[x];
  const float f[6] = {(float)(v0 * 0.01), (float)((v0 - v1) * 0.01), (float)((v1 - v2) * 0.01),
                      (float)(ue0[x] * 0.01), (float)((ue0[x] - ue1[x]) * 0.01), (float)((ue1[x] - ue2[x]) * 0.01)};
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const __nv_bfloat16 b = __float2bfloat16(f[q]);
    Xb[(long long)j * ld_in + 6 * a + q] = b;
    XbT[(long long)(6 * a + q) * ld_b + j] = b;
  }
  if (ti) {
    const long long o = (long long)j * n_out + 2 * a;
    T[o] = (float)(ti[x] - ui0[x]);
    T[o + 1] = (float)(te[x] - ue0[x]);
    mask[o] = 1.f;
    mask[o + 1] = 1.f;
  }
}

// FP32 inputs [B][n_in] -> Xb [B][ld_in], XbT [n_in][ld_b]
__global__ void k_inputs_bf16(int B, int n_in, int ld_in, int ld_b, const float *__restrict__ X,
                              __nv_bfloat16 *__restrict__ Xb, __nv_bfloat16 *__restrict__ XbT) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * n_in) return;
  const int j = (int)(i / n_in), c = (int)(i % n_in);
  const __nv_bfloat16 b = __float2bfloat16(X[i]);
  Xb[(long long)j * ld_in + c] = b;
  XbT[(long long)c * ld_b + j] = b;
}

// dG[2g + f] = mean over the subdomains holding interface node g of their predicted
// increments (ent = j * n_tr + a)
__global__ void k_mlp_trace_increment(int n, int n_tr, int n_out, const int *__restrict__ ptr,
                                      const int *__restrict__ ent, const float *__restrict__ Y,
                                      double *__restrict__ dG) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  double si = 0.0, se = 0.0;
  const int b = ptr[g], e = ptr[g + 1];
  for (int k = b; k < e; ++k) {
    const int j = ent[k] / n_tr, a = ent[k] % n_tr;
    const long long o = (long long)j * n_out + 2 * a;
    si += Y[o];
    se += Y[o + 1];
  }
  const double inv = e > b ? 1.0 / (e - b) : 0.0;
  dG[2 * g] = si * inv;
  dG[2 * g + 1] = se * inv;
}

// ---- host side ------------------------------------------------------------------
void mlp_forward(const MlpDev &m, int *err, cudaStream_t s) {
  const int H = m.n_hidden, B = m.batch;
  GemmEpi e1;
  e1.mode = 0; e1.relu = 1; e1.bias = m.b1; e1.Z = m.Z1; e1.ldz = H;
  e1.Hb = m.H1b; e1.ldh = H; e1.HbT = m.H1bT; e1.ldht = m.ld_b;
  launch_gemm_bf16(B, H, m.ld_in, m.Xb, m.ld_in, m.W1b, m.ld_in, e1, err, s);
  GemmEpi e2 = e1;
  e2.bias = m.b2; e2.Z = m.Z2; e2.Hb = m.H2b; e2.HbT = m.H2bT;
  launch_gemm_bf16(B, H, H, m.H1b, H, m.W2b, H, e2, err, s);
  GemmEpi e3;
  e3.mode = 0; e3.relu = 0; e3.bias = m.b3; e3.Z = m.Y; e3.ldz = m.n_out;
  launch_gemm_bf16(B, m.n_out, H, m.H2b, H, m.W3b, H, e3, err, s);
}

void mlp_backward(const MlpDev &m, float inv_cnt, double *partial, int *err, cudaStream_t s) {
  const int H = m.n_hidden, B = m.batch;
  k_mlp_loss<<<kRedBlocks, 256, 0, s>>>(B, m.n_out, m.ld_out, m.ld_b, m.Y, m.T, m.mask, inv_cnt, m.dY, m.dYb,
                                        m.dYbT, partial);
  count_launch();
  GemmEpi w3;  // dW3 = dYb^T H2b: (n_out x B) (B x H)
  w3.mode = 2; w3.Z = m.g + m.off_W3; w3.ldz = H;
  launch_gemm_bf16(m.n_out, H, m.ld_b, m.dYbT, m.ld_b, m.H2bT, m.ld_b, w3, err, s);
  GemmEpi b3;  // dZ2 = (dYb W3b) * (Z2 > 0)
  b3.mode = 1; b3.Zprev = m.Z2; b3.ldzp = H; b3.Z = m.dZ2; b3.ldz = H;
  b3.Hb = m.dZ2b; b3.ldh = H; b3.HbT = m.dZ2bT; b3.ldht = m.ld_b;
  launch_gemm_bf16(B, H, m.ld_out, m.dYb, m.ld_out, m.W3bT, m.ld_out, b3, err, s);
  GemmEpi w2;  // dW2 = dZ2b^T H1b
  w2.mode = 2; w2.Z = m.g + m.off_W2; w2.ldz = H;
  launch_gemm_bf16(H, H, m.ld_b, m.dZ2bT, m.ld_b, m.H1bT, m.ld_b, w2, err, s);
  GemmEpi b2;  // dZ1 = (dZ2b W2b) * (Z1 > 0)
  b2.mode = 1; b2.Zprev = m.Z1; b2.ldzp = H; b2.Z = m.dZ1; b2.ldz = H;
  b2.HbT = m.dZ1bT; b2.ldht = m.ld_b;
  launch_gemm_bf16(B, H, H, m.dZ2b, H, m.W2bT, H, b2, err, s);
  GemmEpi w1;  // dW1 = dZ1b^T Xb
  w1.mode = 2; w1.Z = m.g + m.off_W1; w1.ldz = m.n_in;
  launch_gemm_bf16(H, m.n_in, m.ld_b, m.dZ1bT, m.ld_b, m.XbT, m.ld_b, w1, err, s);
  k_colsum<<<ceil_div(m.n_out, 256), 256, 0, s>>>(B, m.n_out, m.dY, m.g + m.off_b3);
  k_colsum<<<ceil_div(H, 256), 256, 0, s>>>(B, H, m.dZ2, m.g + m.off_b2);
  k_colsum<<<ceil_div(H, 256), 256, 0, s>>>(B, H, m.dZ1, m.g + m.off_b1);
  count_launch(3);
}

void mlp_adam(MlpDev &m, float lr, cudaStream_t s) {
  m.t += 1;
  // bias corrections 1 - beta^t in FP64: in FP32, 1 - 0.999^t loses about five digits
  // to cancellation at small t
  const float c1 = (float)(1.0 - std::pow(0.9, (double)m.t)), c2 = (float)(1.0 - std::pow(0.999, (double)m.t));
  const long long n = m.n_params;
  k_mlp_adam<<<(int)((n + 255) / 256), 256, 0, s>>>(n, m.w, m.g, m.am, m.av, lr, c1, c2);
  count_launch();
  mlp_refresh_bf16(m, s);
}

void mlp_refresh_bf16(const MlpDev &m, cudaStream_t s) {
  const int H = m.n_hidden;
  auto cv = [&](int rows, int cols, long long off, __nv_bfloat16 *dst, int ld, __nv_bfloat16 *dstT, int ldT) {
    const long long n = (long long)rows * cols;
    k_to_bf16<<<(int)((n + 255) / 256), 256, 0, s>>>(rows, cols, m.w + off, dst, ld, dstT, ldT);
  };
  cv(H, m.n_in, m.off_W1, m.W1b, m.ld_in, nullptr, 0);
  cv(H, H, m.off_W2, m.W2b, H, m.W2bT, H);
  cv(m.n_out, H, m.off_W3, m.W3b, H, m.W3bT, m.ld_out);
  count_launch(3);
}

void mlp_inputs_from_f32(const MlpDev &m, cudaStream_t s) {
  const long long n = (long long)m.batch * m.n_in;
  k_inputs_bf16<<<(int)((n + 255) / 256), 256, 0, s>>>(m.batch, m.n_in, m.ld_in, m.ld_b, m.Xf, m.Xb, m.XbT);
  count_launch();
}

void mlp_features(const MlpDev &m, int nt, const int *t_sub, const int *t_pos, const int *t_node, const double *ui0,
                  const double *ue0, const double *ui1, const double *ue1, const double *ui2, const double *ue2,
                  const double *ti, const double *te, cudaStream_t s) {
  k_mlp_features<<<ceil_div(nt, 256), 256, 0, s>>>(nt, m.ld_in, m.ld_b, m.n_out, t_sub, t_pos, t_node, ui0, ue0,
                                                   ui1, ue1, ui2, ue2, m.Xb, m.XbT, ti, te, m.T, m.mask);
  count_launch();
}

void mlp_trace_increment(const MlpDev &m, int n_if_nodes, const int *ptr, const int *ent, double *dG,
                         cudaStream_t s) {
  k_mlp_trace_increment<<<ceil_div(n_if_nodes, 256), 256, 0, s>>>(n_if_nodes, m.n_tr, m.n_out, ptr, ent, m.Y, dG);
  count_launch();
}

}  // namespace bd
