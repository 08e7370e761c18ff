// Learned initial guess: a per-subdomain MLP (features -> 256 -> 256 -> outputs,
// ReLU) with bfloat16 weights, float32 accumulation, MSE loss and Adam.  Not in
// the paper (it only requires some Newton starting value, Section 3c).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "mlp.cuh"

namespace bd {

// C[m][n] = act(sum_k A[m][k] W[n][k] + b[n]); one warp per (m, 4 consecutive n), lanes
// over k: every A value is loaded once for the four outputs.
__global__ void k_mlp_fwd(int M, int N, int K, const float *__restrict__ A, const __nv_bfloat16 *__restrict__ W,
                          const float *__restrict__ b, float *__restrict__ Z, float *__restrict__ H, int relu) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nq = (N + 3) / 4;
  if (gw >= M * nq) return;
  const int m = gw / nq, n0 = (gw % nq) * 4;
  const float *a = A + (long long)m * K;
  const __nv_bfloat16 *w[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) w[j] = W + (long long)min(n0 + j, N - 1) * K;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = lane; k < K; k += 32) {
    const float av = a[k];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += av * __bfloat162float(w[j][k]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j] = warp_sum(acc[j]);
  if (lane < 4 && n0 + lane < N) {
    float v = acc[0];
#pragma unroll
    for (int j = 1; j < 4; ++j)
      if (lane == j) v = acc[j];
    const int n = n0 + lane;
    const float z = v + b[n];
    if (Z) Z[(long long)m * N + n] = z;
    H[(long long)m * N + n] = relu ? fmaxf(z, 0.f) : z;
  }
}

// dY = 2 mask (Y - T) / count, and per-block partial sums of mask (Y - T)^2.
__global__ void k_mlp_loss(int total, const float *__restrict__ Y, const float *__restrict__ T,
                           const float *__restrict__ mask, float inv_cnt, float *__restrict__ dY,
                           double *__restrict__ partial) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const float r = (Y[i] - T[i]) * mask[i];
    dY[i] = 2.f * r * inv_cnt;
    acc += (double)r * r;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc * inv_cnt;
}

// dW[n][k] = sum_m dZ[m][n] A[m][k]; db[n] = sum_m dZ[m][n]  (M = batch, small).
// One thread per (k, 4 consecutive n): every A value is loaded once for four outputs.
__global__ void k_mlp_wgrad(int M, int N, int K, const float *__restrict__ dZ, const float *__restrict__ A,
                            float *__restrict__ dW, float *__restrict__ db) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nq = (N + 3) / 4;
  if (t >= (long long)nq * (K + 1)) return;
  const int n0 = (int)(t / (K + 1)) * 4, k = (int)(t % (K + 1));
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int m = 0; m < M; ++m) {
    const float av = (k < K) ? A[(long long)m * K + k] : 1.f;
    const float *dz = dZ + (long long)m * N;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (n0 + j < N) acc[j] += dz[n0 + j] * av;
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (n0 + j >= N) continue;
    if (k < K) dW[(long long)(n0 + j) * K + k] = acc[j];
    else db[n0 + j] = acc[j];
  }
}

// dA[m][k] = (sum_n dZ[m][n] W[n][k]) * (Zprev[m][k] > 0)   (ReLU backward of the previous layer).
// One CTA per (m, 32 consecutive k): the 8 warps split the n range, lane = k, and their
// partial sums are added in a fixed order.
__global__ void __launch_bounds__(256) k_mlp_bgrad(int M, int N, int K, const float *__restrict__ dZ,
                                                   const __nv_bfloat16 *__restrict__ W,
                                                   const float *__restrict__ Zprev, float *__restrict__ dA) {
  __shared__ float part[8][33];
  const int m = blockIdx.y, k = blockIdx.x * 32 + (threadIdx.x & 31), wid = threadIdx.x >> 5;
  const float *dz = dZ + (long long)m * N;
  float a0 = 0.f, a1 = 0.f;
  if (k < K) {
    int n = wid;
    for (; n + 8 < N; n += 16) {
      a0 += dz[n] * __bfloat162float(W[(long long)n * K + k]);
      a1 += dz[n + 8] * __bfloat162float(W[(long long)(n + 8) * K + k]);
    }
    for (; n < N; n += 8) a0 += dz[n] * __bfloat162float(W[(long long)n * K + k]);
  }
  part[wid][threadIdx.x & 31] = a0 + a1;
  __syncthreads();
  if (wid == 0 && k < K) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += part[q][threadIdx.x];
    const long long t = (long long)m * K + k;
    dA[t] = Zprev[t] > 0.f ? acc : 0.f;
  }
}

// Adam with bias correction; refreshes the bfloat16 copy used by the forward pass.
__global__ void k_mlp_adam(long long n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                           float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, float lr, float c1, float c2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(long long n, const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16(w[i]);
}

// Features of local node a of subdomain j (inputs padded to maxq nodes, zero outside):
// [V^n, V^n - V^{n-1}, V^{n-1} - V^{n-2}, u_e^n, u_e^n - u_e^{n-1}, u_e^{n-1} - u_e^{n-2}] / 100,
// V = u_i - u_e.  Targets / mask for the same layout when t_i is given: (u^{n+1} - u^n) per field.
__global__ void k_mlp_features(int nq, int maxq, const int *__restrict__ q_sub, const int *__restrict__ q_loc,
                               const int *__restrict__ q_node, const double *__restrict__ ui0,
                               const double *__restrict__ ue0, const double *__restrict__ ui1,
                               const double *__restrict__ ue1, const double *__restrict__ ui2,
                               const double *__restrict__ ue2, float *__restrict__ X, const double *__restrict__ ti,
                               const double *__restrict__ te, float *__restrict__ T, float *__restrict__ mask) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int j = q_sub[q], a = q_loc[q], x = q_node[q];
  const double v0 = ui0[x] - ue0[x], v1 = ui1[x] - ue1[x], v2 = ui2[x] - ue2[x];
  float *f = X + ((long long)j * maxq + a) * 6;
  f[0] = (float)(v0 * 0.01);
  f[1] = (float)((v0 - v1) * 0.01);
  f[2] = (float)((v1 - v2) * 0.01);
  f[3] = (float)(ue0[x] * 0.01);
  f[4] = (float)((ue0[x] - ue1[x]) * 0.01);
  f[5] = (float)((ue1[x] - ue2[x]) * 0.01);
  if (ti) {
    float *t = T + ((long long)j * maxq + a) * 2;
    t[0] = (float)(ti[x] - ui0[x]);
    t[1] = (float)(te[x] - ue0[x]);
    mask[((long long)j * maxq + a) * 2] = 1.f;
    mask[((long long)j * maxq + a) * 2 + 1] = 1.f;
  }
}

// Guess u0 = u^n + mean over the subdomains holding node x of their predicted increments.
__global__ void k_mlp_guess(int n, int maxq, const int *__restrict__ ptr, const int *__restrict__ ent,
                            const float *__restrict__ Y, const double *__restrict__ ui, const double *__restrict__ ue,
                            double *__restrict__ gi, double *__restrict__ ge) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  double si = 0.0, se = 0.0;
  const int b = ptr[x], e = ptr[x + 1];
  for (int k = b; k < e; ++k) {
    const long long o = (long long)ent[k] * 2;  // ent = j * maxq + a
    si += Y[o];
    se += Y[o + 1];
  }
  const double inv = e > b ? 1.0 / (e - b) : 0.0;
  gi[x] = ui[x] + si * inv;
  ge[x] = ue[x] + se * inv;
}

// ---- host side ------------------------------------------------------------------
void mlp_forward(const MlpDev &m, int B, cudaStream_t s) {
  const int H = m.n_hidden;
  auto fwd = [&](int N, int K, const float *A, const __nv_bfloat16 *W, const float *b, float *Z, float *Hh, int relu) {
    const long long warps = (long long)B * ((N + 3) / 4);
    k_mlp_fwd<<<(int)((warps * 32 + 255) / 256), 256, 0, s>>>(B, N, K, A, W, b, Z, Hh, relu);
    count_launch();
  };
  fwd(H, m.n_in, m.X, m.Wb1, m.b1, m.Z1, m.H1, 1);
  fwd(H, H, m.H1, m.Wb2, m.b2, m.Z2, m.H2, 1);
  fwd(m.n_out, H, m.H2, m.Wb3, m.b3, nullptr, m.Y, 0);
}

void mlp_backward(const MlpDev &m, int B, float inv_cnt, double *partial, cudaStream_t s) {
  const int H = m.n_hidden;
  const int total = B * m.n_out;
  k_mlp_loss<<<kRedBlocks, 256, 0, s>>>(total, m.Y, m.T, m.mask, inv_cnt, m.dY, partial);
  auto wg = [&](int N, int K, const float *dZ, const float *A, float *dW, float *db) {
    const long long t = (long long)((N + 3) / 4) * (K + 1);
    k_mlp_wgrad<<<(int)((t + 255) / 256), 256, 0, s>>>(B, N, K, dZ, A, dW, db);
  };
  auto bg = [&](int N, int K, const float *dZ, const __nv_bfloat16 *W, const float *Zp, float *dA) {
    k_mlp_bgrad<<<dim3(ceil_div(K, 32), B), 256, 0, s>>>(B, N, K, dZ, W, Zp, dA);
  };
  wg(m.n_out, H, m.dY, m.H2, m.g + m.off_W3, m.g + m.off_b3);
  bg(m.n_out, H, m.dY, m.Wb3, m.Z2, m.dZ2);
  wg(H, H, m.dZ2, m.H1, m.g + m.off_W2, m.g + m.off_b2);
  bg(H, H, m.dZ2, m.Wb2, m.Z1, m.dZ1);
  wg(H, m.n_in, m.dZ1, m.X, m.g + m.off_W1, m.g + m.off_b1);
  count_launch(6);
}

void mlp_adam(MlpDev &m, float lr, cudaStream_t s) {
  m.t += 1;
  // bias corrections 1 - beta^t in FP64: in FP32, 1 - 0.999^t loses about five digits
  // to cancellation at small t
  const float c1 = (float)(1.0 - std::pow(0.9, (double)m.t)), c2 = (float)(1.0 - std::pow(0.999, (double)m.t));
  const long long n = m.n_params;
  k_mlp_adam<<<(int)((n + 255) / 256), 256, 0, s>>>(n, m.w, m.g, m.am, m.av, nullptr, lr, c1, c2);
  count_launch();
  mlp_refresh_bf16(m, s);
}

void mlp_refresh_bf16(const MlpDev &m, cudaStream_t s) {
  auto cv = [&](long long off, long long n, __nv_bfloat16 *dst) {
    k_to_bf16<<<(int)((n + 255) / 256), 256, 0, s>>>(n, m.w + off, dst);
  };
  cv(m.off_W1, (long long)m.n_hidden * m.n_in, m.Wb1);
  cv(m.off_W2, (long long)m.n_hidden * m.n_hidden, m.Wb2);
  cv(m.off_W3, (long long)m.n_out * m.n_hidden, m.Wb3);
  count_launch(3);
}

void mlp_features(const MlpDev &m, int nq, const int *q_sub, const int *q_loc, const int *q_node, const double *ui0,
                  const double *ue0, const double *ui1, const double *ue1, const double *ui2, const double *ue2,
                  const double *ti, const double *te, cudaStream_t s) {
  k_mlp_features<<<ceil_div(nq, 256), 256, 0, s>>>(nq, m.maxq, q_sub, q_loc, q_node, ui0, ue0, ui1, ue1, ui2, ue2,
                                                   m.X, ti, te, m.T, m.mask);
  count_launch();
}

void mlp_guess(const MlpDev &m, int n, const int *ptr, const int *ent, const double *ui, const double *ue, double *gi,
               double *ge, cudaStream_t s) {
  k_mlp_guess<<<ceil_div(n, 256), 256, 0, s>>>(n, m.maxq, ptr, ent, m.Y, ui, ue, gi, ge);
  count_launch();
}

}  // namespace bd
