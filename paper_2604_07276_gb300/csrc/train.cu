// Training kernels of the distilled student potential (stage a17): weight
// gradients of the energy, the per-frame energy / force loss, Adam, and the
// refresh of the derived weight copies the forward kernels read.
//
// Loss of one frame (N atoms): L = pe ((E - E_ref) / N)^2 + pf mean |F - F_ref|^2.
// dL/dtheta = 2 pe (E - E_ref) / N^2 dE/dtheta
//           - (2 pf / 3N) d/dtheta [ sum_k (F - F_ref)_k . dE/dx_k ],
// and the bracket is the derivative of E along the fixed direction
// v = F - F_ref, whose theta-gradient is taken here as the central difference
// [dE/dtheta(x + s v) - dE/dtheta(x - s v)] / (2 s) of exact energy-weight
// gradients, with s = h / max|v| (largest displacement h).
#include "common.cuh"
#include "kernels.h"

namespace dpa1 {

// C[i][o] += scale * sum_n A[n][i] * B[n][o]; the n range is split over
// grid.z slices that add their parts atomically.
__global__ void __launch_bounds__(256) k_wgrad(const float* __restrict__ A, int lda, const float* __restrict__ B,
                                               int ldb, float* __restrict__ C, int ldc, int I, int O, int N, int chunk,
                                               const float* __restrict__ scale) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * 64, o0 = blockIdx.y * 64;
  const int n_begin = blockIdx.z * chunk;
  const int n_end = min(N, n_begin + chunk);
  float acc[4][4] = {};
  for (int n0 = n_begin; n0 < n_end; n0 += 16) {
    for (int t = threadIdx.x; t < 16 * 64; t += 256) {
      const int k = t / 64, c = t % 64;
      const int n = n0 + k;
      As[k][c] = (n < n_end && i0 + c < I) ? A[(size_t)n * lda + i0 + c] : 0.f;
      Bs[k][c] = (n < n_end && o0 + c < O) ? B[(size_t)n * ldb + o0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[k][ty * 4 + q]; b[q] = Bs[k][tx * 4 + q]; }
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
    }
    __syncthreads();
  }
  const float s = *scale;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = i0 + ty * 4 + p, o = o0 + tx * 4 + q;
      if (i < I && o < O) atomicAdd(&C[(size_t)i * ldc + o], s * acc[p][q]);
    }
}

// c[o] += scale * factor * sum_n B[n][o]
__global__ void k_colsum(const float* __restrict__ B, int ldb, float* __restrict__ c, int O, int N, int chunk,
                         const float* __restrict__ scale, float factor) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= O) return;
  const int n_begin = blockIdx.y * chunk, n_end = min(N, n_begin + chunk);
  float s = 0.f;
  for (int n = n_begin; n < n_end; ++n) s += B[(size_t)n * ldb + o];
  atomicAdd(&c[o], *scale * factor * s);
}

// de_i/d ebias[t_i] = 1 and de_i/d b_out = out_scale for every atom.
__global__ void k_head_bias_grad(const int* __restrict__ atype, int n, float* __restrict__ g_ebias,
                                 float* __restrict__ g_bout, const float* __restrict__ scale, float out_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = *scale;
  atomicAdd(&g_ebias[atype[i]], s);
  atomicAdd(g_bout, s * out_scale);
}

// One block: loss of the frame, the gradient scales and the displaced
// coordinates x +- s (F - F_ref).
__global__ void k_train_prep(int n, const double* __restrict__ energy, double e_ref,
                             const double* __restrict__ force, const double* __restrict__ force_ref,
                             const double* __restrict__ coord, double pe, double pf, double h,
                             double* __restrict__ coord_plus, double* __restrict__ coord_minus,
                             double* __restrict__ loss, float* __restrict__ scales) {
  __shared__ double red_s[32];
  __shared__ double red_m[32];
  __shared__ double s_step;
  double ss = 0.0, mx = 0.0;
  for (int k = threadIdx.x; k < 3 * n; k += blockDim.x) {
    const double d = force[k] - force_ref[k];
    ss += d * d;
    mx = fmax(mx, fabs(d));
  }
  ss = warp_sum_d(ss);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) {
    red_s[threadIdx.x >> 5] = ss;
    red_m[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, M = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      S += red_s[w];
      M = fmax(M, red_m[w]);
    }
    const double nn = n > 0 ? (double)n : 1.0;
    const double de = *energy - e_ref;
    const double lE = pe * (de / nn) * (de / nn);
    const double lF = pf * S / (3.0 * nn);
    loss[0] = lE + lF;
    loss[1] = lE;
    loss[2] = lF;
    const double step = M > 0.0 ? h / M : 0.0;
    s_step = step;
    const double cF = 2.0 * pf / (3.0 * nn);
    scales[0] = 1.0f;
    scales[1] = (float)(2.0 * pe * de / (nn * nn));
    scales[2] = step > 0.0 ? (float)(-cF / (2.0 * step)) : 0.f;
    scales[3] = step > 0.0 ? (float)(cF / (2.0 * step)) : 0.f;
  }
  __syncthreads();
  const double step = s_step;
  for (int k = threadIdx.x; k < 3 * n; k += blockDim.x) {
    const double d = force[k] - force_ref[k];
    coord_plus[k] = coord[k] + step * d;
    coord_minus[k] = coord[k] - step * d;
  }
}

__global__ void k_adam(float* __restrict__ theta, float* __restrict__ g, float* __restrict__ m1, float* __restrict__ m2,
                       int n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = b;
  theta[i] -= lr * (a / bc1) / (sqrtf(b / bc2) + eps);
  g[i] = 0.f;
}

__global__ void k_transpose(const float* __restrict__ W, int R, int C, float* __restrict__ WT) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * C) return;
  const int r = t / C, c = t % C;
  WT[(size_t)c * R + r] = W[t];
}

__global__ void k_scale_copy(const float* __restrict__ src, float* __restrict__ dst, int n, float s) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = s * src[t];
}

static int blocks(long long n, int t) { return (int)((n + t - 1) / t); }

void launch_wgrad(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int I, int O, int N,
                  const float* scale, cudaStream_t st) {
  if (N <= 0 || I <= 0 || O <= 0) return;
  const int splits = std::min(64, std::max(1, N / 256));
  const int chunk = (N + splits - 1) / splits;
  dim3 grid(blocks(I, 64), blocks(O, 64), splits);
  k_wgrad<<<grid, 256, 0, st>>>(A, lda, B, ldb, C, ldc, I, O, N, chunk, scale);
  note_launch();
}

void launch_colsum(const float* B, int ldb, float* c, int O, int N, const float* scale, float factor,
                   cudaStream_t st) {
  if (N <= 0 || O <= 0) return;
  const int splits = std::min(128, std::max(1, N / 128));
  const int chunk = (N + splits - 1) / splits;
  k_colsum<<<dim3(blocks(O, 128), splits), 128, 0, st>>>(B, ldb, c, O, N, chunk, scale, factor);
  note_launch();
}

void launch_head_bias_grad(const int* atype, int n, float* g_ebias, float* g_bout, const float* scale, float out_scale,
                           cudaStream_t st) {
  if (n <= 0) return;
  k_head_bias_grad<<<blocks(n, 256), 256, 0, st>>>(atype, n, g_ebias, g_bout, scale, out_scale);
  note_launch();
}

void launch_train_prep(int n, const double* energy, double e_ref, const double* force, const double* force_ref,
                       const double* coord, double pe, double pf, double h, double* coord_plus, double* coord_minus,
                       double* loss, float* scales, cudaStream_t st) {
  k_train_prep<<<1, 1024, 0, st>>>(n, energy, e_ref, force, force_ref, coord, pe, pf, h, coord_plus, coord_minus,
                                   loss, scales);
  note_launch();
}

void launch_adam(float* theta, float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, cudaStream_t st) {
  if (n <= 0) return;
  k_adam<<<blocks(n, 256), 256, 0, st>>>(theta, g, m1, m2, n, lr, b1, b2, eps, bc1, bc2);
  note_launch();
}

void launch_transpose(const float* W, int R, int C, float* WT, cudaStream_t st) {
  if (R * C <= 0) return;
  k_transpose<<<blocks((long long)R * C, 256), 256, 0, st>>>(W, R, C, WT);
  note_launch();
}

void launch_scale_copy(const float* src, float* dst, int n, float s, cudaStream_t st) {
  if (n <= 0) return;
  k_scale_copy<<<blocks(n, 256), 256, 0, st>>>(src, dst, n, s);
  note_launch();
}

}  // namespace dpa1
