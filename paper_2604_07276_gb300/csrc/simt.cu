// FP32 SIMT kernels of the network stages a5-a13: embedding net, gated
// attention (forward and adjoint), LayerNorm, descriptor, fitting helpers
// and a general FP32 GEMM.  These form the FP32 path and provide the
// stages the tensor-core path shares with it.
#include "common.cuh"
#include "kernels.h"

namespace dpa1 {

static int sm_count();

// ----------------------------------------------------------------- FP32 GEMM
// C = epi(A B + bias (+R)), A [M][K], B [K][N] row-major.  128x128 tile, K
// step 16, 256 threads with 8x8 outputs each (two 4x4 quadrants 64 apart, so
// that the 16 threads of a half warp read 16 consecutive float4 of a shared
// row), shared-memory double buffering with the next tile held in registers.
// VEC: 16-byte global loads and stores (every leading dimension, K and N
// multiples of 4, the arrays 16-byte aligned); otherwise 4-byte ones.
constexpr int GBK = 16, GLD = 128 + 4;

template <int EPI, bool VEC>
__global__ void __launch_bounds__(256, 2)
k_sgemm128(const float* __restrict__ A, int lda, const float* __restrict__ B, int ldb,
           const float* __restrict__ bias, const float* __restrict__ R, int ldr, float* __restrict__ C, int ldc,
           int M, int N, int K) {
  __shared__ __align__(16) float As[2][GBK][GLD];  // k-major: As[k][row]
  __shared__ __align__(16) float Bs[2][GBK][GLD];  // Bs[k][column]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.x * 128;
  const int n0 = blockIdx.y * 128;
  const int ar = tid >> 1, ak = (tid & 1) * 8;   // A: row, first of its 8 k
  const int bk = tid >> 4, bc = (tid & 15) * 8;  // B: k, first of its 8 columns
  float ra[8], rb[8];
  auto load = [&](int k0) {
    const long long gm = m0 + ar;
    const int gka = k0 + ak, gkb = k0 + bk;
    if (VEC) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gm < M && gka + 4 * h < K) x = *reinterpret_cast<const float4*>(A + gm * lda + gka + 4 * h);
        ra[4 * h] = x.x; ra[4 * h + 1] = x.y; ra[4 * h + 2] = x.z; ra[4 * h + 3] = x.w;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
        const int gn = n0 + bc + 4 * h;
        if (gkb < K && gn < N) y = *reinterpret_cast<const float4*>(B + (long long)gkb * ldb + gn);
        rb[4 * h] = y.x; rb[4 * h + 1] = y.y; rb[4 * h + 2] = y.z; rb[4 * h + 3] = y.w;
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int gk = gka + q, gn = n0 + bc + q;
        ra[q] = (gm < M && gk < K) ? A[gm * lda + gk] : 0.f;
        rb[q] = (gkb < K && gn < N) ? B[(long long)gkb * ldb + gn] : 0.f;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) As[buf][ak + q][ar] = ra[q];
    *reinterpret_cast<float4*>(&Bs[buf][bk][bc]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    *reinterpret_cast<float4*>(&Bs[buf][bk][bc + 4]) = make_float4(rb[4], rb[5], rb[6], rb[7]);
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    const bool more = k0 + GBK < K;
    if (more) load(k0 + GBK);
#pragma unroll
    for (int k = 0; k < GBK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const long long m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (m >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int nq = n0 + h * 64 + tx * 4;  // first of this thread's 4 columns
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = nq + j;
        float x = acc[i][4 * h + j];
        if (n < N) {
          if (EPI == EPI_BIAS || EPI == EPI_TANH || EPI == EPI_RES_TANH) x += bias ? bias[n] : 0.f;
          if (EPI == EPI_TANH || EPI == EPI_RES_TANH) x = tanhf(x);
        }
        v[j] = x;
      }
      if (VEC) {
        if (nq < N) {  // N % 4 == 0: the 4 columns are all in range
          float4 o = make_float4(v[0], v[1], v[2], v[3]);
          if (EPI == EPI_RES_TANH || EPI == EPI_RES) {
            const float4 r = *reinterpret_cast<const float4*>(R + m * ldr + nq);
            o.x += r.x; o.y += r.y; o.z += r.z; o.w += r.w;
          }
          float4* c = reinterpret_cast<float4*>(C + m * ldc + nq);
          if (EPI == EPI_ACCUM) {
            const float4 cc = *c;
            o.x += cc.x; o.y += cc.y; o.z += cc.z; o.w += cc.w;
          }
          *c = o;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = nq + j;
          if (n >= N) continue;
          float* c = C + m * ldc + n;
          if (EPI == EPI_RES_TANH || EPI == EPI_RES) *c = R[m * ldr + n] + v[j];
          else if (EPI == EPI_ACCUM) *c = *c + v[j];
          else *c = v[j];
        }
      }
    }
  }
}

template <int EPI>
static void sgemm_launch(dim3 grid, bool vec, const float* A, int lda, const float* B, int ldb, const float* bias,
                         const float* R, int ldr, float* C, int ldc, int M, int N, int K, cudaStream_t st) {
  if (vec)
    k_sgemm128<EPI, true><<<grid, 256, 0, st>>>(A, lda, B, ldb, bias, R, ldr, C, ldc, M, N, K);
  else
    k_sgemm128<EPI, false><<<grid, 256, 0, st>>>(A, lda, B, ldb, bias, R, ldr, C, ldc, M, N, K);
}

void gemm_f32(const float* A, int lda, const float* B, int ldb, const float* bias, const float* R, int ldr,
              float* C, int ldc, int M, int N, int K, int epi, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + 127) / 128));
  const bool res = epi == EPI_RES || epi == EPI_RES_TANH;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
                         reinterpret_cast<uintptr_t>(C) | (res ? reinterpret_cast<uintptr_t>(R) : 0);
  const bool vec = (addr & 15) == 0 && lda % 4 == 0 && ldb % 4 == 0 && ldc % 4 == 0 && (!res || ldr % 4 == 0) &&
                   N % 4 == 0 && K % 4 == 0;
  switch (epi) {
    case EPI_BIAS: sgemm_launch<EPI_BIAS>(grid, vec, A, lda, B, ldb, bias, R, ldr, C, ldc, M, N, K, st); break;
    case EPI_TANH: sgemm_launch<EPI_TANH>(grid, vec, A, lda, B, ldb, bias, R, ldr, C, ldc, M, N, K, st); break;
    case EPI_RES_TANH: sgemm_launch<EPI_RES_TANH>(grid, vec, A, lda, B, ldb, bias, R, ldr, C, ldc, M, N, K, st); break;
    case EPI_ACCUM: sgemm_launch<EPI_ACCUM>(grid, vec, A, lda, B, ldb, bias, R, ldr, C, ldc, M, N, K, st); break;
    default: sgemm_launch<EPI_RES>(grid, vec, A, lda, B, ldb, bias, R, ldr, C, ldc, M, N, K, st); break;
  }
  note_launch();
}

// ------------------------------------------------------------ embedding net
// G0_ij = net_s(R_ij,0) * (1 + Gt[t_i, t_j]); net_s = 1 -> E0 -> E1 -> E2 with
// tanh and the residual rule (keep width: x + f; double: [x, x] + f).
// A CTA takes 64 neighbour rows of one atom; activations of the block live in
// shared memory and every layer is a small tiled product over the block, so
// global rows are read and written whole (coalesced).
template <int E0, int E1, int E2>
struct EmbedLayout {  // packed global weights: W0 b0 W1 b1 W2 b2
  static constexpr int W0 = 0, B0 = E0, W1 = 2 * E0, B1 = W1 + E0 * E1, W2 = B1 + E1, B2 = W2 + E1 * E2,
                       TOTAL = B2 + E2;
};

constexpr int EROWS = 64;  // neighbour rows per CTA
constexpr int ETHREADS = 256;

template <int IN, int OUT>
__device__ __forceinline__ float skip_in(const float* x, int o) {
  return OUT == IN ? x[o] : (OUT == 2 * IN ? x[o % IN] : 0.f);
}

// Shared layout (floats); W2 is kept with row stride E2 + 1 (bank-conflict
// free for both of its access patterns), activations with row stride n + 1.
template <int E0, int E1, int E2>
struct EmbedSmem {
  static constexpr int P2 = E2 + 1;
  static constexpr int W0 = 0, B0 = E0, W1 = 2 * E0, B1 = W1 + E0 * E1, W2 = B1 + E1, B2 = W2 + E1 * P2,
                       X = B2 + E2, H1 = X + EROWS, H2 = H1 + EROWS * (E0 + 1), Z = H2 + EROWS * (E1 + 1),
                       DH2 = Z + EROWS * (E2 + 1), DZ2 = DH2 + EROWS * (E1 + 1), DH1 = DZ2 + EROWS * (E1 + 1),
                       TJ = DH1 + EROWS * (E0 + 1), TOTAL = TJ + EROWS;  // TJ: the rows' neighbour types (int)
};

template <int E0, int E1, int E2>
__device__ __forceinline__ void embed_load(float* sm, const EmbedArgs& a, size_t base, int cnt) {
  using Lw = EmbedLayout<E0, E1, E2>;
  using S = EmbedSmem<E0, E1, E2>;
  for (int t = threadIdx.x; t < Lw::W2; t += ETHREADS) sm[t] = a.w[t];  // W0 b0 W1 b1 share offsets
  for (int t = threadIdx.x; t < E1 * E2; t += ETHREADS) sm[S::W2 + (t / E2) * S::P2 + t % E2] = a.w[Lw::W2 + t];
  for (int t = threadIdx.x; t < E2; t += ETHREADS) sm[S::B2 + t] = a.w[Lw::B2 + t];
  for (int r = threadIdx.x; r < EROWS; r += ETHREADS) {
    sm[S::X + r] = r < cnt ? a.R[(base + r) * 4] : 0.f;
    reinterpret_cast<int*>(sm + S::TJ)[r] = r < cnt ? a.atype[a.nlist[base + r]] : 0;
  }
  __syncthreads();
}

// Layers 1 and 2, then Z = H2 W2 + b2 (4 rows per thread per weight load).
// b0t: the centre type's rows of the concat mode's first-layer bias table
// ([neighbour type][E0]), or null (strip mode: b0).
template <int E0, int E1, int E2>
__device__ __forceinline__ void embed_forward(float* sm, int cnt, const float* b0t) {
  using S = EmbedSmem<E0, E1, E2>;
  const int* tj = reinterpret_cast<const int*>(sm + S::TJ);
  for (int idx = threadIdx.x; idx < EROWS * E0; idx += ETHREADS) {
    const int r = idx / E0, p = idx % E0;
    const float b = b0t ? b0t[tj[r] * E0 + p] : sm[S::B0 + p];
    sm[S::H1 + r * (E0 + 1) + p] = r < cnt ? tanhf(fmaf(sm[S::X + r], sm[S::W0 + p], b)) : 0.f;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < (EROWS / 4) * E1; idx += ETHREADS) {  // four rows per thread
    const int r0 = (idx / E1) * 4, b = idx % E1;
    const float* h1 = sm + S::H1 + r0 * (E0 + 1);
    float z[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) z[u] = sm[S::B1 + b];
#pragma unroll 5
    for (int p = 0; p < E0; ++p) {
      const float w = sm[S::W1 + p * E1 + b];
#pragma unroll
      for (int u = 0; u < 4; ++u) z[u] = fmaf(h1[u * (E0 + 1) + p], w, z[u]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = r0 + u;
      sm[S::H2 + r * (E1 + 1) + b] = r < cnt ? skip_in<E0, E1>(h1 + u * (E0 + 1), b) + tanhf(z[u]) : 0.f;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < (EROWS / 4) * E2; idx += ETHREADS) {
    const int r0 = (idx / E2) * 4, c = idx % E2;
    float z0 = sm[S::B2 + c], z1 = z0, z2 = z0, z3 = z0;
    const float* h = sm + S::H2 + r0 * (E1 + 1);
#pragma unroll 5
    for (int b = 0; b < E1; ++b) {
      const float wv = sm[S::W2 + b * S::P2 + c];
      z0 = fmaf(h[b], wv, z0);
      z1 = fmaf(h[(E1 + 1) + b], wv, z1);
      z2 = fmaf(h[2 * (E1 + 1) + b], wv, z2);
      z3 = fmaf(h[3 * (E1 + 1) + b], wv, z3);
    }
    float* zr = sm + S::Z + r0 * (E2 + 1) + c;
    zr[0] = z0; zr[E2 + 1] = z1; zr[2 * (E2 + 1)] = z2; zr[3 * (E2 + 1)] = z3;
  }
  __syncthreads();
}

template <int E0, int E1, int E2>
__global__ void __launch_bounds__(ETHREADS) k_embed_fwd(EmbedArgs a) {
  using S = EmbedSmem<E0, E1, E2>;
  extern __shared__ float sm[];
  const int atom = blockIdx.x >> 1, part = blockIdx.x & 1;
  const int r0 = part * EROWS;
  const int cnt = max(0, min(EROWS, a.nnei[atom] - r0));
  const size_t base = (size_t)atom * NP + r0;
  if (cnt > 0) {
    embed_load<E0, E1, E2>(sm, a, base, cnt);
    embed_forward<E0, E1, E2>(sm, cnt, a.b0t ? a.b0t + (size_t)a.atype[atom] * a.ntypes * E0 : nullptr);
  }
  const int ti = a.atype[atom];
  for (int idx = threadIdx.x; idx < EROWS * E2; idx += ETHREADS) {
    const int r = idx / E2, c = idx % E2;
    float g = 0.f;
    if (r < cnt) {
      const int tj = a.atype[a.nlist[base + r]];
      const float h3 = skip_in<E1, E2>(sm + S::H2 + r * (E1 + 1), c) + tanhf(sm[S::Z + r * (E2 + 1) + c]);
      g = h3 * (1.f + a.Gt[((size_t)ti * a.ntypes + tj) * E2 + c]);
    }
    a.G0[(base + r) * a.m1 + c] = g;
  }
}

// Adjoint: dR[:,0] += d net_s / dx . (dG0 * (1 + Gt)), recomputing the
// forward activations of the block.
template <int E0, int E1, int E2>
__global__ void __launch_bounds__(ETHREADS) k_embed_bwd(EmbedArgs a) {
  using S = EmbedSmem<E0, E1, E2>;
  extern __shared__ float sm[];
  const int atom = blockIdx.x >> 1, part = blockIdx.x & 1;
  const int r0 = part * EROWS;
  const int cnt = max(0, min(EROWS, a.nnei[atom] - r0));
  if (cnt == 0) return;
  const size_t base = (size_t)atom * NP + r0;
  embed_load<E0, E1, E2>(sm, a, base, cnt);
  embed_forward<E0, E1, E2>(sm, cnt, a.b0t ? a.b0t + (size_t)a.atype[atom] * a.ntypes * E0 : nullptr);
  const int ti = a.atype[atom];
  // Z <- dZ3 = g (1 - t3^2) with g = dG0 (1 + Gt); the skip part of dH2 is
  // summed from g directly below
  for (int idx = threadIdx.x; idx < EROWS * E2; idx += ETHREADS) {
    const int r = idx / E2, c = idx % E2;
    float dz = 0.f;
    if (r < cnt) {
      const int tj = a.atype[a.nlist[base + r]];
      const float g = a.dG0[(base + r) * a.m1 + c] * (1.f + a.Gt[((size_t)ti * a.ntypes + tj) * E2 + c]);
      const float t = tanhf(sm[S::Z + r * (E2 + 1) + c]);
      dz = g * (1.f - t * t);
    }
    sm[S::Z + r * (E2 + 1) + c] = dz;
  }
  __syncthreads();
  // dH2[r][b] = skip^T(g)[b] + sum_c W2[b][c] dZ3[r][c], four rows per
  // thread so that each weight load serves four products (dZ3 is zero on
  // rows past cnt)
  for (int idx = threadIdx.x; idx < (EROWS / 4) * E1; idx += ETHREADS) {
    const int r0 = (idx / E1) * 4, b = idx % E1;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    if (r0 < cnt) {
      const float* dz = sm + S::Z + r0 * (E2 + 1);
      const float* w2 = sm + S::W2 + b * S::P2;
#pragma unroll 4
      for (int c = 0; c < E2; ++c) {
        const float w = w2[c];
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = fmaf(w, dz[u * (E2 + 1) + c], s[u]);
      }
      if (E2 == E1 || E2 == 2 * E1) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = r0 + u;
          if (r >= cnt) break;
          const int tj = a.atype[a.nlist[base + r]];
          const float* gt = a.Gt + ((size_t)ti * a.ntypes + tj) * E2;
          const float* dg = a.dG0 + (base + r) * a.m1;
          for (int c = b; c < E2; c += E1) s[u] += dg[c] * (1.f + gt[c]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sm[S::DH2 + (r0 + u) * (E1 + 1) + b] = r0 + u < cnt ? s[u] : 0.f;
  }
  __syncthreads();
  // dZ2 = dH2 (1 - t2^2) with t2 = H2 - skip(H1)
  for (int idx = threadIdx.x; idx < EROWS * E1; idx += ETHREADS) {
    const int r = idx / E1, b = idx % E1;
    const float t = sm[S::H2 + r * (E1 + 1) + b] - skip_in<E0, E1>(sm + S::H1 + r * (E0 + 1), b);
    sm[S::DZ2 + r * (E1 + 1) + b] = sm[S::DH2 + r * (E1 + 1) + b] * (1.f - t * t);
  }
  __syncthreads();
  // dH1[r][p] = skip^T(dH2)[p] + sum_b W1[p][b] dZ2[r][b]; term of dx: W0[p]
  // dH1 (1 - H1^2); four rows per thread as above (dZ2 is zero past cnt)
  for (int idx = threadIdx.x; idx < (EROWS / 4) * E0; idx += ETHREADS) {
    const int r0 = (idx / E0) * 4, p = idx % E0;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    if (r0 < cnt) {
      const float* dz2 = sm + S::DZ2 + r0 * (E1 + 1);
      const float* w1 = sm + S::W1 + p * E1;
#pragma unroll 5
      for (int b = 0; b < E1; ++b) {
        const float w = w1[b];
#pragma unroll
        for (int u = 0; u < 4; ++u) s[u] = fmaf(w, dz2[u * (E1 + 1) + b], s[u]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = r0 + u;
        if (E1 == E0 || E1 == 2 * E0)
          for (int b = p; b < E1; b += E0) s[u] += sm[S::DH2 + r * (E1 + 1) + b];
        const float h1 = sm[S::H1 + r * (E0 + 1) + p];
        s[u] = s[u] * (1.f - h1 * h1) * sm[S::W0 + p];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) sm[S::DH1 + (r0 + u) * (E0 + 1) + p] = r0 + u < cnt ? s[u] : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < cnt; r += ETHREADS) {
    float dx = 0.f;
    for (int p = 0; p < E0; ++p) dx += sm[S::DH1 + r * (E0 + 1) + p];
    a.dR[(base + r) * 4] += dx;
  }
}

// Weight gradients of the embedding net, scale * dE/d(W0 b0 W1 b1 W2 b2)
// (packed layout), accumulated over every neighbour row.  Persistent CTAs
// walk the 64-row blocks, keep per-CTA sums in shared memory and add them to
// `grad` once at the end.
template <int E0, int E1, int E2>
__global__ void __launch_bounds__(ETHREADS) k_embed_wgrad(EmbedArgs a, float* grad, const float* scale) {
  using Lw = EmbedLayout<E0, E1, E2>;
  using S = EmbedSmem<E0, E1, E2>;
  extern __shared__ float sm[];
  float* acc = sm + S::TOTAL;
  for (int t = threadIdx.x; t < Lw::TOTAL; t += ETHREADS) acc[t] = 0.f;
  for (int blk = blockIdx.x; blk < 2 * a.n; blk += gridDim.x) {
    const int atom = blk >> 1, part = blk & 1;
    const int r0 = part * EROWS;
    const int cnt = max(0, min(EROWS, a.nnei[atom] - r0));
    if (cnt == 0) continue;  // uniform over the CTA
    const size_t base = (size_t)atom * NP + r0;
    __syncthreads();
    embed_load<E0, E1, E2>(sm, a, base, cnt);
    embed_forward<E0, E1, E2>(sm, cnt, a.b0t ? a.b0t + (size_t)a.atype[atom] * a.ntypes * E0 : nullptr);
    const int ti = a.atype[atom];
    for (int idx = threadIdx.x; idx < EROWS * E2; idx += ETHREADS) {
      const int r = idx / E2, c = idx % E2;
      float dz = 0.f;
      if (r < cnt) {
        const int tj = a.atype[a.nlist[base + r]];
        const float g = a.dG0[(base + r) * a.m1 + c] * (1.f + a.Gt[((size_t)ti * a.ntypes + tj) * E2 + c]);
        const float t = tanhf(sm[S::Z + r * (E2 + 1) + c]);
        dz = g * (1.f - t * t);
      }
      sm[S::Z + r * (E2 + 1) + c] = dz;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < EROWS * E1; idx += ETHREADS) {
      const int r = idx / E1, b = idx % E1;
      float sacc = 0.f;
      if (r < cnt) {
        const float* dz = sm + S::Z + r * (E2 + 1);
        const float* w2 = sm + S::W2 + b * S::P2;
        for (int c = 0; c < E2; ++c) sacc = fmaf(w2[c], dz[c], sacc);
        if (E2 == E1 || E2 == 2 * E1) {
          const int tj = a.atype[a.nlist[base + r]];
          const float* gt = a.Gt + ((size_t)ti * a.ntypes + tj) * E2;
          const float* dg = a.dG0 + (base + r) * a.m1;
          for (int c = b; c < E2; c += E1) sacc += dg[c] * (1.f + gt[c]);
        }
      }
      sm[S::DH2 + r * (E1 + 1) + b] = sacc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < EROWS * E1; idx += ETHREADS) {
      const int r = idx / E1, b = idx % E1;
      const float t = sm[S::H2 + r * (E1 + 1) + b] - skip_in<E0, E1>(sm + S::H1 + r * (E0 + 1), b);
      sm[S::DZ2 + r * (E1 + 1) + b] = r < cnt ? sm[S::DH2 + r * (E1 + 1) + b] * (1.f - t * t) : 0.f;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < EROWS * E0; idx += ETHREADS) {
      const int r = idx / E0, q = idx % E0;
      float sacc = 0.f;
      if (r < cnt) {
        const float* dz2 = sm + S::DZ2 + r * (E1 + 1);
        const float* w1 = sm + S::W1 + q * E1;
        for (int b = 0; b < E1; ++b) sacc = fmaf(w1[b], dz2[b], sacc);
        if (E1 == E0 || E1 == 2 * E0)
          for (int b = q; b < E1; b += E0) sacc += sm[S::DH2 + r * (E1 + 1) + b];
        const float h1 = sm[S::H1 + r * (E0 + 1) + q];
        sacc *= (1.f - h1 * h1);  // dz1
      }
      sm[S::DH1 + r * (E0 + 1) + q] = sacc;
    }
    __syncthreads();
    // accumulate this block's weight gradients (rows >= cnt are zero everywhere)
    for (int t = threadIdx.x; t < Lw::TOTAL; t += ETHREADS) {
      float g = 0.f;
      if (t < Lw::B0) {
        for (int r = 0; r < EROWS; ++r) g = fmaf(sm[S::X + r], sm[S::DH1 + r * (E0 + 1) + t], g);
      } else if (t < Lw::W1) {
        for (int r = 0; r < EROWS; ++r) g += sm[S::DH1 + r * (E0 + 1) + (t - Lw::B0)];
      } else if (t < Lw::B1) {
        const int q = (t - Lw::W1) / E1, b = (t - Lw::W1) % E1;
        for (int r = 0; r < EROWS; ++r) g = fmaf(sm[S::H1 + r * (E0 + 1) + q], sm[S::DZ2 + r * (E1 + 1) + b], g);
      } else if (t < Lw::W2) {
        for (int r = 0; r < EROWS; ++r) g += sm[S::DZ2 + r * (E1 + 1) + (t - Lw::B1)];
      } else if (t < Lw::B2) {
        const int b = (t - Lw::W2) / E2, c = (t - Lw::W2) % E2;
        for (int r = 0; r < EROWS; ++r) g = fmaf(sm[S::H2 + r * (E1 + 1) + b], sm[S::Z + r * (E2 + 1) + c], g);
      } else {
        for (int r = 0; r < EROWS; ++r) g += sm[S::Z + r * (E2 + 1) + (t - Lw::B2)];
      }
      acc[t] += g;
    }
  }
  __syncthreads();
  const float sc = *scale;
  for (int t = threadIdx.x; t < Lw::TOTAL; t += ETHREADS) atomicAdd(&grad[t], sc * acc[t]);
}

template <int E0, int E1, int E2>
static void embed_wgrad_launch(const EmbedArgs& a, float* grad, const float* scale, cudaStream_t st) {
  using Lw = EmbedLayout<E0, E1, E2>;
  using S = EmbedSmem<E0, E1, E2>;
  if (a.n == 0) return;
  const size_t smem = sizeof(float) * (S::TOTAL + Lw::TOTAL);
  cudaFuncSetAttribute(k_embed_wgrad<E0, E1, E2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int grid = std::min(2 * a.n, 2 * sm_count());
  k_embed_wgrad<E0, E1, E2><<<grid, ETHREADS, smem, st>>>(a, grad, scale);
  note_launch();
}

bool launch_embed_wgrad(const EmbedArgs& a, const int* w, float* grad, const float* scale, cudaStream_t st) {
  if (w[0] == 25 && w[1] == 50 && w[2] == 100) { embed_wgrad_launch<25, 50, 100>(a, grad, scale, st); return true; }
  if (w[0] == 16 && w[1] == 32 && w[2] == 64) { embed_wgrad_launch<16, 32, 64>(a, grad, scale, st); return true; }
  if (w[0] == 32 && w[1] == 64 && w[2] == 128) { embed_wgrad_launch<32, 64, 128>(a, grad, scale, st); return true; }
  return false;
}

template <int E0, int E1, int E2>
static void embed_launch(const EmbedArgs& a, bool bwd, cudaStream_t st) {
  using S = EmbedSmem<E0, E1, E2>;
  if (a.n == 0) return;
  const unsigned grid = (unsigned)a.n * 2;
  const size_t sm = sizeof(float) * S::TOTAL;
  if (!bwd) {
    cudaFuncSetAttribute(k_embed_fwd<E0, E1, E2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_embed_fwd<E0, E1, E2><<<grid, ETHREADS, sm, st>>>(a);
  } else {
    cudaFuncSetAttribute(k_embed_bwd<E0, E1, E2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_embed_bwd<E0, E1, E2><<<grid, ETHREADS, sm, st>>>(a);
  }
  note_launch();
}

static bool embed_dispatch(const EmbedArgs& a, const int* w, bool bwd, cudaStream_t st) {
  if (w[0] == 25 && w[1] == 50 && w[2] == 100) { embed_launch<25, 50, 100>(a, bwd, st); return true; }
  if (w[0] == 16 && w[1] == 32 && w[2] == 64) { embed_launch<16, 32, 64>(a, bwd, st); return true; }
  if (w[0] == 32 && w[1] == 64 && w[2] == 128) { embed_launch<32, 64, 128>(a, bwd, st); return true; }
  return false;
}
bool launch_embed_fwd(const EmbedArgs& a, const int* widths, cudaStream_t st) { return embed_dispatch(a, widths, false, st); }
bool launch_embed_bwd(const EmbedArgs& a, const int* widths, cudaStream_t st) { return embed_dispatch(a, widths, true, st); }

// ---------------------------------------------------------------- LayerNorm
// G_out = G_in + LN(Y) on rows with a neighbour, G_out = G_in elsewhere.
__global__ void k_ln_res_fwd(const float* __restrict__ Y, const float* __restrict__ Gin, const int* __restrict__ nlist,
                             const float* __restrict__ gamma, const float* __restrict__ beta, float eps,
                             float* __restrict__ Gout, float* __restrict__ stats, long long rows, int m1) {
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const float* y = Y + row * m1;
  float v[4];
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    v[q] = c < m1 ? y[c] : 0.f;
    s += v[q];
  }
  const float mean = warp_sum(s) / (float)m1;
  float s2 = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    const float d = c < m1 ? v[q] - mean : 0.f;
    s2 += d * d;
  }
  const float var = warp_sum(s2) / (float)m1;
  const float rstd = 1.0f / sqrtf(var + eps);
  const bool valid = nlist[row] >= 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    if (c < m1) {
      const float gin = Gin[row * m1 + c];
      Gout[row * m1 + c] = valid ? gin + (v[q] - mean) * rstd * gamma[c] + beta[c] : gin;
    }
  }
  if (lane == 0) {
    stats[2 * row] = mean;
    stats[2 * row + 1] = rstd;
  }
}

__global__ void k_ln_bwd(const float* __restrict__ dZ, const float* __restrict__ Y, const float* __restrict__ stats,
                         const int* __restrict__ nlist, const float* __restrict__ gamma, float* __restrict__ dY,
                         long long rows, int m1) {
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  const bool valid = nlist[row] >= 0;
  const float mean = stats[2 * row], rstd = stats[2 * row + 1];
  float gz[4], yh[4];
  float s1 = 0.f, s2 = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    if (c < m1 && valid) {
      gz[q] = gamma[c] * dZ[row * m1 + c];
      yh[q] = (Y[row * m1 + c] - mean) * rstd;
    } else {
      gz[q] = 0.f; yh[q] = 0.f;
    }
    s1 += gz[q];
    s2 += gz[q] * yh[q];
  }
  s1 = warp_sum(s1) / (float)m1;
  s2 = warp_sum(s2) / (float)m1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = lane + 32 * q;
    if (c < m1) dY[row * m1 + c] = valid ? rstd * (gz[q] - s1 - yh[q] * s2) : 0.f;
  }
}

void launch_ln_res_fwd(const float* Y, const float* Gin, const int* nlist, const float* gamma, const float* beta,
                       float eps, float* Gout, float* stats, int rows_i, int m1, cudaStream_t st) {
  long long rows = rows_i;
  if (rows == 0) return;
  k_ln_res_fwd<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(Y, Gin, nlist, gamma, beta, eps, Gout, stats,
                                                                      rows, m1);
  note_launch();
}
void launch_ln_bwd(const float* dZ, const float* Y, const float* stats, const int* nlist, const float* gamma,
                   float* dY, int rows_i, int m1, cudaStream_t st) {
  long long rows = rows_i;
  if (rows == 0) return;
  k_ln_bwd<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(dZ, Y, stats, nlist, gamma, dY, rows, m1);
  note_launch();
}

// ------------------------------------------------- gated attention (FP32)
// Per centre atom, over its valid neighbour slots j, k < n_i:
//   l_jk = Q_j.K_k / sqrt(A);  l'_jk = (l_jk + S) w_j w_k - S
//   A_jk = softmax_k(l'_jk);   P_jk = A_jk w_j w_k (rhat_j . rhat_k);  O = P V
// (the forward evaluates O Wo through P G, see k_attn_fwd_f32)

// Smooth logits l'_jk = (l_jk + S) w_j w_k carry the shift S = 20, whose
// FP32 spacing (2e-6) is far coarser than the logit differences that matter.
// They are evaluated as unevaluated float pairs (h + l): l + S exactly by a
// two-sum, the product of the switch weights (FP64, held as float pairs) and
// the final product with their rounding errors by FMA; ~44 bits, without the
// FP64 pipe (narrow on this GPU).  Only differences to the row maximum are
// used, as floats.
__device__ __forceinline__ float2 split_pair(double w) {
  const float h = (float)w;
  return make_float2(h, (float)(w - (double)h));
}

__device__ __forceinline__ float2 smooth_logit(float t, float S, float2 wj, float2 wk) {
  const float uh = t + S;
  const float bb = uh - t;
  const float ul = (t - (uh - bb)) + (S - bb);
  const float ph = wj.x * wk.x;
  float pl = fmaf(wj.x, wk.x, -ph);
  pl = fmaf(wj.x, wk.y, pl);
  pl = fmaf(wj.y, wk.x, pl);
  const float hh = uh * ph;
  float hl = fmaf(uh, ph, -hh);
  hl = fmaf(uh, pl, hl);
  hl = fmaf(ul, ph, hl);
  return make_float2(hh, hl);
}

// the largest pair (ordered by h, then l) over the warp; every lane gets the same
__device__ __forceinline__ float2 warp_max_pair(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, v.x, o);
    const float ol = __shfl_xor_sync(0xffffffffu, v.y, o);
    if (oh > v.x || (oh == v.x && ol > v.y)) v = make_float2(oh, ol);
  }
  return v;
}

__device__ __forceinline__ float pair_diff(float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); }

// Forward, register-tiled: 512 threads as a 32 x 16 grid.  Thread (ty, tx)
// owns rows 4 ty + i (i < 4) and keys t_rc(tx, jj) (jj < 8) of S (128 x
// 128), then the same rows and columns of each 128-column part of PG.  Q and K pass
// through shared memory feature-major, 128 features at a time; P stays
// row-major and [G 1] comes in 128-column parts, key-major.  S sums over the
// features and PG over the keys in order, as a plain loop would.
//
// The kernel writes PG = [P G, rowsum(P)] instead of O = P V: with V = G Wv +
// bv, O Wo + bo = [P G, rowsum(P)] [Wv Wo; bv Wo] + bo, which a GEMM with the
// FP64-formed [Wv Wo; bv Wo] then evaluates.  The two are equal in exact
// arithmetic, but the gate (rhat_j . rhat_k of both signs) makes sum_k P_jk
// V_k cancel, and the accumulation errors of each computed V_k (a 100-term
// FP32 sum) survive that cancellation; the LayerNorm of weakly attended rows
// (variance << eps) then turns them into force errors up to ~5e-4 eV/A on
// a few atoms.  Summing the exact layer input G instead leaves only the
// rounding of the cancelling sum itself (a CPU emulation of both forms on the
// 15,668-atom box: force RMSE 7.5e-6 -> 2.4e-6 eV/A).
constexpr int FTF = 512;       // threads of the forward and the adjoint (4 x 8 tiles)
static_assert(4 * (FTF / 16) == NP, "32 thread rows of 4 rows each cover the 128 rows of an atom");
static_assert((FTF / 16) * NP * 4 <= 128 * (NP + 4), "the adjoint's column parts fit one shared tile");
constexpr int TLD = NP + 4;    // row stride of their shared tiles (16-byte rows)

// Row (or column) i < 8 of thread coordinate t < 16: the quarter tiles
// 4 t .. 4 t + 3 and 64 + 4 t .. 64 + 4 t + 3, so that the 16 threads of a
// half warp read 16 consecutive float4 of a shared row (no bank conflicts).
__device__ __forceinline__ int t_rc(int t, int i) { return i < 4 ? 4 * t + i : 60 + 4 * t + i; }

// Feature-major staging of a 128-row chunk: element idx (0 .. 4095) of the
// CTA's accesses takes row j and features f .. f + 3, 16 rows x 32 bytes per
// warp access (full sectors), and its transposed stores (feature f + u, row
// j) fall on distinct banks.
__device__ __forceinline__ void fm_pos(int idx, int& j, int& f) {
  const int w = idx >> 5, l = idx & 31;
  j = 16 * (w & 7) + (l >> 1);
  f = 4 * ((l & 1) + 2 * (w >> 3));
}

__device__ __forceinline__ void fm_store(float* T, int j, int f, float4 v) {
  T[(f + 0) * TLD + j] = v.x; T[(f + 1) * TLD + j] = v.y;
  T[(f + 2) * TLD + j] = v.z; T[(f + 3) * TLD + j] = v.w;
}

// Row i < TR of thread row coordinate ty: with TR = 8 (16 thread rows) the
// quarter tiles of t_rc; with TR = 4 (32 thread rows) rows 4 ty .. 4 ty + 3.
template <int TR>
__device__ __forceinline__ int r_of(int ty, int i) { return TR == 8 ? t_rc(ty, i) : 4 * ty + i; }

// The TR x 8 outer-product step of a register tile: acc[i][jj] += a[i] b[jj],
// with a = (A[ra .. ra + 3] (, A[ra + 64 .. ra + 67] for TR = 8)) and b =
// (B[rb .. rb + 3], B[rb + 64 .. rb + 67]).
template <int TR>
__device__ __forceinline__ void tile_fma(float (&acc)[TR][8], const float* A, int ra, const float* B, int rb) {
  float av[TR];
  const float4 a0 = *reinterpret_cast<const float4*>(A + ra);
  av[0] = a0.x; av[1] = a0.y; av[2] = a0.z; av[3] = a0.w;
  if constexpr (TR == 8) {
    const float4 a1 = *reinterpret_cast<const float4*>(A + ra + 64);
    av[4] = a1.x; av[5] = a1.y; av[6] = a1.z; av[7] = a1.w;
  }
  const float4 b0 = *reinterpret_cast<const float4*>(B + rb);
  const float4 b1 = *reinterpret_cast<const float4*>(B + rb + 64);
  const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fmaf(av[i], bv[jj], acc[i][jj]);
}

// acc[i][jj] += sum over k0 .. k0 + 3 of A[r_of(ty, i)][k] B[k][t_rc(tx, jj)]
// (A row-major, B key-major, both with row stride TLD).
template <int TR>
__device__ __forceinline__ void tile_fma4(float (&acc)[TR][8], const float* A, const float* B, int k0, int ty,
                                          int tx) {
  float4 pa[TR];
#pragma unroll
  for (int i = 0; i < TR; ++i) pa[i] = *reinterpret_cast<const float4*>(A + r_of<TR>(ty, i) * TLD + k0);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float4 v0 = *reinterpret_cast<const float4*>(B + (k0 + u) * TLD + 4 * tx);
    const float4 v1 = *reinterpret_cast<const float4*>(B + (k0 + u) * TLD + 64 + 4 * tx);
    const float vb[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
    for (int i = 0; i < TR; ++i) {
      const float p = u == 0 ? pa[i].x : u == 1 ? pa[i].y : u == 2 ? pa[i].z : pa[i].w;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fmaf(p, vb[jj], acc[i][jj]);
    }
  }
}

// One row of a register tile -> dst row (columns 4 tx .. and 64 + 4
// tx .. from col0, each float4 only below ncols).
__device__ __forceinline__ void tile_store_row(float* dst, const float* accrow, int col0, int tx, int ncols) {
  if (col0 + 4 * tx < ncols)
    *reinterpret_cast<float4*>(dst + col0 + 4 * tx) = make_float4(accrow[0], accrow[1], accrow[2], accrow[3]);
  if (col0 + 64 + 4 * tx < ncols)
    *reinterpret_cast<float4*>(dst + col0 + 64 + 4 * tx) = make_float4(accrow[4], accrow[5], accrow[6], accrow[7]);
}

template <int A>
__global__ void __launch_bounds__(FTF, 1) k_attn_fwd_f32(AttnArgs a, float scale) {
  extern __shared__ float sm[];
  float* X = sm;                 // [128][TLD]: Q chunk (feature-major), then P (row-major)
  float* Y = X + 128 * TLD;      // [128][TLD]: K chunk (feature-major), then a part of [G 1] (key-major)
  float4* rws = reinterpret_cast<float4*>(Y + 128 * TLD);  // [NP]
  float2* w2s = reinterpret_cast<float2*>(rws + NP);       // [NP] switch weights as float pairs
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int ld = a.ldq;  // Q | K
  for (int atom = blockIdx.x; atom < a.n; atom += gridDim.x) {
    const int nn = a.nnei[atom];
    const size_t base = (size_t)atom * NP;
    __syncthreads();  // the previous atom is done with every shared array
    for (int r = tid; r < NP; r += FTF) {
      rws[r] = r < nn ? reinterpret_cast<const float4*>(a.rw)[base + r] : make_float4(0.f, 0.f, 0.f, 0.f);
      w2s[r] = split_pair(r < nn ? a.w64[base + r] : 0.0);
    }
    float s[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) s[i][jj] = 0.f;
    const bool live = 4 * ty < nn && 4 * tx < nn;
    for (int c0 = 0; c0 < A; c0 += 128) {
      if (c0 > 0) __syncthreads();  // the previous chunk's products are done
      for (int idx = tid; idx < NP * 32; idx += FTF) {
        int j, f;
        fm_pos(idx, j, f);
        float4 qv = make_float4(0.f, 0.f, 0.f, 0.f), kv = qv;
        if (j < nn) {
          qv = *reinterpret_cast<const float4*>(a.QK + (base + j) * ld + c0 + f);
          kv = *reinterpret_cast<const float4*>(a.QK + (base + j) * ld + A + c0 + f);
        }
        fm_store(X, j, f, qv);
        fm_store(Y, j, f, kv);
      }
      __syncthreads();
      if (live)
        for (int f = 0; f < 128; ++f) tile_fma<4>(s, X, f * TLD + 4 * ty, Y, f * TLD + 4 * tx);
    }
    __syncthreads();  // X and Y are free: P goes to X
    // softmax per row over the 16 threads of a half warp (every lane takes
    // part in the shuffles; rows and keys past nnei come out zero)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = 4 * ty + i;
      const float4 rj = rws[j];
      const float2 wj = w2s[j];
      float2 lp[8], mx = make_float2(-3.0e38f, 0.f);
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int k = t_rc(tx, jj);
        lp[jj] = make_float2(-3.0e38f, 0.f);
        if (k < nn) {
          lp[jj] = smooth_logit(s[i][jj] * scale, a.shift, wj, w2s[k]);
          if (lp[jj].x > mx.x || (lp[jj].x == mx.x && lp[jj].y > mx.y)) mx = lp[jj];
        }
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, mx.x, o);
        const float ol = __shfl_xor_sync(0xffffffffu, mx.y, o);
        if (oh > mx.x || (oh == mx.x && ol > mx.y)) mx = make_float2(oh, ol);
      }
      float e[8], sum = 0.f;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        e[jj] = t_rc(tx, jj) < nn ? expf(pair_diff(lp[jj], mx)) : 0.f;
        sum += e[jj];
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      const float inv = sum > 0.f ? 1.0f / sum : 0.f;
      float pv[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int k = t_rc(tx, jj);
        pv[jj] = 0.f;
        if (j < nn && k < nn) {
          const float4 rk = rws[k];
          pv[jj] = e[jj] * inv * (rj.w * rk.w) * (rj.x * rk.x + rj.y * rk.y + rj.z * rk.z);
        }
      }
      tile_store_row(X + j * TLD, pv, 0, tx, 128);
    }
    // PG = P [G 1], 128 columns at a time (column m1 of [G 1] is 1, later
    // ones 0; m1 % 4 == 0)
    const int nn4 = (nn + 3) & ~3;
    for (int c0 = 0; c0 < a.ldpg; c0 += 128) {
      if (c0 > 0) __syncthreads();  // the previous part's products are done
      for (int idx = tid; idx < NP * 32; idx += FTF) {
        const int k = idx >> 5, f = c0 + 4 * (idx & 31);
        float4 vv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < nn) {
          if (f < a.m1) vv = *reinterpret_cast<const float4*>(a.G + (base + k) * a.m1 + f);
          else if (f == a.m1) vv.x = 1.f;
        }
        *reinterpret_cast<float4*>(Y + k * TLD + f - c0) = vv;
      }
      __syncthreads();  // P (first part) and this part of [G 1] are in place
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.f;
      if (4 * ty < nn)
        for (int k = 0; k < nn4; k += 4) tile_fma4<4>(acc, X, Y, k, ty, tx);
#pragma unroll
      for (int i = 0; i < 4; ++i) tile_store_row(a.PG + (base + 4 * ty + i) * a.ldpg, acc[i], c0, tx, a.ldpg);
    }
  }
}

// Adjoint of one attention layer for one centre, register-tiled like the
// forward (512 threads as a 32 x 16 grid; thread (ty, tx) owns rows 4 ty + i
// (i < 4) and keys or columns t_rc(tx, jj) (jj < 8) of each 128 x 128 product),
// in the form of the forward's output Y = [P G, rowsum P] [Wv Wo; bv Wo] +
// bo: with dPG = dE/d[P G, rowsum P] (a GEMM of dY with [Wv Wo; bv Wo]^T),
//   dP_jk = sum_c dPG_jc G_kc + dPG_j,m1        (the values V never appear)
//   softmax adjoint: dS, and the row / column parts of dE/dw and dE/drhat
//   dQ = dS K,  dK = dS^T Q,  dE/dG += P^T dPG (columns below m1).
// S and dP stay in registers through the softmax adjoint; dS and P then go to
// shared memory (row-major), where the three last products read them.  The
// column parts are summed over the 16 row groups in a fixed order.
template <int A>
__global__ void __launch_bounds__(FTF, 1) k_attn_bwd_f32(AttnArgs a, float scale) {
  extern __shared__ float sm[];
  float* B0 = sm;               // [128][TLD] operand chunks
  float* B1 = B0 + 128 * TLD;   // [128][TLD] K / G chunk, then dS (row-major)
  float* B2 = B1 + 128 * TLD;   // [128][TLD] P (row-major)
  float4* rws = reinterpret_cast<float4*>(B2 + 128 * TLD);  // [NP]
  float2* w2s = reinterpret_cast<float2*>(rws + NP);         // [NP] switch weights as float pairs
  float4* rowg = reinterpret_cast<float4*>(w2s + NP);        // [NP] row parts of (d rhat, d w)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int ld = a.ldq;  // Q | K, and dQ | dK
  for (int atom = blockIdx.x; atom < a.n; atom += gridDim.x) {
    const int nn = a.nnei[atom];
    const size_t base = (size_t)atom * NP;
    __syncthreads();  // the previous atom is done with every shared array
    for (int r = tid; r < NP; r += FTF) {
      rws[r] = r < nn ? reinterpret_cast<const float4*>(a.rw)[base + r] : make_float4(0.f, 0.f, 0.f, 0.f);
      w2s[r] = split_pair(r < nn ? a.w64[base + r] : 0.0);
    }
    const bool live = 4 * ty < nn && 4 * tx < nn;
    float s[4][8], dp[4][8];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) { s[i][jj] = 0.f; dp[i][jj] = 0.f; }
    // S = Q K^T over feature chunks of 128 (feature-major in B0, B1)
    for (int c0 = 0; c0 < A; c0 += 128) {
      if (c0 > 0) __syncthreads();
      for (int idx = tid; idx < NP * 32; idx += FTF) {
        int j, f;
        fm_pos(idx, j, f);
        float4 qv = make_float4(0.f, 0.f, 0.f, 0.f), kv = qv;
        if (j < nn) {
          qv = *reinterpret_cast<const float4*>(a.QK + (base + j) * ld + c0 + f);
          kv = *reinterpret_cast<const float4*>(a.QK + (base + j) * ld + A + c0 + f);
        }
        fm_store(B0, j, f, qv);
        fm_store(B1, j, f, kv);
      }
      __syncthreads();
      if (live)
        for (int f = 0; f < 128; ++f) tile_fma<4>(s, B0, f * TLD + 4 * ty, B1, f * TLD + 4 * tx);
    }
    __syncthreads();
    // dP = dPG G^T over the m1 columns (feature-major: dPG in B0, G in B1;
    // m1 % 4 == 0)
    for (int idx = tid; idx < NP * 32; idx += FTF) {
      int j, f;
      fm_pos(idx, j, f);
      float4 dv = make_float4(0.f, 0.f, 0.f, 0.f), gv = dv;
      if (j < nn && f < a.m1) {
        dv = *reinterpret_cast<const float4*>(a.dPG + (base + j) * a.ldpg + f);
        gv = *reinterpret_cast<const float4*>(a.G + (base + j) * a.m1 + f);
      }
      fm_store(B0, j, f, dv);
      fm_store(B1, j, f, gv);
    }
    __syncthreads();
    if (live)
      for (int f = 0; f < a.m1; ++f) tile_fma<4>(dp, B0, f * TLD + 4 * ty, B1, f * TLD + 4 * tx);
    __syncthreads();  // B0 and B1 are free: dS goes to B1, P to B2, column parts to B0
    // softmax adjoint per row over the 16 threads of a half warp (every lane
    // takes part in the shuffles; rows and keys past nnei come out zero)
    float cw[8], cx[8], cy[8], cz[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) { cw[jj] = 0.f; cx[jj] = 0.f; cy[jj] = 0.f; cz[jj] = 0.f; }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = 4 * ty + i;
      const float4 rj = rws[j];
      const float2 wj = w2s[j];
      const float dpg1 = j < nn ? a.dPG[(base + j) * a.ldpg + a.m1] : 0.f;  // adjoint of rowsum P
      float2 lp[8], mx = make_float2(-3.0e38f, 0.f);
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int k = t_rc(tx, jj);
        lp[jj] = make_float2(-3.0e38f, 0.f);
        if (k < nn) {
          lp[jj] = smooth_logit(s[i][jj] * scale, a.shift, wj, w2s[k]);  // as in the forward kernel
          if (lp[jj].x > mx.x || (lp[jj].x == mx.x && lp[jj].y > mx.y)) mx = lp[jj];
        }
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, mx.x, o);
        const float ol = __shfl_xor_sync(0xffffffffu, mx.y, o);
        if (oh > mx.x || (oh == mx.x && ol > mx.y)) mx = make_float2(oh, ol);
      }
      float e[8], sum = 0.f;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        e[jj] = t_rc(tx, jj) < nn ? expf(pair_diff(lp[jj], mx)) : 0.f;
        sum += e[jj];
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      const float inv = sum > 0.f ? 1.0f / sum : 0.f;
      float At[8], dA[8], tsum = 0.f;
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int k = t_rc(tx, jj);
        const float4 rk = rws[k];
        At[jj] = e[jj] * inv;
        dA[jj] = k < nn ? (dp[i][jj] + dpg1) * (rj.w * rk.w) * (rj.x * rk.x + rj.y * rk.y + rj.z * rk.z) : 0.f;
        tsum += At[jj] * dA[jj];
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
      float rw_ = 0.f, rx = 0.f, ry = 0.f, rz = 0.f, ds[8], pv[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int k = t_rc(tx, jj);
        ds[jj] = 0.f;
        pv[jj] = 0.f;
        if (j < nn && k < nn) {
          const float4 rk = rws[k];
          const float ww = rj.w * rk.w;
          const float c = rj.x * rk.x + rj.y * rk.y + rj.z * rk.z;
          const float dpv = dp[i][jj] + dpg1;
          const float dLp = At[jj] * (dA[jj] - tsum);
          ds[jj] = dLp * ww * scale;
          pv[jj] = At[jj] * ww * c;
          const float H = dpv * At[jj] * c + dLp * (s[i][jj] * scale + a.shift);  // dE/d(w_j w_k)
          const float dc = dpv * At[jj] * ww;                                      // dE/dc_jk
          rw_ += H * rk.w;
          rx += dc * rk.x; ry += dc * rk.y; rz += dc * rk.z;
          cw[jj] += H * rj.w;
          cx[jj] += dc * rj.x; cy[jj] += dc * rj.y; cz[jj] += dc * rj.z;
        }
      }
      tile_store_row(B1 + j * TLD, ds, 0, tx, 128);
      tile_store_row(B2 + j * TLD, pv, 0, tx, 128);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        rw_ += __shfl_xor_sync(0xffffffffu, rw_, o);
        rx += __shfl_xor_sync(0xffffffffu, rx, o);
        ry += __shfl_xor_sync(0xffffffffu, ry, o);
        rz += __shfl_xor_sync(0xffffffffu, rz, o);
      }
      if (tx == 0) rowg[j] = make_float4(rx, ry, rz, rw_);
    }
    // column parts of this thread's 4 rows -> B0 as [ty][key] (32 x 128 float4)
    float4* colp = reinterpret_cast<float4*>(B0);
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) colp[ty * NP + t_rc(tx, jj)] = make_float4(cx[jj], cy[jj], cz[jj], cw[jj]);
    __syncthreads();
    if (tid < nn) {
      float4 acc = rowg[tid];
      for (int q = 0; q < 32; ++q) {
        const float4 c = colp[q * NP + tid];
        acc.x += c.x; acc.y += c.y; acc.z += c.z; acc.w += c.w;
      }
      // one writer per row in a launch: a reduction without a return
      atomicAdd(reinterpret_cast<float4*>(a.dgeo) + base + tid, acc);
    }
    const int nn4 = (nn + 3) & ~3;
    for (int c0 = 0; c0 < A; c0 += 128) {
      // dQ = dS K: K key-major in B0
      __syncthreads();
      for (int idx = tid; idx < NP * 32; idx += FTF) {
        const int k = idx >> 5, f = 4 * (idx & 31);
        *reinterpret_cast<float4*>(B0 + k * TLD + f) =
            k < nn ? *reinterpret_cast<const float4*>(a.QK + (base + k) * ld + A + c0 + f) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.f;
      if (4 * ty < nn)
        for (int k = 0; k < nn4; k += 4) tile_fma4<4>(acc, B1, B0, k, ty, tx);
#pragma unroll
      for (int i = 0; i < 4; ++i) tile_store_row(a.dQK + (base + 4 * ty + i) * ld, acc[i], c0, tx, A);
      // dK = dS^T Q: Q row-major in B0
      __syncthreads();
      for (int idx = tid; idx < NP * 32; idx += FTF) {
        const int j = idx >> 5, f = 4 * (idx & 31);
        *reinterpret_cast<float4*>(B0 + j * TLD + f) =
            j < nn ? *reinterpret_cast<const float4*>(a.QK + (base + j) * ld + c0 + f) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.f;
      if (4 * ty < nn)
        for (int j = 0; j < nn; ++j) tile_fma<4>(acc, B1, j * TLD + 4 * ty, B0, j * TLD + 4 * tx);
#pragma unroll
      for (int i = 0; i < 4; ++i) tile_store_row(a.dQK + (base + 4 * ty + i) * ld + A, acc[i], c0, tx, A);
    }
    // dE/dG += P^T dPG: dPG row-major in B0 (columns below m1; m1 <= 128)
    __syncthreads();
    for (int idx = tid; idx < NP * 32; idx += FTF) {
      const int j = idx >> 5, f = 4 * (idx & 31);
      *reinterpret_cast<float4*>(B0 + j * TLD + f) = j < nn && f < a.m1
                                                         ? *reinterpret_cast<const float4*>(a.dPG + (base + j) * a.ldpg + f)
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    if (4 * ty < nn && 4 * tx < a.m1) {
      float acc[4][8];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.f;
      for (int j = 0; j < nn; ++j) tile_fma<4>(acc, B2, j * TLD + 4 * ty, B0, j * TLD + 4 * tx);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * ty + i;
        if (k >= nn) continue;
        float* dgrow = a.dG + (base + k) * a.m1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 64 * h + 4 * tx;
          if (c < a.m1) {
            float4* dg = reinterpret_cast<float4*>(dgrow + c);
            float4 x = *dg;
            x.x += acc[i][4 * h]; x.y += acc[i][4 * h + 1]; x.z += acc[i][4 * h + 2]; x.w += acc[i][4 * h + 3];
            *dg = x;
          }
        }
      }
    }
  }
}

static int sm_count() {
  static int count = 0;
  if (count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
    if (count <= 0) count = 1;
  }
  return count;
}

template <int A>
static void attn_f32_launch(const AttnArgs& a, bool bwd, cudaStream_t st) {
  const float scale = (float)(1.0 / sqrt((double)A));
  const int grid = a.n < sm_count() ? a.n : sm_count();
  if (!bwd) {
    const size_t smem = sizeof(float) * (2 * 128 * TLD + 4 * NP) + sizeof(float2) * NP;
    cudaFuncSetAttribute(k_attn_fwd_f32<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_attn_fwd_f32<A><<<grid, FTF, smem, st>>>(a, scale);
  } else {
    const size_t smem = sizeof(float) * (3 * 128 * TLD + 8 * NP) + sizeof(float2) * NP;
    cudaFuncSetAttribute(k_attn_bwd_f32<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_attn_bwd_f32<A><<<grid, FTF, smem, st>>>(a, scale);
  }
  note_launch();
}

// Attention widths with a kernel instance: 128 (the measured model) and 256
// (the paper's own model size).
void launch_attn_fwd_f32(const AttnArgs& a, cudaStream_t st) {
  if (a.n == 0) return;
  if (a.A == 256) attn_f32_launch<256>(a, false, st);
  else attn_f32_launch<128>(a, false, st);
}

void launch_attn_bwd_f32(const AttnArgs& a, cudaStream_t st) {
  if (a.n == 0) return;
  if (a.A == 256) attn_f32_launch<256>(a, true, st);
  else attn_f32_launch<128>(a, true, st);
}

// ------------------------------------------------------------- descriptor
// T = R^T G / sel (4 x m1); D = T^T T[:, :axis]; X = [D (row-major), Z[t_i]].
// A block of 128 threads per atom, 10 blocks per SM (48 registers): the kernel
// waits on its loads, and more resident warps hide more of them.
__global__ void __launch_bounds__(128, 10) k_desc_fwd(DescArgs a) {
  extern __shared__ float sm[];
  float* Ts = sm;  // [4][m1]
  const int atom = blockIdx.x;
  const int nn = a.nnei[atom];
  const size_t base = (size_t)atom * NP;
  const float inv_sel = 1.0f / (float)a.sel;
  if (a.cq) {
    // a warp per column quad, its lanes over the rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const float4* G4 = reinterpret_cast<const float4*>(a.G + base * a.m1);
    const float4* R4 = reinterpret_cast<const float4*>(a.R) + base;
    for (int q = warp; q < a.m1 / 4; q += nw) {
      float t[4][4] = {};
      // the lane's (at most NP / 32) rows, their loads issued together
      float4 rq[NP / 32], gq[NP / 32];
#pragma unroll
      for (int it = 0; it < NP / 32; ++it) {
        const int s = lane + 32 * it;
        rq[it] = s < nn ? R4[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        gq[it] = s < nn ? G4[(size_t)q * NP + s] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int it = 0; it < NP / 32; ++it) {
        const float rr[4] = {rq[it].x, rq[it].y, rq[it].z, rq[it].w};
        const float gg[4] = {gq[it].x, gq[it].y, gq[it].z, gq[it].w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int k = 0; k < 4; ++k) t[c][k] = fmaf(rr[c], gg[k], t[c][k]);
      }
      float tv[16];
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int k = 0; k < 4; ++k) tv[4 * c + k] = t[c][k];
      const float v = warp_reduce_scatter16(tv);  // lane l: entry l % 16 = (c, k) = (l / 4, l % 4)
      if (lane < 16) Ts[(lane >> 2) * a.m1 + 4 * q + (lane & 3)] = v * inv_sel;
    }
  } else {
    for (int c = threadIdx.x; c < a.m1; c += blockDim.x) {
      float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
      for (int s = 0; s < nn; ++s) {
        const float4 r = reinterpret_cast<const float4*>(a.R)[base + s];
        const float gv = a.G[(base + s) * a.m1 + c];
        t0 = fmaf(r.x, gv, t0); t1 = fmaf(r.y, gv, t1); t2 = fmaf(r.z, gv, t2); t3 = fmaf(r.w, gv, t3);
      }
      Ts[c] = t0 * inv_sel; Ts[a.m1 + c] = t1 * inv_sel; Ts[2 * a.m1 + c] = t2 * inv_sel; Ts[3 * a.m1 + c] = t3 * inv_sel;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * a.m1; t += blockDim.x) a.T[(size_t)atom * 4 * a.m1 + t] = Ts[t];
  float* x = a.X + (size_t)atom * a.fit_in;
  for (int idx = threadIdx.x; idx < a.m1 * a.axis; idx += blockDim.x) {
    const int p = idx / a.axis, b = idx % a.axis;
    float d = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) d = fmaf(Ts[c * a.m1 + p], Ts[c * a.m1 + b], d);
    x[idx] = d;
  }
  const int ti = a.atype[atom];
  for (int t = threadIdx.x; t < a.tebd_dim; t += blockDim.x) x[a.m1 * a.axis + t] = a.tebd[ti * a.tebd_dim + t];
}

// dT[c][p] = sum_b<axis dD[p][b] T[c][b] + (p < axis) sum_q dD[q][p] T[c][q];
// dG_s = R_s dT / sel; dR_s = G_s dT^T / sel.
__global__ void k_desc_bwd(DescArgs a) {
  extern __shared__ float sm[];
  const int m1 = a.m1, ax = a.axis;
  float* Ts = sm;              // [4][m1]
  float* dTs = Ts + 4 * m1;    // [4][m1]
  float* dD = dTs + 4 * m1;    // [m1][axis]
  float* dDt = dD + m1 * ax;   // [axis][m1]: dD transposed, so that threads with consecutive p read consecutive words
  const int atom = blockIdx.x;
  const int nn = a.nnei[atom];
  const size_t base = (size_t)atom * NP;
  const float inv_sel = 1.0f / (float)a.sel;
  for (int t = threadIdx.x; t < 4 * m1; t += blockDim.x) Ts[t] = a.T[(size_t)atom * 4 * m1 + t];
  for (int t = threadIdx.x; t < m1 * ax; t += blockDim.x) {
    const float v = a.dX[(size_t)atom * a.fit_in + t];
    dD[t] = v;
    dDt[(t % ax) * m1 + t / ax] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * m1; t += blockDim.x) {
    const int c = t / m1, p = t % m1;
    float v = 0.f;
    for (int b = 0; b < ax; ++b) v = fmaf(dDt[b * m1 + p], Ts[c * m1 + b], v);
    if (p < ax)
      for (int q = 0; q < m1; ++q) v = fmaf(dD[q * ax + p], Ts[c * m1 + q], v);
    dTs[t] = v * inv_sel;
  }
  __syncthreads();
  if (a.cq) {
    // A thread per row: its dG row in column quads (consecutive threads ->
    // consecutive rows; live rows only: the fused layer kernels and the
    // embedding adjoint read no others) and its dR row, with the columns of
    // dT read as float4 broadcasts (m1 % 4 == 0)
    const int q4 = m1 / 4;
    float4* dG4 = reinterpret_cast<float4*>(a.dG + base * m1);
    const float4* G4 = reinterpret_cast<const float4*>(a.G + base * m1);
    const float4* dT4 = reinterpret_cast<const float4*>(dTs);
    for (int s = threadIdx.x; s < NP; s += blockDim.x) {
      float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
      if (s < nn) {
        const float4 r = reinterpret_cast<const float4*>(a.R)[base + s];
#pragma unroll 1  // at 48 registers 10 blocks fit per SM (unrolled: 66 and 7, 30 % slower)
        for (int q = 0; q < q4; ++q) {
          const float4 g = G4[(size_t)q * NP + s];
          const float4 t[4] = {dT4[q], dT4[q4 + q], dT4[2 * q4 + q], dT4[3 * q4 + q]};
          const float gg[4] = {g.x, g.y, g.z, g.w};
          float4 v;
          float* vp = &v.x;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float t0 = (&t[0].x)[k], t1 = (&t[1].x)[k], t2 = (&t[2].x)[k], t3 = (&t[3].x)[k];
            vp[k] = r.x * t0 + r.y * t1 + r.z * t2 + r.w * t3;
            d0 = fmaf(gg[k], t0, d0); d1 = fmaf(gg[k], t1, d1);
            d2 = fmaf(gg[k], t2, d2); d3 = fmaf(gg[k], t3, d3);
          }
          dG4[(size_t)q * NP + s] = v;
        }
      }
      reinterpret_cast<float4*>(a.dR)[base + s] = make_float4(d0, d1, d2, d3);
    }
    return;
  }
  // dG rows (all NP rows; zero on padding), a column quad per thread (m1 % 4 == 0)
  const int q4 = m1 / 4;
  float4* dG4 = reinterpret_cast<float4*>(a.dG + base * m1);
  for (int idx = threadIdx.x; idx < NP * q4; idx += blockDim.x) {
    const int s = idx / q4, q = idx % q4;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (s < nn) {
      const float4 r = reinterpret_cast<const float4*>(a.R)[base + s];
      float* vp = &v.x;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int p = 4 * q + k;
        vp[k] = r.x * dTs[p] + r.y * dTs[m1 + p] + r.z * dTs[2 * m1 + p] + r.w * dTs[3 * m1 + p];
      }
    }
    dG4[idx] = v;
  }
  // dR rows: a warp per row, a column quad per lane
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const float4* G4 = reinterpret_cast<const float4*>(a.G + base * m1);
  for (int s = warp; s < NP; s += nw) {
    float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
    if (s < nn) {
      for (int q = lane; q < q4; q += 32) {
        const float4 g = G4[(size_t)s * q4 + q];
        const float gg[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int p = 4 * q + k;
          d0 = fmaf(gg[k], dTs[p], d0); d1 = fmaf(gg[k], dTs[m1 + p], d1);
          d2 = fmaf(gg[k], dTs[2 * m1 + p], d2); d3 = fmaf(gg[k], dTs[3 * m1 + p], d3);
        }
      }
    }
    d0 = warp_sum(d0); d1 = warp_sum(d1); d2 = warp_sum(d2); d3 = warp_sum(d3);
    if (lane == 0) reinterpret_cast<float4*>(a.dR)[base + s] = make_float4(d0, d1, d2, d3);
  }
}

void launch_desc_fwd(const DescArgs& a, cudaStream_t st) {
  if (a.n == 0) return;
  k_desc_fwd<<<a.n, 128, sizeof(float) * 4 * a.m1, st>>>(a);
  note_launch();
}
void launch_desc_bwd(const DescArgs& a, cudaStream_t st) {
  if (a.n == 0) return;
  size_t sm = sizeof(float) * (8 * a.m1 + 2 * a.m1 * a.axis);
  k_desc_bwd<<<a.n, 128, sm, st>>>(a);
  note_launch();
}

// ------------------------------------------------------------ fitting head
__global__ void k_energy_head(const float* __restrict__ H, int n, int width, const float* __restrict__ w,
                              const float* __restrict__ bptr, float out_scale, const float* __restrict__ ebias,
                              const int* __restrict__ atype, float* __restrict__ e) {
  const int atom = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (atom >= n) return;
  float s = 0.f;
  for (int c = lane; c < width; c += 32) s = fmaf(H[(size_t)atom * width + c], w[c], s);
  s = warp_sum(s);
  if (lane == 0) e[atom] = out_scale * (s + *bptr) + ebias[atype[atom]];
}

void launch_energy_head(const float* H, int n, int width, const float* w_out, const float* b_out, float out_scale,
                        const float* ebias, const int* atype, float* e, cudaStream_t st) {
  if (n == 0) return;
  k_energy_head<<<(unsigned)(((long long)n * 32 + 255) / 256), 256, 0, st>>>(H, n, width, w_out, b_out, out_scale,
                                                                          ebias, atype, e);
  note_launch();
}

__global__ void k_tanh_bwd(const float* __restrict__ dH, const float* __restrict__ Hc, const float* __restrict__ Hp,
                           float* __restrict__ dZ, long long count) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float t = Hp ? Hc[i] - Hp[i] : Hc[i];
  dZ[i] = dH[i] * (1.f - t * t);
}

void launch_tanh_bwd(const float* dH, const float* Hcur, const float* Hprev, float* dZ, long long count,
                     cudaStream_t st) {
  if (count == 0) return;
  k_tanh_bwd<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(dH, Hcur, Hprev, dZ, count);
  note_launch();
}

__global__ void k_fill_rows(float* __restrict__ dst, const float* __restrict__ row, long long count, long long nlocal_el,
                            int width) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  dst[i] = i < nlocal_el ? row[i % width] : 0.f;
}

void launch_fill_rows(float* dst, const float* row, int n, int nlocal, int width, cudaStream_t st) {
  long long count = (long long)n * width;
  if (count == 0) return;
  k_fill_rows<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(dst, row, count, (long long)nlocal * width, width);
  note_launch();
}

}  // namespace dpa1
