// Training kernels of the distilled student potential (stage a17): weight
// gradients of the energy, the per-frame energy / force loss, Adam, and the
// refresh of the derived weight copies the forward kernels read.
//
// Loss of one frame (N atoms): L = pe ((E - E_ref) / N)^2 + pf mean |F - F_ref|^2.
// dL/dtheta = 2 pe (E - E_ref) / N^2 dE/dtheta
//           - (2 pf / 3N) d/dtheta [ sum_k (F - F_ref)_k . dE/dx_k ],
// and the bracket's theta-gradient is the derivative of dE/dtheta along the
// fixed displacement field v = F - F_ref: d/de dE/dtheta(x + e v) at e = 0.
// It is evaluated exactly in forward mode over the adjoint: every quantity q
// of the energy evaluation and of its adjoint gets its tangent q' = dq/de,
// and the weight gradients (sums over rows of input (x) adjoint) get theirs by
// the product rule.
#include <algorithm>

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

// One block: loss of the frame, the gradient scales and the direction
// v = F - F_ref.
__global__ void k_train_prep(int n, const double* __restrict__ energy, double e_ref,
                             const double* __restrict__ force, const double* __restrict__ force_ref, double pe,
                             double pf, double* __restrict__ v, double* __restrict__ loss,
                             float* __restrict__ scales) {
  __shared__ double red_s[32];
  double ss = 0.0;
  for (int k = threadIdx.x; k < 3 * n; k += blockDim.x) {
    const double d = force[k] - force_ref[k];
    v[k] = d;
    ss += d * d;
  }
  ss = warp_sum_d(ss);
  if ((threadIdx.x & 31) == 0) red_s[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) S += red_s[w];
    const double nn = n > 0 ? (double)n : 1.0;
    const double de = *energy - e_ref;
    const double lE = pe * (de / nn) * (de / nn);
    const double lF = pf * S / (3.0 * nn);
    loss[0] = lE + lF;
    loss[1] = lE;
    loss[2] = lF;
    scales[0] = 1.0f;
    scales[1] = (float)(2.0 * pe * de / (nn * nn));
    scales[2] = (float)(-2.0 * pf / (3.0 * nn));
    scales[3] = 0.f;
  }
}

__global__ void k_axpy(float* __restrict__ g, const float* __restrict__ src, int n, const float* __restrict__ scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g[i] += *scale * src[i];
}

// ------------------------------------------------------------------ tangents
// R'_ij = dR_ij/dr_ij . (v_j - v_i), in FP64 like the FP32 path's environment
// rows: with d = |r|, s = sw(d)/d, q = s/d, R = ((s - avg0)/std0,
// (q r_a - avg_a)/std_a): s' = s_d d', (q r_a)' = q_d d' r_a + q r_a',
// d' = r.r'/d.  (The image shift of r is constant.)
__global__ void k_env_jvp(JvpArgs a) {
  const long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long long)a.n * NP) return;
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  const int j = a.nlist[row];
  if (j >= 0) {
    const int i = (int)(row / NP);
    const CellGrid g = *a.grid;
    const double rx = mic(a.coord[3 * j] - a.coord[3 * i], g.L[0]);
    const double ry = mic(a.coord[3 * j + 1] - a.coord[3 * i + 1], g.L[1]);
    const double rz = mic(a.coord[3 * j + 2] - a.coord[3 * i + 2], g.L[2]);
    const double vx = a.v[3 * j] - a.v[3 * i], vy = a.v[3 * j + 1] - a.v[3 * i + 1], vz = a.v[3 * j + 2] - a.v[3 * i + 2];
    const double d = sqrt(rx * rx + ry * ry + rz * rz), inv = 1.0 / d;
    const double dd = (rx * vx + ry * vy + rz * vz) * inv;
    const double rcs = a.rcs, rc = a.rc;
    double sw, dsw;
    if (d < rcs) {
      sw = 1.0; dsw = 0.0;
    } else if (d < rc) {
      const double wdt = rc - rcs, u = (d - rcs) / wdt;
      sw = u * u * u * (-6.0 * u * u + 15.0 * u - 10.0) + 1.0;
      dsw = -30.0 * u * u * (u - 1.0) * (u - 1.0) / wdt;
    } else {
      sw = 0.0; dsw = 0.0;
    }
    const double s_d = dsw * inv - sw * inv * inv;
    const double q = sw * inv * inv, q_d = dsw * inv * inv - 2.0 * sw * inv * inv * inv;
    const float* sv = a.dstd + 4 * a.atype[i];
    out.x = (float)(s_d * dd / (double)sv[0]);
    out.y = (float)((q_d * dd * rx + q * vx) / (double)sv[1]);
    out.z = (float)((q_d * dd * ry + q * vy) / (double)sv[2]);
    out.w = (float)((q_d * dd * rz + q * vz) / (double)sv[3]);
  }
  reinterpret_cast<float4*>(a.Rd)[row] = out;
}

// The embedding net G = net(s) (1 + Gt[t_i][t_j]), net: 1 -> E0 -> E1 -> E2,
// tanh layers with the residual rule (same width: x + f; double: [x, x] + f),
// input s = R_ij,0.  A CTA takes JROWS neighbour rows of one atom and
// evaluates the activations and their tangents (s' = R'_ij,0).  Mode 0 writes
// G'.  Mode 1 also runs the adjoint from dE/dG and (dE/dG)' and adds
// *scale times the tangents of the weight gradients to grad (per-CTA sums,
// one atomic add per weight at the end).
constexpr int JROWS = 32;
constexpr int JTHREADS = 256;

template <int E0, int E1, int E2>
struct JvpEmbedSmem {
  static constexpr int P2 = E2 + 1, Q0 = E0 + 1, Q1 = E1 + 1;
  // packed weights as in the parameter vector, W2 rows padded to P2
  static constexpr int W0 = 0, B0 = E0, W1 = 2 * E0, B1 = W1 + E0 * E1, W2 = B1 + E1, B2 = W2 + E1 * P2;
  static constexpr int X = B2 + E2, XD = X + JROWS;
  static constexpr int H1 = XD + JROWS, H1D = H1 + JROWS * Q0;
  static constexpr int H2 = H1D + JROWS * Q0, H2D = H2 + JROWS * Q1;
  static constexpr int Z3 = H2D + JROWS * Q1, Z3D = Z3 + JROWS * P2;
  static constexpr int FWD_TOTAL = Z3D + JROWS * P2;
  // mode 1 only
  static constexpr int DH2 = FWD_TOTAL, DH2D = DH2 + JROWS * Q1, DZ2 = DH2D + JROWS * Q1, DZ2D = DZ2 + JROWS * Q1;
  static constexpr int DZ1 = DZ2D + JROWS * Q1, DZ1D = DZ1 + JROWS * Q0;
  static constexpr int NW = B2 + E2 - E1 * (P2 - E2);  // packed weight count
  static constexpr int ACC = DZ1D + JROWS * Q0, TOTAL = ACC + NW;
};

template <int IN, int OUT>
__device__ __forceinline__ float jskip(const float* x, int o) {
  return OUT == IN ? x[o] : (OUT == 2 * IN ? x[o % IN] : 0.f);
}

template <int E0, int E1, int E2>
__global__ void __launch_bounds__(JTHREADS) k_embed_jvp(JvpArgs a, int mode, float* __restrict__ grad,
                                                         const float* __restrict__ scale) {
  using S = JvpEmbedSmem<E0, E1, E2>;
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  // weights (packed W0 b0 W1 b1 | W2 | b2)
  for (int t = tid; t < S::W2; t += JTHREADS) sm[t] = a.w[t];
  for (int t = tid; t < E1 * E2; t += JTHREADS) sm[S::W2 + (t / E2) * S::P2 + t % E2] = a.w[S::W2 + t];
  for (int t = tid; t < E2; t += JTHREADS) sm[S::B2 + t] = a.w[S::W2 + E1 * E2 + t];
  if (mode == 1)
    for (int t = tid; t < S::NW; t += JTHREADS) sm[S::ACC + t] = 0.f;
  const int per_atom = NP / JROWS;
  const int nblk = a.n * per_atom;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int atom = blk / per_atom, r0 = (blk % per_atom) * JROWS;
    const int cnt = max(0, min(JROWS, a.nnei[atom] - r0));
    const size_t base = (size_t)atom * NP + r0;
    if (cnt == 0) {  // uniform over the CTA
      if (mode == 0)
        for (int idx = tid; idx < JROWS * E2; idx += JTHREADS) a.Gd[(base + idx / E2) * a.m1 + idx % E2] = 0.f;
      continue;
    }
    const int ti = a.atype[atom];
    __syncthreads();  // the previous block is done with the activations
    for (int r = tid; r < JROWS; r += JTHREADS) {
      sm[S::X + r] = r < cnt ? a.R[(base + r) * 4] : 0.f;
      sm[S::XD + r] = r < cnt ? a.Rd[(base + r) * 4] : 0.f;
    }
    __syncthreads();
    // layer 1: h1 = tanh(s W0 + b0), h1' = (1 - h1^2) s' W0
    for (int idx = tid; idx < JROWS * E0; idx += JTHREADS) {
      const int r = idx / E0, p = idx % E0;
      float h = 0.f, hd = 0.f;
      if (r < cnt) {
        const float b0 = a.b0t ? a.b0t[((size_t)ti * a.ntypes + a.atype[a.nlist[base + r]]) * E0 + p] : sm[S::B0 + p];
        h = tanhf(fmaf(sm[S::X + r], sm[S::W0 + p], b0));
        hd = (1.f - h * h) * sm[S::XD + r] * sm[S::W0 + p];
      }
      sm[S::H1 + r * S::Q0 + p] = h;
      sm[S::H1D + r * S::Q0 + p] = hd;
    }
    __syncthreads();
    // layer 2: H2 = skip(h1) + tanh(h1 W1 + b1), and its tangent
    for (int idx = tid; idx < JROWS * E1; idx += JTHREADS) {
      const int r = idx / E1, b = idx % E1;
      float h = 0.f, hd = 0.f;
      if (r < cnt) {
        const float* h1 = sm + S::H1 + r * S::Q0;
        const float* h1d = sm + S::H1D + r * S::Q0;
        float z = sm[S::B1 + b], zd = 0.f;
        for (int p = 0; p < E0; ++p) {
          const float wv = sm[S::W1 + p * E1 + b];
          z = fmaf(h1[p], wv, z);
          zd = fmaf(h1d[p], wv, zd);
        }
        const float t = tanhf(z);
        h = jskip<E0, E1>(h1, b) + t;
        hd = jskip<E0, E1>(h1d, b) + (1.f - t * t) * zd;
      }
      sm[S::H2 + r * S::Q1 + b] = h;
      sm[S::H2D + r * S::Q1 + b] = hd;
    }
    __syncthreads();
    // layer 3 pre-activation: t3 = tanh(H2 W2 + b2) and t3'
    for (int idx = tid; idx < JROWS * E2; idx += JTHREADS) {
      const int r = idx / E2, c = idx % E2;
      float t = 0.f, td = 0.f;
      if (r < cnt) {
        const float* h2 = sm + S::H2 + r * S::Q1;
        const float* h2d = sm + S::H2D + r * S::Q1;
        float z = sm[S::B2 + c], zd = 0.f;
        for (int b = 0; b < E1; ++b) {
          const float wv = sm[S::W2 + b * S::P2 + c];
          z = fmaf(h2[b], wv, z);
          zd = fmaf(h2d[b], wv, zd);
        }
        t = tanhf(z);
        td = (1.f - t * t) * zd;
      }
      sm[S::Z3 + r * S::P2 + c] = t;
      sm[S::Z3D + r * S::P2 + c] = td;
    }
    __syncthreads();
    if (mode == 0) {
      for (int idx = tid; idx < JROWS * E2; idx += JTHREADS) {
        const int r = idx / E2, c = idx % E2;
        float gd = 0.f;
        if (r < cnt) {
          const int tj = a.atype[a.nlist[base + r]];
          const float f = 1.f + a.Gt[((size_t)ti * a.ntypes + tj) * E2 + c];
          gd = (jskip<E1, E2>(sm + S::H2D + r * S::Q1, c) + sm[S::Z3D + r * S::P2 + c]) * f;
        }
        a.Gd[(base + r) * a.m1 + c] = gd;
      }
      continue;
    }
    // adjoint of layer 3 with g = dE/dG (1 + Gt): dz3 = g (1 - t3^2),
    // dz3' = g' (1 - t3^2) - 2 g t3 t3' (in place of t3, t3')
    for (int idx = tid; idx < JROWS * E2; idx += JTHREADS) {
      const int r = idx / E2, c = idx % E2;
      float dz = 0.f, dzd = 0.f;
      if (r < cnt) {
        const int tj = a.atype[a.nlist[base + r]];
        const float f = 1.f + a.Gt[((size_t)ti * a.ntypes + tj) * E2 + c];
        const float g = a.dG[(base + r) * a.m1 + c] * f, gd = a.dGd[(base + r) * a.m1 + c] * f;
        const float t = sm[S::Z3 + r * S::P2 + c], td = sm[S::Z3D + r * S::P2 + c];
        dz = g * (1.f - t * t);
        dzd = gd * (1.f - t * t) - 2.f * g * t * td;
      }
      sm[S::Z3 + r * S::P2 + c] = dz;
      sm[S::Z3D + r * S::P2 + c] = dzd;
    }
    __syncthreads();
    // dH2 = W2 dz3 + skip^T(g), dz2 = dH2 (1 - t2^2) with t2 = H2 - skip(h1)
    for (int idx = tid; idx < JROWS * E1; idx += JTHREADS) {
      const int r = idx / E1, b = idx % E1;
      float dh = 0.f, dhd = 0.f, dz = 0.f, dzd = 0.f;
      if (r < cnt) {
        const float* dz3 = sm + S::Z3 + r * S::P2;
        const float* dz3d = sm + S::Z3D + r * S::P2;
        for (int c = 0; c < E2; ++c) {
          const float wv = sm[S::W2 + b * S::P2 + c];
          dh = fmaf(wv, dz3[c], dh);
          dhd = fmaf(wv, dz3d[c], dhd);
        }
        if (E2 == E1 || E2 == 2 * E1) {
          const int tj = a.atype[a.nlist[base + r]];
          const float* gt = a.Gt + ((size_t)ti * a.ntypes + tj) * E2;
          for (int c = b; c < E2; c += E1) {
            const float f = 1.f + gt[c];
            dh += a.dG[(base + r) * a.m1 + c] * f;
            dhd += a.dGd[(base + r) * a.m1 + c] * f;
          }
        }
        const float t = sm[S::H2 + r * S::Q1 + b] - jskip<E0, E1>(sm + S::H1 + r * S::Q0, b);
        const float td = sm[S::H2D + r * S::Q1 + b] - jskip<E0, E1>(sm + S::H1D + r * S::Q0, b);
        dz = dh * (1.f - t * t);
        dzd = dhd * (1.f - t * t) - 2.f * dh * t * td;
      }
      sm[S::DH2 + r * S::Q1 + b] = dh;
      sm[S::DH2D + r * S::Q1 + b] = dhd;
      sm[S::DZ2 + r * S::Q1 + b] = dz;
      sm[S::DZ2D + r * S::Q1 + b] = dzd;
    }
    __syncthreads();
    // dh1 = W1 dz2 + skip^T(dH2), dz1 = dh1 (1 - h1^2)
    for (int idx = tid; idx < JROWS * E0; idx += JTHREADS) {
      const int r = idx / E0, p = idx % E0;
      float dz = 0.f, dzd = 0.f;
      if (r < cnt) {
        float dh = 0.f, dhd = 0.f;
        for (int b = 0; b < E1; ++b) {
          const float wv = sm[S::W1 + p * E1 + b];
          dh = fmaf(wv, sm[S::DZ2 + r * S::Q1 + b], dh);
          dhd = fmaf(wv, sm[S::DZ2D + r * S::Q1 + b], dhd);
        }
        if (E1 == E0 || E1 == 2 * E0)
          for (int b = p; b < E1; b += E0) {
            dh += sm[S::DH2 + r * S::Q1 + b];
            dhd += sm[S::DH2D + r * S::Q1 + b];
          }
        const float h = sm[S::H1 + r * S::Q0 + p], hd = sm[S::H1D + r * S::Q0 + p];
        dz = dh * (1.f - h * h);
        dzd = dhd * (1.f - h * h) - 2.f * dh * h * hd;
      }
      sm[S::DZ1 + r * S::Q0 + p] = dz;
      sm[S::DZ1D + r * S::Q0 + p] = dzd;
    }
    __syncthreads();
    // tangents of the weight gradients: (sum_r in (x) dz)' = sum_r in' (x) dz + in (x) dz'
    for (int t = tid; t < S::NW; t += JTHREADS) {
      float g = 0.f;
      if (t < S::B0) {
        for (int r = 0; r < cnt; ++r)
          g += sm[S::XD + r] * sm[S::DZ1 + r * S::Q0 + t] + sm[S::X + r] * sm[S::DZ1D + r * S::Q0 + t];
      } else if (t < S::W1) {
        for (int r = 0; r < cnt; ++r) g += sm[S::DZ1D + r * S::Q0 + (t - S::B0)];
      } else if (t < S::B1) {
        const int p = (t - S::W1) / E1, b = (t - S::W1) % E1;
        for (int r = 0; r < cnt; ++r)
          g += sm[S::H1D + r * S::Q0 + p] * sm[S::DZ2 + r * S::Q1 + b] +
               sm[S::H1 + r * S::Q0 + p] * sm[S::DZ2D + r * S::Q1 + b];
      } else if (t < S::W2) {
        for (int r = 0; r < cnt; ++r) g += sm[S::DZ2D + r * S::Q1 + (t - S::B1)];
      } else if (t < S::W2 + E1 * E2) {
        const int b = (t - S::W2) / E2, c = (t - S::W2) % E2;
        for (int r = 0; r < cnt; ++r)
          g += sm[S::H2D + r * S::Q1 + b] * sm[S::Z3 + r * S::P2 + c] +
               sm[S::H2 + r * S::Q1 + b] * sm[S::Z3D + r * S::P2 + c];
      } else {
        const int c = t - S::W2 - E1 * E2;
        for (int r = 0; r < cnt; ++r) g += sm[S::Z3D + r * S::P2 + c];
      }
      sm[S::ACC + t] += g;
    }
  }
  if (mode == 1) {
    __syncthreads();
    const float sc = *scale;
    for (int t = tid; t < S::NW; t += JTHREADS) atomicAdd(&grad[t], sc * sm[S::ACC + t]);
  }
}

// T' = (R'^T G + R^T G') / sel and D' = T'^T T_< + T^T T'_< (the type row of
// X is constant).  One CTA per atom.
__global__ void k_desc_jvp_fwd(JvpArgs a) {
  extern __shared__ float sm[];
  const int m1 = a.m1, ax = a.axis;
  float* Ts = sm;            // [4][m1]
  float* Tds = Ts + 4 * m1;  // [4][m1]
  const int atom = blockIdx.x;
  const int nn = a.nnei[atom];
  const size_t base = (size_t)atom * NP;
  const float inv_sel = 1.0f / (float)a.sel;
  for (int t = threadIdx.x; t < 4 * m1; t += blockDim.x) {
    const int c = t / m1, p = t % m1;
    float v = 0.f;
    for (int s = 0; s < nn; ++s) {
      const float* r = a.R + (base + s) * 4;
      const float* rd = a.Rd + (base + s) * 4;
      v = fmaf(rd[c], a.G[(base + s) * m1 + p], v);
      v = fmaf(r[c], a.Gd[(base + s) * m1 + p], v);
    }
    Tds[t] = v * inv_sel;
    Ts[t] = a.T[(size_t)atom * 4 * m1 + t];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * m1; t += blockDim.x) a.Td[(size_t)atom * 4 * m1 + t] = Tds[t];
  float* xd = a.Xd + (size_t)atom * a.fit_in;
  for (int idx = threadIdx.x; idx < m1 * ax; idx += blockDim.x) {
    const int p = idx / ax, b = idx % ax;
    float d = 0.f;
    for (int c = 0; c < 4; ++c) d += Tds[c * m1 + p] * Ts[c * m1 + b] + Ts[c * m1 + p] * Tds[c * m1 + b];
    xd[idx] = d;
  }
  for (int t = m1 * ax + threadIdx.x; t < a.fit_in; t += blockDim.x) xd[t] = 0.f;
}

// dT = (dD T_< + [p < axis] dD^T T) / sel as in the descriptor adjoint, its
// tangent by the product rule, and (dE/dG)' = R' dT + R dT'.
__global__ void k_desc_jvp_bwd(JvpArgs a) {
  extern __shared__ float sm[];
  const int m1 = a.m1, ax = a.axis;
  float* Ts = sm;
  float* Tds = Ts + 4 * m1;
  float* dTs = Tds + 4 * m1;
  float* dTds = dTs + 4 * m1;
  float* dD = dTds + 4 * m1;  // [m1][axis]
  float* dDd = dD + m1 * ax;
  const int atom = blockIdx.x;
  const int nn = a.nnei[atom];
  const size_t base = (size_t)atom * NP;
  const float inv_sel = 1.0f / (float)a.sel;
  for (int t = threadIdx.x; t < 4 * m1; t += blockDim.x) {
    Ts[t] = a.T[(size_t)atom * 4 * m1 + t];
    Tds[t] = a.Td[(size_t)atom * 4 * m1 + t];
  }
  for (int t = threadIdx.x; t < m1 * ax; t += blockDim.x) {
    dD[t] = a.dX[(size_t)atom * a.fit_in + t];
    dDd[t] = a.dXd[(size_t)atom * a.fit_in + t];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 4 * m1; t += blockDim.x) {
    const int c = t / m1, p = t % m1;
    float v = 0.f, vd = 0.f;
    for (int b = 0; b < ax; ++b) {
      v = fmaf(dD[p * ax + b], Ts[c * m1 + b], v);
      vd += dDd[p * ax + b] * Ts[c * m1 + b] + dD[p * ax + b] * Tds[c * m1 + b];
    }
    if (p < ax)
      for (int q = 0; q < m1; ++q) {
        v = fmaf(dD[q * ax + p], Ts[c * m1 + q], v);
        vd += dDd[q * ax + p] * Ts[c * m1 + q] + dD[q * ax + p] * Tds[c * m1 + q];
      }
    dTs[t] = v * inv_sel;
    dTds[t] = vd * inv_sel;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < NP * m1; idx += blockDim.x) {
    const int s = idx / m1, p = idx % m1;
    float v = 0.f;
    if (s < nn) {
      const float* r = a.R + (base + s) * 4;
      const float* rd = a.Rd + (base + s) * 4;
      for (int c = 0; c < 4; ++c) v += rd[c] * dTs[c * m1 + p] + r[c] * dTds[c * m1 + p];
    }
    a.dGd[(base + s) * m1 + p] = v;
  }
}

__global__ void k_tanh_jvp(const float* __restrict__ Zd, const float* __restrict__ H, const float* __restrict__ Hprev,
                           const float* __restrict__ Hprevd, float* __restrict__ Hd, long long count) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const float t = Hprev ? H[k] - Hprev[k] : H[k];
  Hd[k] = (1.f - t * t) * Zd[k] + (Hprevd ? Hprevd[k] : 0.f);
}

__global__ void k_tanh_bwd_jvp(const float* __restrict__ dH, const float* __restrict__ dHd, const float* __restrict__ H,
                               const float* __restrict__ Hprev, const float* __restrict__ Hd,
                               const float* __restrict__ Hprevd, float* __restrict__ dZ, float* __restrict__ dZd,
                               long long count) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const float t = Hprev ? H[k] - Hprev[k] : H[k];
  const float td = Hprevd ? Hd[k] - Hprevd[k] : Hd[k];
  const float d = dH[k];
  dZ[k] = d * (1.f - t * t);
  dZd[k] = dHd[k] * (1.f - t * t) - 2.f * d * t * td;
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

__global__ void k_add_rows(const float* __restrict__ rows, const float* __restrict__ vec, int nrows, int width,
                           float* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nrows * width) out[t] = rows[t] + vec[t % width];
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
                       double pe, double pf, double* v, double* loss, float* scales, cudaStream_t st) {
  k_train_prep<<<1, 1024, 0, st>>>(n, energy, e_ref, force, force_ref, pe, pf, v, loss, scales);
  note_launch();
}

void launch_axpy(float* g, const float* src, int n, const float* scale, cudaStream_t st) {
  if (n <= 0) return;
  k_axpy<<<blocks(n, 256), 256, 0, st>>>(g, src, n, scale);
  note_launch();
}

void launch_env_jvp(const JvpArgs& a, cudaStream_t st) {
  const long long rows = (long long)a.n * NP;
  if (rows == 0) return;
  k_env_jvp<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a);
  note_launch();
}

template <int E0, int E1, int E2>
static void embed_jvp_launch(const JvpArgs& a, int mode, float* grad, const float* scale, cudaStream_t st) {
  using S = JvpEmbedSmem<E0, E1, E2>;
  const size_t smem = sizeof(float) * (mode == 1 ? S::TOTAL : S::FWD_TOTAL);
  cudaFuncSetAttribute(k_embed_jvp<E0, E1, E2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float) * S::TOTAL));
  const int nblk = a.n * (NP / JROWS);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = mode == 1 ? std::min(nblk, 2 * std::max(1, sms)) : nblk;
  k_embed_jvp<E0, E1, E2><<<grid, JTHREADS, smem, st>>>(a, mode, grad, scale);
  note_launch();
}

bool launch_embed_jvp(const JvpArgs& a, const int* w, int mode, float* grad, const float* scale, cudaStream_t st) {
  if (a.n == 0) return true;
  if (w[0] == 16 && w[1] == 32 && w[2] == 64) { embed_jvp_launch<16, 32, 64>(a, mode, grad, scale, st); return true; }
  if (w[0] == 25 && w[1] == 50 && w[2] == 100) { embed_jvp_launch<25, 50, 100>(a, mode, grad, scale, st); return true; }
  if (w[0] == 32 && w[1] == 64 && w[2] == 128) { embed_jvp_launch<32, 64, 128>(a, mode, grad, scale, st); return true; }
  return false;
}

void launch_desc_jvp_fwd(const JvpArgs& a, cudaStream_t st) {
  if (a.n == 0) return;
  k_desc_jvp_fwd<<<a.n, 128, sizeof(float) * 8 * a.m1, st>>>(a);
  note_launch();
}

void launch_desc_jvp_bwd(const JvpArgs& a, cudaStream_t st) {
  if (a.n == 0) return;
  const size_t smem = sizeof(float) * (16 * a.m1 + 2 * a.m1 * a.axis);
  k_desc_jvp_bwd<<<a.n, 128, smem, st>>>(a);
  note_launch();
}

void launch_tanh_jvp(const float* Zd, const float* H, const float* Hprev, const float* Hprevd, float* Hd,
                     long long count, cudaStream_t st) {
  if (count <= 0) return;
  k_tanh_jvp<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(Zd, H, Hprev, Hprevd, Hd, count);
  note_launch();
}

void launch_tanh_bwd_jvp(const float* dH, const float* dHd, const float* H, const float* Hprev, const float* Hd,
                         const float* Hprevd, float* dZ, float* dZd, long long count, cudaStream_t st) {
  if (count <= 0) return;
  k_tanh_bwd_jvp<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(dH, dHd, H, Hprev, Hd, Hprevd, dZ, dZd, count);
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

void launch_add_rows(const float* rows, const float* vec, int nrows, int width, float* out, cudaStream_t st) {
  if (nrows * width <= 0) return;
  k_add_rows<<<blocks((long long)nrows * width, 256), 256, 0, st>>>(rows, vec, nrows, width, out);
  note_launch();
}

}  // namespace dpa1
