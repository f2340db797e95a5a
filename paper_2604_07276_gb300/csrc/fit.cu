// Stages a8 / a10 on the tensor cores: the fitting-net products of the
// 16-bit paths, C = epi(A B + bias (+ R)) with A [M][K] FP32 activations
// (row-major) and B [K][N] FP32 weights, as tcgen05 kind::tf32 MMAs with
// two-term splits of both operands: A = A_hi + A_lo, B = B_hi + B_lo, where
// x_hi is x with its low 13 mantissa bits cleared (an exact TF32 value) and
// x_lo the TF32 truncation of x - x_hi.  A_hi B_hi + A_lo B_hi + A_hi B_lo
// misses A_lo B_lo and the truncation of the low parts, ~2^-20 relative:
// the products stay at FP32 accuracy.
//
// One CTA computes a 128-row x (<= 256)-column tile with the full K:
//   warp 0      : producer.  A tiles (128 rows x 32 K, FP32) by TMA with the
//                 128-byte swizzle, B_hi / B_lo tiles by 1D bulk copies of
//                 pre-swizzled images; two pipeline stages.
//   warps 4-7   : split each A tile in place (A_hi) and into its A_lo tile.
//   warp 1      : issues the MMAs (one thread), accumulator in TMEM.
//   warp 2      : allocates / frees TMEM.
//   all 8 warps : the epilogue (TMEM -> bias, tanh, residual -> global); warp
//                 w reads TMEM lane quadrant w % 4 and every other 16-column
//                 chunk, starting at chunk w / 4.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "dpa1.h"
#include "kernels.h"
#include "model.h"
#include "tc_ptx.cuh"

namespace dpa1 {

using namespace tc;

namespace {

constexpr int FBM = 128;            // rows per tile
constexpr int FBK = 32;             // K per stage (one 128-byte swizzle row of FP32)
constexpr int FNMAX = 256;          // output columns per tile
constexpr int FSTAGES = 2;
constexpr int FA_TILE = FBM * FBK * 4;  // 16 KB
constexpr int FTHREADS = 256;

struct FitGemmArgs {
  const uint8_t* bimg;  // B images: [n block][k block][hi, lo] tiles of bn_max rows x 128 bytes
  const float* bias;    // [N] or null
  const float* R;       // residual [M][ldr] or null
  float* C;             // [M][ldc]
  int ldr, ldc;
  int M, N, nkb;        // rows, output columns, K blocks of 32
  int bn_max;           // rows of one B image tile (multiple of 16, <= 256)
  int epi;
  int* err;
};

__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  // D = F32 (bit 4), A and B = TF32 (2 at bits 7 and 10), both K-major, N >> 3, M >> 4
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 2D tiled TMA load of box {32 K, 128 rows} at (x = k, y = row) into dst.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ uint32_t tf32_trunc(uint32_t bits) { return bits & 0xFFFFE000u; }

// Per-thread bounded wait that gives up for good after the first time-out.
struct Waiter {
  int* err;
  bool ok = true;
  __device__ void wait(uint64_t* bar, uint32_t parity) {
    if (ok) ok = mbar_wait(bar, parity, err);
  }
};

__global__ void __launch_bounds__(FTHREADS, 1)
k_fit_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ FitGemmArgs a) {
  extern __shared__ uint8_t fsm_raw[];
  const uint32_t raw = smem_u32(fsm_raw);
  uint8_t* sm = fsm_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned tiles
  const int bn = min(FNMAX, ((a.N - (int)blockIdx.y * FNMAX) + 15) & ~15);  // MMA width of this tile
  const int b_tile = a.bn_max * 128;
  const int stage_bytes = 2 * FA_TILE + 2 * b_tile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + FSTAGES * stage_bytes);
  uint64_t* full = bars;              // [FSTAGES]
  uint64_t* conv = bars + FSTAGES;    // [FSTAGES]
  uint64_t* empty = bars + 2 * FSTAGES;
  uint64_t* done = bars + 3 * FSTAGES;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(done + 1);
  auto sA = [&](int s) { return sm + s * stage_bytes; };
  auto sAl = [&](int s) { return sm + s * stage_bytes + FA_TILE; };
  auto sBh = [&](int s) { return sm + s * stage_bytes + 2 * FA_TILE; };
  auto sBl = [&](int s) { return sm + s * stage_bytes + 2 * FA_TILE + b_tile; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < FSTAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(conv + s, 128);
      mbar_init(empty + s, 1);
    }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 2) tmem_alloc(s_tmem, 256);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = *s_tmem;
  const int mb = blockIdx.x, nb = blockIdx.y;
  Waiter wt{a.err};

  if (warp == 0 && lane == 0) {
    // producer
    const uint8_t* img = a.bimg + (size_t)nb * a.nkb * 2 * b_tile;
    for (int kb = 0; kb < a.nkb && wt.ok; ++kb) {
      const int s = kb % FSTAGES, u = kb / FSTAGES;
      if (kb >= FSTAGES) wt.wait(empty + s, (u - 1) & 1);
      if (!wt.ok) break;
      mbar_expect_tx(full + s, FA_TILE + 2 * bn * 128);
      tma_load_2d(sA(s), &tmA, kb * FBK, mb * FBM, full + s);
      bulk_g2s(sBh(s), img + (size_t)(2 * kb) * b_tile, bn * 128, full + s);
      bulk_g2s(sBl(s), img + (size_t)(2 * kb + 1) * b_tile, bn * 128, full + s);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    const uint32_t id = idesc_tf32(FBM, bn);
    for (int kb = 0; kb < a.nkb && wt.ok; ++kb) {
      const int s = kb % FSTAGES, u = kb / FSTAGES;
      wt.wait(conv + s, u & 1);
      fence_after_sync();
      if (wt.ok) {
        const uint32_t ah = smem_u32(sA(s)), al = smem_u32(sAl(s));
        const uint32_t bh = smem_u32(sBh(s)), bl = smem_u32(sBl(s));
#pragma unroll
        for (int ks = 0; ks < FBK / 8; ++ks) {
          const uint64_t dah = kmajor_desc(ah, ks, FBM), dal = kmajor_desc(al, ks, FBM);
          const uint64_t dbh = kmajor_desc(bh, ks, bn), dbl = kmajor_desc(bl, ks, bn);
          mma_tf32(tm, dah, dbh, id, (kb > 0 || ks > 0) ? 1u : 0u);
          mma_tf32(tm, dal, dbh, id, 1u);
          mma_tf32(tm, dah, dbl, id, 1u);
        }
      }
      mma_commit(empty + s);
    }
    mma_commit(done);
  } else if (warp >= 4) {
    // split A in place; thread t takes 16-byte pieces t, t + 128, ... of the
    // tile, so that a warp touches 512 contiguous bytes (the swizzle only
    // permutes pieces within a row, and the split is element-wise)
    const int t = threadIdx.x - 128;
    for (int kb = 0; kb < a.nkb && wt.ok; ++kb) {
      const int s = kb % FSTAGES, u = kb / FSTAGES;
      wt.wait(full + s, u & 1);
      uint4* hi = reinterpret_cast<uint4*>(sA(s));
      uint4* lo = reinterpret_cast<uint4*>(sAl(s));
#pragma unroll
      for (int i = 0; i < FA_TILE / 16 / 128; ++i) {
        const int q = i * 128 + t;
        const uint4 x = hi[q];
        uint4 h, l;
        h.x = tf32_trunc(x.x); l.x = tf32_trunc(__float_as_uint(__uint_as_float(x.x) - __uint_as_float(h.x)));
        h.y = tf32_trunc(x.y); l.y = tf32_trunc(__float_as_uint(__uint_as_float(x.y) - __uint_as_float(h.y)));
        h.z = tf32_trunc(x.z); l.z = tf32_trunc(__float_as_uint(__uint_as_float(x.z) - __uint_as_float(h.z)));
        h.w = tf32_trunc(x.w); l.w = tf32_trunc(__float_as_uint(__uint_as_float(x.w) - __uint_as_float(h.w)));
        hi[q] = h;
        lo[q] = l;
      }
      fence_async_smem();
      mbar_arrive(conv + s);
    }
  }
  // epilogue, all warps
  __syncwarp();
  Waiter wd{a.err};
  wd.wait(done, 0);
  fence_after_sync();
  {
    const int r = (warp & 3) * 32 + lane;  // row in the tile = TMEM lane
    const long long m = (long long)mb * FBM + r;
    const uint32_t taddr = tm + ((uint32_t)((warp & 3) * 32) << 16);
    for (int c0 = (warp >> 2) * 16; c0 < bn; c0 += 32) {
      float v[16];
      tmem_ld16(taddr + c0, v);
      const int n0 = nb * FNMAX + c0;
      if (m >= a.M) continue;
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const int n = n0 + q;
        if (n >= a.N) break;  // N % 4 == 0
        float4 o = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
        float* op = &o.x;
        if (a.bias) {
#pragma unroll
          for (int t = 0; t < 4; ++t) op[t] += a.bias[n + t];
        }
        if (a.epi == EPI_TANH || a.epi == EPI_RES_TANH) {
#pragma unroll
          for (int t = 0; t < 4; ++t) op[t] = tanhf(op[t]);
        }
        if (a.epi == EPI_RES_TANH || a.epi == EPI_RES) {
          const float4 rr = *reinterpret_cast<const float4*>(a.R + m * a.ldr + n);
          o.x += rr.x; o.y += rr.y; o.z += rr.z; o.w += rr.w;
        }
        *reinterpret_cast<float4*>(a.C + m * a.ldc + n) = o;
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tm, 256);
}

// B image of one product: B [K][N] row-major FP32 -> per (n block, k block) a
// hi and a lo tile of bn_max rows (output columns) x 32 K in the K-major
// 128-byte-swizzled layout, zero outside B.
__global__ void k_fit_image(const float* __restrict__ B, int K, int N, int nkb, int bn_max, uint8_t* __restrict__ img) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nnb = (N + FNMAX - 1) / FNMAX;
  const long long total = (long long)nnb * nkb * bn_max * FBK;
  if (t >= total) return;
  const int k_local = (int)(t % FBK);
  const int n_local = (int)((t / FBK) % bn_max);
  const int kb = (int)((t / ((long long)FBK * bn_max)) % nkb);
  const int nb = (int)(t / ((long long)FBK * bn_max * nkb));
  const int k = kb * FBK + k_local, n = nb * FNMAX + n_local;
  const bool in = k < K && n < N && n_local < FNMAX;
  const uint32_t x = in ? __float_as_uint(B[(size_t)k * N + n]) : 0u;
  const uint32_t h = tf32_trunc(x);
  const uint32_t l = tf32_trunc(__float_as_uint(__uint_as_float(x) - __uint_as_float(h)));
  const size_t tile = (size_t)bn_max * 128;
  uint8_t* base = img + ((size_t)nb * nkb + kb) * 2 * tile;
  const uint32_t off = sw128_offset(n_local, 2 * k_local, bn_max);  // FP32 element k = 16-bit column 2k
  *reinterpret_cast<uint32_t*>(base + off) = h;
  *reinterpret_cast<uint32_t*>(base + tile + off) = l;
}

struct ImageShape {
  int K, N, nkb, nnb, bn_max;
  size_t bytes() const { return (size_t)nnb * nkb * 2 * bn_max * 128; }
};

ImageShape image_shape(int K, int N) {
  ImageShape s;
  s.K = K;
  s.N = N;
  s.nkb = (K + FBK - 1) / FBK;
  s.nnb = (N + FNMAX - 1) / FNMAX;
  s.bn_max = std::min(FNMAX, (N + 15) & ~15);
  return s;
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

int fit_smem(int bn_max) { return FSTAGES * (2 * FA_TILE + 2 * bn_max * 128) + 1024 + 128; }

}  // namespace

bool fit_tc_supported(const dp_model* m) {
  int fan = m->fit_in;
  if (fan % 4) return false;
  for (int l = 0; l < m->nfit; ++l) {
    if (m->fit[l] % 4) return false;
    fan = m->fit[l];
  }
  return true;
}

int fit_tc_init(dp_model* m, std::string& msg) {
  TcWeights& w = m->tcw;
  w.fitW_t.clear();
  w.fitWT_t.clear();
  if (!fit_tc_supported(m)) return DP_OK;  // the SIMT products serve other widths
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      msg = "cuTensorMapEncodeTiled is not available from the driver";
      return DP_ERR_CUDA;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  int fan = m->fit_in;
  for (int l = 0; l < m->nfit; ++l) {
    const int out = m->fit[l];
    for (int dir = 0; dir < 2; ++dir) {
      const ImageShape s = dir == 0 ? image_shape(fan, out) : image_shape(out, fan);
      void* d = nullptr;
      if (cudaMalloc(&d, s.bytes()) != cudaSuccess) {
        msg = "cudaMalloc of the fitting-net weight images failed";
        return DP_ERR_CUDA;
      }
      w.allocations.push_back(d);
      (dir == 0 ? w.fitW_t : w.fitWT_t).push_back(d);
      const int smem = fit_smem(s.bn_max);
      cudaFuncSetAttribute(k_fit_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, std::max(smem, fit_smem(FNMAX)));
    }
    fan = out;
  }
  fit_tc_refresh(m, nullptr);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    msg = "building the fitting-net weight images failed";
    return DP_ERR_CUDA;
  }
  return DP_OK;
}

void fit_tc_refresh(dp_model* m, cudaStream_t st) {
  const TcWeights& w = m->tcw;
  if (w.fitW_t.empty()) return;
  int fan = m->fit_in;
  for (int l = 0; l < m->nfit; ++l) {
    const int out = m->fit[l];
    for (int dir = 0; dir < 2; ++dir) {
      // forward: B = W_l [fan][out]; backward: B = W_l^T [out][fan]
      const ImageShape s = dir == 0 ? image_shape(fan, out) : image_shape(out, fan);
      const float* B = dir == 0 ? m->fitW[l] : m->fitWT[l];
      uint8_t* img = reinterpret_cast<uint8_t*>(dir == 0 ? w.fitW_t[l] : w.fitWT_t[l]);
      const long long total = (long long)s.nnb * s.nkb * s.bn_max * FBK;
      k_fit_image<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(B, s.K, s.N, s.nkb, s.bn_max, img);
      note_launch();
    }
    fan = out;
  }
}

int fit_gemm_tc(dp_model* m, int layer, bool backward, const float* A, int lda, const float* bias, const float* R,
                int ldr, float* C, int ldc, int M, int epi, cudaStream_t st) {
  if (M <= 0) return DP_OK;
  const int fan = layer == 0 ? m->fit_in : m->fit[layer - 1];
  const int out = m->fit[layer];
  const ImageShape s = backward ? image_shape(out, fan) : image_shape(fan, out);
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)s.K, (cuuint64_t)M};
  const cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(float)};
  const cuuint32_t box[2] = {FBK, FBM};
  const cuuint32_t estr[2] = {1, 1};
  if (g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return DP_ERR_CUDA;
  FitGemmArgs a;
  a.bimg = reinterpret_cast<const uint8_t*>(backward ? m->tcw.fitWT_t[layer] : m->tcw.fitW_t[layer]);
  a.bias = bias;
  a.R = R;
  a.C = C;
  a.ldr = ldr;
  a.ldc = ldc;
  a.M = M;
  a.N = s.N;
  a.nkb = s.nkb;
  a.bn_max = s.bn_max;
  a.epi = epi;
  a.err = m->d_err;
  dim3 grid((unsigned)((M + FBM - 1) / FBM), (unsigned)s.nnb);
  k_fit_gemm<<<grid, FTHREADS, fit_smem(s.bn_max), st>>>(map, a);
  note_launch();
  return DP_OK;
}

}  // namespace dpa1
