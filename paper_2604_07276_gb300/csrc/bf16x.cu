// The BF16-operand precision mode ("bf16x"): every matrix product of the
// attention layers (stages a6, a12) and of the fitting net (a8, a10) runs on
// tcgen05 with BF16 operands and FP32 accumulation in TMEM, with two-term
// splits of both operands, x = x_hi + x_lo (x_hi = bf16(x), x_lo =
// bf16(x - x_hi)), evaluated as the three products x_hi y_hi + x_lo y_hi +
// x_hi y_lo.  The dropped x_lo y_lo and the rounding of the low parts leave
// about 2^-16 relative error per product.  A CPU emulation of the layer's
// rounding points shows that BF16 operands meet force RMSE <= 5e-3 eV/A and
// atomic energies <= 1e-3 eV against FP64 only when every forward operand is
// split this way; in the adjoint the attention weights P and dS may stay
// single BF16 (force RMSE ~1e-3 eV/A on the model with perturbed biases).
//
// The layer is organised as in the FP32 path (stored projections, O through
// P G, LayerNorm kernels), for attention widths 128 and 256 (the cores take
// the features in halves of 128), with:
//   k_gemm_bf16x          the projections [Q K] = G [Wq Wk] + b (V only
//                         enters through [Wv Wo; bv Wo]),
//                         Y = [P G, rowsum P] [Wv Wo; bv Wo] + bo,
//                         dPG = dY [Wv Wo; bv Wo]^T, dG += [dQ dK] [Wq Wk]^T,
//                         and the fitting
//                         net's products (A by TMA as FP32, split in shared
//                         memory; B from pre-split images);
//   k_attn_core_fwd_bf16x per atom: S = Q K^T, smooth softmax and gate,
//                         [P G, rowsum P] (P G on the tensor cores, the row
//                         sums in FP32);
//   k_attn_core_bwd_bf16x per atom: dP = dPG [G 1]^T, S recomputed, the
//                         softmax adjoint (dE/drhat, dE/dw), dE/dG += P^T dPG,
//                         dQ = dS K, dK = dS^T Q, with dPG = dE/d[P G,
//                         rowsum P] from a GEMM of dY with [Wv Wo; bv Wo]^T.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "dpa1.h"
#include "kernels.h"
#include "model.h"
#include "tc_layer.cuh"
#include "tc_ptx.cuh"

namespace dpa1 {

using namespace tc;

namespace {

// ------------------------------------------------------------------- GEMM
// C = epi(A B + bias (+ R)), A [M][K] FP32 row-major, B [K][N] from a
// pre-split image.  Persistent: CTA (x, y) keeps N block y (<= 144 columns)
// and walks the 128-row tiles x, x + gridDim.x, ...; the K loop runs in
// stages of 64 through a two-stage ring that continues across tiles, and
// the accumulator alternates between two TMEM buffers, so that the epilogue
// of one tile overlaps the loads and products of the next.
//   warp 0      : producer.  Two TMA boxes of A (128 rows x 32 K FP32,
//                 128-byte swizzle) and the B hi / lo tiles (bulk copies).
//   warps 4-7   : split the stage's FP32 A into its BF16 hi and lo tiles
//                 (K-major, 128-byte swizzle); thread t owns row t.
//   warp 1      : issues the MMAs (one thread).
//   warp 2      : allocates / frees TMEM.
//   warps 8-11  : epilogue (TMEM lane quadrant w - 8 -> bias, tanh,
//                 residual / accumulate -> global).  A warp takes its 32
//                 rows 32 columns at a time through a shared staging block,
//                 so that each global access covers 4 rows x 128 bytes.
constexpr int XBM = 128, XBK = 64, XBN = 144, XSTAGES = 2, XTHREADS = 384;
constexpr int XF32 = 2 * XBM * 32 * 4;  // FP32 staging of one stage: two TMA boxes (32 KB)
constexpr int XAT = XBM * XBK * 2;      // one BF16 A tile (hi or lo): 16 KB
constexpr int XSLD = 36;                // row stride (floats) of an epilogue warp's 32 x 32 staging block
constexpr int XSTG = 32 * XSLD * 4;     // bytes of one staging block

struct XGemmArgs {
  const uint8_t* bimg;  // [n block][k block][hi, lo] tiles of bn_max rows x 64 K (BF16, K-major, SW128)
  const float* bias;    // [N] or null
  const float* R;       // residual [M][ldr] or null
  float* C;             // [M][ldc]
  int ldr, ldc;
  int M, N, nkb, bn_max, epi, mtiles;
  int* err;
};

__device__ __forceinline__ void x_tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// 8 FP32 values -> their BF16 high parts and the BF16 rounding of the residues.
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat16 a = __float2bfloat16_rn(v[2 * i]), b = __float2bfloat16_rn(v[2 * i + 1]);
    h[i] = pack_bf16(__bfloat162float(a), __bfloat162float(b));
    l[i] = pack_bf16(v[2 * i] - __bfloat162float(a), v[2 * i + 1] - __bfloat162float(b));
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

__global__ void __launch_bounds__(XTHREADS, 1)
k_gemm_bf16x(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ XGemmArgs a) {
  extern __shared__ uint8_t xsm_raw[];
  const uint32_t raw = smem_u32(xsm_raw);
  uint8_t* sm = xsm_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned tiles
  const int nb = blockIdx.y;
  const int bn = min(XBN, ((a.N - nb * XBN) + 15) & ~15);  // MMA width of this N block
  const int b_tile = a.bn_max * 128;
  const int stage_bytes = XF32 + 2 * XAT + 2 * b_tile;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + XSTAGES * stage_bytes);
  uint64_t* full = bars;                 // [XSTAGES] A boxes and B tiles arrived
  uint64_t* conv = bars + XSTAGES;       // [XSTAGES] A split into hi / lo (128 arrivals)
  uint64_t* empty = bars + 2 * XSTAGES;  // [XSTAGES] the stage's MMAs are done
  uint64_t* tfull = bars + 3 * XSTAGES;  // [2] accumulator buffer complete
  uint64_t* tempty = tfull + 2;          // [2] accumulator buffer read out (4 warp arrivals)
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(tempty + 2);
  // [XBN + 32] this N block's bias (0 without one, and past the block: the
  // epilogue's last 32-column chunk may reach past it)
  float* s_bias = reinterpret_cast<float*>(bars + 16);
  float* s_stg = s_bias + XBN + 32;  // [4][32][XSLD] epilogue staging
  auto sF = [&](int s) { return sm + s * stage_bytes; };
  auto sAh = [&](int s) { return sm + s * stage_bytes + XF32; };
  auto sAl = [&](int s) { return sm + s * stage_bytes + XF32 + XAT; };
  auto sBh = [&](int s) { return sm + s * stage_bytes + XF32 + 2 * XAT; };
  auto sBl = [&](int s) { return sm + s * stage_bytes + XF32 + 2 * XAT + b_tile; };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < XSTAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(conv + s, 128);
      mbar_init(empty + s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull + b, 1);
      mbar_init(tempty + b, 4);
    }
    fence_mbar_init();
  }
  if (warp == 2) tmem_alloc(s_tmem, 512);
  for (int c = threadIdx.x; c < XBN + 32; c += blockDim.x) {
    const int n = nb * XBN + c;
    s_bias[c] = (a.bias && c < bn && n < a.N) ? a.bias[n] : 0.f;
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tm = *s_tmem;
  bool ok = true;
  auto wait = [&](uint64_t* bar, uint32_t parity) {
    if (ok) ok = mbar_wait(bar, parity, a.err);
  };
  const int ntile = a.mtiles > (int)blockIdx.x ? (a.mtiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 0 && lane == 0) {
    const uint8_t* img = a.bimg + (size_t)nb * a.nkb * 2 * b_tile;
    for (int it = 0; it < ntile && ok; ++it) {
      const int mb = blockIdx.x + it * gridDim.x;
      for (int kb = 0; kb < a.nkb && ok; ++kb) {
        const int g = it * a.nkb + kb, s = g % XSTAGES, u = g / XSTAGES;
        if (g >= XSTAGES) wait(empty + s, (u - 1) & 1);
        if (!ok) break;
        mbar_expect_tx(full + s, XF32 + 2 * bn * 128);
        x_tma_load_2d(sF(s), &tmA, kb * XBK, mb * XBM, full + s);
        x_tma_load_2d(sF(s) + XF32 / 2, &tmA, kb * XBK + 32, mb * XBM, full + s);
        bulk_g2s(sBh(s), img + (size_t)(2 * kb) * b_tile, bn * 128, full + s);
        bulk_g2s(sBl(s), img + (size_t)(2 * kb + 1) * b_tile, bn * 128, full + s);
      }
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t id = idesc_16(XBM, bn, false, false, false);
    for (int it = 0; it < ntile && ok; ++it) {
      const int b = it & 1;
      const uint32_t acc = tm + (uint32_t)(b * 256);
      if (it >= 2) wait(tempty + b, ((it >> 1) - 1) & 1);
      fence_after_sync();
      for (int kb = 0; kb < a.nkb && ok; ++kb) {
        const int g = it * a.nkb + kb, s = g % XSTAGES, u = g / XSTAGES;
        wait(conv + s, u & 1);
        fence_after_sync();
        if (ok) {
          const uint32_t ah = smem_u32(sAh(s)), al = smem_u32(sAl(s));
          const uint32_t bh = smem_u32(sBh(s)), bl = smem_u32(sBl(s));
#pragma unroll
          for (int ks = 0; ks < XBK / 16; ++ks) {
            const uint64_t dah = kmajor_desc(ah, ks, XBM), dal = kmajor_desc(al, ks, XBM);
            const uint64_t dbh = kmajor_desc(bh, ks, bn), dbl = kmajor_desc(bl, ks, bn);
            mma_bf16(acc, dah, dbh, id, (kb > 0 || ks > 0) ? 1u : 0u);
            mma_bf16(acc, dal, dbh, id, 1u);
            mma_bf16(acc, dah, dbl, id, 1u);
          }
        }
        mma_commit(empty + s);
      }
      mma_commit(tfull + b);
    }
  } else if (warp >= 4 && warp < 8) {
    // row r of the stage: FP32 K 0..31 in box 0, 32..63 in box 1, each row a
    // 128-byte line whose 16-byte pieces are permuted by XOR with r % 8; its
    // BF16 row is one 128-byte line with the same permutation
    const int r = threadIdx.x - 128;
    const uint32_t line = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128);
    for (int g = 0; g < ntile * a.nkb && ok; ++g) {
      const int s = g % XSTAGES, u = g / XSTAGES;
      wait(full + s, u & 1);
      const uint8_t* f = sF(s);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint8_t* box = f + (q >> 2) * (XF32 / 2) + line;
        const int p0 = 2 * (q & 3);
        const float4 x0 = *reinterpret_cast<const float4*>(box + ((p0 ^ (r & 7)) << 4));
        const float4 x1 = *reinterpret_cast<const float4*>(box + (((p0 + 1) ^ (r & 7)) << 4));
        const float v[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        uint4 hi, lo;
        split8(v, hi, lo);
        const uint32_t off = line + ((q ^ (r & 7)) << 4);
        *reinterpret_cast<uint4*>(sAh(s) + off) = hi;
        *reinterpret_cast<uint4*>(sAl(s) + off) = lo;
      }
      fence_async_smem();
      mbar_arrive(conv + s);
    }
  } else if (warp >= 8) {
    const int quad = warp - 8;
    float* stg = s_stg + quad * 32 * XSLD;
    for (int it = 0; it < ntile && ok; ++it) {
      const int b = it & 1;
      wait(tfull + b, (it >> 1) & 1);
      fence_after_sync();
      const long long m0 = (long long)(blockIdx.x + it * gridDim.x) * XBM + quad * 32;  // this warp's first row
      const uint32_t taddr = tm + (uint32_t)(b * 256) + ((uint32_t)(quad * 32) << 16);
      for (int c0 = 0; c0 < bn; c0 += 32) {
        float v[32];
        tmem_ld32(taddr + c0, v);
        // lane = row: bias and tanh, then the row into the staging block
#pragma unroll
        for (int q = 0; q < 32; q += 4) {
          const float4 bb = *reinterpret_cast<const float4*>(s_bias + c0 + q);
          float4 o = make_float4(v[q] + bb.x, v[q + 1] + bb.y, v[q + 2] + bb.z, v[q + 3] + bb.w);
          if (a.epi == EPI_TANH || a.epi == EPI_RES_TANH) {
            o.x = tanhf(o.x); o.y = tanhf(o.y); o.z = tanhf(o.z); o.w = tanhf(o.w);
          }
          *reinterpret_cast<float4*>(stg + lane * XSLD + q) = o;
        }
        __syncwarp();
        // 8 lanes per row, 4 rows per access: residual / accumulate, store
        const int q = 4 * (lane & 7);
        const int nl = c0 + q;  // column within the N block
        const int n = nb * XBN + nl;
        if (ok && nl < bn && n < a.N) {  // N % 4 == 0
          // four rows at a time: the residual / accumulator loads, then the stores
          const bool res = a.epi == EPI_RES_TANH || a.epi == EPI_RES, acc = a.epi == EPI_ACCUM;
#pragma unroll
          for (int k0 = 0; k0 < 8; k0 += 4) {
            float4 o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int rr = 4 * (k0 + k) + (lane >> 3);
              const long long m = m0 + rr;
              o[k] = *reinterpret_cast<const float4*>(stg + rr * XSLD + q);
              if (m < a.M && (res || acc)) {
                const float4 e = res ? *reinterpret_cast<const float4*>(a.R + m * a.ldr + n)
                                     : *reinterpret_cast<const float4*>(a.C + m * a.ldc + n);
                o[k].x += e.x; o[k].y += e.y; o[k].z += e.z; o[k].w += e.w;
              }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const long long m = m0 + 4 * (k0 + k) + (lane >> 3);
              if (m < a.M) *reinterpret_cast<float4*>(a.C + m * a.ldc + n) = o[k];
            }
          }
        }
        __syncwarp();
      }
      // the buffer is read: the MMAs of tile it + 2 may overwrite it
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty + b);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tm, 512);
}

// B image of one product, built on the device from B [K][N] (FP32,
// row-major): per (n block, k block) a hi and a lo tile of bn_max rows
// (output columns) x 64 K, BF16, K-major with the 128-byte swizzle, zero
// outside B.
__global__ void k_x_image(const float* __restrict__ B, int ldb, int K, int N, int nkb, int bn_max,
                          uint8_t* __restrict__ img) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int nnb = (N + XBN - 1) / XBN;
  const long long total = (long long)nnb * nkb * bn_max * XBK;
  if (t >= total) return;
  const int k_local = (int)(t % XBK);
  const int n_local = (int)((t / XBK) % bn_max);
  const int kb = (int)((t / ((long long)XBK * bn_max)) % nkb);
  const int nb = (int)(t / ((long long)XBK * bn_max * nkb));
  const int k = kb * XBK + k_local, n = nb * XBN + n_local;
  const float x = (k < K && n < N && n_local < XBN) ? B[(size_t)k * ldb + n] : 0.f;
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  const size_t tile = (size_t)bn_max * 128;
  uint8_t* base = img + ((size_t)nb * nkb + kb) * 2 * tile;
  const uint32_t off = sw128_offset(n_local, k_local, bn_max);
  *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(base + tile + off) = l;
}

PFN_cuTensorMapEncodeTiled_v12000 g_x_encode = nullptr;

// the stages, 1024 bytes of alignment slack, the barriers (128 bytes), the
// bias (XBN + 32 floats) and the epilogue staging (4 blocks)
int x_smem(int bn_max) {
  return XSTAGES * (XF32 + 2 * XAT + 2 * bn_max * 128) + 1024 + 128 + (XBN + 32) * 4 + 4 * XSTG;
}

int x_sm_count(int dev) {
  int c = 0;
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

// ------------------------------------------------------ attention cores
// One persistent CTA of 512 threads per SM walks over centre atoms; warp w
// owns TMEM lane quadrant w % 4 (rows 32 (w % 4) .. +31) and column quarter
// w / 4 (32 columns), as in the fused layer kernels.  Tiles are 128 x 128
// BF16 with the 128-byte swizzle (32 KB).
constexpr int XC_NT = 512;
constexpr int XT = 32768;

struct XCoreArgs {
  const float* QK;   // [rows][ldq]: Q | K (attention width each)
  const float* G;    // [rows][m1] layer input
  float* PG;         // fwd: [rows][ldpg] = [P G, rowsum(P), 0 ...]
  const float* dPG;  // bwd: [rows][ldpg] dE/d[P G, rowsum P]
  float* dQK;        // bwd: [rows][ldq] dQ | dK
  float* dG;         // bwd: [rows][m1] += P^T dE/d(P G) (the path through the values)
  float* dgeo;       // bwd: [rows][4] += (d rhat, d w)
  const float* rw;   // [rows][4] (rhat, w)
  const int* nnei;
  int n, m1, ldpg, npg, ldq;  // npg: MMA width of P G (m1 rounded up to 16)
  float scale, shift;
  int* err;
};

__device__ __forceinline__ void store_split32(uint8_t* hi, uint8_t* lo, int r, int c0, const float* v) {
  store_row32<false>(hi, r, c0, v);
  store_row32<false, true>(lo, r, c0, v);
}

// Coalesced block access of the cores: in access t (0..7) warp w (of 16)
// takes row w + 16 t and lane l columns 4 l .. 4 l + 3 of a 128-column
// block, so that each warp access is one row's 512 contiguous bytes.
static_assert(XC_NT == 512, "block accesses: 16 warps x 8 accesses cover the 128 rows");
__device__ __forceinline__ int blk_row(int t) { return (int)(threadIdx.x >> 5) + 16 * t; }

// v[4 t .. 4 t + 3] = src[r][c .. c + 3] (r = blk_row(t), c = 4 lane), zero
// for rows at or past nrows and columns at or past ncols (ncols % 4 == 0).
__device__ __forceinline__ void load_blk(const float* src, size_t ld, int nrows, int ncols, float* v) {
  const int c = 4 * (threadIdx.x & 31);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int r = blk_row(t);
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < nrows && c < ncols) x = *reinterpret_cast<const float4*>(src + (size_t)r * ld + c);
    v[4 * t] = x.x; v[4 * t + 1] = x.y; v[4 * t + 2] = x.z; v[4 * t + 3] = x.w;
  }
}

// The BF16 high parts (LO = false) or the BF16 roundings of the residues of a
// block loaded by load_blk, into a 128 x 128 SW128 tile.
template <bool LO>
__device__ __forceinline__ void store_blk(uint8_t* tile, const float* v) {
  const int c = 4 * (threadIdx.x & 31);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    float x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = LO ? v[4 * t + i] - round16<false>(v[4 * t + i]) : v[4 * t + i];
    *reinterpret_cast<uint2*>(tile + sw128_offset(blk_row(t), c, 128)) =
        make_uint2(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]));
  }
}

__device__ __forceinline__ void store_blk_split(uint8_t* hi, uint8_t* lo, const float* v) {
  store_blk<false>(hi, v);
  store_blk<true>(lo, v);
}

// FP32 staging of a 128 x 128 block in shared memory (64 KB): float4 q of
// row r at r * 128 + 4 (q ^ (r % 8)), free of bank conflicts both for a warp
// writing one float4 column of 32 rows and for a warp reading one row.
__device__ __forceinline__ float4* stg4(float* s, int r, int q) {
  return reinterpret_cast<float4*>(s + r * 128 + 4 * (q ^ (r & 7)));
}

// TMEM columns [taddr, taddr + 32) of this thread's lane (row) -> the staging
// block, columns c0 .. c0 + 31.
__device__ __forceinline__ void tmem_to_stg(uint32_t taddr, float* s, int row, int c0) {
  float v[32];
  tmem_ld32(taddr, v);
#pragma unroll
  for (int q = 0; q < 8; ++q) *stg4(s, row, (c0 >> 2) + q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
}

// Rows [0, nrows), columns [0, ncols) of a staged block -> dst (row stride
// ld), one row per warp access; ACC: dst += (a thread's loads are issued four
// rows at a time before their stores).  ncols % 4 == 0, ncols <= 128.
template <bool ACC>
__device__ __forceinline__ void stg_to_global(float* s, float* dst, size_t ld, int nrows, int ncols) {
  const int q = threadIdx.x & 31;
  if (4 * q >= ncols) return;
#pragma unroll
  for (int t0 = 0; t0 < 8; t0 += 4) {
    float4 x[4], y[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int r = blk_row(t0 + t);
      if (r < nrows) {
        x[t] = *stg4(s, r, q);
        if (ACC) y[t] = *reinterpret_cast<const float4*>(dst + (size_t)r * ld + 4 * q);
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int r = blk_row(t0 + t);
      if (r < nrows) {
        if (ACC) { x[t].x += y[t].x; x[t].y += y[t].y; x[t].z += y[t].z; x[t].w += y[t].w; }
        *reinterpret_cast<float4*>(dst + (size_t)r * ld + 4 * q) = x[t];
      }
    }
  }
}

constexpr int XF_SMEM = 6 * XT + 2048 + 64;

// NH feature halves of 128 (attention width 128 NH).  Tiles: Q hi / lo of
// one half (then P hi / lo), K hi / lo of one half, G hi / lo.  S is summed
// over the halves in TMEM [0, 128); P G goes to TMEM [128, 128 + npg); the
// row sums of P are taken in FP32 by the threads.
template <int NH>
__global__ void __launch_bounds__(XC_NT, 1) k_attn_core_fwd_bf16x(const __grid_constant__ XCoreArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {  // tiles need 1024-byte alignment
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint8_t* sQh = sm;
  uint8_t* sQl = sm + XT;
  uint8_t* sKh = sm + 2 * XT;
  uint8_t* sKl = sm + 3 * XT;
  uint8_t* sGh = sm + 4 * XT;
  uint8_t* sGl = sm + 5 * XT;
  float4* s_key = reinterpret_cast<float4*>(sm + 6 * XT);  // [128] (rhat, w)
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_key + 128);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2;
  const int row = quad * 32 + lane, c0 = part * 32;
  const bool issuer = tid == XC_NT - 32;
  if (issuer) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(s_tmem, 256);
  handoff();
  const uint32_t tm = *s_tmem;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  const uint32_t tQh = smem_u32(sQh), tQl = smem_u32(sQl), tKh = smem_u32(sKh), tKl = smem_u32(sKl);
  const uint32_t tGh = smem_u32(sGh), tGl = smem_u32(sGl);
  Sync sy{bar, 0u, a.err};
  const int ld = a.ldq;  // Q | K, 128 NH columns each
  for (int atom = blockIdx.x; atom < a.n && sy.ok; atom += gridDim.x) {
    const int nn = a.nnei[atom];
    const size_t base = (size_t)atom * NP;
    const bool rv = row < nn;
    // the next atom's Q and K rows and its layer input into L2
    if (atom + (int)gridDim.x < a.n) {
      const size_t nb = (size_t)(atom + gridDim.x) * NP;
      if (tid < NP) prefetch_l2(a.QK + (nb + tid) * ld, (uint32_t)(2 * NH * 128 * sizeof(float)));
      if (issuer) prefetch_l2(a.G + nb * a.m1, (uint32_t)(NP * a.m1 * sizeof(float)));
    }
    float v[32];
    // two blocks in flight: each block's loads are issued before the
    // previous block is split into its tiles
    float w[32];
    load_blk(a.G + base * a.m1, a.m1, nn, a.m1, v);
    load_blk(a.QK + base * ld, ld, nn, 128, w);  // Q, first half
    store_blk_split(sGh, sGl, v);
    if (tid < 128) s_key[tid] = tid < nn ? reinterpret_cast<const float4*>(a.rw)[base + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    // S = sum over the halves of Q_h K_h^T (three split products each) -> TMEM [0, 128)
#pragma unroll 1
    for (int h = 0; h < NH; ++h) {
      if (h > 0) load_blk(a.QK + base * ld + h * 128, ld, nn, 128, w);
      load_blk(a.QK + base * ld + NH * 128 + h * 128, ld, nn, 128, v);
      store_blk_split(sQh, sQl, w);
      store_blk_split(sKh, sKl, v);
      handoff();
      if (issuer) {
        mma_block<false>(tm, tQh, false, 128, tKh, false, 128, 128, 8, h > 0);
        mma_block<false>(tm, tQl, false, 128, tKh, false, 128, 128, 8, true);
        mma_block<false>(tm, tQh, false, 128, tKl, false, 128, 128, 8, true);
      }
      commit_and_sync(sy, issuer);
    }
    // smooth softmax and gate: P_jk = A_jk w_j w_k (rhat_j . rhat_k) -> Q's tiles
    tmem_ld32(tm + lane_off + c0, v);
    float psum;
    {
      const RowXchg xr(sQh, row, part, lane, quad);  // P hi is stored after the exchanges
      const float4 kj = s_key[row];
      const float wj = kj.w;
      const bool live = c0 < nn;
      float mx = -INFINITY;
      if (live) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int k = c0 + i;
          const float l = (k < nn && rv) ? (v[i] * a.scale + a.shift) * (wj * s_key[k].w) : -INFINITY;
          v[i] = l;
          mx = fmaxf(mx, l);
        }
      }
      mx = xr.max(mx);
      const float mxs = mx == -INFINITY ? 0.f : mx;  // a row without neighbours: every term -inf
      float sum = 0.f;
      if (live) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float e = exp_sfu(v[i] - mxs);
          v[i] = e;
          sum += e;
        }
      }
      sum = xr.sum(sum);
      const float inv = sum > 0.f ? 1.0f / sum : 0.f;
      psum = 0.f;
      if (live) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float4 kk = s_key[c0 + i];
          const float c = kj.x * kk.x + kj.y * kk.y + kj.z * kk.z;
          v[i] = v[i] * inv * (wj * kk.w) * c;
          psum += v[i];
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      psum = xr.sum(psum);
      store_split32(sQh, sQl, row, c0, v);
    }
    handoff();
    // P G = P G ([G] as an MN-major operand) -> TMEM [128, 128 + npg)
    if (issuer) {
      mma_block<false>(tm + 128, tQh, false, 128, tGh, true, 128, a.npg, 8, false);
      mma_block<false>(tm + 128, tQl, false, 128, tGh, true, 128, a.npg, 8, true);
      mma_block<false>(tm + 128, tQh, false, 128, tGl, true, 128, a.npg, 8, true);
    }
    commit_and_sync(sy, issuer);
    // [P G, rowsum P, 0 ...] (ldpg columns) -> staging over the dead Q tiles
    // (the first 128 columns) -> PG, a row per warp access
    float* stg = reinterpret_cast<float*>(sm);
    {
      if (c0 < a.m1) tmem_ld32(tm + lane_off + 128 + c0, v);  // warp-uniform
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = c0 + 4 * q + i;
          o[i] = c < a.m1 ? v[4 * q + i] : (c == a.m1 ? psum : 0.f);
        }
        *stg4(stg, row, (c0 >> 2) + q) = make_float4(o[0], o[1], o[2], o[3]);
      }
      if (part == 0 && row < nn) {  // columns past 128 (m1 = 128: the row sum and padding)
        float4* out = reinterpret_cast<float4*>(a.PG + (base + row) * a.ldpg);
        for (int c = 128; c < a.ldpg; c += 4) out[c >> 2] = make_float4(c == a.m1 ? psum : 0.f, 0.f, 0.f, 0.f);
      }
    }
    __syncthreads();
    // live rows only: every later reader of P G works row by row, and the
    // cores read no row past the last neighbour.  (The adjoint core's dE/dQ,
    // dE/dK stores stay whole-block: restricted to the live rows they made
    // the width-256 core 16 % slower.)
    stg_to_global<false>(stg, a.PG + base * a.ldpg, a.ldpg, nn, a.ldpg < 128 ? a.ldpg : 128);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// The softmax adjoint over this thread's 32 keys of its row, S and dP
// re-read from TMEM in pieces of 8: A is recomputed with its row max and
// normaliser; tsum = sum_k A_jk dA_jk with dA = dP w_j w_k c_jk; then per key
// dLp = A (dA - tsum), dS = dLp w_j w_k scale -> TMEM over S, P -> the tile
// pt, dE/d(w_j w_k) = dP A c + dLp (l + shift), dE/dc = dP A w_j w_k.  dP
// includes dpg1, the adjoint of the row sum of P (the same for every key).
// The row part (this thread's row) and column parts (lanes 0-15: key c0 + h
// + lane) of dE/drhat and dE/dw are returned.  pt's row lines also carry the
// row exchanges, before P is stored.
__device__ __forceinline__ void softmax_adjoint(const XCoreArgs& a, uint8_t* pt, const float4* s_key, uint32_t tS,
                                                uint32_t tP, int row, int part, int lane, int quad, int nn, float dpg1,
                                                float4& rpart, float4* cpart) {
  const int c0 = part * 32;
  const bool rv = row < nn;
  const RowXchg xr(pt, row, part, lane, quad);
  const float4 kj = s_key[row];
  const float wj = kj.w;
  // the TMEM loads are warp-collective: their condition is uniform over the
  // warp (c0), the row mask (rv) is applied per lane
  const bool wlive = c0 < nn;
  const bool live = wlive && rv;
  float mx = -INFINITY;
  if (wlive) {
#pragma unroll
    for (int e8 = 0; e8 < 32; e8 += 8) {
      float t[8];
      tmem_ld8(tS + e8, t);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = c0 + e8 + i;
        if (k < nn && rv) mx = fmaxf(mx, (t[i] * a.scale + a.shift) * (wj * s_key[k].w));
      }
    }
  }
  mx = xr.max(mx);
  const float mxs = mx == -INFINITY ? 0.f : mx;
  float sum = 0.f, esum = 0.f;  // sum_k e_k and sum_k e_k dA_k
  if (wlive) {
#pragma unroll
    for (int e8 = 0; e8 < 32; e8 += 8) {
      float t[8], u[8];
      tmem_ld8(tS + e8, t);
      tmem_ld8(tP + e8, u);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = c0 + e8 + i;
        if (k < nn && rv) {
          const float4 kk = s_key[k];
          const float ww = wj * kk.w;
          const float e = exp_sfu((t[i] * a.scale + a.shift) * ww - mxs);
          sum += e;
          esum += e * (u[i] + dpg1) * ww * (kj.x * kk.x + kj.y * kk.y + kj.z * kk.z);
        }
      }
    }
  }
  const float2 ss = xr.sum2(make_float2(sum, esum));
  const float inv = ss.x > 0.f ? 1.0f / ss.x : 0.f;
  const float tsum = ss.y * inv;
  float rw_ = 0.f, rx = 0.f, ry = 0.f, rz = 0.f;
#pragma unroll 1
  for (int h = 0; h < 32; h += 16) {
    float4 cph = make_float4(0.f, 0.f, 0.f, 0.f);
    float cw[16], dcv[16];
#pragma unroll
    for (int e8 = 0; e8 < 16; e8 += 8) {
      float t[8], u[8], pv[8];
      tmem_ld8(tS + h + e8, t);
      tmem_ld8(tP + h + e8, u);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = c0 + h + e8 + i;
        const float4 kk = s_key[k];
        const float ww = wj * kk.w;
        const float c = kj.x * kk.x + kj.y * kk.y + kj.z * kk.z;
        const float lg = t[i] * a.scale + a.shift;
        const float A = (live && k < nn) ? exp_sfu(lg * ww - mxs) * inv : 0.f;
        const float dp = u[i] + dpg1;
        const float dA = dp * ww * c;
        const float dLp = A * (dA - tsum);
        const float H = fmaf(dLp, lg, dp * A * c);  // dE/d(w_j w_k)
        const float dc = dp * A * ww;               // dE/dc_jk
        rw_ += H * kk.w;
        rx += dc * kk.x; ry += dc * kk.y; rz += dc * kk.z;
        cw[e8 + i] = H * wj;
        dcv[e8 + i] = dc;
        pv[i] = A * ww * c;
        t[i] = dLp * ww * a.scale;  // dS
      }
      uint4 w4;
      w4.x = pack_bf16(pv[0], pv[1]);
      w4.y = pack_bf16(pv[2], pv[3]);
      w4.z = pack_bf16(pv[4], pv[5]);
      w4.w = pack_bf16(pv[6], pv[7]);
      sw128_store8(pt, row, c0 + h + e8, 128, w4);
      tmem_st8_async(tS + h + e8, t);
    }
    cph.w = warp_reduce_scatter16(cw);
    float tmp[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) tmp[i] = dcv[i] * kj.x;
    cph.x = warp_reduce_scatter16(tmp);
#pragma unroll
    for (int i = 0; i < 16; ++i) tmp[i] = dcv[i] * kj.y;
    cph.y = warp_reduce_scatter16(tmp);
#pragma unroll
    for (int i = 0; i < 16; ++i) tmp[i] = dcv[i] * kj.z;
    cph.z = warp_reduce_scatter16(tmp);
    cpart[h >> 4] = cph;
  }
  rpart = make_float4(rx, ry, rz, rw_);
  tmem_wait_st();
}

// Adjoint core, in the form of the forward (Y = [P G, rowsum P] [Wv Wo; bv Wo]
// + bo): with dPG = dE/d[P G, rowsum P] (a GEMM of dY with [Wv Wo; bv Wo]^T),
// dP_jk = (dPG G^T)_jk + dPG_j,m1 and dE/dG += P^T dPG (columns below m1), so
// the values V and their adjoint never appear.  NH feature halves of 128.
// Tiles T0 .. T6:
//   NH = 1: T0 / T1 dPG hi / lo, T2 G hi then Q lo, T3 G lo then P then dS,
//           T4 Q hi, T5 / T6 K hi / lo.
//   NH = 2: T0 / T1 dPG hi / lo (then K0, then Q0 hi / lo), T2 G hi then Q0 lo
//           then P then dS, T3 G lo then Q1 hi, T4 Q0 hi then K1 hi, T5 K0 hi
//           then Q1 lo, T6 K0 lo then K1 lo; the first half's K and Q come in
//           again (from L2) for dQ and dK.
// TMEM: [0, 128) S, then dS, then dQ (first half); [128, 256) dP, then dQ of
// the second half; [256, 256 + npg) P^T dPG, then dK of the first half (NH =
// 2); [384, 512) dK (of the last half).
constexpr int XB_SMEM = 7 * XT + 2048 + 64;

template <int NH>
__global__ void __launch_bounds__(XC_NT, 1) k_attn_core_bwd_bf16x(const __grid_constant__ XCoreArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint8_t* T[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) T[i] = sm + i * XT;
  float4* s_key = reinterpret_cast<float4*>(sm + 7 * XT);  // [128] (rhat, w)
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_key + 128);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2;
  const int row = quad * 32 + lane, c0 = part * 32;
  const bool issuer = tid == XC_NT - 32;
  if (issuer) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(s_tmem, 512);
  handoff();
  const uint32_t tm = *s_tmem;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  uint32_t t[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) t[i] = smem_u32(T[i]);
  const int kg = a.npg / 16;  // K-steps of dPG G^T
  Sync sy{bar, 0u, a.err};
  const int ld = a.ldq;        // Q | K, 128 NH columns each; dQ | dK likewise
  constexpr int AW = NH * 128;  // attention width
  for (int atom = blockIdx.x; atom < a.n && sy.ok; atom += gridDim.x) {
    const int nn = a.nnei[atom];
    const size_t base = (size_t)atom * NP;
    const bool rv = row < nn;
    const float* qk0 = a.QK + base * ld;  // this atom's Q | K block
    // the next atom's Q and K rows, dPG and layer input into L2
    if (atom + (int)gridDim.x < a.n) {
      const size_t nb = (size_t)(atom + gridDim.x) * NP;
      if (tid < NP) prefetch_l2(a.QK + (nb + tid) * ld, (uint32_t)(2 * AW * sizeof(float)));
      if (issuer) {
        prefetch_l2(a.dPG + nb * a.ldpg, (uint32_t)(NP * a.ldpg * sizeof(float)));
        prefetch_l2(a.G + nb * a.m1, (uint32_t)(NP * a.m1 * sizeof(float)));
      }
    }
    float v[32], q32[32];
    // dPG (columns below m1; the row-sum adjoint, column m1, separately) and
    // G, then K and Q of the first half, in coalesced block accesses
    // two blocks in flight: each block's loads are issued before the previous
    // block is split into its tiles
    load_blk(a.dPG + base * a.ldpg, a.ldpg, nn, a.m1, v);
    load_blk(a.G + base * a.m1, a.m1, nn, a.m1, q32);
    const float dpg1 = rv ? a.dPG[(base + row) * a.ldpg + a.m1] : 0.f;
    store_blk_split(T[0], T[1], v);
    load_blk(qk0 + AW, ld, nn, 128, v);  // K, first half
    store_blk_split(T[2], T[3], q32);
    load_blk(qk0, ld, nn, 128, q32);  // Q, first half
    store_blk_split(T[5], T[6], v);
    store_blk<false>(T[4], q32);
    if (tid < 128) s_key[tid] = tid < nn ? reinterpret_cast<const float4*>(a.rw)[base + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    handoff();
    // dP = dPG G^T -> [128, 256); S = Q0_hi K0^T -> [0, 128)
    if (issuer) {
      mma_block<false>(tm + 128, t[0], false, 128, t[2], false, 128, 128, kg, false);
      mma_block<false>(tm + 128, t[1], false, 128, t[2], false, 128, 128, kg, true);
      mma_block<false>(tm + 128, t[0], false, 128, t[3], false, 128, 128, kg, true);
      mma_block<false>(tm, t[4], false, 128, t[5], false, 128, 128, 8, false);
      mma_block<false>(tm, t[4], false, 128, t[6], false, 128, 128, 8, true);
    }
    commit_and_sync(sy, issuer);
    // G is dead: Q0 lo -> T2, S += Q0_lo K0_hi (NH = 2: with the second half's
    // Q hi, K hi / lo, then its Q lo)
    store_blk<true>(T[2], q32);
    int pti;  // the P / dS tile
    if constexpr (NH == 1) {
      handoff();
      if (issuer) mma_block<false>(tm, t[2], false, 128, t[5], false, 128, 128, 8, true);
      commit_and_sync(sy, issuer);
      pti = 3;
    } else {
      load_blk(qk0 + 128, ld, nn, 128, q32);  // Q1
      load_blk(qk0 + AW + 128, ld, nn, 128, v);  // K1 (hi -> T4 over Q0 hi, lo -> T6 over K0 lo)
      store_blk<false>(T[3], q32);
      store_blk<false>(T[4], v);
      store_blk<true>(T[6], v);
      handoff();
      if (issuer) {
        mma_block<false>(tm, t[2], false, 128, t[5], false, 128, 128, 8, true);  // Q0_lo K0_hi
        mma_block<false>(tm, t[3], false, 128, t[4], false, 128, 128, 8, true);  // Q1_hi K1_hi
        mma_block<false>(tm, t[3], false, 128, t[6], false, 128, 128, 8, true);  // Q1_hi K1_lo
      }
      commit_and_sync(sy, issuer);
      store_blk<true>(T[5], q32);  // Q1 lo over K0 hi
      handoff();
      if (issuer) mma_block<false>(tm, t[5], false, 128, t[4], false, 128, 128, 8, true);  // Q1_lo K1_hi
      commit_and_sync(sy, issuer);
      pti = 2;
    }
    float4 rpart, cpart[2];
    softmax_adjoint(a, T[pti], s_key, tm + lane_off + c0, tm + lane_off + 128 + c0, row, part, lane, quad, nn, dpg1,
                    rpart, cpart);
    handoff();
    // P^T dPG -> [256, 256 + npg) (P^T and dPG as MN-major operands)
    if (issuer) {
      mma_block<false>(tm + 256, t[pti], true, 128, t[0], true, 128, a.npg, 8, false);
      mma_block<false>(tm + 256, t[pti], true, 128, t[1], true, 128, a.npg, 8, true);
    }
    commit_and_sync(sy, issuer);
    // P^T dPG -> staging over T0 / T1 (dPG is dead), dS -> the P tile
    float* stg01 = reinterpret_cast<float*>(T[0]);
    if (c0 < a.m1) tmem_to_stg(tm + lane_off + 256 + c0, stg01, row, c0);  // warp-uniform
    tmem_ld32(tm + lane_off + c0, v);
    store_row32<false>(T[pti], row, c0, v);
    float* dqk = a.dQK + base * ld;
    if constexpr (NH == 1) {
      handoff();
      // dQ = dS K -> [0, 128); dK = dS^T Q -> [384, 512), while the threads
      // add P^T dPG to dE/dG (this atom's rows, columns below m1)
      if (issuer) {
        mma_block<false>(tm, t[3], false, 128, t[5], true, 128, 128, 8, false);
        mma_block<false>(tm, t[3], false, 128, t[6], true, 128, 128, 8, true);
        mma_block<false>(tm + 384, t[3], true, 128, t[4], true, 128, 128, 8, false);
        mma_block<false>(tm + 384, t[3], true, 128, t[2], true, 128, 128, 8, true);
      }
      stg_to_global<true>(stg01, a.dG + base * a.m1, a.m1, nn, a.m1);
      commit_and_sync(sy, issuer);
      // every thread's reads of the staging (the dE/dG update) are done before
      // it takes dQ: the MMA wait above is not a CTA barrier
      __syncthreads();
      // dQ -> staging over T0 / T1, dK over T2 / T3
      float* stg23 = reinterpret_cast<float*>(T[2]);
      tmem_to_stg(tm + lane_off + c0, stg01, row, c0);
      tmem_to_stg(tm + lane_off + 384 + c0, stg23, row, c0);
    } else {
      handoff();
      stg_to_global<true>(stg01, a.dG + base * a.m1, a.m1, nn, a.m1);
      handoff();
      load_blk(qk0 + AW, ld, nn, 128, v);  // K0 again -> T0 / T1
      store_blk_split(T[0], T[1], v);
      handoff();
      // dQ0 = dS K0 -> [0, 128), dQ1 = dS K1 -> [128, 256), dK1 = dS^T Q1 -> [384, 512)
      if (issuer) {
        mma_block<false>(tm, t[2], false, 128, t[0], true, 128, 128, 8, false);
        mma_block<false>(tm, t[2], false, 128, t[1], true, 128, 128, 8, true);
        mma_block<false>(tm + 128, t[2], false, 128, t[4], true, 128, 128, 8, false);
        mma_block<false>(tm + 128, t[2], false, 128, t[6], true, 128, 128, 8, true);
        mma_block<false>(tm + 384, t[2], true, 128, t[3], true, 128, 128, 8, false);
        mma_block<false>(tm + 384, t[2], true, 128, t[5], true, 128, 128, 8, true);
      }
      commit_and_sync(sy, issuer);
      load_blk(qk0, ld, nn, 128, v);  // Q0 again -> T0 / T1
      store_blk_split(T[0], T[1], v);
      handoff();
      // dK0 = dS^T Q0 -> [256, 384)
      if (issuer) {
        mma_block<false>(tm + 256, t[2], true, 128, t[0], true, 128, 128, 8, false);
        mma_block<false>(tm + 256, t[2], true, 128, t[1], true, 128, 128, 8, true);
      }
      commit_and_sync(sy, issuer);
      // dQ0, dQ1 -> staging over T0 - T3 -> dQ; then dK0, dK1 the same way
      float* stg23 = reinterpret_cast<float*>(T[2]);
      tmem_to_stg(tm + lane_off + c0, stg01, row, c0);
      tmem_to_stg(tm + lane_off + 128 + c0, stg23, row, c0);
      __syncthreads();
      stg_to_global<false>(stg01, dqk, ld, 128, 128);
      stg_to_global<false>(stg23, dqk + 128, ld, 128, 128);
      __syncthreads();
      tmem_to_stg(tm + lane_off + 256 + c0, stg01, row, c0);
      tmem_to_stg(tm + lane_off + 384 + c0, stg23, row, c0);
    }
    // the row and column parts of dE/drhat, dE/dw -> T4 (dead): [quadrant][128
    // keys] column parts, then [quarter][128 rows] row parts
    float4* parts = reinterpret_cast<float4*>(T[4]);
    if (lane < 16) {
      parts[quad * 128 + c0 + lane] = cpart[0];
      parts[quad * 128 + c0 + 16 + lane] = cpart[1];
    }
    parts[512 + part * 128 + row] = rpart;
    __syncthreads();
    // dK (NH = 1: dQ | dK; NH = 2: dK0 | dK1) from the staging, and dgeo
    if constexpr (NH == 1) {
      stg_to_global<false>(stg01, dqk, ld, 128, 128);
      stg_to_global<false>(reinterpret_cast<float*>(T[2]), dqk + AW, ld, 128, 128);
    } else {
      stg_to_global<false>(stg01, dqk + AW, ld, 128, 128);
      stg_to_global<false>(reinterpret_cast<float*>(T[2]), dqk + AW + 128, ld, 128, 128);
    }
    if (tid < nn) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 r = parts[512 + q * 128 + tid];
        const float4 c = parts[q * 128 + tid];
        s.x += r.x + c.x; s.y += r.y + c.y; s.z += r.z + c.z; s.w += r.w + c.w;
      }
      // one writer per row in a launch: a reduction without a return
      atomicAdd(reinterpret_cast<float4*>(a.dgeo) + base + tid, s);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}

}  // namespace

// ------------------------------------------------------------------ host

bool bf16x_supported(const dp_model* m) {
  if (m->nattn > 0 && ((m->A != 128 && m->A != 256) || m->m1 > 128 || m->m1 % 4 != 0)) return false;
  int fan = m->fit_in;
  if (fan % 4) return false;
  for (int l = 0; l < m->nfit; ++l) {
    if (m->fit[l] % 4) return false;
    fan = m->fit[l];
  }
  return true;
}

namespace {

XImage x_image_shape(int K, int N) {
  XImage s;
  s.K = K;
  s.N = N;
  s.nkb = (K + XBK - 1) / XBK;
  s.nnb = (N + XBN - 1) / XBN;
  s.bn_max = std::min(XBN, (N + 15) & ~15);
  return s;
}

// B: [K][ldb] row-major, the image's N columns taken from the left.
int x_image_build(dp_model* m, XImage& im, const float* B, int ldb, cudaStream_t st, std::string& msg) {
  if (!im.d) {
    void* d = nullptr;
    if (cudaMalloc(&d, im.bytes()) != cudaSuccess) {
      msg = "cudaMalloc of a BF16 weight image failed";
      return DP_ERR_CUDA;
    }
    m->xw.allocations.push_back(d);
    im.d = d;
  }
  const long long total = (long long)im.nnb * im.nkb * im.bn_max * XBK;
  k_x_image<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(B, ldb, im.K, im.N, im.nkb, im.bn_max,
                                                             reinterpret_cast<uint8_t*>(im.d));
  note_launch();
  return DP_OK;
}

}  // namespace

int bf16x_init_weights(dp_model* m, std::string& msg) {
  XWeights& w = m->xw;
  if (!bf16x_supported(m)) {
    msg = "the BF16-split path needs attention width 128 or 256, an embedding width <= 128 divisible by 4 and "
          "fitting widths divisible by 4";
    return DP_ERR_UNSUPPORTED;
  }
  if (!g_x_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      msg = "cuTensorMapEncodeTiled is not available from the driver";
      return DP_ERR_CUDA;
    }
    g_x_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const int A = m->A, m1 = m->m1;
  w.layers.assign(m->nattn, XWeights::Layer{});
  for (int l = 0; l < m->nattn; ++l) {
    XWeights::Layer& L = w.layers[l];
    const AttnLayerW& aw = m->attn[l];
    // V only enters through [Wv Wo; bv Wo], so the projection stops at [Q K]
    L.qk = x_image_shape(m1, 2 * A);    // [Wq Wk]
    L.vo = x_image_shape(pg_ld(m1), m1);
    L.voT = x_image_shape(m1, pg_ld(m1));
    L.qkT = x_image_shape(2 * A, m1);   // [Wq Wk]^T
    int rc;
    if ((rc = x_image_build(m, L.qk, aw.Wqk, 2 * A, nullptr, msg)) != DP_OK) return rc;
    if ((rc = x_image_build(m, L.vo, aw.Wvo, m1, nullptr, msg)) != DP_OK) return rc;
    if ((rc = x_image_build(m, L.voT, aw.WvoT, pg_ld(m1), nullptr, msg)) != DP_OK) return rc;
    if ((rc = x_image_build(m, L.qkT, aw.WqkT, m1, nullptr, msg)) != DP_OK) return rc;
  }
  w.fit.assign(m->nfit, XImage{});
  w.fitT.assign(m->nfit, XImage{});
  int fan = m->fit_in;
  for (int l = 0; l < m->nfit; ++l) {
    w.fit[l] = x_image_shape(fan, m->fit[l]);
    w.fitT[l] = x_image_shape(m->fit[l], fan);
    fan = m->fit[l];
  }
  bf16x_refresh(m, nullptr);
  cudaFuncSetAttribute(k_gemm_bf16x, cudaFuncAttributeMaxDynamicSharedMemorySize, x_smem(XBN));
  cudaFuncSetAttribute(k_attn_core_fwd_bf16x<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, XF_SMEM);
  cudaFuncSetAttribute(k_attn_core_fwd_bf16x<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, XF_SMEM);
  cudaFuncSetAttribute(k_attn_core_bwd_bf16x<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, XB_SMEM);
  cudaFuncSetAttribute(k_attn_core_bwd_bf16x<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, XB_SMEM);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    msg = "building the BF16 weight images failed";
    return DP_ERR_CUDA;
  }
  w.ready = true;
  return DP_OK;
}

// The fitting images follow the (trainable) FP32 fitting weights.
void bf16x_refresh(dp_model* m, cudaStream_t st) {
  XWeights& w = m->xw;
  std::string msg;
  for (int l = 0; l < (int)w.fit.size(); ++l) {
    x_image_build(m, w.fit[l], m->fitW[l], w.fit[l].N, st, msg);
    x_image_build(m, w.fitT[l], m->fitWT[l], w.fitT[l].N, st, msg);
  }
}

void bf16x_free(dp_model* m) {
  for (void* p : m->xw.allocations) cudaFree(p);
  m->xw = XWeights{};
}

int gemm_bf16x(dp_model* m, const XImage& im, const float* A, int lda, const float* bias, const float* R, int ldr,
               float* C, int ldc, int M, int epi, cudaStream_t st) {
  if (M <= 0) return DP_OK;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)im.K, (cuuint64_t)M};
  const cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(float)};
  const cuuint32_t box[2] = {32, XBM};
  const cuuint32_t estr[2] = {1, 1};
  if (g_x_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), dims, strides, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return DP_ERR_CUDA;
  XGemmArgs a;
  a.bimg = reinterpret_cast<const uint8_t*>(im.d);
  a.bias = bias;
  a.R = R;
  a.C = C;
  a.ldr = ldr;
  a.ldc = ldc;
  a.M = M;
  a.N = im.N;
  a.nkb = im.nkb;
  a.bn_max = im.bn_max;
  a.epi = epi;
  a.mtiles = (M + XBM - 1) / XBM;
  a.err = m->d_err;
  // persistent: about one CTA per SM over the N blocks
  const int per_n = std::max(1, x_sm_count(m->device) / im.nnb);
  dim3 grid((unsigned)std::min(a.mtiles, per_n), (unsigned)im.nnb);
  k_gemm_bf16x<<<grid, XTHREADS, x_smem(im.bn_max), st>>>(map, a);
  note_launch();
  return DP_OK;
}

namespace {
XCoreArgs core_args(dp_model* m, int n, int l) {
  Workspace& ws = m->ws;
  XCoreArgs a{};
  a.QK = ws.QK[l];  // [rows][2A]: Q | K
  a.G = ws.G[l];
  a.PG = ws.PG[l];
  a.dPG = ws.dPG;  // dE/d[P G, rowsum P], [rows][ldpg]
  a.dQK = ws.dQK;
  a.dG = ws.dG;
  a.dgeo = ws.dgeo;
  a.rw = ws.rw;
  a.nnei = ws.nnei;
  a.n = n;
  a.m1 = m->m1;
  a.ldpg = pg_ld(m->m1);
  a.npg = (m->m1 + 15) & ~15;
  a.ldq = 2 * m->A;
  a.scale = (float)(1.0 / std::sqrt((double)m->A));
  a.shift = (float)m->shift;
  a.err = m->d_err;
  return a;
}
}  // namespace

void attn_core_fwd_bf16x(dp_model* m, int n, int l, cudaStream_t st) {
  if (n == 0) return;
  const int grid = std::min(n, x_sm_count(m->device));
  if (m->A == 256)
    k_attn_core_fwd_bf16x<2><<<grid, XC_NT, XF_SMEM, st>>>(core_args(m, n, l));
  else
    k_attn_core_fwd_bf16x<1><<<grid, XC_NT, XF_SMEM, st>>>(core_args(m, n, l));
  note_launch();
}

void attn_core_bwd_bf16x(dp_model* m, int n, int l, cudaStream_t st) {
  if (n == 0) return;
  const int grid = std::min(n, x_sm_count(m->device));
  if (m->A == 256)
    k_attn_core_bwd_bf16x<2><<<grid, XC_NT, XB_SMEM, st>>>(core_args(m, n, l));
  else
    k_attn_core_bwd_bf16x<1><<<grid, XC_NT, XB_SMEM, st>>>(core_args(m, n, l));
  note_launch();
}

}  // namespace dpa1
