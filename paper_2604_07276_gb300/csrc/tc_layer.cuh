// Device helpers shared by the per-atom tensor-core kernels of the attention
// layers (the fused layer kernels and the BF16-split attention cores): a
// bounded mbarrier wait with phase tracking, the hand-offs between the
// element-wise threads and the MMA issuer, 16-bit (hi / lo) row stores into
// SW128 tiles, the MMA block issue and the row exchange among the four
// threads that own one TMEM lane.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace dpa1 {
namespace tc {

struct Sync {
  uint64_t* bar;
  uint32_t phase;
  int* err;
  bool ok = true;
  __device__ bool wait() {
    if (ok) ok = mbar_wait(bar, phase & 1u, err);
    ++phase;
    fence_after_sync();
    return ok;
  }
};

__device__ __forceinline__ void commit_and_sync(Sync& s, bool issuer) {
  if (issuer) mma_commit(s.bar);
  s.wait();
}

// All threads: make their generic shared-memory writes visible to the tensor
// cores and finish their TMEM loads, then meet.
__device__ __forceinline__ void handoff() {
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
}

// A warp's share of a handoff to the MMA issuer through an mbarrier that
// expects one arrival per warp: its shared-memory writes made visible to the
// tensor cores and its TMEM accesses ordered, then lane 0 arrives.  Unlike
// handoff(), no thread waits.
__device__ __forceinline__ void warp_arrive(uint64_t* bar) {
  fence_async_smem();
  fence_before_sync();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

__device__ __forceinline__ void copy_image(uint8_t* dst, const uint4* src, int bytes) {
  uint4* d = reinterpret_cast<uint4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = src[i];
}

// Store 32 FP32 values (cols c0..c0+31 of row r) as the 16-bit operand type
// into an SW128 tile; LO = true stores the rounding residue v - round16(v)
// instead (the low part of a two-term split).
template <bool F16, bool LO = false>
__device__ __forceinline__ void store_row32(uint8_t* tile, int r, int c0, const float* v) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = LO ? v[8 * q + i] - round16<F16>(v[8 * q + i]) : v[8 * q + i];
    uint4 u;
    u.x = pack16<F16>(x[0], x[1]);
    u.y = pack16<F16>(x[2], x[3]);
    u.z = pack16<F16>(x[4], x[5]);
    u.w = pack16<F16>(x[6], x[7]);
    sw128_store8(tile, r, c0 + 8 * q, 128, u);
  }
}

// Load row r, columns c0..c0+31 (zero past m1), of an atom's column-quad
// interleaved FP32 block; a row that is not live (past the last neighbour,
// whose content is not kept) reads as zeros without a load.
__device__ __forceinline__ void load_cq32(const float* blk, int m1, int r, int c0, float* v, bool live = true) {
  const float4* b4 = reinterpret_cast<const float4*>(blk);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int c = c0 + 4 * q;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c < m1 && live) x = b4[(c >> 2) * NP + r];  // m1 % 4 == 0
    v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
  }
}

// e^x as 2^(x log2 e) on the special-function unit, subnormal results
// flushed to zero (the attention weights are normalised by sums >= 1, so
// that loses nothing), exp(-inf) = 0.  Relative error a few units in the
// last place of FP32 for the arguments of the softmax (|x| below ~100).
__device__ __forceinline__ float exp_sfu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * 1.4426950408889634f));
  return y;
}

// Columns m1 and m1 + 1 of a layer-input row carry the constant 1 that picks
// up the Q, K, V biases stored in the weight tiles (the columns are zero
// padding of the embedding width otherwise).
__device__ __forceinline__ void set_bias_ones(float* v, int c0, int m1) {
#pragma unroll
  for (int i = 0; i < 32; ++i)
    if (c0 + i == m1 || c0 + i == m1 + 1) v[i] = 1.f;
}

// Issue D = sum over K-steps of A * B for one 128 x N block.
template <bool F16>
__device__ __forceinline__ void mma_block(uint32_t d, uint32_t a, bool a_mn, int a_rows, uint32_t b, bool b_mn,
                                          int b_rows, int N, int ksteps, bool accumulate_first) {
  const uint32_t id = idesc_16(128, N, a_mn, b_mn, F16);
  for (int s = 0; s < ksteps; ++s) {
    const uint64_t ad = a_mn ? mnmajor_desc(a, s, a_rows) : kmajor_desc(a, s, a_rows);
    const uint64_t bd = b_mn ? mnmajor_desc(b, s, b_rows) : kmajor_desc(b, s, b_rows);
    mma_bf16(d, ad, bd, id, (s > 0 || accumulate_first) ? 1u : 0u);
  }
}

// Row exchange among the four threads (column quarters) that own a row.  The
// four warps of one TMEM lane quadrant meet on their own named barrier; the
// values are parked in the row's own 128-byte line of chunk 0 of an SW128
// tile that only this row's threads write afterwards, at a word offset that
// differs between the 32 rows of a warp (no bank conflicts).
struct RowXchg {
  uint8_t* line;  // this row's line in the parking tile
  int part, lane, quad;
  __device__ RowXchg(uint8_t* tile, int row, int part_, int lane_, int quad_)
      : line(tile + (row >> 3) * 1024 + (row & 7) * 128), part(part_), lane(lane_), quad(quad_) {}
  __device__ void sync() const { asm volatile("bar.sync %0, 128;" ::"r"(1 + quad) : "memory"); }
  __device__ float* slot(int p) const { return reinterpret_cast<float*>(line) + ((lane + 8 * p) & 31); }
  __device__ float2* slot2(int p) const { return reinterpret_cast<float2*>(line) + ((lane + 4 * p) & 15); }
  __device__ float sum(float v) const {
    *slot(part) = v;
    sync();
    const float r = (*slot(0) + *slot(1)) + (*slot(2) + *slot(3));
    sync();
    return r;
  }
  __device__ float max(float v) const {
    *slot(part) = v;
    sync();
    const float r = fmaxf(fmaxf(*slot(0), *slot(1)), fmaxf(*slot(2), *slot(3)));
    sync();
    return r;
  }
  __device__ float2 sum2(float2 v) const {
    *slot2(part) = v;
    sync();
    const float2 a = *slot2(0), b = *slot2(1), c = *slot2(2), d = *slot2(3);
    sync();
    return make_float2((a.x + b.x) + (c.x + d.x), (a.y + b.y) + (c.y + d.y));
  }
};

}  // namespace tc
}  // namespace dpa1
