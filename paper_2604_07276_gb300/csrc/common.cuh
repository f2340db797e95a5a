// Shared definitions of the DPA-1 CUDA path (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace dpa1 {

// Rows reserved per centre atom: the neighbour cap sel (<= 128) padded to one
// 128-row tile, so that every per-atom matrix has a fixed 128-row shape.
constexpr int NP = 128;
// Per-atom [NP][W] FP32 matrices of the tensor-core path (the layer inputs
// G_l and dE/dG) are stored column-quad interleaved: the 4 columns
// 4q..4q+3 of a row are contiguous and the NP rows of one column quad follow
// each other, so that one thread per row reading or writing 16 bytes makes a
// warp access 512 contiguous bytes.  The atom block keeps the size NP * W.
__host__ __device__ __forceinline__ size_t cq_off(int r, int c) {
  return ((size_t)(c >> 2) * NP + (size_t)r) * 4 + (size_t)(c & 3);
}

// Candidate capacity of the neighbour search per centre (before the sel cap).
constexpr int NBR_CAP = 256;
// Capacity of the reverse neighbour list per atom (centres that list it).
constexpr int REV_CAP = 256;

// Bits of the device status flag.
enum ErrBits : int {
  ERR_BOX = 1,       // box not orthorhombic or an edge <= 2 rcut
  ERR_CAPACITY = 2,  // candidate / reverse-list / workspace overflow
  ERR_NAN = 4,       // non-finite coordinate
  ERR_TIMEOUT = 8,   // a bounded wait gave up
  ERR_TYPE = 16,     // atom type out of range
};

// Cell grid derived on the device from the (device) box.
struct CellGrid {
  double L[3];
  int nc[3];
  int ncells;
  int ok;
};

__device__ __forceinline__ void set_err(int* err, int bits) { atomicOr(err, bits); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the 32 lanes of a warp of 16 values per lane; lanes l and l + 16
// return the sum of value l % 16 (butterfly reduce-scatter, fixed order;
// 16 shuffles instead of 16 full reductions).
__device__ __forceinline__ float warp_reduce_scatter16(float* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1) {
    const bool up = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float send = up ? v[i] : v[i + w];
      const float keep = up ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// Minimum-image displacement component d - L * rint(d / L), every operation
// rounded separately (no FMA contraction) so that the host can reproduce it
// bit for bit.
__device__ __forceinline__ double mic(double d, double L) {
  return __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
}

// (dx*dx + dy*dy) + dz*dz without contraction.
__device__ __forceinline__ double sqdist(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

}  // namespace dpa1
