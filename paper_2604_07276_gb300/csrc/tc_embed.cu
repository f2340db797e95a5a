// The embedding net (stages a5, a13) on the tensor cores: tcgen05 products
// with FP16 or BF16 two-term operand splits, FP32 element-wise work, for the
// 25-50-100 net and the paper's 32-64-128 net.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dpa1.h"
#include "kernels.h"
#include "model.h"
#include "tc_ptx.cuh"
#include "tc_layer.cuh"

namespace dpa1 {

using namespace tc;

namespace {

int emb_sm_count(int dev) {
  int c = 0;
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

// ----------------------------------------------------------- embedding net
// Stage a5 / a13 on the tensor cores: net_s = 1 -> E0 -> E1 -> E2 (tanh,
// residual rule) for the 128 neighbour rows of an atom, G0 = net_s * (1 + Gt).
// The two matrix products per direction run in FP16 (or BF16) with hi + lo
// splits of both operands (three products each), which keeps them within
// FP32-level accuracy; the 1 -> E0 layer and all element-wise work are FP32.
// Two net shapes have instances: the measured 25-50-100 net and the paper's
// 32-64-128 net (both double their width per layer, E1 = 2 E0, E2 = 2 E1).
constexpr int EMB_TA = 128 * 64 * 2;    // activation tile: 128 rows x 64 cols
constexpr int EMB_TD = 128 * 128 * 2;   // dZ3 tile: 128 rows x 128 cols
constexpr int EMB_MAXT = 8;             // atom types the staged type-pair rows allow
constexpr int EMB_THREADS = 256;
static_assert(2 * EMB_TD == 4 * EMB_TA, "the dZ3 hi / lo tiles fill the activation tiles");

template <int E0_, int E1_, int E2_>
struct EmbShape {
  static constexpr int E0 = E0_, E1 = E1_, E2 = E2_;
  static_assert(E0 > 16 && E0 <= 32 && E1 == 2 * E0 && E2 == 2 * E1, "a doubling net of first width 17 .. 32");
  static constexpr int E2P = (E2 + 15) & ~15;          // W2 rows, Z3 columns
  static constexpr int T1 = 64 * 64 * 2;               // W1 tile: 64 (E1 padded) rows x 64 cols
  static constexpr int T2 = E2P * 64 * 2;              // W2 tile: E2P rows x 64 cols
  static constexpr int WIMG = 2 * T1 + 2 * T2;         // W1 hi, W1 lo, W2 hi, W2 lo
  static constexpr int GT = EMB_MAXT * E2 * 4;         // this atom's rows of the type-pair table
  static constexpr int B0T = EMB_MAXT * E0 * 4;        // concat mode: this atom's rows of the first-layer bias table
  static constexpr int F_B0 = WIMG + 4 * EMB_TA + GT;  // forward: bias rows after the type-pair rows
  static constexpr int F_SMEM = F_B0 + B0T + 64;
  // the adjoint reads layers 1 and 2 as stored (no bias rows); its dZ3 tiles
  // reuse the four activation tiles
  static constexpr int B_SMEM = WIMG + 4 * EMB_TA + GT + 512 + 64;
  static constexpr int SPLIT = (E1 / 2) & ~7;          // first layer-2 unit of half 1 (24 / 32)
  static constexpr int G2 = (E1 + 7) / 8;              // 8-column groups of layer 2
  static constexpr int G3 = (E2 + 7) / 8;              // 8-column groups of layer 3
  static constexpr int GS = (G3 + 1) / 2;              // dZ3 groups stored by half 0 ([0, GS)), half 1 the rest
  static constexpr int NK3 = E2P / 16;                 // 16-column chunks of Z3
  static constexpr int TM_H1 = 64 + E2P;               // TMEM columns of the layer-1 exchange (32)
  // CTAs per SM the shared memory allows (228 KB per SM, 1 KB of it reserved per CTA)
  static constexpr int MIN_CTAS = 2 * ((F_SMEM > B_SMEM ? F_SMEM : B_SMEM) + 1024) <= 228 * 1024 ? 2 : 1;
  static_assert(TM_H1 + 32 <= 256, "TMEM columns");
};
using EmbS100 = EmbShape<25, 50, 100>;
using EmbS128 = EmbShape<32, 64, 128>;

struct EmbedTcArgs {
  const float* R;
  const int* nlist;
  const int* nnei;
  const int* atype;
  const float* Gt;        // [ntypes][ntypes][E2]
  float* G0;              // fwd out, column-quad interleaved per atom (rm: row-major [rows][E2])
  const float* dG0;       // bwd in, same layout as G0
  float* dR;              // bwd: dR[:,0] +=
  const float* b0t;       // concat type-embedding mode: first-layer bias per (centre,
                          // neighbour) type [ntypes][ntypes][E0]; null: b0 below
  float* H12;             // [atom][E0 + E1 units][NP rows]: layers 1 and 2 of the net,
                          // written by the forward, read by the adjoint
  const uint4* wimg;      // W1/W2 hi/lo tiles (FP16 or BF16, as the kernel's operands)
  int n, ntypes;
  int rm;                 // G0 and dG0 row-major (the modular layer layout) instead of interleaved
  int live_only;          // G0's rows past the last neighbour are not written (their content is
                          // undefined: the fused layer kernels never read them); else zeros.
                          // The live-row kernels need 1 (a row past the list's end stores nothing)
  const int* rowmap;      // live-row kernels: the live rows (atom * NP + slot) in tile order
  const int* nrows;       // live-row kernels: their number (device)
  int* err;
  float W0[32], b0[32], b1[64], b2[128];  // the net's first layer and biases (first E0 / E1 / E2 used)
};

// Thread layout (256 threads): warp w owns TMEM lane quadrant w % 4 (rows
// 32 (w % 4) .. +31) and half H = w / 4 of the work of its row.  Half 0 owns
// the layer-2 units b in [0, SPLIT), half 1 those in [SPLIT, E1); a layer-3
// output c belongs to the owner of c % E1 (the residual input it needs), so no
// row data crosses between the halves except one partial sum at the end of
// the adjoint.  Layer 1 is split between the halves (units 0-15 and the
// rest), which exchange their units through TMEM.
template <bool F16>
__device__ __forceinline__ void emb_store8(uint8_t* tile, int r, int c0, int R, const float* v, bool lo) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = lo ? v[i] - round16<F16>(v[i]) : v[i];
  uint4 u;
  u.x = pack16<F16>(x[0], x[1]); u.y = pack16<F16>(x[2], x[3]);
  u.z = pack16<F16>(x[4], x[5]); u.w = pack16<F16>(x[6], x[7]);
  sw128_store8(tile, r, c0, R, u);
}

// D (+)= A * B with A = Ah + Al and B = Bh + Bl, dropping Al * Bl.
template <bool F16>
__device__ __forceinline__ void mma_split(uint32_t d, uint32_t ah, uint32_t al, int a_rows, uint32_t bh, uint32_t bl,
                                          bool b_mn, int b_rows, int N, int ksteps) {
  mma_block<F16>(d, ah, false, a_rows, bh, b_mn, b_rows, N, ksteps, false);
  mma_block<F16>(d, al, false, a_rows, bh, b_mn, b_rows, N, ksteps, true);
  mma_block<F16>(d, ah, false, a_rows, bl, b_mn, b_rows, N, ksteps, true);
}

template <class S, int H>
struct EmbOwn {
  static constexpr int b0 = H == 0 ? 0 : S::SPLIT;          // first owned layer-2 unit
  static constexpr int nb = H == 0 ? S::SPLIT : S::E1 - S::SPLIT;
  static constexpr int g_lo = b0 / 8, g_hi = H == 0 ? S::SPLIT / 8 : S::G2;  // layer-2 8-column groups stored
  __host__ __device__ static constexpr bool owns_b(int b) { return b >= b0 && b < b0 + nb; }
  __host__ __device__ static constexpr bool owns_c(int c) { return c < S::E2 && owns_b(c % S::E1); }
};

// Layers 1 and 2 of a row and the issue of Z3 = H2 W2; returns once Z3 is in
// TMEM columns [64, 64 + E2P).  h1 gets all E0 layer-1 units, h2 the owned
// layer-2 units.
template <class S, bool F16, int H, class BeforeZ3>
__device__ __forceinline__ void embed_tc_front(const EmbedTcArgs& a, uint8_t* sm, uint32_t tm, uint32_t lane_off,
                                               Sync& sy, int row, bool rv, float x, const float* b0row, float* h1,
                                               float* h2, BeforeZ3 before_z3) {
  using O = EmbOwn<S, H>;
  uint8_t* sW1h = sm;
  uint8_t* sW1l = sW1h + S::T1;
  uint8_t* sW2h = sW1l + S::T1;
  uint8_t* sW2l = sW2h + S::T2;
  uint8_t* sH1h = sm + S::WIMG;
  uint8_t* sH1l = sH1h + EMB_TA;
  uint8_t* sH2h = sH1l + EMB_TA;
  uint8_t* sH2l = sH2h + EMB_TA;
  const bool issuer = threadIdx.x == 0;
  // layer 1: half 0 evaluates units 0-15, half 1 units 16 .. E0 - 1; each
  // stores the hi and lo parts of its 8-column groups of H1 (K = E0, read as
  // 32) and leaves its units in TMEM columns [TM_H1, TM_H1 + 32) (free in
  // both kernels), where the other half reads them after the hand-off
  constexpr int p0 = H == 0 ? 0 : 16, np = H == 0 ? 16 : S::E0 - 16;
#pragma unroll
  for (int p = p0; p < p0 + np; ++p) h1[p] = rv ? tanhf(fmaf(x, a.W0[p], b0row ? b0row[p] : a.b0[p])) : 0.f;
  {
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = p0 + i < S::E0 ? h1[p0 + i] : 0.f;
    emb_store8<F16>(sH1h, row, p0, 128, v, false);
    emb_store8<F16>(sH1l, row, p0, 128, v, true);
    emb_store8<F16>(sH1h, row, p0 + 8, 128, v + 8, false);
    emb_store8<F16>(sH1l, row, p0 + 8, 128, v + 8, true);
    tmem_st16(tm + lane_off + S::TM_H1 + p0, v);
  }
  handoff();
  if (issuer)
    mma_split<F16>(tm + 0, smem_u32(sH1h), smem_u32(sH1l), 128, smem_u32(sW1h), smem_u32(sW1l), false, 64, 64, 2);
  {
    constexpr int q0 = H == 0 ? 16 : 0, nq = H == 0 ? S::E0 - 16 : 16;
    float v[16];
    tmem_ld16(tm + lane_off + S::TM_H1 + q0, v);
#pragma unroll
    for (int i = 0; i < nq; ++i) h1[q0 + i] = v[i];
  }
  commit_and_sync(sy, issuer);
  // layer 2, owned units: h2 = h1[b % E0] + tanh(z2 + b1)
#pragma unroll
  for (int k = 0; k < 4; ++k) {  // 16-column TMEM chunks
    if (16 * k + 15 < O::b0 || 16 * k >= 8 * O::g_hi) continue;
    float z[16];
    tmem_ld16(tm + lane_off + 16 * k, z);
#pragma unroll
    for (int gg = 0; gg < 2; ++gg) {
      const int g = 2 * k + gg;
      if (g < O::g_lo || g >= O::g_hi) continue;
      float v[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int b = 8 * g + i;
        float hb = 0.f;
        if (b < S::E1 && rv) hb = h1[b % S::E0] + tanhf(z[8 * gg + i] + a.b1[b]);
        if (O::owns_b(b)) h2[b - O::b0] = hb;
        v[i] = hb;
      }
      emb_store8<F16>(sH2h, row, 8 * g, 128, v, false);
      emb_store8<F16>(sH2l, row, 8 * g, 128, v, true);
    }
  }
  handoff();
  if (issuer) {
    mma_split<F16>(tm + 64, smem_u32(sH2h), smem_u32(sH2l), 128, smem_u32(sW2h), smem_u32(sW2l), false, S::E2P,
                   S::E2P, 4);
    mma_commit(sy.bar);
  }
  before_z3();  // work that does not need Z3 (the adjoint's first dE/dG0 loads)
  sy.wait();
}

// The adjoint's front: layers 1 and 2 as the forward stored them (all E0
// layer-1 units, the owned layer-2 units), the H2 tiles, and the issue of
// Z3 = H2 W2; returns once Z3 is in TMEM columns [64, 64 + E2P).
template <class S, bool F16, int H, class BeforeZ3>
__device__ __forceinline__ void embed_bwd_front(const EmbedTcArgs& a, uint8_t* sm, uint32_t tm, Sync& sy, int row,
                                                bool rv, int atom, int slot, float* h1, float* h2,
                                                BeforeZ3 before_z3) {
  using O = EmbOwn<S, H>;
  uint8_t* sW2h = sm + 2 * S::T1;
  uint8_t* sW2l = sW2h + S::T2;
  uint8_t* sH2h = sm + S::WIMG + 2 * EMB_TA;
  uint8_t* sH2l = sH2h + EMB_TA;
  const bool issuer = threadIdx.x == 0;
  const float* hs = a.H12 + (size_t)atom * (S::E0 + S::E1) * NP + slot;  // live rows only were stored
#pragma unroll
  for (int p = 0; p < S::E0; ++p) h1[p] = rv ? hs[p * NP] : 0.f;
#pragma unroll
  for (int i = 0; i < O::nb; ++i) h2[i] = rv ? hs[(S::E0 + O::b0 + i) * NP] : 0.f;
#pragma unroll
  for (int g = O::g_lo; g < O::g_hi; ++g) {
    float v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int b = 8 * g + i;
      v[i] = b < S::E1 ? h2[b - O::b0] : 0.f;
    }
    emb_store8<F16>(sH2h, row, 8 * g, 128, v, false);
    emb_store8<F16>(sH2l, row, 8 * g, 128, v, true);
  }
  handoff();
  if (issuer) {
    mma_split<F16>(tm + 64, smem_u32(sH2h), smem_u32(sH2l), 128, smem_u32(sW2h), smem_u32(sW2l), false, S::E2P,
                   S::E2P, 4);
    mma_commit(sy.bar);
  }
  before_z3();
  sy.wait();
}

// A row's inputs of the embedding net (s of the neighbour, its type), read
// for the next atom while the current one is processed: the neighbour
// count, s and the neighbour index at its start, the type at its end.
struct EmbRowIn {
  int nn = 0, nl = 0, tj = 0;
  float x = 0.f;
  __device__ void count(const EmbedTcArgs& a, int atom) { nn = atom < a.n ? a.nnei[atom] : 0; }
  __device__ void rows(const EmbedTcArgs& a, int atom, int row) {
    if (atom < a.n) {  // R and nlist are written for all NP rows: read unmasked, used masked
      const size_t rg = (size_t)atom * NP + row;
      x = a.R[rg * 4];
      nl = a.nlist[rg];
    }
  }
  __device__ void type(const EmbedTcArgs& a, int row) {
    const bool rv = row < nn;
    x = rv ? x : 0.f;
    tj = rv ? a.atype[nl] : 0;
  }
};

template <class S>
__device__ __forceinline__ void embed_tc_setup(const EmbedTcArgs& a, uint8_t* sm, uint64_t*& bar, uint32_t*& s_tmem,
                                               int smem_bytes) {
  bar = reinterpret_cast<uint64_t*>(sm + smem_bytes - 64);
  s_tmem = reinterpret_cast<uint32_t*>(bar + 1);
  uint4* d = reinterpret_cast<uint4*>(sm);
  for (int i = threadIdx.x; i < S::WIMG / 16; i += blockDim.x) d[i] = a.wimg[i];
  // activation tiles start at zero: columns never written later are read
  // only against zero weight rows, which needs finite values there
  for (int i = threadIdx.x; i < 4 * EMB_TA / 16; i += blockDim.x) d[S::WIMG / 16 + i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(s_tmem, 256);
  handoff();
}

// Per atom: copy the centre type's rows of the type-pair table Gt[t_i][*]
// (and, in concat mode and given s_b0, of the first-layer bias table) to
// shared memory, read by neighbour type afterwards, and bring the next atom's
// per-row inputs into L2.
template <class S>
__device__ __forceinline__ void embed_tc_atom_start(const EmbedTcArgs& a, float* s_gt, float* s_b0, int atom,
                                                    bool bwd) {
  const float4* src = reinterpret_cast<const float4*>(a.Gt + (size_t)a.atype[atom] * a.ntypes * S::E2);
  float4* dst = reinterpret_cast<float4*>(s_gt);
  for (int i = threadIdx.x; i < a.ntypes * S::E2 / 4; i += blockDim.x) dst[i] = src[i];
  if (a.b0t && s_b0) {  // read by layer 1 right away: a barrier of its own
    const float* b0 = a.b0t + (size_t)a.atype[atom] * a.ntypes * S::E0;
    for (int i = threadIdx.x; i < a.ntypes * S::E0; i += blockDim.x) s_b0[i] = b0[i];
    __syncthreads();
  }
  const int next = atom + gridDim.x;
  if (threadIdx.x == 0 && next < a.n) {
    const size_t base = (size_t)next * NP;
    prefetch_l2(a.R + base * 4, NP * 4 * sizeof(float));
    prefetch_l2(a.nlist + base, NP * sizeof(int));
    if (bwd) {
      prefetch_l2(a.dG0 + base * S::E2, NP * S::E2 * sizeof(float));
      prefetch_l2(a.H12 + base * (S::E0 + S::E1), NP * (S::E0 + S::E1) * sizeof(float));
    }
  }
}

// Layer 3 forward of the owned outputs: G0[c] = (h2[c % E1] + tanh(z3 + b2)) (1 + Gt[t_i][t_j][c]).
template <class S, int H>
__device__ __forceinline__ void embed_fwd_out(const EmbedTcArgs& a, uint32_t taddr, const float* gt, const float* h2,
                                              bool rv, float* out_blk, int row) {
  using O = EmbOwn<S, H>;
#pragma unroll
  for (int k = 0; k < S::NK3; ++k) {
    bool any = false;
#pragma unroll
    for (int i = 0; i < 16; ++i) any |= O::owns_c(16 * k + i);
    if (!any) continue;
    float z[16];
    tmem_ld16(taddr + 64 + 16 * k, z);
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      const int c = 16 * k + i;
      if (!O::owns_c(c)) continue;  // pairs never straddle an ownership boundary (SPLIT, E1, E1 + SPLIT even)
      const float2 g2 = *reinterpret_cast<const float2*>(gt + c);
      float2 o;
      o.x = rv ? (h2[c % S::E1 - O::b0] + tanhf(z[i] + a.b2[c])) * (1.f + g2.x) : 0.f;
      o.y = rv ? (h2[(c + 1) % S::E1 - O::b0] + tanhf(z[i + 1] + a.b2[c + 1])) * (1.f + g2.y) : 0.f;
      if (rv || !a.live_only)
        __stcs(reinterpret_cast<float2*>(out_blk + (a.rm ? (size_t)row * S::E2 + c : cq_off(row, c))), o);
    }
  }
}

template <class S, bool F16>
__global__ void __launch_bounds__(EMB_THREADS, S::MIN_CTAS) k_embed_tc_fwd(const __grid_constant__ EmbedTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint64_t* bar;
  uint32_t* s_tmem;
  embed_tc_setup<S>(a, sm, bar, s_tmem, S::F_SMEM);
  const uint32_t tm = *s_tmem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  float* s_gt = reinterpret_cast<float*>(sm + S::WIMG + 4 * EMB_TA);
  float* s_b0 = reinterpret_cast<float*>(sm + S::F_B0);
  Sync sy{bar, 0u, a.err};
  float h1[S::E0], h2[S::E1 - S::SPLIT];
  EmbRowIn in;
  in.count(a, blockIdx.x);
  in.rows(a, blockIdx.x, row);
  in.type(a, row);
  for (int atom = blockIdx.x; atom < a.n && sy.ok; atom += gridDim.x) {
    const EmbRowIn cur = in;
    const int nn = cur.nn, tj = cur.tj, next = atom + gridDim.x;
    const bool rv = row < nn;
    in.count(a, next);
    embed_tc_atom_start<S>(a, s_gt, s_b0, atom, false);  // visible after the front's barriers
    auto rows_next = [&] { in.rows(a, next, row); };
    const float* b0row = a.b0t ? s_b0 + tj * S::E0 : nullptr;
    if (half == 0)
      embed_tc_front<S, F16, 0>(a, sm, tm, lane_off, sy, row, rv, cur.x, b0row, h1, h2, rows_next);
    else
      embed_tc_front<S, F16, 1>(a, sm, tm, lane_off, sy, row, rv, cur.x, b0row, h1, h2, rows_next);
    if (rv) {  // layers 1 and 2 of a live row for the adjoint: this half's layer-1 units, its layer-2 units
      float* hs = a.H12 + (size_t)atom * (S::E0 + S::E1) * NP + row;
      if (half == 0) {
#pragma unroll
        for (int p = 0; p < 16; ++p) hs[p * NP] = h1[p];
#pragma unroll
        for (int i = 0; i < S::SPLIT; ++i) hs[(S::E0 + i) * NP] = h2[i];
      } else {
#pragma unroll
        for (int p = 16; p < S::E0; ++p) hs[p * NP] = h1[p];
#pragma unroll
        for (int i = 0; i < S::E1 - S::SPLIT; ++i) hs[(S::E0 + S::SPLIT + i) * NP] = h2[i];
      }
    }
    float* out = a.G0 + (size_t)atom * NP * S::E2;
    if (half == 0)
      embed_fwd_out<S, 0>(a, tm + lane_off, s_gt + tj * S::E2, h2, rv, out, row);
    else
      embed_fwd_out<S, 1>(a, tm + lane_off, s_gt + tj * S::E2, h2, rv, out, row);
    in.type(a, row);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// Adjoint of layer 3 for one half: dZ3 = g (1 - t3^2) with g = dG0 (1 + Gt)
// into the dZ3 tiles (8-column groups: half 0 takes groups [0, GS), half 1
// [GS, G3)), and the skip part dh2[c % E1] += g of the owned units.
template <class S, int H>
struct EmbDz3 {
  using O = EmbOwn<S, H>;
  static constexpr int gs_lo = H == 0 ? 0 : S::GS, gs_hi = H == 0 ? S::GS : S::G3;  // stored 8-column groups
  // column quad c4 of dE/dG0 is read by this half
  __host__ __device__ static constexpr bool need4(int c4) {
    return c4 < S::E2 && ((((c4 >> 3) >= gs_lo && (c4 >> 3) < gs_hi)) || O::owns_c(c4) || O::owns_c(c4 + 1) ||
                          O::owns_c(c4 + 2) || O::owns_c(c4 + 3));
  }
  __host__ __device__ static constexpr bool any16(int k) {
    return need4(16 * k) || need4(16 * k + 4) || need4(16 * k + 8) || need4(16 * k + 12);
  }
};

// Index of column quad c4 of a row of an atom's dE/dG0 block (rm: row-major
// [NP][E2], else column-quad interleaved).
template <class S>
__device__ __forceinline__ int emb_dg4(bool rm, int c4, int row) {
  return rm ? row * (S::E2 / 4) + (c4 >> 2) : (c4 >> 2) * NP + row;
}

// This half's dE/dG0 column quads of 16-column chunk k of a row (zero where
// not read, or past nnei).
template <class S, int H>
__device__ __forceinline__ void embed_bwd_load16(const float4* dg, bool rm, int k, int row, bool rv, float4* d) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c4 = 16 * k + 4 * q;
    d[q] = EmbDz3<S, H>::need4(c4) && rv ? dg[emb_dg4<S>(rm, c4, row)] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Bring this half's dE/dG0 column quads of chunk k of a row into L1.
template <class S, int H>
__device__ __forceinline__ void embed_bwd_prefetch16(const float4* dg, bool rm, int k, int row, bool rv) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c4 = 16 * k + 4 * q;
    if (EmbDz3<S, H>::need4(c4) && rv)
      asm volatile("prefetch.global.L1 [%0];" ::"l"(dg + emb_dg4<S>(rm, c4, row)));
  }
}

// dE/dG0 of chunk 0 is loaded (and chunk 1 brought into L1) by the caller
// before it waits for Z3; chunk k + 1 is brought into L1 while chunk k is
// processed.
template <class S, bool F16, int H>
__device__ __forceinline__ void embed_bwd_dz3(const EmbedTcArgs& a, uint32_t taddr, const float* gt, const float4* dg,
                                              bool rv, int row, int slot, uint8_t* sDZ3h, uint8_t* sDZ3l, float* dh2,
                                              float4* dcur) {
  using O = EmbOwn<S, H>;
  using D = EmbDz3<S, H>;
#pragma unroll
  for (int k = 0; k < S::NK3; ++k) {
    if (k > 0 && D::any16(k)) embed_bwd_load16<S, H>(dg, a.rm, k, slot, rv, dcur);
    if (k + 2 < S::NK3 && D::any16(k + 2)) embed_bwd_prefetch16<S, H>(dg, a.rm, k + 2, slot, rv);
    if (D::any16(k)) {
    float z[16];
    tmem_ld16(taddr + 64 + 16 * k, z);
#pragma unroll
    for (int gg = 0; gg < 2; ++gg) {
      const int g = 2 * k + gg;
      const bool store = g >= D::gs_lo && g < D::gs_hi;
      float dz[8];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int c4 = 8 * g + 4 * q;
        bool need = store;
#pragma unroll
        for (int t = 0; t < 4; ++t) need |= O::owns_c(c4 + t);
        float gq[4] = {0.f, 0.f, 0.f, 0.f};
        if (need && c4 < S::E2 && rv) {
          const float4 d4 = dcur[2 * gg + q];
          const float4 t4 = *reinterpret_cast<const float4*>(gt + c4);
          gq[0] = d4.x * (1.f + t4.x); gq[1] = d4.y * (1.f + t4.y);
          gq[2] = d4.z * (1.f + t4.z); gq[3] = d4.w * (1.f + t4.w);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int c = c4 + t;
          if (O::owns_c(c)) dh2[c % S::E1 - O::b0] += gq[t];
          float d = 0.f;
          if (store && c < S::E2 && rv) {
            const float th = tanhf(z[8 * gg + 4 * q + t] + a.b2[c]);
            d = gq[t] * (1.f - th * th);
          }
          dz[4 * q + t] = d;
        }
      }
      if (store) {
        emb_store8<F16>(sDZ3h, row, 8 * g, 128, dz, false);
        emb_store8<F16>(sDZ3l, row, 8 * g, 128, dz, true);
      }
    }
    }
  }
}

// Adjoint of layer 2 for one half: d = dh2 (skip) + dH2 (product), the skip
// part of dh1, and dZ2 = d (1 - t2^2) into the dZ2 tiles for the owned units.
template <class S, bool F16, int H>
__device__ __forceinline__ void embed_bwd_dz2(uint32_t taddr, const float* h1, const float* h2, const float* dh2,
                                              bool rv, int row, uint8_t* sDZ2h, uint8_t* sDZ2l, float* dh1) {
  using O = EmbOwn<S, H>;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (16 * k + 15 < O::b0 || 16 * k >= 8 * O::g_hi) continue;
    float v[16];
    tmem_ld16(taddr + 16 * k, v);
#pragma unroll
    for (int gg = 0; gg < 2; ++gg) {
      const int g = 2 * k + gg;
      if (g < O::g_lo || g >= O::g_hi) continue;
      float dz[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int b = 8 * g + i;
        float d2 = 0.f;
        if (O::owns_b(b) && rv) {
          const float d = dh2[b - O::b0] + v[8 * gg + i];
          dh1[b % S::E0] += d;  // skip path of layer 2
          const float t = h2[b - O::b0] - h1[b % S::E0];
          d2 = d * (1.f - t * t);
        }
        dz[i] = d2;
      }
      emb_store8<F16>(sDZ2h, row, 8 * g, 128, dz, false);
      emb_store8<F16>(sDZ2l, row, 8 * g, 128, dz, true);
    }
  }
}

// rowg = atom * NP + slot: the row's place in the atom blocks (row is its
// place in the tile); pre() runs with the row's first loads, before the wait
// for Z3.
template <class S, bool F16, int H, class Pre>
__device__ __forceinline__ void embed_bwd_tail(const EmbedTcArgs& a, uint8_t* sm, uint32_t tm, uint32_t lane_off,
                                               Sync& sy, int row, bool rv, size_t rowg, const float* gt,
                                               const float4* dg, float* xch, Pre pre) {
  using O = EmbOwn<S, H>;
  const bool issuer = threadIdx.x == 0;
  uint8_t* sW1h = sm;
  uint8_t* sW1l = sW1h + S::T1;
  uint8_t* sW2h = sW1l + S::T1;
  uint8_t* sW2l = sW2h + S::T2;
  // the activation tiles are dead once Z3 = H2 W2 is in TMEM: dZ3 (hi, lo)
  // takes all four, then dZ2 (hi, lo) the first two once dH2 is computed
  uint8_t* sDZ3h = sm + S::WIMG;
  uint8_t* sDZ3l = sDZ3h + EMB_TD;
  uint8_t* sDZ2h = sm + S::WIMG;
  uint8_t* sDZ2l = sDZ2h + EMB_TA;
  float h1[S::E0], h2[O::nb];
  float4 d0[4];
  const int atom = (int)(rowg / NP), slot = (int)(rowg - (size_t)atom * NP);
  embed_bwd_front<S, F16, H>(a, sm, tm, sy, row, rv, atom, slot, h1, h2, [&] {
    embed_bwd_load16<S, H>(dg, a.rm, 0, slot, rv, d0);
    embed_bwd_prefetch16<S, H>(dg, a.rm, 1, slot, rv);
    pre();
  });
  float dh2[O::nb];
#pragma unroll
  for (int b = 0; b < O::nb; ++b) dh2[b] = 0.f;
  embed_bwd_dz3<S, F16, H>(a, tm + lane_off, gt, dg, rv, row, slot, sDZ3h, sDZ3l, dh2, d0);
  handoff();
  // dH2 (product part) = dZ3 W2^T -> TMEM [0, 64)
  if (issuer)
    mma_split<F16>(tm + 0, smem_u32(sDZ3h), smem_u32(sDZ3l), 128, smem_u32(sW2h), smem_u32(sW2l), true, S::E2P, 64,
                   S::NK3);
  commit_and_sync(sy, issuer);
  float dh1[S::E0];
#pragma unroll
  for (int p = 0; p < S::E0; ++p) dh1[p] = 0.f;
  embed_bwd_dz2<S, F16, H>(tm + lane_off, h1, h2, dh2, rv, row, sDZ2h, sDZ2l, dh1);
  handoff();
  // dH1 (product part) = dZ2 W1^T -> TMEM [64, 96)
  if (issuer)
    mma_split<F16>(tm + 64, smem_u32(sDZ2h), smem_u32(sDZ2l), 128, smem_u32(sW1h), smem_u32(sW1l), true, 64, 32, 4);
  commit_and_sync(sy, issuer);
  float v[32];
  tmem_ld16(tm + lane_off + 64, v);
  tmem_ld16(tm + lane_off + 80, v + 16);
  float dx = 0.f;
  if (rv) {
#pragma unroll
    for (int p = 0; p < S::E0; ++p) dx = fmaf(a.W0[p] * (1.f - h1[p] * h1[p]), dh1[p] + (H == 0 ? v[p] : 0.f), dx);
  }
  // half 1 hands its part to half 0, which owns the row's dR update
  if (H == 1) xch[row] = dx;
  __syncthreads();
  // one writer per row in a launch: a reduction without a return (the same
  // FP32 add as a load, add and store, without waiting for the load)
  if (H == 0 && rv) atomicAdd(a.dR + rowg * 4, dx + xch[row]);
}

template <class S, bool F16>
__global__ void __launch_bounds__(EMB_THREADS, S::MIN_CTAS) k_embed_tc_bwd(const __grid_constant__ EmbedTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint64_t* bar;
  uint32_t* s_tmem;
  embed_tc_setup<S>(a, sm, bar, s_tmem, S::B_SMEM);
  const uint32_t tm = *s_tmem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  float* s_gt = reinterpret_cast<float*>(sm + S::WIMG + 4 * EMB_TA);
  float* xch = s_gt + EMB_MAXT * S::E2;  // [128] half 1's part of dE/dx
  Sync sy{bar, 0u, a.err};
  if (threadIdx.x == 0 && blockIdx.x < a.n)
    prefetch_l2(a.dG0 + (size_t)blockIdx.x * NP * S::E2, NP * S::E2 * sizeof(float));
  EmbRowIn in;
  in.count(a, blockIdx.x);
  in.rows(a, blockIdx.x, row);
  in.type(a, row);
  for (int atom = blockIdx.x; atom < a.n && sy.ok; atom += gridDim.x) {
    const EmbRowIn cur = in;
    const int nn = cur.nn, tj = cur.tj, next = atom + gridDim.x;
    in.count(a, next);
    in.rows(a, next, row);
    if (nn == 0) {  // uniform over the CTA
      in.type(a, row);
      continue;
    }
    const bool rv = row < nn;
    const size_t rowg = (size_t)atom * NP + row;
    embed_tc_atom_start<S>(a, s_gt, nullptr, atom, true);  // visible after the front's barriers
    const float4* dg = reinterpret_cast<const float4*>(a.dG0 + (size_t)atom * NP * S::E2);
    if (half == 0)
      embed_bwd_tail<S, F16, 0>(a, sm, tm, lane_off, sy, row, rv, rowg, s_gt + tj * S::E2, dg, xch, [] {});
    else
      embed_bwd_tail<S, F16, 1>(a, sm, tm, lane_off, sy, row, rv, rowg, s_gt + tj * S::E2, dg, xch, [] {});
    in.type(a, row);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

// ------------------------------------------------- live-row tiles
// The net treats every neighbour row on its own, so its tiles need not
// follow the atoms: the live-row kernels below take 128 live rows at a time
// from one list of all atoms' live rows (atom * NP + slot), so that no lane
// of a tile holds a row past its atom's last neighbour (with 72-103
// neighbours per atom, per-atom tiles leave lane quadrant 3, and with it
// one of the SM's four schedulers, idle).  A row's results do not depend on
// where in the list it is or which rows share its tile: every product row
// and every element-wise step is the row's own.

constexpr int LR_THREADS = 256;

// The list: each block takes LR_THREADS atoms, reserves room for their live
// rows with one atomic add and writes them, an atom's slots in order.  The
// blocks' order in the list is that of their reservations.
__global__ void __launch_bounds__(LR_THREADS) k_live_rows(const int* __restrict__ nnei, int n, int* __restrict__ count,
                                                          int* __restrict__ rows) {
  __shared__ int s_warp[LR_THREADS / 32];
  __shared__ int s_base;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int first = blockIdx.x * LR_THREADS;
  const int nn = first + t < n ? nnei[first + t] : 0;
  int x = nn;  // inclusive sum over the warp's atoms
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (t == 0) {
    int tot = 0;
    for (int k = 0; k < LR_THREADS / 32; ++k) {
      const int c = s_warp[k];
      s_warp[k] = tot;
      tot += c;
    }
    s_base = tot > 0 ? atomicAdd(count, tot) : 0;
  }
  __syncthreads();
  const int off = s_base + s_warp[w] + x - nn;  // this atom's first place in the list
  for (int j = 0; j < 32; ++j) {                // the warp writes its atoms one at a time
    const int nj = __shfl_sync(0xffffffffu, nn, j), oj = __shfl_sync(0xffffffffu, off, j);
    const int aj = first + 32 * w + j;
    for (int s = lane; s < nj; s += 32) rows[oj + s] = aj * NP + s;
  }
}

// A row of a live-row tile: its place in the atom blocks (rg = atom * NP +
// slot, -1 past the end of the list), s, and the centre and neighbour types.
// map() reads the list for the next tile, rows() its s and neighbour index
// once map's load is back, type() the types at the end of the current tile.
struct LiveRowIn {
  int rg = -1, nl = 0, atom = 0, slot = 0, ti = 0, tj = 0;
  float x = 0.f;
  __device__ void map(const EmbedTcArgs& a, int nrows, int tile, int row) {
    const long long r = (long long)tile * 128 + row;
    rg = r < nrows ? a.rowmap[r] : -1;
  }
  __device__ void rows(const EmbedTcArgs& a, bool need_x) {
    if (rg >= 0) {
      if (need_x) x = a.R[(size_t)rg * 4];
      nl = a.nlist[rg];
    }
  }
  __device__ void type(const EmbedTcArgs& a) {
    const bool v = rg >= 0;
    atom = v ? rg / NP : 0;
    slot = v ? rg - atom * NP : 0;
    ti = v ? a.atype[atom] : 0;
    tj = v ? a.atype[nl] : 0;
    x = v ? x : 0.f;
  }
  // the row's entry of the type-pair table (and of the first-layer bias
  // table in concat mode): small tables, read through L1
  __device__ const float* gt(const EmbedTcArgs& a, int e2) const {
    return a.Gt + ((size_t)ti * a.ntypes + tj) * e2;
  }
};

template <class S>
__global__ void __launch_bounds__(EMB_THREADS, S::MIN_CTAS) k_embed_tc_fwd_live(const __grid_constant__ EmbedTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint64_t* bar;
  uint32_t* s_tmem;
  embed_tc_setup<S>(a, sm, bar, s_tmem, S::F_SMEM);
  const uint32_t tm = *s_tmem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  Sync sy{bar, 0u, a.err};
  const int nrows = *a.nrows;
  const int ntiles = (nrows + 127) / 128;
  float h1[S::E0], h2[S::E1 - S::SPLIT];
  LiveRowIn in;
  in.map(a, nrows, blockIdx.x, row);
  in.rows(a, true);
  in.type(a);
  for (int tile = blockIdx.x; tile < ntiles && sy.ok; tile += gridDim.x) {
    const LiveRowIn cur = in;
    const bool rv = cur.rg >= 0;
    in.map(a, nrows, tile + gridDim.x, row);
    auto rows_next = [&] { in.rows(a, true); };
    const float* b0row = a.b0t && rv ? a.b0t + ((size_t)cur.ti * a.ntypes + cur.tj) * S::E0 : nullptr;
    if (half == 0)
      embed_tc_front<S, true, 0>(a, sm, tm, lane_off, sy, row, rv, cur.x, b0row, h1, h2, rows_next);
    else
      embed_tc_front<S, true, 1>(a, sm, tm, lane_off, sy, row, rv, cur.x, b0row, h1, h2, rows_next);
    if (rv) {  // layers 1 and 2 of the row for the adjoint, as the per-atom kernel stores them
      float* hs = a.H12 + (size_t)cur.atom * (S::E0 + S::E1) * NP + cur.slot;
      if (half == 0) {
#pragma unroll
        for (int p = 0; p < 16; ++p) __stcs(hs + p * NP, h1[p]);
#pragma unroll
        for (int i = 0; i < S::SPLIT; ++i) __stcs(hs + (S::E0 + i) * NP, h2[i]);
      } else {
#pragma unroll
        for (int p = 16; p < S::E0; ++p) __stcs(hs + p * NP, h1[p]);
#pragma unroll
        for (int i = 0; i < S::E1 - S::SPLIT; ++i) __stcs(hs + (S::E0 + S::SPLIT + i) * NP, h2[i]);
      }
    }
    float* out = a.G0 + (size_t)cur.atom * NP * S::E2;
    if (half == 0)
      embed_fwd_out<S, 0>(a, tm + lane_off, cur.gt(a, S::E2), h2, rv, out, cur.slot);
    else
      embed_fwd_out<S, 1>(a, tm + lane_off, cur.gt(a, S::E2), h2, rv, out, cur.slot);
    in.type(a);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

template <class S>
__global__ void __launch_bounds__(EMB_THREADS, S::MIN_CTAS) k_embed_tc_bwd_live(const __grid_constant__ EmbedTcArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint64_t* bar;
  uint32_t* s_tmem;
  embed_tc_setup<S>(a, sm, bar, s_tmem, S::B_SMEM);
  const uint32_t tm = *s_tmem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  float* xch = reinterpret_cast<float*>(sm + S::WIMG + 4 * EMB_TA) + EMB_MAXT * S::E2;  // [128] half 1's dE/dx
  Sync sy{bar, 0u, a.err};
  const int nrows = *a.nrows;
  const int ntiles = (nrows + 127) / 128;
  LiveRowIn in;
  in.map(a, nrows, blockIdx.x, row);
  in.rows(a, false);
  in.type(a);
  for (int tile = blockIdx.x; tile < ntiles && sy.ok; tile += gridDim.x) {
    const LiveRowIn cur = in;
    const bool rv = cur.rg >= 0;
    in.map(a, nrows, tile + gridDim.x, row);
    // with the row's first loads: the next tile's neighbour indices, and its
    // atoms' dE/dG0 and layer blocks brought into L2 (by the thread of an
    // atom's first row in that tile)
    auto pre = [&] {
      in.rows(a, false);
      if (half == 0 && in.rg >= 0) {
        const int at = in.rg / NP;
        if (row == 0 || in.rg == at * NP) {
          prefetch_l2(a.dG0 + (size_t)at * NP * S::E2, NP * S::E2 * sizeof(float));
          prefetch_l2(a.H12 + (size_t)at * (S::E0 + S::E1) * NP, NP * (S::E0 + S::E1) * sizeof(float));
        }
      }
    };
    const size_t rowg = rv ? (size_t)cur.rg : 0;
    const float4* dg = reinterpret_cast<const float4*>(a.dG0 + (size_t)cur.atom * NP * S::E2);
    if (half == 0)
      embed_bwd_tail<S, true, 0>(a, sm, tm, lane_off, sy, row, rv, rowg, cur.gt(a, S::E2), dg, xch, pre);
    else
      embed_bwd_tail<S, true, 1>(a, sm, tm, lane_off, sy, row, rv, rowg, cur.gt(a, S::E2), dg, xch, pre);
    in.type(a);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 256);
}

}  // namespace

namespace {
// The hi and lo parts of W1 and W2 of a net of shape S as swizzled K-major
// tiles (W1 as [E1 (64 rows)][E0 (K)], W2 as [E2P rows][E1 (K)]), in FP16
// (f16) or BF16.
template <class S>
std::vector<uint8_t> emb_image(const std::vector<double>& W1, const std::vector<double>& W2, bool f16) {
  std::vector<uint8_t> img(S::WIMG, 0);
  auto put = [&](int off, int r, int c, int R, double x, bool lo) {
    if (f16) {
      const __half hi = __float2half((float)x);
      const __half v = lo ? __float2half((float)(x - (double)__half2float(hi))) : hi;
      memcpy(img.data() + off + sw128_offset(r, c, R), &v, 2);
    } else {
      const __nv_bfloat16 hi = __float2bfloat16((float)x);
      const __nv_bfloat16 v = lo ? __float2bfloat16((float)(x - (double)__bfloat162float(hi))) : hi;
      memcpy(img.data() + off + sw128_offset(r, c, R), &v, 2);
    }
  };
  for (int b = 0; b < S::E1; ++b)
    for (int p = 0; p < S::E0; ++p) {
      put(0, b, p, 64, W1[(size_t)p * S::E1 + b], false);
      put(S::T1, b, p, 64, W1[(size_t)p * S::E1 + b], true);
    }
  for (int c = 0; c < S::E2; ++c)
    for (int b = 0; b < S::E1; ++b) {
      put(2 * S::T1, c, b, S::E2P, W2[(size_t)b * S::E2 + c], false);
      put(2 * S::T1 + S::T2, c, b, S::E2P, W2[(size_t)b * S::E2 + c], true);
    }
  return img;
}

template <class S>
void emb_set_smem() {
  cudaFuncSetAttribute(k_embed_tc_fwd<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::F_SMEM);
  cudaFuncSetAttribute(k_embed_tc_bwd<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::B_SMEM);
  cudaFuncSetAttribute(k_embed_tc_fwd_live<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::F_SMEM);
  cudaFuncSetAttribute(k_embed_tc_bwd_live<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::B_SMEM);
}

template <class S>
bool emb_is(const dp_model* m) {
  return m->emb[0] == S::E0 && m->emb[1] == S::E1 && m->emb[2] == S::E2;
}
}  // namespace

// Weight images of the tensor-core embedding net (the 25-50-100 and
// 32-64-128 nets with at most EMB_MAXT types): the hi and lo parts of W1 and
// W2 in FP16 (the fused 16-bit paths) and in BF16 (the bf16x mode), and its
// per-unit vectors.  Other nets keep both images null (FP32 SIMT kernels).
int tc_init_embedding(dp_model* m, const HostArrays& arrays, std::string& msg) {
  auto get = [&](const std::string& name) -> const std::vector<double>& {
    for (auto& kv : arrays)
      if (kv.first == name) return kv.second;
    static std::vector<double> empty;
    return empty;
  };
  TcWeights& w = m->tcw;
  w.emb_W1_t = nullptr;
  w.emb_W2_t = nullptr;
  const bool s100 = emb_is<EmbS100>(m), s128 = emb_is<EmbS128>(m);
  if (!(s100 || s128) || m->nt > EMB_MAXT) return DP_OK;
  const std::vector<double>& W1 = get("em_W1");  // [E0][E1]
  const std::vector<double>& W2 = get("em_W2");  // [E1][E2]
  for (int f16 = 1; f16 >= 0; --f16) {  // FP16 image (fused paths), BF16 image (bf16x)
    const std::vector<uint8_t> img = s100 ? emb_image<EmbS100>(W1, W2, f16 != 0) : emb_image<EmbS128>(W1, W2, f16 != 0);
    void* d = nullptr;
    if (cudaMalloc(&d, img.size()) != cudaSuccess ||
        cudaMemcpy(d, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      msg = "cudaMalloc of the embedding weight image failed";
      return DP_ERR_CUDA;
    }
    w.allocations.push_back(d);
    (f16 ? w.emb_W1_t : w.emb_W2_t) = d;
  }
  const std::vector<double>& W0 = get("em_W0");
  const std::vector<double>& b0 = get("em_b0");
  const std::vector<double>& b1 = get("em_b1");
  const std::vector<double>& b2 = get("em_b2");
  for (int q = 0; q < m->emb[0]; ++q) { w.emb_vec.W0[q] = (float)W0[q]; w.emb_vec.b0[q] = (float)b0[q]; }
  for (int q = 0; q < m->emb[1]; ++q) w.emb_vec.b1[q] = (float)b1[q];
  for (int q = 0; q < m->emb[2]; ++q) w.emb_vec.b2[q] = (float)b2[q];
  if (s100)
    emb_set_smem<EmbS100>();
  else
    emb_set_smem<EmbS128>();
  return DP_OK;
}

namespace {
// One launch of the tensor-core embedding net, forward or adjoint: live-row
// tiles with FP16 operand splits (the fused 16-bit paths, given a row list),
// or per-atom tiles with BF16 ones (bf16x).
template <class S>
void tc_embed_launch_s(int grid, const EmbedTcArgs& et, bool bwd, cudaStream_t st) {
  if (et.rowmap) {
    if (!bwd) k_embed_tc_fwd_live<S><<<grid, EMB_THREADS, S::F_SMEM, st>>>(et);
    if (bwd) k_embed_tc_bwd_live<S><<<grid, EMB_THREADS, S::B_SMEM, st>>>(et);
  } else {
    if (!bwd) k_embed_tc_fwd<S, false><<<grid, EMB_THREADS, S::F_SMEM, st>>>(et);
    if (bwd) k_embed_tc_bwd<S, false><<<grid, EMB_THREADS, S::B_SMEM, st>>>(et);
  }
}

void tc_embed_launch(dp_model* m, const EmbedTcArgs& et, bool bwd, cudaStream_t st) {
  const int per_sm = emb_is<EmbS100>(m) ? EmbS100::MIN_CTAS : EmbS128::MIN_CTAS;
  // at most n tiles either way: n atoms, or n * NP live rows at most
  const int grid = std::min(et.n, per_sm * emb_sm_count(m->device));
  if (emb_is<EmbS100>(m))
    tc_embed_launch_s<EmbS100>(grid, et, bwd, st);
  else
    tc_embed_launch_s<EmbS128>(grid, et, bwd, st);
  note_launch();
}

EmbedTcArgs embed_tc_args(dp_model* m, int n, const int* atype) {
  Workspace& ws = m->ws;
  EmbedTcArgs et{};
  et.R = ws.R; et.nlist = ws.nlist; et.nnei = ws.nnei; et.atype = atype; et.Gt = m->Gt;
  et.n = n; et.ntypes = m->nt; et.err = m->d_err; et.b0t = m->b0t;
  memcpy(et.W0, m->tcw.emb_vec.W0, sizeof(et.W0));
  memcpy(et.b0, m->tcw.emb_vec.b0, sizeof(et.b0));
  memcpy(et.b1, m->tcw.emb_vec.b1, sizeof(et.b1));
  memcpy(et.b2, m->tcw.emb_vec.b2, sizeof(et.b2));
  return et;
}
}  // namespace

// The embedding net of the bf16x mode on the tensor cores (BF16 hi + lo
// splits of both operands), G0 and dE/dG0 row-major: forward, or adjoint
// (dR[:, 0] +=).  H12 holds the layers the adjoint reads back.
void tc_embed_bf16(dp_model* m, int n, const int* atype, bool bwd, float* G0, const float* dG0, float* dR,
                   float* H12, cudaStream_t st) {
  if (n == 0) return;
  EmbedTcArgs et = embed_tc_args(m, n, atype);
  et.G0 = G0; et.dG0 = dG0; et.dR = dR; et.H12 = H12; et.rm = 1;
  et.wimg = reinterpret_cast<const uint4*>(m->tcw.emb_W2_t);
  tc_embed_launch(m, et, bwd, st);
}


// The list of live neighbour rows the fused paths' embedding net runs over
// (after the neighbour list, before the net's forward; its adjoint reads the
// same list).
void tc_live_rows(dp_model* m, int n, cudaStream_t st) {
  if (n == 0) return;
  Workspace& ws = m->ws;
  int* count = reinterpret_cast<int*>(ws.tc.p[7]);
  cudaMemsetAsync(count, 0, sizeof(int), st);
  k_live_rows<<<(n + LR_THREADS - 1) / LR_THREADS, LR_THREADS, 0, st>>>(ws.nnei, n, count,
                                                                          reinterpret_cast<int*>(ws.tc.p[6]));
  note_launch();
}

// The embedding net of the fused 16-bit paths on the tensor cores (FP16 hi +
// lo splits) over the live-row tiles of tc_live_rows, G0 and dE/dG0
// column-quad interleaved per atom: forward (G0 -> G[0]), or adjoint (dE/dG0
// from dG, dR[:, 0] +=).
void tc_embed_fused(dp_model* m, int n, const int* atype, bool bwd, cudaStream_t st) {
  if (n == 0) return;
  Workspace& ws = m->ws;
  EmbedTcArgs et = embed_tc_args(m, n, atype);
  et.G0 = ws.G[0]; et.dG0 = ws.dG; et.dR = ws.dR; et.rm = 0; et.live_only = 1;
  et.rowmap = reinterpret_cast<const int*>(ws.tc.p[6]);
  et.nrows = reinterpret_cast<const int*>(ws.tc.p[7]);
  et.H12 = reinterpret_cast<float*>(ws.tc.p[5]);
  et.wimg = reinterpret_cast<const uint4*>(m->tcw.emb_W1_t);
  tc_embed_launch(m, et, bwd, st);
}

}  // namespace dpa1
