// Tensor-core (tcgen05, 16-bit operands, FP32 accumulation in TMEM) path of
// the gated attention layers (stage a6) and their adjoint (stage a12).
// Two operand modes: plain BF16, and FP16 with two-term (hi + lo) splits of
// the layer input G, the attention weights P and the output weights Wvo in the
// forward products, whose rounding the LayerNorm of weakly attended rows
// amplifies.
//
// One persistent CTA per SM walks over centre atoms; an atom is one 128-row
// tile (its neighbour slots).  Every product of a layer runs on the tensor
// cores from 128x128 16-bit tiles in shared memory.  With V = G Wv + bv,
// O Wo = P V Wo = [P G, rowsum P] [Wv Wo; bv Wo], so the values V are never
// formed:
//   forward : [Q K] = G [Wq Wk], S = Q K^T, PG = P [G 1], Y = PG Wvo
//   backward: [Q K] and S recomputed, dPG = dY Wvo^T, dP = dPG [G 1]^T,
//             dQ = dS K, dK = dS^T Q,
//             dG = dQ Wq^T + dK Wk^T + P^T dPG
// The transposed operands are MN-major views of the same tiles, so no
// transpose is ever materialised.  Softmax, LayerNorm and all element-wise
// work run in FP32 on 512 threads (a thread owns a quarter of a row: 32
// columns of one TMEM lane).  The embedding net (stages a5, a13) is in
// tc_embed.cu.
#include <cuda_bf16.h>

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

constexpr int NT = 512;           // threads per CTA of the layer kernels
constexpr int TILE = 32768;       // 128 x 128 bf16 SW128 tile
constexpr int WO_ROWS = 112;      // Wvo tile: M1 = 100 output rows padded to 112
constexpr int WO_TILE = 2 * WO_ROWS * 128;  // 28 KB
// per-layer weight image (bytes): [Wq; Wk], then Wvo = [Wv Wo; bv Wo] and its
// rounding residue Wvo - round16(Wvo) (the low part of a two-term split)
constexpr int WV_OFF = 2 * TILE;
constexpr int WIMG = WV_OFF + 2 * WO_TILE;
constexpr int KS_M1 = 7;          // K-steps covering the M1 = 100 (<= 112) inputs

struct LayerArgs {
  const float* Gin;        // [rows][m1] layer input
  float* Gout;             // fwd: [rows][m1] layer output
  __nv_bfloat16* yhat;     // normalised LayerNorm input, [NP][yld] per atom in 8-column groups (fwd writes, bwd reads)
  float* rstd;             // [rows]
  float2* smax;            // [rows] softmax row max and 1 / normaliser (fwd writes, bwd reads)
  float* dG;               // bwd: in dE/dG_{l+1}, out dE/dG_l (in place)
  float* dgeo;             // bwd: [rows][4] += (d rhat, d w)
  const float* rw;         // [rows][4] (rhat, w)
  const int* nnei;
  int n, m1, yld;          // yld = m1 rounded up to a multiple of 8
  const uint4* wimg;       // swizzled weight image of this layer
  float scale, shift, eps;
  int* err;
  // per-feature vectors, passed by value (constant bank: every lane of a warp
  // reads the same feature at the same time)
  float bo[128];
  float gamma[128];
  float beta[128];
};

// G_l, G_{l+1} and dE/dG are column-quad interleaved per atom (cq_off);
// yhat likewise in groups of 8 bf16 columns: element (r, c) of an atom at
// ((c / 8) * NP + r) * 8 + c % 8.  A warp's per-row 16-byte accesses are then
// 512 contiguous bytes.  Only an atom's live rows (its first nnei) of these
// blocks and of rstd and smax are read or written: the rows past them stay
// as they were (the layer input's are treated as zeros), which leaves every
// live row's result unchanged, since the attention weights of keys past the
// last neighbour are exact zeros.
__host__ __device__ constexpr int yhat_ld(int m1) { return (m1 + 7) & ~7; }

// Bring the per-row inputs of centre atom `atom` (if it exists) into L2 ahead
// of its turn: one thread, bulk prefetches of whole blocks.  (Prefetching the
// live rows alone takes one prefetch per column quad, ~60 instead of 6 per
// atom, and the issuing warp, which holds the MMA issuer, then stalls for
// longer than the prefetches save.)
__device__ __forceinline__ void prefetch_atom(const LayerArgs& a, int atom, bool bwd) {
  if (atom >= a.n) return;
  const size_t base = (size_t)atom * NP;
  prefetch_l2(a.Gin + base * a.m1, (uint32_t)(NP * a.m1 * sizeof(float)));
  prefetch_l2(a.rw + base * 4, (uint32_t)(NP * 4 * sizeof(float)));
  if (bwd) {
    prefetch_l2(a.dG + base * a.m1, (uint32_t)(NP * a.m1 * sizeof(float)));
    prefetch_l2(a.yhat + base * a.yld, (uint32_t)(NP * a.yld * sizeof(__nv_bfloat16)));
    prefetch_l2(a.rstd + base, (uint32_t)(NP * sizeof(float)));
    prefetch_l2(a.smax + base, (uint32_t)(NP * sizeof(float2)));
  }
}

// ------------------------------------------------------------------ forward
// Shared memory: slots A-D [0,128K), Wq, Wk [128K,192K), then the per-key
// (rhat, w) table and the barriers.  Slot use per atom: G (hi, lo) in A, B
// until P G is formed; Q, K in C, D; P (hi, lo) in C, D; then P G in A and
// Wvo, streamed per atom by a bulk asynchronous copy, in D (its residue in
// C).  TMEM columns: [Q K] accumulators 0-255 (S and P G reuse 0-127) and Y
// at 256-367, where it waits for its LayerNorm: an atom's LayerNorm runs
// while the next atom's [Q K] product is on the tensor cores.
// Thread layout: warp w owns TMEM lane quadrant w % 4 (rows 32 (w % 4) ..
// +31) and column quarter w / 4 (32 columns).
constexpr int F_SLOT_A = 0, F_SLOT_B = TILE, F_SLOT_C = 2 * TILE, F_SLOT_D = 3 * TILE, F_W = 4 * TILE;
constexpr int F_SMALL = 6 * TILE;
constexpr int F_SMEM = F_SMALL + 2048 + 64;

// F16 = true: FP16 operands with two-term splits of G (in [Q K] = G [Wq Wk]
// and P G) and of P; F16 = false: plain BF16 operands.
template <bool F16>
__global__ void __launch_bounds__(NT, 1) k_layer_fwd_tc(const __grid_constant__ LayerArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {  // tiles need 1024-byte alignment
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint8_t* sA = sm + F_SLOT_A;
  uint8_t* sB = sm + F_SLOT_B;
  uint8_t* sC = sm + F_SLOT_C;
  uint8_t* sD = sm + F_SLOT_D;
  uint8_t* sWqk = sm + F_W;  // [Wq; Wk], 256 rows
  float4* s_key = reinterpret_cast<float4*>(sm + F_SMALL);  // [128] (rhat_x, rhat_y, rhat_z, w)
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_key + 128);  // [6]: general, Wvo copy, Q K, Q K out, (unused), inputs
  uint64_t* bar_ld = bar + 1;
  uint64_t* bar_q = bar + 2;
  uint64_t* bar_in = bar + 5;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 6);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2;
  const int row = quad * 32 + lane;
  const int c0 = part * 32;
  // The MMA issuer stalls while the tensor pipe's queue is full: it lives in
  // the warp with the least element-wise work (rows 96-127 are past the
  // last neighbour of most atoms, columns 96-127 past the embedding width)
  const bool issuer = tid == NT - 32;

  copy_image(sWqk, a.wimg, 2 * TILE);
  if (issuer) {
    for (int i = 0; i < 6; ++i) mbar_init(bar + i, i == 3 ? NT / 32 : 1);  // [3]: one arrival per warp
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(s_tmem, 512);
  handoff();
  const uint32_t tm = *s_tmem;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  const uint32_t tA = smem_u32(sA), tB = smem_u32(sB), tC = smem_u32(sC), tD = smem_u32(sD);
  const uint32_t tWqk = smem_u32(sWqk);
  const uint4* wo_img = a.wimg + WV_OFF / 16;
  Sync sy{bar, 0u, a.err};
  Sync sl{bar_ld, 0u, a.err};
  Sync sq{bar_q, 0u, a.err};
  Sync so{bar_q + 1, 0u, a.err};  // Q and K are out of TMEM: waited on by the issuer only
  Sync si{bar_in, 0u, a.err};
  const uint32_t g_bytes = (uint32_t)(NP * a.m1 * sizeof(float)), k_bytes = NP * sizeof(float4);
  // An atom's layer input (its column-quad interleaved block, as stored) and
  // its per-key (rhat, w) rows (zero past nnei) arrive by bulk copies: into
  // slots C..D and the key table, during the previous atom's LayerNorm.  One
  // copy of the whole block: its rows past the last neighbour hold whatever
  // was there and are replaced by zeros when read.
  auto fetch_inputs = [&](int at) {
    const size_t b = (size_t)at * NP;
    mbar_expect_tx(bar_in, g_bytes + k_bytes);
    bulk_g2s(sC, a.Gin + b * a.m1, g_bytes, bar_in);
    bulk_g2s(s_key, a.rw + b * 4, k_bytes, bar_in);
  };
  if (issuer && (int)blockIdx.x < a.n) fetch_inputs(blockIdx.x);
  // neighbour counts are read one atom ahead
  int nn_next = (int)blockIdx.x < a.n ? a.nnei[blockIdx.x] : 0;
  // LayerNorm and residual of an atom whose Y = P G Wvo is in TMEM [256,
  // 368): G_l+1 = G_l + LN(w_j Y + bo) on its live rows (G_l read again, from
  // L2), and the normalised input yhat and 1 / sigma for the adjoint.  The
  // row exchanges park in slot C, which is free between the layer input's
  // copy and Q (a row's line is only touched by that row's four threads, and
  // each exchange ends with their barrier).
  auto layer_norm_out = [&](size_t lbase, int lnn, float lw) {
    const bool lrv = row < lnn;
    const RowXchg xr(sC, row, part, lane, quad);
    float v[32];
    tmem_ld32(tm + lane_off + 256 + c0, v);
    float s1 = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int c = c0 + i;
      v[i] = c < a.m1 ? lw * v[i] + a.bo[c] : 0.f;
      s1 += v[i];
    }
    const float mean = xr.sum(s1) / (float)a.m1;
    float s2 = 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const int c = c0 + i;
      const float d = c < a.m1 ? v[i] - mean : 0.f;
      s2 += d * d;
    }
    const float var = xr.sum(s2) / (float)a.m1;
    const float rs = 1.0f / sqrtf(var + a.eps);
    float4* gout = reinterpret_cast<float4*>(a.Gout + lbase * a.m1);
    uint4* yh = reinterpret_cast<uint4*>(a.yhat + lbase * a.yld);
    float gin[32];
    load_cq32(a.Gin + lbase * a.m1, a.m1, row, c0, gin, lrv);
#pragma unroll
    for (int i = 0; i < 32; i += 8) {
      const int c = c0 + i;
      if (c < a.m1 && lrv) {
        float y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) y[k] = c + k < a.m1 ? (v[i + k] - mean) * rs : 0.f;
#pragma unroll
        for (int h = 0; h < 8; h += 4) {
          const int cc = c + h;
          if (cc < a.m1) {
            float4 g = make_float4(gin[i + h], gin[i + h + 1], gin[i + h + 2], gin[i + h + 3]);
            g.x += y[h] * a.gamma[cc] + a.beta[cc];
            g.y += y[h + 1] * a.gamma[cc + 1] + a.beta[cc + 1];
            g.z += y[h + 2] * a.gamma[cc + 2] + a.beta[cc + 2];
            g.w += y[h + 3] * a.gamma[cc + 3] + a.beta[cc + 3];
            gout[(cc >> 2) * NP + row] = g;
          }
        }
        uint4 u;
        u.x = pack_bf16(y[0], y[1]);
        u.y = pack_bf16(y[2], y[3]);
        u.z = pack_bf16(y[4], y[5]);
        u.w = pack_bf16(y[6], y[7]);
        yh[(c >> 3) * NP + row] = u;
      }
    }
    if (part == 0 && lrv) a.rstd[lbase + row] = rs;
  };
  // the atom whose LayerNorm is pending
  bool have_prev = false;
  size_t prev_base = 0;
  int prev_nn = 0;
  float prev_w = 0.f;

  for (int atom = blockIdx.x; atom < a.n && sy.ok; atom += gridDim.x) {
    const int nn = nn_next;
    const size_t base = (size_t)atom * NP;
    const int next = atom + (int)gridDim.x;
    const bool rv = row < nn;
    if (issuer) prefetch_atom(a, next, false);
    si.wait();
    float v[32];
    // G_l (FP32) -> 16-bit slot A (+ its rounding residue in slot B); rows
    // past the last neighbour as zeros
    load_cq32(reinterpret_cast<const float*>(sC), a.m1, row, c0, v, rv);
    set_bias_ones(v, c0, a.m1);
    store_row32<F16>(sA, row, c0, v);
    if (F16) store_row32<F16, true>(sB, row, c0, v);
    handoff();
    // [Q K] = G [Wq Wk] (N = 256, + the G_lo product)
    if (issuer) {
      mma_block<F16>(tm + 0, tA, false, 128, tWqk, false, 256, 256, KS_M1, false);
      if (F16) mma_block<F16>(tm + 0, tB, false, 128, tWqk, false, 256, 256, KS_M1, true);
      mma_commit(bar_q);
    }
    // meanwhile: the previous atom's LayerNorm
    if (have_prev) layer_norm_out(prev_base, prev_nn, prev_w);
    // Q -> C, K -> D (G stays in A, B for P G)
    sq.wait();
    tmem_ld32(tm + lane_off + 0 + c0, v);
    store_row32<F16>(sC, row, c0, v);
    tmem_ld32(tm + lane_off + 128 + c0, v);
    store_row32<F16>(sD, row, c0, v);
    // an arrival per warp, then S = Q K^T -> TMEM [0,128)
    warp_arrive(bar_q + 1);
    if (issuer) {
      if (so.wait()) mma_block<F16>(tm + 0, tC, false, 128, tD, false, 128, 128, 8, false);
      mma_commit(bar);
    }
    sy.wait();
    // smooth softmax and gate: P -> slot C (+ P_lo -> slot D); Q and K are dead.
    // Row j of P carries the factor w_j, which vanishes for neighbours near
    // rcut; the tiles hold P / w_j instead (no FP16 subnormals), and w_j is
    // applied to Y = (P / w_j) G Wvo in FP32 before the LayerNorm.
    tmem_ld32(tm + lane_off + 0 + c0, v);
    float w_row;
    {
      const RowXchg xr(sC, row, part, lane, quad);
      const float4 kj = s_key[row];
      const float wj = kj.w;
      w_row = wj;
      // a column quarter past the last neighbour, or a lane quadrant whose
      // rows are all past it, has nothing to compute
      const bool live = c0 < nn && quad * 32 < nn;
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
      if (part == 0 && rv) a.smax[base + row] = make_float2(mx, inv);
      if (live) {
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float4 kk = s_key[c0 + i];
          const float c = kj.x * kk.x + kj.y * kk.y + kj.z * kk.z;
          v[i] = v[i] * inv * kk.w * c;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      store_row32<F16>(sC, row, c0, v);
      if (F16) store_row32<F16, true>(sD, row, c0, v);
    }
    handoff();
    // P G = P [G 1 1] (+ P_lo G + P G_lo) -> TMEM [0, 112) (G as an MN-major
    // operand; its columns M1, M1 + 1 are 1, so those of P G are rowsum P)
    if (issuer) {
      mma_block<F16>(tm + 0, tC, false, 128, tA, true, 128, WO_ROWS, 8, false);
      if (F16) {
        mma_block<F16>(tm + 0, tD, false, 128, tA, true, 128, WO_ROWS, 8, true);
        mma_block<F16>(tm + 0, tC, false, 128, tB, true, 128, WO_ROWS, 8, true);
      }
    }
    commit_and_sync(sy, issuer);
    // Wvo -> slot D (bulk copy, P_lo is dead) while P G leaves TMEM -> A; with
    // FP16 operands also the residue of Wvo -> slot C (P is dead): rounding the
    // weights themselves to FP16 would shift the atomic energies by up to
    // ~1e-3 eV.  Columns past 112 of the P G tile are never read (K = 112).
    if (issuer) {
      mbar_expect_tx(bar_ld, F16 ? 2 * WO_TILE : WO_TILE);
      bulk_g2s(sD, wo_img, WO_TILE, bar_ld);
      if (F16) bulk_g2s(sC, wo_img + WO_TILE / 16, WO_TILE, bar_ld);
    }
    tmem_ld32(tm + lane_off + 0 + c0, v);
    store_row32<F16>(sA, row, c0, v);
    handoff();
    // Y = P G Wvo (+ P G Wvo_lo) -> TMEM [256, 368)
    if (issuer && sl.wait()) {
      mma_block<F16>(tm + 256, tA, false, 128, tD, false, WO_ROWS, WO_ROWS, KS_M1, false);
      if (F16) mma_block<F16>(tm + 256, tA, false, 128, tC, false, WO_ROWS, WO_ROWS, KS_M1, true);
    }
    commit_and_sync(sy, issuer);
    // C, D and the key table are dead: the next atom's inputs start to arrive
    // (no thread reads C, D or the key table again for this atom; its
    // LayerNorm runs during the next atom's [Q K] product)
    if (issuer && next < a.n) fetch_inputs(next);
    if (next < a.n) nn_next = a.nnei[next];
    have_prev = true;
    prev_base = base;
    prev_nn = nn;
    prev_w = w_row;
  }
  if (have_prev && sy.ok) layer_norm_out(prev_base, prev_nn, prev_w);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// ----------------------------------------------------------------- backward
// Shared memory: slots A-D [0,128K), Wq, Wk [128K, 192K), slot E [192K,
// 224K), per-key table, barriers.  Wvo is streamed per atom into slot D.
// Same thread layout as the forward kernel.
constexpr int B_SLOT_A = 0, B_SLOT_B = TILE, B_SLOT_C = 2 * TILE, B_SLOT_D = 3 * TILE, B_W = 4 * TILE;
constexpr int B_SMALL = 4 * TILE + 3 * TILE;
constexpr int B_SMEM = B_SMALL + 2048 + 64;

template <bool F16>
__global__ void __launch_bounds__(NT, 1) k_layer_bwd_tc(const __grid_constant__ LayerArgs a) {
  extern __shared__ __align__(1024) uint8_t sm[];
  if ((smem_u32(sm) & 1023u) != 0) {
    if (threadIdx.x == 0) set_err(a.err, ERR_CAPACITY);
    return;
  }
  uint8_t* sA = sm + B_SLOT_A;
  uint8_t* sB = sm + B_SLOT_B;
  uint8_t* sC = sm + B_SLOT_C;
  uint8_t* sD = sm + B_SLOT_D;
  uint8_t* sWqk = sm + B_W;  // [Wq; Wk], 256 rows
  uint8_t* sE = sWqk + 2 * TILE;
  float4* s_key = reinterpret_cast<float4*>(sm + B_SMALL);  // [128] (rhat_x, rhat_y, rhat_z, w)
  // [5]: general, Wvo copy, Q K, G ready, dY ready (the last two take one
  // arrival per warp; each sees exactly one phase per atom)
  uint64_t* bar = reinterpret_cast<uint64_t*>(s_key + 128);
  uint64_t* bar_ld = bar + 1;
  uint64_t* bar_q = bar + 2;
  uint64_t* bar_g = bar + 3;
  uint64_t* bar_dy = bar + 4;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bar + 5);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2;
  const int row = quad * 32 + lane;
  const int c0 = part * 32;
  // The MMA issuer stalls while the tensor pipe's queue is full: it lives in
  // the warp with the least element-wise work (rows 96-127 are past the
  // last neighbour of most atoms, columns 96-127 past the embedding width)
  const bool issuer = tid == NT - 32;

  copy_image(sWqk, a.wimg, 2 * TILE);
  if (issuer) {
    for (int i = 0; i < 3; ++i) mbar_init(bar + i, 1);
    mbar_init(bar_g, NT / 32);
    mbar_init(bar_dy, NT / 32);
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(s_tmem, 512);
  handoff();
  const uint32_t tm = *s_tmem;
  const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
  const uint32_t tA = smem_u32(sA), tB = smem_u32(sB), tC = smem_u32(sC), tD = smem_u32(sD);
  const uint32_t tWqk = smem_u32(sWqk), tE = smem_u32(sE);
  const uint32_t tWk = tWqk + 128 * 128;  // rows 128-255 of the [Wq; Wk] tile
  Sync sy{bar, 0u, a.err};
  Sync sl{bar_ld, 0u, a.err};
  Sync sq{bar_q, 0u, a.err};
  Sync sg{bar_g, 0u, a.err}, sd{bar_dy, 0u, a.err};  // waited on by the issuer only
  const uint8_t* wo_img = reinterpret_cast<const uint8_t*>(a.wimg) + WV_OFF;
  // An atom's Wvo copy (slot D) and its layer-input rows (parked in TMEM
  // columns [0, 128)) arrive during the previous atom's last phase; the
  // first atom's here
  int nn_next = (int)blockIdx.x < a.n ? a.nnei[blockIdx.x] : 0;
  if ((int)blockIdx.x < a.n) {
    if (issuer) {
      mbar_expect_tx(bar_ld, WO_TILE);
      bulk_g2s(sD, wo_img, WO_TILE, bar_ld);
      prefetch_atom(a, blockIdx.x, true);
    }
    float gn[32];
    load_cq32(a.Gin + (size_t)blockIdx.x * NP * a.m1, a.m1, row, c0, gn, row < nn_next);
    tmem_st32(tm + lane_off + 0 + c0, gn);
  }

  for (int atom = blockIdx.x; atom < a.n && sy.ok; atom += gridDim.x) {
    const int nn = nn_next;
    const size_t base = (size_t)atom * NP;
    const bool rv = row < nn;
    const int next = atom + (int)gridDim.x;
    if (issuer) prefetch_atom(a, next, true);  // the next atom's inputs -> L2
    // Every per-row input of the atom in one round trip (live rows only: the
    // rows past the last neighbour are not kept).  With FP16 operands the
    // loads are issued before the TMEM read of the layer-input row, which the
    // compiler does not move loads across (with BF16 that order spills)
    float v[32];
    if constexpr (!F16) tmem_ld32(tm + lane_off + 0 + c0, v);
    const float rs = rv ? a.rstd[base + row] : 0.f;
    const float2 sst = rv ? a.smax[base + row] : make_float2(0.f, 0.f);
    float4 kr = make_float4(0.f, 0.f, 0.f, 0.f);
    if (tid < nn) kr = reinterpret_cast<const float4*>(a.rw)[base + tid];
    if (next < a.n) nn_next = a.nnei[next];
    float4 dz[8];
    uint4 yy[4];
    {
      const float4* dz4 = reinterpret_cast<const float4*>(a.dG + base * a.m1);
      const uint4* yh8 = reinterpret_cast<const uint4*>(a.yhat + base * a.yld);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + 4 * q;
        dz[q] = c < a.m1 && rv ? dz4[(c >> 2) * NP + row] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + 8 * q;
        yy[q] = c < a.m1 && rv ? yh8[(c >> 3) * NP + row] : make_uint4(0u, 0u, 0u, 0u);
      }
    }
    if constexpr (F16) tmem_ld32(tm + lane_off + 0 + c0, v);
    if (tid < 128) s_key[tid] = kr;
    // P0a: G_l -> A (+ G_lo -> B), the bias columns set to 1
    set_bias_ones(v, c0, a.m1);
    store_row32<F16>(sA, row, c0, v);
    if (F16) store_row32<F16, true>(sB, row, c0, v);
    // The two handoffs to the issuer in P0 are arrivals on mbarriers, not CTA
    // barriers: no warp waits while the issuer is held up issuing M0a
    warp_arrive(bar_g);
    // M0a: [Q K] = G [Wq Wk] (N = 256, + the G_lo product) -> [0, 256)
    if (issuer) {
      if (sg.wait()) {
        mma_block<F16>(tm + 0, tA, false, 128, tWqk, false, 256, 256, KS_M1, false);
        if (F16) mma_block<F16>(tm + 0, tB, false, 128, tWqk, false, 256, 256, KS_M1, true);
      }
      mma_commit(bar_q);
    }
    // P0b, while M0a runs: dY = LayerNorm adjoint of dZ -> C.  A lane
    // quadrant whose rows are all past the last neighbour (the same for its
    // four warps) stores zeros and skips the exchange: the issuer's quadrant
    // then does not hold M0b back while the issuer waits to queue M0a.
    if (quad * 32 >= nn) {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = 0.f;
      store_row32<F16>(sC, row, c0, v);
    } else {
      const RowXchg xr(sC, row, part, lane, quad);  // dY is stored after the exchange
      float yv[32];
      float s1 = 0.f, s2 = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t yw[4] = {yy[q].x, yy[q].y, yy[q].z, yy[q].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const __nv_bfloat162 p2 = *reinterpret_cast<const __nv_bfloat162*>(&yw[k]);
          yv[8 * q + 2 * k] = __low2float(p2);
          yv[8 * q + 2 * k + 1] = __high2float(p2);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + 4 * q;
        const float4 g4 = dz[q];
        float* g = v + 4 * q;
        if (c < a.m1 && rv) {
          g[0] = g4.x * a.gamma[c];
          g[1] = g4.y * a.gamma[c + 1];
          g[2] = g4.z * a.gamma[c + 2];
          g[3] = g4.w * a.gamma[c + 3];
        } else {
          g[0] = g[1] = g[2] = g[3] = 0.f;
        }
        s1 += (g[0] + g[1]) + (g[2] + g[3]);
        s2 += (g[0] * yv[4 * q] + g[1] * yv[4 * q + 1]) + (g[2] * yv[4 * q + 2] + g[3] * yv[4 * q + 3]);
      }
      const float2 ss = xr.sum2(make_float2(s1, s2));
      s1 = ss.x / (float)a.m1;
      s2 = ss.y / (float)a.m1;
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = rv ? rs * (v[i] - s1 - yv[i] * s2) : 0.f;
      store_row32<F16>(sC, row, c0, v);
    }
    warp_arrive(bar_dy);
    // M0b: dPG = dY Wvo^T -> [256, 368) (Wvo tile as MN-major)
    if (issuer) {
      if (sd.wait() && sl.wait()) mma_block<F16>(tm + 256, tC, false, 128, tD, true, WO_ROWS, WO_ROWS, KS_M1, false);
      mma_commit(bar);
    }
    // P1: Q -> B, K -> E once M0a is done (G_lo is dead; G stays in A); dPG
    // -> D once M0b is done (Wvo is dead; its columns past 112 are never read)
    sq.wait();
    tmem_ld32(tm + lane_off + 0 + c0, v);
    store_row32<F16>(sB, row, c0, v);
    tmem_ld32(tm + lane_off + 128 + c0, v);
    store_row32<F16>(sE, row, c0, v);
    sy.wait();
    tmem_ld32(tm + lane_off + 256 + c0, v);
    store_row32<F16>(sD, row, c0, v);
    handoff();
    // M1: S = Q K^T -> [384,512) ; dP = dPG [G 1 1]^T -> [0,128) (the ones
    // columns of G give the row-sum term dPG_j,M1 + dPG_j,M1+1 of every key)
    if (issuer) {
      mma_block<F16>(tm + 384, tB, false, 128, tE, false, 128, 128, 8, false);
      mma_block<F16>(tm + 0, tD, false, 128, tA, false, 128, 128, KS_M1, false);
    }
    commit_and_sync(sy, issuer);
    // P2: softmax adjoint over this thread's 32 keys, with the row max and
    // normaliser the forward pass stored: A and sum_k A_jk dA_jk first, then
    // the main pass in 8-key pieces that reload S, dP, A and the gate cosine
    // from TMEM; P -> slot C, dS -> TMEM over the consumed S columns.  Key
    // halves past the last neighbour only write their zeros.  The row parts
    // (this thread's row) and column parts (lanes 0-15: key c0 + h + lane)
    // of dE/drhat and dE/dw stay in registers until slot C is free.
    float4 rpart, cpart[2];
    {
      const RowXchg xr(sC, row, part, lane, quad);  // dY is dead after dPG
      const uint32_t tS = tm + lane_off + 384 + c0, tP = tm + lane_off + 0 + c0;
      const float4 kj = s_key[row];
      const float wj = kj.w;
      const float mx = sst.x, inv = sst.y;
      // A and the gate cosine c of this thread's keys, kept in the dead K and
      // dPG accumulator columns for the main pass
      const uint32_t tAw = tm + lane_off + 128 + c0, tCs = tm + lane_off + 256 + c0;
      float wsum = 0.f;
      if (c0 < nn) {
        float t[32], u[32];
        tmem_ld32x2(tS, tP, t, u);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int k = c0 + i;
          const float4 kk = s_key[k];
          const float c = kj.x * kk.x + kj.y * kk.y + kj.z * kk.z;
          float A = 0.f;
          if (k < nn && rv) {
            const float ww = wj * kk.w;
            A = exp_sfu((t[i] * a.scale + a.shift) * ww - mx) * inv;
            wsum += A * u[i] * ww * c;
          }
          t[i] = A;
          u[i] = c;
        }
        tmem_st32(tAw, t);
        tmem_st32(tCs, u);
      }
      const float tsum = xr.sum(wsum);  // sum_k A_jk dA_jk; ends with the quadrant's barrier
      float rw_ = 0.f, rx = 0.f, ry = 0.f, rz = 0.f;
#pragma unroll 1
      for (int h = 0; h < 32; h += 16) {
        float4 cph = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c0 + h < nn) {
          float cw[16], dcv[16];
#pragma unroll
          for (int e8 = 0; e8 < 16; e8 += 8) {
            float t[8], u[8], Av[8], cv[8], pv[8];
            tmem_ld8x4(tS + h + e8, tP + h + e8, tAw + h + e8, tCs + h + e8, t, u, Av, cv);
            // No masks: A is 0 past the last neighbour and on rows past it
            // (first pass), and S, dP and c are finite there, so every term
            // below vanishes on its own
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float4 kk = s_key[c0 + h + e8 + i];
              const float A = Av[i], c = cv[i];
              const float ww = wj * kk.w;
              const float e = A * u[i];                           // A dP
              const float dc = e * ww;                            // dE/dc_jk
              const float dLp = fmaf(dc, c, -A * tsum);           // A (dA - sum_k A dA), dA = dP ww c
              const float H = fmaf(dLp, fmaf(t[i], a.scale, a.shift), e * c);  // dE/d(w_j w_k)
              const float P = A * ww * c;
              const float dS = dLp * ww * a.scale;
              rw_ += H * kk.w;
              rx += dc * kk.x; ry += dc * kk.y; rz += dc * kk.z;
              cw[e8 + i] = H * wj;
              dcv[e8 + i] = dc;
              pv[i] = P;
              t[i] = dS;
            }
            uint4 w4;
            w4.x = pack16<F16>(pv[0], pv[1]);
            w4.y = pack16<F16>(pv[2], pv[3]);
            w4.z = pack16<F16>(pv[4], pv[5]);
            w4.w = pack16<F16>(pv[6], pv[7]);
            sw128_store8(sC, row, c0 + h + e8, 128, w4);
            tmem_st8_async(tS + h + e8, t);  // dS over these consumed S columns
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
        } else {
          const float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
          for (int e8 = 0; e8 < 16; e8 += 8) {
            sw128_store8(sC, row, c0 + h + e8, 128, make_uint4(0u, 0u, 0u, 0u));
            tmem_st8_async(tS + h + e8, z);
          }
        }
        cpart[h >> 4] = cph;
      }
      rpart = make_float4(rx, ry, rz, rw_);
      tmem_wait_st();
    }
    handoff();
    // M2: P^T dPG -> [128, 240) (kept in TMEM until P5)
    if (issuer) mma_block<F16>(tm + 128, tC, true, 128, tD, true, 128, WO_ROWS, 8, false);
    commit_and_sync(sy, issuer);
    tmem_ld32(tm + lane_off + 384 + c0, v);  // dS
    store_row32<F16>(sC, row, c0, v);
    handoff();
    // M3: dQ = dS K -> [0,128) ; dK = dS^T Q -> [256,384)
    if (issuer) {
      mma_block<F16>(tm + 0, tC, false, 128, tE, true, 128, 128, 8, false);
      mma_block<F16>(tm + 256, tC, true, 128, tB, true, 128, 128, 8, false);
    }
    commit_and_sync(sy, issuer);
    // P4: dQ -> B, dK -> A (G is dead); the row and column parts -> slot C
    // (dS is dead): [quadrant][128 keys] column parts, then [quarter][128
    // rows] row parts, float4 (x, y, z, w) each
    tmem_ld32(tm + lane_off + 0 + c0, v);
    store_row32<F16>(sB, row, c0, v);
    tmem_ld32(tm + lane_off + 256 + c0, v);
    store_row32<F16>(sA, row, c0, v);
    float4* parts = reinterpret_cast<float4*>(sC);
    if (lane < 16) {
      parts[quad * 128 + c0 + lane] = cpart[0];
      parts[quad * 128 + c0 + 16 + lane] = cpart[1];
    }
    parts[512 + part * 128 + row] = rpart;
    handoff();
    // M4: dQ Wq^T + dK Wk^T -> [384, 496)
    if (issuer) {
      mma_block<F16>(tm + 384, tB, false, 128, tWqk, true, 256, WO_ROWS, 8, false);
      mma_block<F16>(tm + 384, tA, false, 128, tWk, true, 256, WO_ROWS, 8, true);
      mma_commit(bar);
    }
    // while M4 runs: dZ for the residual, and dgeo of this atom (key `tid`:
    // the four quarters' row parts + the four quadrants' column parts)
    float4* dg4 = reinterpret_cast<float4*>(a.dG + base * a.m1);
    float4 g[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int c = c0 + 4 * q;
      g[q] = c < a.m1 && rv ? dg4[(c >> 2) * NP + row] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // the next atom's layer-input row, parked in TMEM [0, 128) (dQ is dead
    // since P4)
    if (next < a.n) {
      float gn[32];
      load_cq32(a.Gin + (size_t)next * NP * a.m1, a.m1, row, c0, gn, row < nn_next);
      tmem_st32(tm + lane_off + 0 + c0, gn);
    }
    if (tid < nn) {
      float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 r = parts[512 + q * 128 + tid];
        const float4 c = parts[q * 128 + tid];
        s.x += r.x + c.x; s.y += r.y + c.y; s.z += r.z + c.z; s.w += r.w + c.w;
      }
      // one writer per row in a launch: a reduction without a return (the
      // same FP32 adds as a load, add and store, without the round trip)
      atomicAdd(reinterpret_cast<float4*>(a.dgeo) + base + tid, s);
    }
    sy.wait();
    // Slot D is free: the next atom's Wvo copy
    if (issuer && next < a.n) {
      mbar_expect_tx(bar_ld, WO_TILE);
      bulk_g2s(sD, wo_img, WO_TILE, bar_ld);
    }
    // P5: dG_l = dZ + (dQ Wq^T + dK Wk^T + P^T dPG), in place, 16 columns at a time
#pragma unroll
    for (int h = 0; h < 32; h += 16) {
      float u[16];
      tmem_ld16(tm + lane_off + 384 + c0 + h, v);
      tmem_ld16(tm + lane_off + 128 + c0 + h, u);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + h + 4 * q, i = 4 * q;
        float4& gq = g[(h >> 2) + q];
        if (c < a.m1 && rv) {
          gq.x += v[i] + u[i]; gq.y += v[i + 1] + u[i + 1]; gq.z += v[i + 2] + u[i + 2]; gq.w += v[i + 3] + u[i + 3];
          dg4[(c >> 2) * NP + row] = gq;
        }
      }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tm, 512);
}

// Row-major [rows][m1] <-> column-quad interleaved per atom (to_cq = 1: row-major
// src to interleaved dst), one float4 per thread in the interleaved order.
__global__ void k_relayout(const float4* __restrict__ src, float4* __restrict__ dst, long long total4, int m1,
                           int to_cq) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total4) return;
  const int q4 = m1 / 4;
  const long long per_atom = (long long)NP * q4;
  const long long atom = i / per_atom;
  const int rem = (int)(i % per_atom), q = rem / NP, r = rem % NP;
  const long long rm = atom * per_atom + (long long)r * q4 + q;
  if (to_cq)
    dst[i] = src[rm];
  else
    dst[rm] = src[i];
}

void relayout(const float* src, float* dst, int n, int m1, bool to_cq, cudaStream_t st) {
  const long long total4 = (long long)n * NP * (m1 / 4);
  if (total4 == 0) return;
  k_relayout<<<(unsigned)((total4 + 255) / 256), 256, 0, st>>>(reinterpret_cast<const float4*>(src),
                                                               reinterpret_cast<float4*>(dst), total4, m1,
                                                               to_cq ? 1 : 0);
  note_launch();
}

int sm_count_dev(int dev) {
  int c = 0;
  cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
  return c > 0 ? c : 1;
}

// Build the swizzled shared-memory image of one layer's weights: [Wq; Wk]
// as a [256 out][128 in] K-major tile (in = M1 padded with zeros), then
// Wvo = [Wv Wo; (bv Wo)_hi; (bv Wo)_lo] (formed in FP64) as a [112 out][128
// in] tile and the 16-bit rounding residue of Wvo in the same layout.  Inputs
// M1 and M1 + 1 of Wq, Wk hold the 16-bit high and low parts of the biases
// bq, bk: the kernels set the layer input's columns M1 and M1 + 1 to 1, so the
// products carry the biases (to about 22 bits in FP16, 16 in BF16); the same
// columns of P G are then the row sums of P, which rows M1 and M1 + 1 of Wvo
// turn into rowsum(P) bv Wo.
std::vector<uint8_t> layer_image(const std::vector<double>* Ws[3], const std::vector<double>* bs[3],
                                 const std::vector<double>& Wo, int m1, int A, bool f16) {
  std::vector<uint8_t> img(WIMG, 0);
  auto r16 = [&](double x) -> double {
    return f16 ? (double)__half2float(__float2half((float)x)) : (double)__bfloat162float(__float2bfloat16((float)x));
  };
  auto put = [&](uint8_t* tile, int r, int c, int R, double x) {
    if (f16) {
      __half h = __float2half((float)x);
      memcpy(tile + sw128_offset(r, c, R), &h, 2);
    } else {
      __nv_bfloat16 h = __float2bfloat16((float)x);
      memcpy(tile + sw128_offset(r, c, R), &h, 2);
    }
  };
  for (int t = 0; t < 2; ++t) {
    // Wq and Wk form one 256-row tile (outputs 0-127: Q, 128-255: K), so that
    // [Q K] is one N = 256 product
    const int r0 = t == 1 ? 128 : 0;
    for (int f = 0; f < A; ++f) {
      for (int m = 0; m < m1; ++m) put(img.data(), r0 + f, m, 256, (*Ws[t])[(size_t)m * A + f]);
      const double b = (*bs[t])[f], hi = r16(b);
      put(img.data(), r0 + f, m1, 256, hi);
      put(img.data(), r0 + f, m1 + 1, 256, b - hi);
    }
  }
  const std::vector<double>& Wv = *Ws[2];
  const std::vector<double>& bv = *bs[2];
  for (int c = 0; c < m1; ++c) {
    for (int p = 0; p < m1; ++p) {
      double x = 0.0;
      for (int f = 0; f < A; ++f) x += Wv[(size_t)p * A + f] * Wo[(size_t)f * m1 + c];
      put(img.data() + WV_OFF, c, p, WO_ROWS, x);
      put(img.data() + WV_OFF + WO_TILE, c, p, WO_ROWS, x - r16(x));
    }
    double b = 0.0;
    for (int f = 0; f < A; ++f) b += bv[f] * Wo[(size_t)f * m1 + c];
    const double bh = r16(b), bl = b - bh;
    put(img.data() + WV_OFF, c, m1, WO_ROWS, bh);
    put(img.data() + WV_OFF, c, m1 + 1, WO_ROWS, r16(bl));
    put(img.data() + WV_OFF + WO_TILE, c, m1 + 1, WO_ROWS, bl - r16(bl));
  }
  return img;
}

}  // namespace

int tc_init_weights(dp_model* m, const HostArrays& arrays, std::string& msg) {
  if (m->A != 128 || m->m1 + 2 > 16 * KS_M1 || m->m1 % 4 != 0) {
    msg = "the tensor-core path needs attention width 128 and an embedding width <= 108 divisible by 4";
    return DP_ERR_UNSUPPORTED;
  }
  auto get = [&](const std::string& name) -> const std::vector<double>& {
    for (auto& kv : arrays)
      if (kv.first == name) return kv.second;
    static std::vector<double> empty;
    return empty;
  };
  TcWeights& w = m->tcw;
  for (int f16 = 0; f16 < 2; ++f16)
    for (int l = 0; l < m->nattn; ++l) {
      const std::string p = "at" + std::to_string(l) + "_";
      const std::vector<double>* Ws[3] = {&get(p + "Wq"), &get(p + "Wk"), &get(p + "Wv")};
      const std::vector<double>* bs[3] = {&get(p + "bq"), &get(p + "bk"), &get(p + "bv")};
      std::vector<uint8_t> img = layer_image(Ws, bs, get(p + "Wo"), m->m1, m->A, f16 != 0);
      void* d = nullptr;
      if (cudaMalloc(&d, img.size()) != cudaSuccess ||
          cudaMemcpy(d, img.data(), img.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        msg = "cudaMalloc of the 16-bit weight image failed";
        return DP_ERR_CUDA;
      }
      w.allocations.push_back(d);
      (f16 ? w.layer_f16_t : w.layer_bf16_t).push_back(d);
    }
  if (int rc = tc_init_embedding(m, arrays, msg)) return rc;
  w.vectors.assign(m->nattn, TcWeights::Vectors{});
  for (int l = 0; l < m->nattn; ++l) {
    const std::string p = "at" + std::to_string(l) + "_";
    TcWeights::Vectors& v = w.vectors[l];
    for (int c = 0; c < m->m1; ++c) {
      v.bo[c] = (float)get(p + "bo")[c];
      v.gamma[c] = (float)get(p + "ln_g")[c];
      v.beta[c] = (float)get(p + "ln_b")[c];
    }
  }
  const int smem = std::max(F_SMEM, B_SMEM);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
  if (optin < smem) {
    msg = "device shared memory per block is below the tensor-core kernels' need";
    return DP_ERR_UNSUPPORTED;
  }
  cudaFuncSetAttribute(k_layer_fwd_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM);
  cudaFuncSetAttribute(k_layer_bwd_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM);
  cudaFuncSetAttribute(k_layer_fwd_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM);
  cudaFuncSetAttribute(k_layer_bwd_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, B_SMEM);
  if (int rc = fit_tc_init(m, msg)) return rc;
  w.ready = true;
  return DP_OK;
}

void tc_plan_buffers(dp_model* m, Arena& a, int cap) {
  Workspace& ws = m->ws;
  const size_t rows = (size_t)cap * NP;
  ws.tc.p[0] = a.take<__nv_bfloat16>(rows * yhat_ld(m->m1) * (size_t)std::max(1, m->nattn));  // yhat per layer
  ws.tc.p[1] = a.take<float>(rows * (size_t)std::max(1, m->nattn));                // rstd per layer
  ws.tc.p[4] = a.take<float2>(rows * (size_t)std::max(1, m->nattn));               // softmax stats per layer
  ws.tc.p[2] = nullptr;
  // row-major staging of G0 / dE/dG0 for the SIMT embedding net (nets other than 25-50-100)
  ws.tc.p[3] = m->tcw.emb_W1_t ? nullptr : a.take<float>(rows * m->m1);
  // layers 1 and 2 of the tensor-core embedding net, for its adjoint
  ws.tc.p[5] = m->tcw.emb_W1_t ? a.take<float>(rows * (size_t)(m->emb[0] + m->emb[1])) : nullptr;
  // the live neighbour rows the tensor-core embedding net runs over, and their number
  ws.tc.p[6] = m->tcw.emb_W1_t ? a.take<int>(rows) : nullptr;
  ws.tc.p[7] = m->tcw.emb_W1_t ? a.take<int>(64) : nullptr;
}


void tc_run_network(dp_model* m, int n, const int* atype, cudaStream_t st) {
  Workspace& ws = m->ws;
  const size_t rows = (size_t)n * NP;
  const int L = m->nattn;
  const int grid = std::min(n, sm_count_dev(m->device));
  const bool f16 = m->precision == DP_PREC_FP16X;
  auto largs = [&](int l) {
    LayerArgs la{};
    la.Gin = ws.G[l];
    la.Gout = ws.G[l + 1];
    la.yhat = reinterpret_cast<__nv_bfloat16*>(ws.tc.p[0]) + (size_t)l * rows * yhat_ld(m->m1);
    la.rstd = reinterpret_cast<float*>(ws.tc.p[1]) + (size_t)l * rows;
    la.smax = reinterpret_cast<float2*>(ws.tc.p[4]) + (size_t)l * rows;
    la.dG = ws.dG;
    la.dgeo = ws.dgeo;
    la.rw = ws.rw;
    la.nnei = ws.nnei;
    la.n = n;
    la.m1 = m->m1;
    la.yld = yhat_ld(m->m1);
    la.wimg = reinterpret_cast<const uint4*>(f16 ? m->tcw.layer_f16_t[l] : m->tcw.layer_bf16_t[l]);
    const TcWeights::Vectors& vec = m->tcw.vectors[l];
    memcpy(la.bo, vec.bo, sizeof(la.bo));
    memcpy(la.gamma, vec.gamma, sizeof(la.gamma));
    memcpy(la.beta, vec.beta, sizeof(la.beta));
    la.scale = (float)(1.0 / std::sqrt((double)m->A));
    la.shift = (float)m->shift;
    la.eps = (float)m->ln_eps;
    la.err = m->d_err;
    return la;
  };
  // embedding, then the attention layers forward
  EmbedArgs ea{};
  float* rm_stage = reinterpret_cast<float*>(ws.tc.p[3]);
  ea.R = ws.R; ea.nlist = ws.nlist; ea.nnei = ws.nnei; ea.atype = atype; ea.n = n; ea.ntypes = m->nt; ea.m1 = m->m1;
  ea.w = m->emb_packed; ea.Gt = m->Gt; ea.b0t = m->b0t; ea.G0 = rm_stage;
  const bool emb_tc = m->tcw.emb_W1_t != nullptr;
  if (emb_tc) {
    tc_live_rows(m, n, st);
    tc_embed_fused(m, n, atype, false, st);
  } else {
    launch_embed_fwd(ea, m->emb, st);
    relayout(rm_stage, ws.G[0], n, m->m1, true, st);
  }
  prof_mark(m, "embed_fwd", st);
  for (int l = 0; l < L && n > 0; ++l) {
    if (f16)
      k_layer_fwd_tc<true><<<grid, NT, F_SMEM, st>>>(largs(l));
    else
      k_layer_fwd_tc<false><<<grid, NT, F_SMEM, st>>>(largs(l));
    note_launch();
    prof_mark(m, "attn_fwd_tc", st);
  }
  run_descriptor_fitting(m, n, atype, st);
  cudaMemsetAsync(ws.dgeo, 0, sizeof(float) * rows * 4, st);
  for (int l = L - 1; l >= 0 && n > 0; --l) {
    if (f16)
      k_layer_bwd_tc<true><<<grid, NT, B_SMEM, st>>>(largs(l));
    else
      k_layer_bwd_tc<false><<<grid, NT, B_SMEM, st>>>(largs(l));
    note_launch();
    prof_mark(m, "attn_bwd_tc", st);
  }
  if (emb_tc) {
    tc_embed_fused(m, n, atype, true, st);
  } else {
    relayout(ws.dG, rm_stage, n, m->m1, false, st);
    ea.dG0 = rm_stage;
    ea.dR = ws.dR;
    launch_embed_bwd(ea, m->emb, st);
  }
  prof_mark(m, "embed_bwd", st);
}

void tc_free_weights(dp_model* m) {
  for (void* p : m->tcw.allocations) cudaFree(p);
  m->tcw.allocations.clear();
  m->tcw.layer_bf16_t.clear();
  m->tcw.layer_f16_t.clear();
  m->tcw.fitW_t.clear();
  m->tcw.fitWT_t.clear();
  m->tcw.ready = false;
}

}  // namespace dpa1
