// Internal model and workspace layout of the DPA-1 engine, shared by the
// C ABI (api.cu) and the tensor-core path (tc.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "dpa1.h"

namespace dpa1 {

struct Arena {
  char* base = nullptr;
  size_t off = 0, cap = 0;
  template <class T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};


struct AttnLayerW {
  float *Wqk, *bqk, *WqkT, *bo, *ln_g, *ln_b;  // [Wq Wk] [m1][2A], [bq bk], [Wq Wk]^T
  // [Wv Wo; bv Wo; 0...] ([pg_ld(m1)][m1]), formed in FP64, so that
  // Y = O Wo + bo = [P G, rowsum(P)] Wvo + bo (see launch_attn_fwd_f32); and
  // its transpose [m1][pg_ld(m1)] (the adjoints of the FP32 and bf16x paths)
  float* Wvo;
  float* WvoT;
};
// Row stride of [P G, rowsum(P)]: M1 + 1 columns rounded up to 8.
inline int pg_ld(int m1) { return (m1 + 1 + 7) & ~7; }

struct TcWeights {
  bool ready = false;
  std::vector<void*> allocations;
  // per attention layer: the swizzled weight image of the fused layer kernels
  // ([Wq; Wk], Wvo and its residue, K-major tcgen05 B operands), with BF16
  // (plain bf16 mode) and with FP16 entries (fp16x)
  std::vector<void*> layer_bf16_t, layer_f16_t;
  std::vector<void*> fitW_t, fitWT_t;
  void* emb_W1_t = nullptr;  // embedding net W1 / W2 hi + lo tiles, FP16 (fused 16-bit paths)
  void* emb_W2_t = nullptr;  // the same in BF16 (bf16x)
  struct Vectors {
    float bo[128] = {};
    float gamma[128] = {};
    float beta[128] = {};
  };
  std::vector<Vectors> vectors;  // per attention layer, host copies passed as kernel parameters
  struct EmbVectors {
    float W0[32] = {}, b0[32] = {}, b1[64] = {}, b2[128] = {};
  } emb_vec;  // the tensor-core embedding net's 1 -> E0 layer and biases
};

// BF16 two-term-split image of one GEMM operand B [K][N] (bf16x.cu).
struct XImage {
  void* d = nullptr;
  int K = 0, N = 0, nkb = 0, nnb = 0, bn_max = 0;
  size_t bytes() const { return (size_t)nnb * nkb * 2 * bn_max * 128; }
};

// Weight images of the BF16-split precision mode ("bf16x").
struct XWeights {
  bool ready = false;
  std::vector<void*> allocations;
  struct Layer {
    XImage qk;    // [Wq Wk] [m1][2A]
    XImage vo;    // [Wv Wo; bv Wo; 0] [pg_ld(m1)][m1]
    XImage voT;   // [Wv Wo; bv Wo]^T [m1][pg_ld(m1)]
    XImage qkT;   // [Wq Wk]^T [2A][m1]
  };
  std::vector<Layer> layers;
  std::vector<XImage> fit, fitT;  // fitting layers, forward and transposed
};

struct TcBuffers {
  void* p[32] = {};
};

struct Workspace {
  int cap = 0;  // atoms
  void* mem = nullptr;
  size_t bytes = 0;
  // neighbour search
  CellGrid* grid;
  int *cell_of, *cell_count, *cell_start, *cell_cursor, *cell_atoms;
  int cell_cap, cap_dim;
  int *nlist, *nnei, *ncand, *rev_cnt, *rev_rows;
  int* atype_c;  // device-checked copy of the atom types
  float4* coordf;  // FP32 coordinates (neighbour screen)
  // environment
  float *R, *rw, *rv, *dR, *dgeo, *g;
  double* w64;
  // network
  // modular layer layout (FP32, bf16x): per layer Q | K, [P G, rowsum P], Y and
  // the LayerNorm statistics; dE/d[P G, rowsum P] and dE/d[Q K] for the adjoint
  std::vector<float*> G, QK, PG, Y, stats;
  float *dG, *dY, *dPG, *dQK;
  float *T, *X, *dX, *e;
  std::vector<float*> H;
  float *dHa, *dHb, *dZ;
  double* partials;
  // host-API staging
  double *coord, *box, *force, *virial, *energy, *atom_energy;
  int* atype;
  // tensor-core path buffers
  TcBuffers tc;
};

// Per-stage CUDA-event timing of one call (enabled with dp_set_profiling).
// Stage boundaries accumulate over calls until profiling is switched on again.
struct Profiler {
  static constexpr int MAXEV = 8192;
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<const char*> name;
  int count = 0;
};

}  // namespace dpa1

struct dp_model {
  int call_nlocal = 0;  // local atoms of the running evaluation (the rest are ghosts)
  using AttnLayerW = dpa1::AttnLayerW;
  using Workspace = dpa1::Workspace;
  using TcWeights = dpa1::TcWeights;
  int device = 0;
  int precision = DP_PREC_FP32;
  int ints[16];
  double dbls[8];
  std::vector<std::string> type_map;
  int nt, td, sel, axis, nattn, A, nfit, m1, fit_in;
  int emb[3], fit[3];
  double rcut, rcs, shift, ln_eps, out_scale;
  float* d_b_out = nullptr;  // output bias times out_scale (device scalar)
  // trainable parameters as one FP32 vector: the embedding net (packed W0 b0
  // W1 b1 W2 b2), the fitting layers (W b per layer), the output layer (w,
  // b) and the per-type energy bias.  The forward kernels read the embedding,
  // fitting and bias weights from it; transposes and scaled copies are
  // refreshed after every update.
  float* theta = nullptr;
  int ntheta = 0;
  std::vector<int> off_fitW, off_fitb;
  int off_wout = 0, off_bout = 0, off_ebias = 0;
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  int adam_t = 0;
  const float* grad_scale = nullptr;  // non-null: the next evaluation adds scale * dE/dtheta to grad
  float* d_scales = nullptr;          // [4]: 1, energy-loss scale, force-loss scale, 0
  void* t_buf = nullptr;              // training scratch: energy, virial, forces, the direction
                                      // v = F - F_ref, dE/dtheta, and the tangents of the evaluation
  int t_cap = 0;                      // atoms t_buf is laid out for
  // device weights
  float *emb_packed, *Gt, *tebd, *davg, *dstd, *ebias, *w_out;
  bool concat = false;     // type-embedding mode: the embedding net reads [s, T_j, T_i]
  float* b0t = nullptr;    // concat mode: first-layer bias per (centre, neighbour) type [nt][nt][E0]
  float* b0t_type = nullptr;  // concat mode: the types' part of b0t (b0t = b0t_type + em_b0)
  std::vector<AttnLayerW> attn;
  std::vector<float*> fitW, fitWT, fitb;
  TcWeights tcw;
  dpa1::XWeights xw;
  std::vector<void*> allocations;
  Workspace ws;
  int* d_err = nullptr;
  cudaStream_t stream = nullptr;  // own stream of the host API
  cudaStream_t last_stream = nullptr;
  int last_natoms = 0;
  dpa1::Profiler prof;
  // velocity-Verlet: step counter, the kick's per-block kinetic energies and
  // the cached graph of one step
  int* d_md_counter = nullptr;
  double* d_md_partial = nullptr;
  int md_partial_cap = 0;
  // dp_compute_batch: device copies of a batch's inputs and results, grown on demand
  void* batch_buf = nullptr;
  size_t batch_cap = 0;
  cudaGraphExec_t md_exec = nullptr;
  cudaGraph_t md_graph = nullptr;
  std::vector<const void*> md_key;
};

namespace dpa1 {
// Record a stage boundary on the stream (no-op unless profiling is on).
void prof_mark(dp_model* m, const char* stage, cudaStream_t st);
}  // namespace dpa1


namespace dpa1 {
using HostArrays = std::vector<std::pair<std::string, std::vector<double>>>;
// fused 16-bit tensor-core path, tc.cu
int tc_init_weights(dp_model* m, const HostArrays& arrays, std::string& msg);
// tensor-core embedding net, tc_embed.cu
int tc_init_embedding(dp_model* m, const HostArrays& arrays, std::string& msg);
void tc_embed_bf16(dp_model* m, int n, const int* atype, bool bwd, float* G0, const float* dG0, float* dR,
                   float* H12, cudaStream_t st);
void tc_live_rows(dp_model* m, int n, cudaStream_t st);
void tc_embed_fused(dp_model* m, int n, const int* atype, bool bwd, cudaStream_t st);
void tc_plan_buffers(dp_model* m, Arena& a, int cap);
void tc_run_network(dp_model* m, int n, const int* atype, cudaStream_t st);
void tc_free_weights(dp_model* m);
// tcgen05 TF32 (two-term split) fitting-net products of the 16-bit paths (fit.cu)
bool fit_tc_supported(const dp_model* m);
int fit_tc_init(dp_model* m, std::string& msg);
void fit_tc_refresh(dp_model* m, cudaStream_t st);
// BF16 two-term-split precision mode (bf16x.cu)
bool bf16x_supported(const dp_model* m);
int bf16x_init_weights(dp_model* m, std::string& msg);
void bf16x_refresh(dp_model* m, cudaStream_t st);
void bf16x_free(dp_model* m);
int gemm_bf16x(dp_model* m, const XImage& im, const float* A, int lda, const float* bias, const float* R, int ldr,
               float* C, int ldc, int M, int epi, cudaStream_t st);
void attn_core_fwd_bf16x(dp_model* m, int n, int l, cudaStream_t st);
void attn_core_bwd_bf16x(dp_model* m, int n, int l, cudaStream_t st);
// the fused 16-bit layer kernels (tc.cu) serve DP_PREC_BF16 and DP_PREC_FP16X;
// DP_PREC_FP32 and DP_PREC_BF16X share the modular layer layout (row-major G,
// stored Q | K and [P G, rowsum P], LayerNorm kernels)
inline bool fused_tc_precision(int p) { return p == DP_PREC_BF16 || p == DP_PREC_FP16X; }
int fit_gemm_tc(dp_model* m, int layer, bool backward, const float* A, int lda, const float* bias, const float* R,
                int ldr, float* C, int ldc, int M, int epi, cudaStream_t st);
// stages a7-a11 (descriptor, fitting forward / backward, descriptor backward)
void run_descriptor_fitting(dp_model* m, int n, const int* atype, cudaStream_t st);
}  // namespace dpa1
