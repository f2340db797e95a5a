// Host-side launchers of the DPA-1 kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>

namespace dpa1 {

// Process-wide count of kernel launches made by this library.
void note_launch(int count = 1);

struct CellGrid;

struct NbrArgs {
  const double* coord;
  const double* box;
  const int* atype;
  int n, ntypes, sel;
  double rcut;
  int cap_dim, cell_cap;
  CellGrid* grid;
  int *cell_of, *cell_count, *cell_start, *cell_cursor, *cell_atoms;
  int *nlist, *nnei, *ncand;
  int* atype_c;    // out: types clamped to [0, ntypes)
  float4* coordf;  // scratch [n]: FP32 copy of the coordinates for the candidate screen
  int* err;
  // packed batches, one frame per call: atoms [n, n_out) are padding (no
  // neighbours, type 0) and base is added to every neighbour index written
  // (0 and 0: plain call)
  int n_out = 0, base = 0;
};
void launch_neighbors(const NbrArgs& a, cudaStream_t st);
// Packed batches, all frames of a pass in one search: slot i belongs to frame
// frame[i] (-1: padding), whose cell grid is grid[frame[i]] (set up by the
// caller) and whose cells are [cell_base[f] - cb0, + ncells) of the pass's cell
// arrays (ncells_total of them, at most cell_cap).  n is the pass's slots.
void launch_neighbors_packed(const NbrArgs& a, const int* frame, const int* cell_base, int cb0, int ncells_total,
                             cudaStream_t st);
void launch_reverse(const int* nlist, int n, int* rev_cnt, int* rev_rows, int* err, cudaStream_t st);

// --- environment matrix and its adjoint, forces, reductions (env.cu)
struct EnvArgs {
  const double* coord;
  const int* atype;
  const CellGrid* grid;
  const int* nlist;
  int n;
  const float* davg;  // [ntypes][4]
  const float* dstd;  // [ntypes][4]
  float rcs, rc;
  float* R;   // [n*NP][4] normalised environment rows
  float* rw;  // [n*NP][4] (rhat_x, rhat_y, rhat_z, w)
  float* rv;  // [n*NP][4] (x, y, z, |r|)
  double* w64;  // [n*NP] switch weight in FP64
  int fp64;     // evaluate in FP64 (else FP32 from the FP64 displacement)
  const int* frame = nullptr;  // packed batches: frame of each atom, indexing grid[]
};
void launch_env(const EnvArgs& a, cudaStream_t st);

struct EnvBwdArgs {
  const double* coord;
  const CellGrid* grid;
  int fp64;  // 1: recompute r_ij and the chain rule in FP64
  const float* rv;
  const int* nlist;
  const int* atype;
  int n;
  const float* dstd;
  float rcs, rc;
  const float* dR;    // [rows][4]
  const float* dgeo;  // [rows][4] (d rhat xyz, d w)
  float* g;           // [rows][4] dE/dr_ij (xyz, 0)
  const int* frame = nullptr;  // packed batches: frame of each atom, indexing grid[]
};
void launch_env_bwd(const EnvBwdArgs& a, cudaStream_t st);

// atoms per block of the force kernel: a packed batch pads every frame to a
// multiple of it, so that no block holds atoms of two frames
constexpr int FORCE_BLOCK_ATOMS = 4;
struct ForceArgs {
  const float* g;
  const float* rv;
  const int* nnei;
  const int* rev_cnt;
  const int* rev_rows;
  const float* e;  // [n] atomic energies
  int n;
  int nlocal;           // atoms [0, nlocal) are local: only their energies count
  double* force;        // [n][3]
  double* atom_energy;  // [n] or null
  double* partials;     // [blocks][10] (9 virial + energy)
  double* energy;       // [1], or [nseg] with seg
  double* virial;       // [9], or [nseg][9] with seg
  int* err;
  // packed batches: atoms whose frame is < 0 are padding (their energies do
  // not count); frame f owns the force blocks [seg[f] - seg[0], seg[f+1] - seg[0])
  // and gets energy[f] and virial[9f..9f+8]
  const int* frame = nullptr;
  const int* seg = nullptr;
  int nseg = 0;
};
void launch_force_virial(const ForceArgs& a, cudaStream_t st);

// --- FP32 SIMT network kernels (simt.cu)
enum Epi { EPI_BIAS = 0, EPI_TANH = 1, EPI_RES_TANH = 2, EPI_ACCUM = 3, EPI_RES = 4 };
// C[M][N] (ldc) = epi(A[M][K] (lda) * B[K][N] (ldb) + bias[N]); R is the residual (ldr).
void gemm_f32(const float* A, int lda, const float* B, int ldb, const float* bias, const float* R, int ldr,
              float* C, int ldc, int M, int N, int K, int epi, cudaStream_t st);

struct EmbedArgs {
  const float* R;
  const int* nlist;
  const int* nnei;
  const int* atype;
  int n, ntypes, m1;
  const float* w;   // packed embedding-net weights (W0 b0 W1 b1 W2 b2)
  const float* Gt;  // [ntypes][ntypes][m1]
  const float* b0t; // concat type-embedding mode: first-layer bias per (centre, neighbour)
                    // type [ntypes][ntypes][E0]; null: the b0 of the packed weights
  float* G0;        // [rows][m1]
  const float* dG0;  // backward only
  float* dR;         // backward only: dR[:,0] +=
};
bool launch_embed_fwd(const EmbedArgs& a, const int* widths, cudaStream_t st);
bool launch_embed_bwd(const EmbedArgs& a, const int* widths, cudaStream_t st);

void launch_ln_res_fwd(const float* Y, const float* Gin, const int* nlist, const float* gamma, const float* beta,
                       float eps, float* Gout, float* stats, int rows, int m1, cudaStream_t st);
void launch_ln_bwd(const float* dZ, const float* Y, const float* stats, const int* nlist, const float* gamma,
                   float* dY, int rows, int m1, cudaStream_t st);

struct AttnArgs {
  const float* QK;   // [rows][ldq]: Q | K (A columns each)
  const float* rw;   // [rows][4]
  const double* w64; // [rows] switch weights in FP64
  const int* nnei;
  int n, A, ldq;
  float shift;
  const float* G;    // [rows][m1] layer input
  int m1, ldpg;      // width of G, row stride of PG and dPG (pg_ld(m1))
  float* PG;         // fwd: [rows][ldpg] = [P G, rowsum(P), 0 ...]
  const float* dPG;  // bwd: [rows][ldpg] dE/d[P G, rowsum P]
  float* dQK;        // bwd: [rows][ldq] dQ | dK
  float* dG;         // bwd: [rows][m1] += P^T dE/d(P G)
  float* dgeo;       // bwd: [rows][4] +=
};
void launch_attn_fwd_f32(const AttnArgs& a, cudaStream_t st);
void launch_attn_bwd_f32(const AttnArgs& a, cudaStream_t st);

struct DescArgs {
  const float* R;
  const float* G;
  const int* nnei;
  const int* atype;
  const float* tebd;  // [ntypes][tebd_dim]
  int n, m1, axis, tebd_dim, sel, fit_in;
  float* T;   // [n][4][m1]
  float* X;   // [n][fit_in]
  const float* dX;  // bwd
  float* dG;        // bwd [rows][m1]
  float* dR;        // bwd [rows][4] (written)
  int cq;           // G and dG column-quad interleaved per atom (else row-major)
};
void launch_desc_fwd(const DescArgs& a, cudaStream_t st);
void launch_desc_bwd(const DescArgs& a, cudaStream_t st);

void launch_energy_head(const float* H, int n, int width, const float* w_out, const float* b_out, float out_scale,
                        const float* ebias, const int* atype, float* e, cudaStream_t st);
// dZ = dH * (1 - t^2) with t = Hcur - Hprev (Hprev may be null: t = Hcur)
void launch_tanh_bwd(const float* dH, const float* Hcur, const float* Hprev, float* dZ, long long count,
                     cudaStream_t st);
// dst[i][:] = row for i < nlocal, 0 for nlocal <= i < n (ghost atoms seed no energy)
void launch_fill_rows(float* dst, const float* row, int n, int nlocal, int width, cudaStream_t st);

// --- training of the student (train.cu, simt.cu)
bool launch_embed_wgrad(const EmbedArgs& a, const int* widths, float* grad, const float* scale, cudaStream_t st);
void launch_wgrad(const float* A, int lda, const float* B, int ldb, float* C, int ldc, int I, int O, int N,
                  const float* scale, cudaStream_t st);
void launch_colsum(const float* B, int ldb, float* c, int O, int N, const float* scale, float factor, cudaStream_t st);
void launch_head_bias_grad(const int* atype, int n, float* g_ebias, float* g_bout, const float* scale, float out_scale,
                           cudaStream_t st);
// loss of one frame, the gradient scales (1, energy term, force term) and
// the direction v = F - F_ref of the force term
void launch_train_prep(int n, const double* energy, double e_ref, const double* force, const double* force_ref,
                       double pe, double pf, double* v, double* loss, float* scales, cudaStream_t st);
// g[i] += *scale * src[i]
void launch_axpy(float* g, const float* src, int n, const float* scale, cudaStream_t st);

// Tangents (forward mode) of an energy evaluation of the FP32 path without
// attention layers, along the atom displacement field v, and of its adjoint.
struct JvpArgs {
  const double* coord;  // [n][3]
  const CellGrid* grid;
  const int* nlist;     // [rows]
  const int* nnei;      // [n]
  const int* atype;     // [n] (range-checked)
  int n, ntypes, m1, axis, fit_in, sel;
  const float* dstd;    // [ntypes][4]
  float rcs, rc;
  const float* R;       // [rows][4] environment rows
  const float* G;       // [rows][m1] embedding output (row-major)
  const float* T;       // [n][4][m1]
  const float* dX;      // [n][fit_in] dE/dX
  const float* dG;      // [rows][m1] dE/dG
  const float* w;       // packed embedding-net weights (W0 b0 W1 b1 W2 b2)
  const float* Gt;      // [ntypes][ntypes][m1]
  const float* b0t;     // concat mode: first-layer bias per (centre, neighbour) type, or null
  const double* v;      // [n][3] the direction
  float* Rd;            // [rows][4]   R'
  float* Gd;            // [rows][m1]  G'
  float* Td;            // [n][4][m1]  T'
  float* Xd;            // [n][fit_in] X'
  const float* dXd;     // [n][fit_in] (dE/dX)'
  float* dGd;           // [rows][m1]  (dE/dG)'
};
void launch_env_jvp(const JvpArgs& a, cudaStream_t st);
// mode 0: G'; mode 1: grad += *scale * (dE/d(embedding weights))'
bool launch_embed_jvp(const JvpArgs& a, const int* widths, int mode, float* grad, const float* scale,
                      cudaStream_t st);
void launch_desc_jvp_fwd(const JvpArgs& a, cudaStream_t st);
void launch_desc_jvp_bwd(const JvpArgs& a, cudaStream_t st);
// H' = (1 - t^2) Z' + Hprev' with t = H - Hprev (Hprev, Hprev' null: t = H, no skip)
void launch_tanh_jvp(const float* Zd, const float* H, const float* Hprev, const float* Hprevd, float* Hd,
                     long long count, cudaStream_t st);
// dZ = dH (1 - t^2), dZ' = dH' (1 - t^2) - 2 dH t t' with t = H - Hprev, t' = H' - Hprev'
void launch_tanh_bwd_jvp(const float* dH, const float* dHd, const float* H, const float* Hprev, const float* Hd,
                         const float* Hprevd, float* dZ, float* dZd, long long count, cudaStream_t st);
void launch_adam(float* theta, float* g, float* m1, float* m2, int n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, cudaStream_t st);
void launch_transpose(const float* W, int R, int C, float* WT, cudaStream_t st);
void launch_scale_copy(const float* src, float* dst, int n, float s, cudaStream_t st);
// out[r][p] = rows[r][p] + vec[p] for r < nrows, p < width
void launch_add_rows(const float* rows, const float* vec, int nrows, int width, float* out, cudaStream_t st);

// --- velocity-Verlet MD (md.cu)
void launch_verlet_drift(int n, double dt, const double* mass, const double* f, double* v, double* x, cudaStream_t st);
// Blocks of the second half kick for n atoms (one partial kinetic energy each).
int verlet_kick_blocks(int n);
void launch_verlet_kick(int n, double dt, const double* mass, const double* f, double* v, double* partial,
                        const double* energy, int* counter, double* thermo, int nrec, cudaStream_t st);

}  // namespace dpa1
