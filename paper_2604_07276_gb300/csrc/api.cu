// C ABI of the DPA-1 engine: model loading, device workspace and the
// orchestration of stages a1-a15 on one CUDA stream.
#include <cuda_runtime.h>

#include <atomic>
#include <climits>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "dpa1.h"
#include "kernels.h"
#include "model.h"

using namespace dpa1;

namespace {

// dp_compute_batch packs its frames into passes of up to this many atom slots
// (more when the workspace already holds more)
constexpr long long BATCH_PACK_ATOMS = 65536;

thread_local std::string g_last_error;

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) return fail(DP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct HostWeights {
  int ints[16];
  double dbls[8];
  std::vector<std::string> type_map;
  std::vector<std::pair<std::string, std::vector<double>>> arrays;
  const std::vector<double>* get(const std::string& name) const {
    for (auto& kv : arrays)
      if (kv.first == name) return &kv.second;
    return nullptr;
  }
};

struct Shape {
  std::string name;
  size_t count;
};

std::vector<Shape> tensor_order(const int* I) {
  const int nt = I[1], td = I[2], nemb = I[5], nattn = I[9], A = I[10], nfit = I[11];
  const int* emb = I + 6;
  const int* fit = I + 12;
  const int m1 = emb[nemb - 1], axis = I[4];
  std::vector<Shape> out;
  out.push_back({"te_W", (size_t)nt * td});
  out.push_back({"te_b", (size_t)td});
  const bool concat = I[15] == 1;  // the embedding net reads [s, T_j, T_i]; no type-pair net
  int fan = 2 * td;
  for (int l = 0; l < nemb && !concat; ++l) {
    out.push_back({"tt_W" + std::to_string(l), (size_t)fan * emb[l]});
    out.push_back({"tt_b" + std::to_string(l), (size_t)emb[l]});
    fan = emb[l];
  }
  fan = concat ? 1 + 2 * td : 1;
  for (int l = 0; l < nemb; ++l) {
    out.push_back({"em_W" + std::to_string(l), (size_t)fan * emb[l]});
    out.push_back({"em_b" + std::to_string(l), (size_t)emb[l]});
    fan = emb[l];
  }
  out.push_back({"davg", (size_t)nt * 4});
  out.push_back({"dstd", (size_t)nt * 4});
  for (int l = 0; l < nattn; ++l) {
    std::string p = "at" + std::to_string(l) + "_";
    out.push_back({p + "Wq", (size_t)m1 * A}); out.push_back({p + "bq", (size_t)A});
    out.push_back({p + "Wk", (size_t)m1 * A}); out.push_back({p + "bk", (size_t)A});
    out.push_back({p + "Wv", (size_t)m1 * A}); out.push_back({p + "bv", (size_t)A});
    out.push_back({p + "Wo", (size_t)A * m1}); out.push_back({p + "bo", (size_t)m1});
    out.push_back({p + "ln_g", (size_t)m1}); out.push_back({p + "ln_b", (size_t)m1});
  }
  fan = m1 * axis + td;
  for (int l = 0; l < nfit; ++l) {
    out.push_back({"fit_W" + std::to_string(l), (size_t)fan * fit[l]});
    out.push_back({"fit_b" + std::to_string(l), (size_t)fit[l]});
    fan = fit[l];
  }
  out.push_back({"fit_W" + std::to_string(nfit), (size_t)fan});
  out.push_back({"fit_b" + std::to_string(nfit), (size_t)1});
  out.push_back({"ebias", (size_t)nt});
  return out;
}

int read_weights(const char* path, HostWeights& w, bool header_only) {
  if (!path) return fail(DP_ERR_ARG, "weights_path is null");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(DP_ERR_IO, std::string("cannot open ") + path);
  char magic[8];
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "DPA1WTS1", 8) == 0;
  ok = ok && fread(w.ints, sizeof(int), 16, f) == 16 && fread(w.dbls, sizeof(double), 8, f) == 8;
  if (!ok) { fclose(f); return fail(DP_ERR_IO, "bad weight file header"); }
  const int* I = w.ints;
  if (I[0] != 1 || I[1] < 1 || I[1] > 64 || I[2] < 1 || I[2] > 16 || I[3] < 1 || I[5] != 3 || I[9] < 0 ||
      I[9] > 8 || I[11] < 1 || I[11] > 3 || I[4] < 1 || I[4] > I[8] || I[15] < 0 || I[15] > 1) {
    fclose(f);
    return fail(DP_ERR_IO, "weight file header out of range");
  }
  for (int t = 0; t < I[1]; ++t) {
    char name[8];
    if (fread(name, 1, 8, f) != 8) { fclose(f); return fail(DP_ERR_IO, "truncated type map"); }
    name[7] = 0;
    w.type_map.emplace_back(name);
  }
  if (header_only) { fclose(f); return DP_OK; }
  for (auto& s : tensor_order(I)) {
    std::vector<double> v(s.count);
    if (fread(v.data(), sizeof(double), s.count, f) != s.count) {
      fclose(f);
      return fail(DP_ERR_IO, "truncated weight array " + s.name);
    }
    for (double x : v)
      if (!std::isfinite(x)) { fclose(f); return fail(DP_ERR_IO, "non-finite weight in " + s.name); }
    w.arrays.emplace_back(s.name, std::move(v));
  }
  fclose(f);
  return DP_OK;
}

// Init-time type tables on the device (a4): Z[t] = tanh(onehot(t) W + b) and
// Gt[a][b] = net_t([Z[b], Z[a]]), evaluated in FP64 and stored in FP32.
__global__ void k_type_tables(const double* __restrict__ teW, const double* __restrict__ teb,
                              const double* __restrict__ tt, int nt, int td, int e0, int e1, int e2,
                              float* __restrict__ tebd, float* __restrict__ Gt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nt * nt) return;
  const int a = p / nt, b = p % nt;
  double x[256], y[256];
  for (int c = 0; c < td; ++c) {
    x[c] = tanh(teW[b * td + c] + teb[c]);       // neighbour type first
    x[td + c] = tanh(teW[a * td + c] + teb[c]);  // centre type second
  }
  if (b == 0)
    for (int c = 0; c < td; ++c) tebd[a * td + c] = (float)x[td + c];
  const int widths[3] = {e0, e1, e2};
  int in = 2 * td;
  const double* wp = tt;
  for (int l = 0; l < 3; ++l) {
    const int out = widths[l];
    const double* W = wp;
    const double* bb = wp + (size_t)in * out;
    for (int o = 0; o < out; ++o) {
      double z = bb[o];
      for (int i = 0; i < in; ++i) z += x[i] * W[(size_t)i * out + o];
      const double t = tanh(z);
      y[o] = (out == in) ? x[o] + t : (out == 2 * in) ? x[o % in] + t : t;
    }
    for (int o = 0; o < out; ++o) x[o] = y[o];
    wp = bb + out;
    in = out;
  }
  for (int o = 0; o < e2; ++o) Gt[(size_t)p * e2 + o] = (float)x[o];
}

}  // namespace

namespace dpa1 {
static std::atomic<long long> g_launches{0};
void note_launch(int count) { g_launches += count; }

void prof_mark(dp_model* m, const char* stage, cudaStream_t st) {
  Profiler& p = m->prof;
  if (!p.on || p.count >= Profiler::MAXEV) return;
  if ((int)p.ev.size() <= p.count) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    p.ev.push_back(e);
    p.name.push_back(nullptr);
  }
  cudaEventRecord(p.ev[p.count], st);
  p.name[p.count] = stage;
  ++p.count;
}
}  // namespace dpa1

namespace {

template <class T>
int dev_upload(dp_model* m, T** out, const std::vector<T>& host) {
  void* p = nullptr;
  CUDA_TRY(cudaMalloc(&p, std::max<size_t>(host.size(), 1) * sizeof(T)));
  m->allocations.push_back(p);
  if (!host.empty()) CUDA_TRY(cudaMemcpy(p, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice));
  *out = reinterpret_cast<T*>(p);
  return DP_OK;
}

std::vector<float> to_f(const std::vector<double>& v) { return std::vector<float>(v.begin(), v.end()); }
std::vector<float> transpose_f(const std::vector<double>& v, int rows, int cols) {
  std::vector<float> t((size_t)rows * cols);
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) t[(size_t)c * rows + r] = (float)v[(size_t)r * cols + c];
  return t;
}

// Transposed fitting weights and the output layer scaled by out_scale, from
// the parameter vector.
void refresh_derived(dp_model* m, cudaStream_t st) {
  int fan = m->fit_in;
  for (int l = 0; l < m->nfit; ++l) {
    launch_transpose(m->fitW[l], fan, m->fit[l], m->fitWT[l], st);
    fan = m->fit[l];
  }
  launch_scale_copy(m->theta + m->off_wout, m->w_out, fan, (float)m->out_scale, st);
  launch_scale_copy(m->theta + m->off_bout, m->d_b_out, 1, (float)m->out_scale, st);
  // concat mode: the first-layer bias per type pair follows em_b0 (entries E0 .. 2 E0 of the vector)
  if (m->concat && m->b0t_type)
    launch_add_rows(m->b0t_type, m->theta + m->emb[0], m->nt * m->nt, m->emb[0], m->b0t, st);
  fit_tc_refresh(m, st);  // tensor-core weight images of the 16-bit paths, if built
  if (m->xw.ready) bf16x_refresh(m, st);
}

void free_workspace(Workspace& ws) {
  if (ws.mem) cudaFree(ws.mem);
  ws.mem = nullptr;
  ws.cap = 0;
}

int alloc_workspace(dp_model* m, int cap) {
  Workspace& ws = m->ws;
  free_workspace(ws);
  if (cap < 1) cap = 1;
  const size_t rows = (size_t)cap * NP;
  const int L = m->nattn, A = m->A, m1 = m->m1;
  int fmax = m->fit_in;
  for (int l = 0; l < m->nfit; ++l) fmax = std::max(fmax, m->fit[l]);
  // cells: edge >= rcut and at most ~2 atoms per cell on average
  int cap_dim = (int)std::cbrt((double)cap * 2.0);
  cap_dim = std::max(3, std::min(cap_dim, 1024));
  ws.cap_dim = cap_dim;
  ws.cell_cap = cap_dim * cap_dim * cap_dim;
  auto plan = [&](Arena& a) {
    ws.grid = a.take<CellGrid>(1);
    ws.cell_of = a.take<int>(cap);
    ws.cell_count = a.take<int>(ws.cell_cap);
    ws.cell_start = a.take<int>(ws.cell_cap + 1);
    ws.cell_cursor = a.take<int>(ws.cell_cap);
    ws.cell_atoms = a.take<int>(cap);
    ws.coordf = a.take<float4>(cap);
    ws.nlist = a.take<int>(rows);
    ws.nnei = a.take<int>(cap);
    ws.ncand = a.take<int>(cap);
    ws.atype_c = a.take<int>(cap);
    ws.rev_cnt = a.take<int>(cap);
    ws.rev_rows = a.take<int>((size_t)cap * REV_CAP);
    ws.R = a.take<float>(rows * 4);
    ws.rw = a.take<float>(rows * 4);
    ws.rv = a.take<float>(rows * 4);
    ws.w64 = a.take<double>(rows);
    ws.dR = a.take<float>(rows * 4);
    ws.dgeo = a.take<float>(rows * 4);
    ws.g = a.take<float>(rows * 4);
    ws.G.assign(L + 1, nullptr);
    for (int l = 0; l <= L; ++l) ws.G[l] = a.take<float>(rows * m1);
    ws.QK.assign(L, nullptr); ws.PG.assign(L, nullptr); ws.Y.assign(L, nullptr); ws.stats.assign(L, nullptr);
    if (!fused_tc_precision(m->precision)) {
      // Q | K only (V enters through [Wv Wo; bv Wo])
      const size_t nqk = 2 * (size_t)A;
      for (int l = 0; l < L; ++l) {
        ws.QK[l] = a.take<float>(rows * nqk);
        ws.PG[l] = a.take<float>(rows * pg_ld(m1));  // [P G, rowsum(P)]
        ws.Y[l] = a.take<float>(rows * m1);
        ws.stats[l] = a.take<float>(rows * 2);
      }
      ws.dY = a.take<float>(rows * m1);
      // dE/d[P G, rowsum P]
      ws.dPG = a.take<float>(rows * (L > 0 ? pg_ld(m1) : 1));
      ws.dQK = a.take<float>(rows * (L > 0 ? nqk : 1));
    }
    ws.dG = a.take<float>(rows * m1);
    ws.T = a.take<float>((size_t)cap * 4 * m1);
    ws.X = a.take<float>((size_t)cap * m->fit_in);
    ws.dX = a.take<float>((size_t)cap * m->fit_in);
    ws.e = a.take<float>(cap);
    ws.H.assign(m->nfit, nullptr);
    for (int l = 0; l < m->nfit; ++l) ws.H[l] = a.take<float>((size_t)cap * m->fit[l]);
    ws.dHa = a.take<float>((size_t)cap * fmax);
    ws.dHb = a.take<float>((size_t)cap * fmax);
    ws.dZ = a.take<float>((size_t)cap * fmax);
    ws.partials = a.take<double>((size_t)((cap + 3) / 4 + 1) * 10);
    ws.coord = a.take<double>((size_t)cap * 3);
    ws.box = a.take<double>(9);
    ws.force = a.take<double>((size_t)cap * 3);
    ws.virial = a.take<double>(9);
    ws.energy = a.take<double>(1);
    ws.atom_energy = a.take<double>(cap);
    ws.atype = a.take<int>(cap);
    if (fused_tc_precision(m->precision)) tc_plan_buffers(m, a, cap);
    // bf16x with the tensor-core embedding net: its layers 1 and 2 for the adjoint
    if (m->precision == DP_PREC_BF16X && m->tcw.emb_W2_t)
      ws.tc.p[5] = a.take<float>(rows * (size_t)(m->emb[0] + m->emb[1]));
  };
  Arena probe;
  plan(probe);
  const size_t bytes = probe.off;
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(DP_ERR_CUDA, "workspace allocation of " + std::to_string(bytes) + " bytes failed: " +
                                 cudaGetErrorString(e));
  }
  Arena real;
  real.base = reinterpret_cast<char*>(mem);
  real.cap = bytes;
  plan(real);
  ws.mem = mem;
  ws.bytes = bytes;
  ws.cap = cap;
  return DP_OK;
}

int check_model(const dp_model* m) {
  if (!m) return fail(DP_ERR_ARG, "model is null");
  return DP_OK;
}

int translate_err(int bits) {
  if (bits & ERR_BOX) return fail(DP_ERR_BOX, "box must be orthorhombic with every edge > 2*rcut");
  if (bits & ERR_NAN) return fail(DP_ERR_NAN, "non-finite coordinate");
  if (bits & ERR_TYPE) return fail(DP_ERR_ARG, "atom type out of range");
  if (bits & ERR_TIMEOUT) return fail(DP_ERR_TIMEOUT, "a device-side wait gave up");
  if (bits & ERR_CAPACITY) return fail(DP_ERR_CAPACITY, "a device-side buffer overflowed (neighbour candidates or reverse list)");
  return DP_OK;
}

// Stages a1-a2 on the stream.
// Neighbour-stage arguments for n atoms at coord, with the list, counts,
// clamped types and FP32 coordinates written from workspace slot rel on.
NbrArgs nbr_args(dp_model* m, int n, const double* coord, const double* box, const int* atype, CellGrid* grid,
                 int rel) {
  Workspace& ws = m->ws;
  NbrArgs a;
  a.coord = coord; a.box = box; a.atype = atype;
  a.n = n; a.ntypes = m->nt; a.sel = m->sel; a.rcut = m->rcut;
  a.cap_dim = ws.cap_dim; a.cell_cap = ws.cell_cap; a.grid = grid;
  a.cell_of = ws.cell_of; a.cell_count = ws.cell_count; a.cell_start = ws.cell_start;
  a.cell_cursor = ws.cell_cursor; a.cell_atoms = ws.cell_atoms;
  a.nlist = ws.nlist + (size_t)rel * NP; a.nnei = ws.nnei + rel; a.ncand = ws.ncand + rel;
  a.atype_c = ws.atype_c + rel; a.coordf = ws.coordf + rel;
  a.err = m->d_err;
  return a;
}

void run_neighbors(dp_model* m, int n, const double* coord, const double* box, const int* atype, cudaStream_t st) {
  launch_neighbors(nbr_args(m, n, coord, box, atype, m->ws.grid, 0), st);
}

// Gathers a batch from the caller's layout (frames back to back) into the
// slots of the packed layout, pos[i] being atom i's slot, and scatters the
// forces back.
__global__ void k_batch_pack(const double* __restrict__ coord, const int* __restrict__ atype,
                             const int* __restrict__ pos, long long total, double* __restrict__ coordP,
                             int* __restrict__ typeP) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long q = pos[i];
  coordP[3 * q] = coord[3 * i];
  coordP[3 * q + 1] = coord[3 * i + 1];
  coordP[3 * q + 2] = coord[3 * i + 2];
  typeP[q] = atype[i];
}

__global__ void k_batch_unpack(const double* __restrict__ forceP, const int* __restrict__ pos, long long total,
                               double* __restrict__ force) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const long long q = pos[i];
  force[3 * i] = forceP[3 * q];
  force[3 * i + 1] = forceP[3 * q + 1];
  force[3 * i + 2] = forceP[3 * q + 2];
}

}  // namespace

namespace dpa1 {
// Stages a7-a11 shared by both precisions: descriptor, fitting forward and
// backward, descriptor backward (dE/dG of the last layer and dE/dR).
void run_descriptor_fitting(dp_model* m, int n, const int* atype, cudaStream_t st) {
  Workspace& ws = m->ws;
  const int L = m->nattn, m1 = m->m1;
  // a7: descriptor
  DescArgs da{};
  da.R = ws.R; da.G = ws.G[L]; da.nnei = ws.nnei; da.atype = atype; da.tebd = m->tebd;
  da.n = n; da.m1 = m1; da.axis = m->axis; da.tebd_dim = m->td; da.sel = m->sel; da.fit_in = m->fit_in;
  da.T = ws.T; da.X = ws.X; da.dX = ws.dX; da.dG = ws.dG; da.dR = ws.dR;
  da.cq = fused_tc_precision(m->precision) ? 1 : 0;  // the fused layer kernels' layout
  launch_desc_fwd(da, st);
  prof_mark(m, "desc_fwd", st);
  // a8: fitting forward
  int fan = m->fit_in;
  const float* hin = ws.X;
  // the 16-bit paths run the products on tcgen05 (TF32 with two-term splits)
  const bool fit_tc = fused_tc_precision(m->precision) && !m->tcw.fitW_t.empty();
  const bool fit_x = m->precision == DP_PREC_BF16X;  // BF16 two-term splits
  for (int l = 0; l < m->nfit; ++l) {
    const int out = m->fit[l];
    const bool res = (l > 0 && out == fan);
    if (fit_x)
      gemm_bf16x(m, m->xw.fit[l], hin, fan, m->fitb[l], res ? hin : nullptr, fan, ws.H[l], out, n,
                 res ? EPI_RES_TANH : EPI_TANH, st);
    else if (fit_tc)
      fit_gemm_tc(m, l, false, hin, fan, m->fitb[l], res ? hin : nullptr, fan, ws.H[l], out, n,
                  res ? EPI_RES_TANH : EPI_TANH, st);
    else
      gemm_f32(hin, fan, m->fitW[l], out, m->fitb[l], res ? hin : nullptr, fan, ws.H[l], out, n, out, fan,
               res ? EPI_RES_TANH : EPI_TANH, st);
    hin = ws.H[l];
    fan = out;
  }
  // w_out and b_out are stored multiplied by out_scale
  launch_energy_head(ws.H[m->nfit - 1], n, fan, m->w_out, m->d_b_out, 1.0f, m->ebias, atype, ws.e, st);
  const float* gs = m->grad_scale;  // non-null: add gs * dE/dtheta to the gradient
  if (gs) {
    launch_colsum(ws.H[m->nfit - 1], fan, m->grad + m->off_wout, fan, n, gs, (float)m->out_scale, st);
    launch_head_bias_grad(atype, n, m->grad + m->off_ebias, m->grad + m->off_bout, gs, (float)m->out_scale, st);
  }
  // a10: fitting backward, seeded with dE/dH_last = out_scale * w_out
  launch_fill_rows(ws.dHa, m->w_out, n, m->call_nlocal, fan, st);
  float* dH = ws.dHa;
  float* dHn = ws.dHb;
  for (int l = m->nfit - 1; l >= 0; --l) {
    const int out = m->fit[l];
    const int in = l > 0 ? m->fit[l - 1] : m->fit_in;
    const bool res = (l > 0 && out == in);
    launch_tanh_bwd(dH, ws.H[l], res ? ws.H[l - 1] : nullptr, ws.dZ, (long long)n * out, st);
    if (gs) {
      const float* input = l > 0 ? ws.H[l - 1] : ws.X;
      launch_wgrad(input, in, ws.dZ, out, m->grad + m->off_fitW[l], out, in, out, n, gs, st);
      launch_colsum(ws.dZ, out, m->grad + m->off_fitb[l], out, n, gs, 1.0f, st);
    }
    float* dst = l > 0 ? dHn : ws.dX;
    if (fit_x)
      gemm_bf16x(m, m->xw.fitT[l], ws.dZ, out, nullptr, res ? dH : nullptr, out, dst, in, n, res ? EPI_RES : EPI_BIAS,
                 st);
    else if (fit_tc)
      fit_gemm_tc(m, l, true, ws.dZ, out, nullptr, res ? dH : nullptr, out, dst, in, n, res ? EPI_RES : EPI_BIAS, st);
    else
      gemm_f32(ws.dZ, out, m->fitWT[l], in, nullptr, res ? dH : nullptr, out, dst, in, n, in, out,
               res ? EPI_RES : EPI_BIAS, st);
    std::swap(dH, dHn);
  }
  prof_mark(m, "fitting", st);
  // a11: descriptor backward -> dG (w.r.t. G_L) and dR
  launch_desc_bwd(da, st);
  prof_mark(m, "desc_bwd", st);
}

}  // namespace dpa1

namespace {

// The FP32 network path (stages a5-a13) between the environment matrix and
// the per-pair gradient.
void run_network_f32(dp_model* m, int n, const int* atype, cudaStream_t st) {
  Workspace& ws = m->ws;
  const int rows = n * NP, L = m->nattn, A = m->A, m1 = m->m1;
  // a5: embedding
  EmbedArgs ea{};
  ea.R = ws.R; ea.nlist = ws.nlist; ea.nnei = ws.nnei; ea.atype = atype; ea.n = n; ea.ntypes = m->nt; ea.m1 = m1;
  ea.w = m->emb_packed; ea.Gt = m->Gt; ea.b0t = m->b0t; ea.G0 = ws.G[0];
  launch_embed_fwd(ea, m->emb, st);
  prof_mark(m, "embed_fwd", st);
  // a6: attention layers
  for (int l = 0; l < L; ++l) {
    const AttnLayerW& w = m->attn[l];
    // [Q K] = G [Wq Wk] + [bq bk] (V only enters through [Wv Wo; bv Wo])
    gemm_f32(ws.G[l], m1, w.Wqk, 2 * A, w.bqk, nullptr, 0, ws.QK[l], 2 * A, rows, 2 * A, m1, EPI_BIAS, st);
    prof_mark(m, "qkv_gemm", st);
    AttnArgs aa{};
    aa.QK = ws.QK[l]; aa.ldq = 2 * A; aa.rw = ws.rw; aa.w64 = ws.w64; aa.nnei = ws.nnei; aa.n = n; aa.A = A;
    aa.shift = (float)m->shift;
    aa.G = ws.G[l]; aa.m1 = m1; aa.ldpg = pg_ld(m1); aa.PG = ws.PG[l];
    launch_attn_fwd_f32(aa, st);
    prof_mark(m, "attn_fwd", st);
    // Y = O Wo + bo = [P G, rowsum(P)] [Wv Wo; bv Wo] + bo
    gemm_f32(ws.PG[l], pg_ld(m1), w.Wvo, m1, w.bo, nullptr, 0, ws.Y[l], m1, rows, m1, pg_ld(m1), EPI_BIAS, st);
    launch_ln_res_fwd(ws.Y[l], ws.G[l], ws.nlist, w.ln_g, w.ln_b, (float)m->ln_eps, ws.G[l + 1], ws.stats[l], rows,
                      m1, st);
    prof_mark(m, "wo_gemm_ln", st);
  }
  run_descriptor_fitting(m, n, atype, st);
  // a12: attention backward
  cudaMemsetAsync(ws.dgeo, 0, sizeof(float) * (size_t)rows * 4, st);
  for (int l = L - 1; l >= 0; --l) {
    const AttnLayerW& w = m->attn[l];
    launch_ln_bwd(ws.dG, ws.Y[l], ws.stats[l], ws.nlist, w.ln_g, ws.dY, rows, m1, st);
    // dE/d[P G, rowsum P] = dY [Wv Wo; bv Wo]^T
    gemm_f32(ws.dY, m1, w.WvoT, pg_ld(m1), nullptr, nullptr, 0, ws.dPG, pg_ld(m1), rows, pg_ld(m1), m1, EPI_BIAS, st);
    prof_mark(m, "ln_wo_bwd", st);
    AttnArgs aa{};
    aa.QK = ws.QK[l]; aa.ldq = 2 * A; aa.rw = ws.rw; aa.w64 = ws.w64; aa.nnei = ws.nnei; aa.n = n; aa.A = A;
    aa.shift = (float)m->shift; aa.G = ws.G[l]; aa.m1 = m1; aa.ldpg = pg_ld(m1);
    aa.dPG = ws.dPG; aa.dQK = ws.dQK; aa.dG = ws.dG; aa.dgeo = ws.dgeo;
    launch_attn_bwd_f32(aa, st);  // dQ, dK; dE/dG += P^T dPG
    prof_mark(m, "attn_bwd", st);
    // dE/dG += [dQ dK] [Wq Wk]^T
    gemm_f32(ws.dQK, 2 * A, w.WqkT, m1, nullptr, nullptr, 0, ws.dG, m1, rows, m1, 2 * A, EPI_ACCUM, st);
    prof_mark(m, "qkv_bwd_gemm", st);
  }
  // a13: embedding backward -> dR[:,0]
  ea.dG0 = ws.dG; ea.dR = ws.dR;
  launch_embed_bwd(ea, m->emb, st);
  if (m->grad_scale) launch_embed_wgrad(ea, m->emb, m->grad, m->grad_scale, st);
  prof_mark(m, "embed_bwd", st);
}

// The BF16-split network path (stages a5-a13): the layout and stage order of
// the FP32 path, with every product of the attention layers, of the fitting
// net and of the embedding net on tcgen05 (bf16x.cu, tc.cu); LayerNorm and
// descriptor in FP32.
void run_network_bf16x(dp_model* m, int n, const int* atype, cudaStream_t st) {
  Workspace& ws = m->ws;
  const int rows = n * NP, L = m->nattn, A = m->A, m1 = m->m1;
  // the 25-50-100 embedding net on the tensor cores (BF16 two-term splits),
  // other nets, and any net while its weight gradient is wanted, in FP32
  const bool emb_tc = m->tcw.emb_W2_t != nullptr && !m->grad_scale;
  float* H12 = reinterpret_cast<float*>(ws.tc.p[5]);
  EmbedArgs ea{};
  ea.R = ws.R; ea.nlist = ws.nlist; ea.nnei = ws.nnei; ea.atype = atype; ea.n = n; ea.ntypes = m->nt; ea.m1 = m1;
  ea.w = m->emb_packed; ea.Gt = m->Gt; ea.b0t = m->b0t; ea.G0 = ws.G[0];
  if (emb_tc)
    tc_embed_bf16(m, n, atype, false, ws.G[0], nullptr, nullptr, H12, st);
  else
    launch_embed_fwd(ea, m->emb, st);
  prof_mark(m, "embed_fwd", st);
  for (int l = 0; l < L; ++l) {
    const AttnLayerW& w = m->attn[l];
    const XWeights::Layer& x = m->xw.layers[l];
    gemm_bf16x(m, x.qk, ws.G[l], m1, w.bqk, nullptr, 0, ws.QK[l], 2 * A, rows, EPI_BIAS, st);
    prof_mark(m, "qkv_gemm", st);
    attn_core_fwd_bf16x(m, n, l, st);
    prof_mark(m, "attn_fwd", st);
    gemm_bf16x(m, x.vo, ws.PG[l], pg_ld(m1), w.bo, nullptr, 0, ws.Y[l], m1, rows, EPI_BIAS, st);
    launch_ln_res_fwd(ws.Y[l], ws.G[l], ws.nlist, w.ln_g, w.ln_b, (float)m->ln_eps, ws.G[l + 1], ws.stats[l], rows,
                      m1, st);
    prof_mark(m, "wo_gemm_ln", st);
  }
  run_descriptor_fitting(m, n, atype, st);
  cudaMemsetAsync(ws.dgeo, 0, sizeof(float) * (size_t)rows * 4, st);
  for (int l = L - 1; l >= 0; --l) {
    const AttnLayerW& w = m->attn[l];
    const XWeights::Layer& x = m->xw.layers[l];
    launch_ln_bwd(ws.dG, ws.Y[l], ws.stats[l], ws.nlist, w.ln_g, ws.dY, rows, m1, st);
    // dE/d[P G, rowsum P] = dY [Wv Wo; bv Wo]^T
    gemm_bf16x(m, x.voT, ws.dY, m1, nullptr, nullptr, 0, ws.dPG, pg_ld(m1), rows, EPI_BIAS, st);
    prof_mark(m, "ln_wo_bwd", st);
    attn_core_bwd_bf16x(m, n, l, st);  // dQ, dK; dE/dG += P^T dPG
    prof_mark(m, "attn_bwd", st);
    gemm_bf16x(m, x.qkT, ws.dQK, 2 * A, nullptr, nullptr, 0, ws.dG, m1, rows, EPI_ACCUM, st);
    prof_mark(m, "qkv_bwd_gemm", st);
  }
  ea.dG0 = ws.dG; ea.dR = ws.dR;
  if (emb_tc) {
    tc_embed_bf16(m, n, atype, true, nullptr, ws.dG, ws.dR, H12, st);
  } else {
    launch_embed_bwd(ea, m->emb, st);
    if (m->grad_scale) launch_embed_wgrad(ea, m->emb, m->grad, m->grad_scale, st);
  }
  prof_mark(m, "embed_bwd", st);
}

// Stages a3-a15 on n atoms whose neighbour list is built.  grid is the cell
// grid of the box (frame non-null: grid[frame[i]] is atom i's box, a packed
// batch); force holds n atoms, energy and virial one frame (seg null) or the
// nseg frames of a packed batch.
int run_after_neighbors(dp_model* m, int n, const double* coord, const CellGrid* grid, const int* frame,
                        const int* seg, int nseg, double* energy, double* force, double* virial,
                        double* atom_energy, cudaStream_t st) {
  Workspace& ws = m->ws;
  const int* atype = ws.atype_c;  // every later stage reads the range-checked types
  // a3: environment matrix
  EnvArgs ea{};
  ea.coord = coord; ea.atype = atype; ea.grid = grid; ea.frame = frame; ea.nlist = ws.nlist; ea.n = n;
  ea.davg = m->davg; ea.dstd = m->dstd; ea.rcs = (float)m->rcs; ea.rc = (float)m->rcut;
  ea.R = ws.R; ea.rw = ws.rw; ea.rv = ws.rv;
  // the FP32 path evaluates R in FP64 and keeps w in FP64 for its smooth logits
  ea.fp64 = m->precision == DP_PREC_FP32 ? 1 : 0;
  ea.w64 = ea.fp64 ? ws.w64 : nullptr;
  launch_env(ea, st);
  prof_mark(m, "env", st);
  if (fused_tc_precision(m->precision))
    tc_run_network(m, n, atype, st);
  else if (m->precision == DP_PREC_BF16X)
    run_network_bf16x(m, n, atype, st);
  else
    run_network_f32(m, n, atype, st);
  // a14: per-pair gradient
  EnvBwdArgs eb{};
  eb.coord = coord; eb.grid = grid; eb.frame = frame; eb.fp64 = m->precision == DP_PREC_FP32 ? 1 : 0;
  eb.rv = ws.rv; eb.nlist = ws.nlist; eb.atype = atype; eb.n = n; eb.dstd = m->dstd;
  eb.rcs = (float)m->rcs; eb.rc = (float)m->rcut; eb.dR = ws.dR; eb.dgeo = ws.dgeo; eb.g = ws.g;
  launch_env_bwd(eb, st);
  prof_mark(m, "env_bwd", st);
  // a15: forces, virial, energy
  launch_reverse(ws.nlist, n, ws.rev_cnt, ws.rev_rows, m->d_err, st);
  ForceArgs fa{};
  fa.g = ws.g; fa.rv = ws.rv; fa.nnei = ws.nnei; fa.rev_cnt = ws.rev_cnt; fa.rev_rows = ws.rev_rows; fa.e = ws.e;
  fa.n = n; fa.nlocal = m->call_nlocal; fa.force = force; fa.atom_energy = atom_energy; fa.partials = ws.partials;
  fa.energy = energy; fa.virial = virial; fa.err = m->d_err;
  fa.frame = frame; fa.seg = seg; fa.nseg = nseg;
  launch_force_virial(fa, st);
  prof_mark(m, "force_virial", st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DP_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
  return DP_OK;
}

int run_device(dp_model* m, int n, int nlocal, const double* coord, const double* box, const int* atype, double* energy,
               double* force, double* virial, double* atom_energy, cudaStream_t st) {
  Workspace& ws = m->ws;
  if (n > ws.cap) return fail(DP_ERR_CAPACITY, "natoms exceeds the reserved workspace (call dp_reserve)");
  m->last_stream = st;
  m->last_natoms = n;
  m->call_nlocal = nlocal;
  prof_mark(m, "start", st);
  run_neighbors(m, n, coord, box, atype, st);
  prof_mark(m, "neighbors", st);
  return run_after_neighbors(m, n, coord, ws.grid, nullptr, nullptr, 0, energy, force, virial, atom_energy, st);
}

// The tangent, along the atom displacement field v, of the energy-weight
// gradient of the evaluation that just ran (FP32 path, no attention layer,
// its intermediates still in the workspace), added to grad times *scale.
void run_force_tangent(dp_model* m, int n, const double* coord, const double* v, float* Rd, float* Gd, float* dGd,
                       float* Td, float* Xd, float* dXd, const std::vector<float*>& Hd, float* const* dH,
                       float* const* dHd, float* dZ, float* dZd, float* Zd, const float* scale, cudaStream_t st) {
  Workspace& ws = m->ws;
  JvpArgs a{};
  a.coord = coord; a.grid = ws.grid; a.nlist = ws.nlist; a.nnei = ws.nnei; a.atype = ws.atype_c;
  a.n = n; a.ntypes = m->nt; a.m1 = m->m1; a.axis = m->axis; a.fit_in = m->fit_in; a.sel = m->sel;
  a.dstd = m->dstd; a.rcs = (float)m->rcs; a.rc = (float)m->rcut;
  a.R = ws.R; a.G = ws.G[0]; a.T = ws.T; a.dX = ws.dX; a.dG = ws.dG; a.w = m->emb_packed; a.Gt = m->Gt;
  a.b0t = m->b0t; a.v = v;
  a.Rd = Rd; a.Gd = Gd; a.Td = Td; a.Xd = Xd; a.dXd = dXd; a.dGd = dGd;
  // the fitting net's products (and their tangents) in the model's mode:
  // FP32, or BF16 two-term splits on the tensor cores
  const bool x16 = m->precision == DP_PREC_BF16X;
  // forward: R', G', T' and X'
  launch_env_jvp(a, st);
  launch_embed_jvp(a, m->emb, 0, nullptr, scale, st);
  launch_desc_jvp_fwd(a, st);
  // fitting forward: H_l' = (1 - t_l^2) H_{l-1}' W_l (+ H_{l-1}')
  const float* hin = Xd;
  int fan = m->fit_in;
  for (int l = 0; l < m->nfit; ++l) {
    const int out = m->fit[l];
    const bool res = (l > 0 && out == fan);
    if (x16)
      gemm_bf16x(m, m->xw.fit[l], hin, fan, nullptr, nullptr, 0, Zd, out, n, EPI_BIAS, st);
    else
      gemm_f32(hin, fan, m->fitW[l], out, nullptr, nullptr, 0, Zd, out, n, out, fan, EPI_BIAS, st);
    launch_tanh_jvp(Zd, ws.H[l], res ? ws.H[l - 1] : nullptr, res ? hin : nullptr, Hd[l], (long long)n * out, st);
    hin = Hd[l];
    fan = out;
  }
  // energy head: (dE/dw_out)' = out_scale sum_i H_last,i'
  launch_colsum(Hd[m->nfit - 1], fan, m->grad + m->off_wout, fan, n, scale, (float)m->out_scale, st);
  // fitting adjoint and its tangent (dE/dH_last = out_scale w_out is constant)
  launch_fill_rows(dH[0], m->w_out, n, n, fan, st);
  cudaMemsetAsync(dHd[0], 0, sizeof(float) * (size_t)n * fan, st);
  int cur = 0;
  for (int l = m->nfit - 1; l >= 0; --l) {
    const int out = m->fit[l];
    const int in = l > 0 ? m->fit[l - 1] : m->fit_in;
    const bool res = (l > 0 && out == in);
    const float* Hprev = res ? ws.H[l - 1] : nullptr;
    const float* Hprevd = res ? Hd[l - 1] : nullptr;
    launch_tanh_bwd_jvp(dH[cur], dHd[cur], ws.H[l], Hprev, Hd[l], Hprevd, dZ, dZd, (long long)n * out, st);
    const float* input = l > 0 ? ws.H[l - 1] : ws.X;
    const float* inputd = l > 0 ? Hd[l - 1] : Xd;
    launch_wgrad(inputd, in, dZ, out, m->grad + m->off_fitW[l], out, in, out, n, scale, st);
    launch_wgrad(input, in, dZd, out, m->grad + m->off_fitW[l], out, in, out, n, scale, st);
    launch_colsum(dZd, out, m->grad + m->off_fitb[l], out, n, scale, 1.0f, st);
    if (l > 0) {
      if (x16) {
        gemm_bf16x(m, m->xw.fitT[l], dZ, out, nullptr, res ? dH[cur] : nullptr, out, dH[1 - cur], in, n,
                   res ? EPI_RES : EPI_BIAS, st);
        gemm_bf16x(m, m->xw.fitT[l], dZd, out, nullptr, res ? dHd[cur] : nullptr, out, dHd[1 - cur], in, n,
                   res ? EPI_RES : EPI_BIAS, st);
      } else {
        gemm_f32(dZ, out, m->fitWT[l], in, nullptr, res ? dH[cur] : nullptr, out, dH[1 - cur], in, n, in, out,
                 res ? EPI_RES : EPI_BIAS, st);
        gemm_f32(dZd, out, m->fitWT[l], in, nullptr, res ? dHd[cur] : nullptr, out, dHd[1 - cur], in, n, in, out,
                 res ? EPI_RES : EPI_BIAS, st);
      }
      cur = 1 - cur;
    } else if (x16) {
      gemm_bf16x(m, m->xw.fitT[l], dZd, out, nullptr, nullptr, 0, dXd, in, n, EPI_BIAS, st);
    } else {
      // dE/dX itself is still in the workspace from the evaluation
      gemm_f32(dZd, out, m->fitWT[l], in, nullptr, nullptr, 0, dXd, in, n, in, out, EPI_BIAS, st);
    }
  }
  // descriptor adjoint's tangent -> (dE/dG)'; the embedding weights' tangent gradients
  launch_desc_jvp_bwd(a, st);
  launch_embed_jvp(a, m->emb, 1, m->grad, scale, st);
}

int read_status(dp_model* m) {
  int bits = 0;
  CUDA_TRY(cudaMemcpy(&bits, m->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(m->d_err, 0, sizeof(int)));
  return translate_err(bits);
}

int check_box_host(const double* box, double rcut) {
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b)
      if (a != b && box[3 * a + b] != 0.0) return fail(DP_ERR_BOX, "box must be orthorhombic");
    if (!(box[4 * a] > 2.0 * rcut)) return fail(DP_ERR_BOX, "every box edge must exceed 2*rcut");
  }
  return DP_OK;
}

}  // namespace

extern "C" {

const char* dp_last_error(void) { return g_last_error.c_str(); }

int dp_inspect_weights(const char* path, int* ints16, double* dbls8) {
  HostWeights w;
  int rc = read_weights(path, w, true);
  if (rc != DP_OK) return rc;
  if (ints16) memcpy(ints16, w.ints, sizeof(w.ints));
  if (dbls8) memcpy(dbls8, w.dbls, sizeof(w.dbls));
  return DP_OK;
}

int dp_init(dp_model** out, const char* weights_path, const char* const* type_map, int ntypes, double rcut,
            double rcut_smth, int sel, int precision, int device) {
  g_last_error.clear();
  if (!out) return fail(DP_ERR_ARG, "out is null");
  *out = nullptr;
  if (precision < DP_PREC_FP32 || precision > DP_PREC_BF16X) return fail(DP_ERR_ARG, "unknown precision");
  HostWeights w;
  int rc = read_weights(weights_path, w, false);
  if (rc != DP_OK) return rc;
  const int* I = w.ints;
  if (type_map) {
    if (ntypes != I[1]) return fail(DP_ERR_ARG, "ntypes differs from the weight file");
    for (int t = 0; t < ntypes; ++t)
      if (!type_map[t] || w.type_map[t] != type_map[t])
        return fail(DP_ERR_ARG, "type map differs from the weight file at type " + std::to_string(t));
  }
  if (rcut >= 0 && rcut != w.dbls[0]) return fail(DP_ERR_ARG, "rcut differs from the weight file");
  if (rcut_smth >= 0 && rcut_smth != w.dbls[1]) return fail(DP_ERR_ARG, "rcut_smth differs from the weight file");
  if (sel >= 0 && sel != I[3]) return fail(DP_ERR_ARG, "sel differs from the weight file");
  if (I[3] > NP) return fail(DP_ERR_UNSUPPORTED, "sel above 128 is not supported");
  if (I[8] > 128) return fail(DP_ERR_UNSUPPORTED, "embedding width above 128 is not supported");
  if (I[9] > 0 && I[10] != 128 && I[10] != 256)
    return fail(DP_ERR_UNSUPPORTED, "attention widths other than 128 and 256 are not supported");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(DP_ERR_CUDA, "CUDA device " + std::to_string(device) + " is not available");
  }
  CUDA_TRY(cudaSetDevice(device));
  dp_model* m = new dp_model();
  m->device = device;
  m->precision = precision;
  memcpy(m->ints, I, sizeof(m->ints));
  memcpy(m->dbls, w.dbls, sizeof(m->dbls));
  m->type_map = w.type_map;
  m->nt = I[1]; m->td = I[2]; m->sel = I[3]; m->axis = I[4];
  m->emb[0] = I[6]; m->emb[1] = I[7]; m->emb[2] = I[8];
  m->nattn = I[9]; m->A = I[10]; m->nfit = I[11];
  for (int l = 0; l < 3; ++l) m->fit[l] = I[12 + l];
  m->m1 = m->emb[2];
  m->fit_in = m->m1 * m->axis + m->td;
  m->rcut = w.dbls[0]; m->rcs = w.dbls[1]; m->shift = w.dbls[2]; m->ln_eps = w.dbls[3]; m->out_scale = w.dbls[4];
  auto fail_free = [&](int code) { dp_free(m); return code; };
  const int probe_widths[3] = {m->emb[0], m->emb[1], m->emb[2]};
  if (!((probe_widths[0] == 25 && probe_widths[1] == 50 && probe_widths[2] == 100) ||
        (probe_widths[0] == 16 && probe_widths[1] == 32 && probe_widths[2] == 64) ||
        (probe_widths[0] == 32 && probe_widths[1] == 64 && probe_widths[2] == 128)))
    return fail_free(fail(DP_ERR_UNSUPPORTED, "embedding widths without a kernel instance"));
  if ((rc = dev_upload(m, &m->davg, to_f(*w.get("davg")))) != DP_OK) return fail_free(rc);
  if ((rc = dev_upload(m, &m->dstd, to_f(*w.get("dstd")))) != DP_OK) return fail_free(rc);
  m->concat = I[15] == 1;
  if (m->concat) {
    // concat mode: the type embedding Z on the host, the type-pair table of
    // strip mode replaced by zeros (G0 = net output), and the part of the
    // first layer that the types contribute folded into a bias per (centre
    // type a, neighbour type b): b0 + Z[b] W0[1 .. td] + Z[a] W0[1 + td ..]
    const std::vector<double>& teW = *w.get("te_W");
    const std::vector<double>& teb = *w.get("te_b");
    const std::vector<double>& W0 = *w.get("em_W0");  // [1 + 2 td][E0]
    const std::vector<double>& b0 = *w.get("em_b0");
    const int nt = m->nt, td = m->td, e0 = m->emb[0];
    std::vector<double> Z((size_t)nt * td);
    for (int t = 0; t < nt; ++t)
      for (int c = 0; c < td; ++c) Z[(size_t)t * td + c] = std::tanh(teW[(size_t)t * td + c] + teb[c]);
    std::vector<float> z((size_t)nt * td), gt((size_t)nt * nt * m->m1, 0.f), b0t((size_t)nt * nt * e0),
        b0t_type((size_t)nt * nt * e0);
    for (size_t i = 0; i < z.size(); ++i) z[i] = (float)Z[i];
    for (int a = 0; a < nt; ++a)
      for (int b = 0; b < nt; ++b)
        for (int p = 0; p < e0; ++p) {
          double v = 0.0;
          for (int c = 0; c < td; ++c)
            v += Z[(size_t)b * td + c] * W0[(size_t)(1 + c) * e0 + p] + Z[(size_t)a * td + c] * W0[(size_t)(1 + td + c) * e0 + p];
          b0t_type[((size_t)a * nt + b) * e0 + p] = (float)v;
          b0t[((size_t)a * nt + b) * e0 + p] = (float)(v + b0[p]);
        }
    if ((rc = dev_upload(m, &m->tebd, z)) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &m->Gt, gt)) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &m->b0t, b0t)) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &m->b0t_type, b0t_type)) != DP_OK) return fail_free(rc);
  }
  // type tables (a4) on the device
  if (!m->concat) {
    std::vector<double> tt;
    for (int l = 0; l < 3; ++l) {
      auto* W = w.get("tt_W" + std::to_string(l));
      auto* b = w.get("tt_b" + std::to_string(l));
      tt.insert(tt.end(), W->begin(), W->end());
      tt.insert(tt.end(), b->begin(), b->end());
    }
    double *dteW, *dteb, *dtt;
    if ((rc = dev_upload(m, &dteW, *w.get("te_W"))) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &dteb, *w.get("te_b"))) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &dtt, tt)) != DP_OK) return fail_free(rc);
    std::vector<float> z((size_t)m->nt * m->td), gt((size_t)m->nt * m->nt * m->m1);
    if ((rc = dev_upload(m, &m->tebd, z)) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &m->Gt, gt)) != DP_OK) return fail_free(rc);
    const int pairs = m->nt * m->nt;
    k_type_tables<<<(pairs + 63) / 64, 64>>>(dteW, dteb, dtt, m->nt, m->td, m->emb[0], m->emb[1], m->emb[2], m->tebd,
                                             m->Gt);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail_free(fail(DP_ERR_CUDA, "type table kernel failed"));
  }
  const int A = m->A, m1 = m->m1;
  m->attn.resize(m->nattn);
  for (int l = 0; l < m->nattn; ++l) {
    std::string p = "at" + std::to_string(l) + "_";
    auto* Wq = w.get(p + "Wq"); auto* Wk = w.get(p + "Wk"); auto* Wv = w.get(p + "Wv");
    // [Wq Wk] [m1][2A] and its transpose; V only enters through [Wv Wo; bv Wo]
    std::vector<double> Wqk((size_t)m1 * 2 * A);
    for (int r = 0; r < m1; ++r)
      for (int c = 0; c < A; ++c) {
        Wqk[(size_t)r * 2 * A + c] = (*Wq)[(size_t)r * A + c];
        Wqk[(size_t)r * 2 * A + A + c] = (*Wk)[(size_t)r * A + c];
      }
    std::vector<double> bqk;
    for (auto nm : {"bq", "bk"}) bqk.insert(bqk.end(), w.get(p + nm)->begin(), w.get(p + nm)->end());
    AttnLayerW& L = m->attn[l];
    if ((rc = dev_upload(m, &L.Wqk, to_f(Wqk))) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &L.WqkT, transpose_f(Wqk, m1, 2 * A))) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &L.bqk, to_f(bqk))) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &L.bo, to_f(*w.get(p + "bo")))) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &L.ln_g, to_f(*w.get(p + "ln_g")))) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &L.ln_b, to_f(*w.get(p + "ln_b")))) != DP_OK) return fail_free(rc);
    // [Wv Wo; bv Wo; 0 ...] in FP64, rounded once to FP32
    {
      const std::vector<double>& Wo = *w.get(p + "Wo");
      const std::vector<double>& bv = *w.get(p + "bv");
      std::vector<double> Wvo((size_t)pg_ld(m1) * m1, 0.0);
      for (int r = 0; r < m1; ++r)
        for (int c = 0; c < m1; ++c) {
          double acc = 0.0;
          for (int f = 0; f < A; ++f) acc += (*Wv)[(size_t)r * A + f] * Wo[(size_t)f * m1 + c];
          Wvo[(size_t)r * m1 + c] = acc;
        }
      for (int c = 0; c < m1; ++c) {
        double acc = 0.0;
        for (int f = 0; f < A; ++f) acc += bv[f] * Wo[(size_t)f * m1 + c];
        Wvo[(size_t)m1 * m1 + c] = acc;
      }
      if ((rc = dev_upload(m, &L.Wvo, to_f(Wvo))) != DP_OK) return fail_free(rc);
      if ((rc = dev_upload(m, &L.WvoT, transpose_f(Wvo, pg_ld(m1), m1))) != DP_OK) return fail_free(rc);
    }
  }
  // trainable parameter vector (layout in model.h) and its derived copies
  {
    std::vector<float> th;
    for (int l = 0; l < 3; ++l) {
      auto* W = w.get("em_W" + std::to_string(l));
      auto* b = w.get("em_b" + std::to_string(l));
      // concat mode: only the s row of the first layer (its type rows are in b0t)
      th.insert(th.end(), W->begin(), l == 0 && m->concat ? W->begin() + m->emb[0] : W->end());
      th.insert(th.end(), b->begin(), b->end());
    }
    m->off_fitW.resize(m->nfit);
    m->off_fitb.resize(m->nfit);
    for (int l = 0; l < m->nfit; ++l) {
      auto* W = w.get("fit_W" + std::to_string(l));
      auto* b = w.get("fit_b" + std::to_string(l));
      m->off_fitW[l] = (int)th.size();
      th.insert(th.end(), W->begin(), W->end());
      m->off_fitb[l] = (int)th.size();
      th.insert(th.end(), b->begin(), b->end());
    }
    auto* Wout = w.get("fit_W" + std::to_string(m->nfit));
    m->off_wout = (int)th.size();
    th.insert(th.end(), Wout->begin(), Wout->end());
    m->off_bout = (int)th.size();
    th.push_back((float)(*w.get("fit_b" + std::to_string(m->nfit)))[0]);
    m->off_ebias = (int)th.size();
    for (double x : *w.get("ebias")) th.push_back((float)x);
    m->ntheta = (int)th.size();
    if ((rc = dev_upload(m, &m->theta, th)) != DP_OK) return fail_free(rc);
    std::vector<float> zeros(th.size(), 0.f);
    if ((rc = dev_upload(m, &m->grad, zeros)) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &m->adam_m, zeros)) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &m->adam_v, zeros)) != DP_OK) return fail_free(rc);
    std::vector<float> sc = {1.f, 0.f, 0.f, 0.f};
    if ((rc = dev_upload(m, &m->d_scales, sc)) != DP_OK) return fail_free(rc);
    m->emb_packed = m->theta;
    m->ebias = m->theta + m->off_ebias;
    m->fitW.resize(m->nfit); m->fitWT.resize(m->nfit); m->fitb.resize(m->nfit);
    int fan = m->fit_in;
    for (int l = 0; l < m->nfit; ++l) {
      m->fitW[l] = m->theta + m->off_fitW[l];
      m->fitb[l] = m->theta + m->off_fitb[l];
      std::vector<float> wt((size_t)fan * m->fit[l], 0.f);
      if ((rc = dev_upload(m, &m->fitWT[l], wt)) != DP_OK) return fail_free(rc);
      fan = m->fit[l];
    }
    std::vector<float> wo((size_t)fan, 0.f), bo(1, 0.f);
    if ((rc = dev_upload(m, &m->w_out, wo)) != DP_OK) return fail_free(rc);
    if ((rc = dev_upload(m, &m->d_b_out, bo)) != DP_OK) return fail_free(rc);
    refresh_derived(m, nullptr);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail_free(fail(DP_ERR_CUDA, "weight refresh failed"));
  }
  if (fused_tc_precision(precision)) {
    std::string msg;
    if ((rc = tc_init_weights(m, w.arrays, msg)) != DP_OK) return fail_free(fail(rc, msg));
  } else if (precision == DP_PREC_BF16X) {
    std::string msg;
    if ((rc = tc_init_embedding(m, w.arrays, msg)) != DP_OK) return fail_free(fail(rc, msg));
    if ((rc = bf16x_init_weights(m, msg)) != DP_OK) return fail_free(fail(rc, msg));
  }
  {
    void* p;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return fail_free(fail(DP_ERR_CUDA, "cudaMalloc failed"));
    m->d_err = reinterpret_cast<int*>(p);
    cudaMemset(m->d_err, 0, sizeof(int));
  }
  if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail_free(fail(DP_ERR_CUDA, "stream creation failed"));
  if ((rc = alloc_workspace(m, 256)) != DP_OK) return fail_free(rc);
  *out = m;
  return DP_OK;
}

int dp_reserve(dp_model* m, int max_atoms) {
  if (check_model(m)) return DP_ERR_ARG;
  if (max_atoms < 0) return fail(DP_ERR_ARG, "max_atoms < 0");
  CUDA_TRY(cudaSetDevice(m->device));
  if (max_atoms <= m->ws.cap) return DP_OK;
  CUDA_TRY(cudaDeviceSynchronize());
  return alloc_workspace(m, max_atoms);
}

int dp_set_precision(dp_model* m, int precision) {
  if (check_model(m)) return DP_ERR_ARG;
  if (precision < DP_PREC_FP32 || precision > DP_PREC_BF16X) return fail(DP_ERR_ARG, "unknown precision");
  if (precision == m->precision) return DP_OK;
  if (fused_tc_precision(precision) && !m->tcw.ready)
    return fail(DP_ERR_UNSUPPORTED, "model was loaded without the 16-bit layer weights; reload with DP_PREC_BF16");
  if (precision == DP_PREC_BF16X && !m->xw.ready)
    return fail(DP_ERR_UNSUPPORTED, "model was loaded without the BF16-split weights; reload with DP_PREC_BF16X");
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaDeviceSynchronize());
  m->precision = precision;
  return alloc_workspace(m, m->ws.cap);
}

int dp_compute_device_local(dp_model* m, int natoms, int nlocal, const double* d_coord, const double* d_box,
                            const int* d_atype, double* d_energy, double* d_force, double* d_virial,
                            double* d_atom_energy, void* stream) {
  if (check_model(m)) return DP_ERR_ARG;
  if (natoms < 0) return fail(DP_ERR_ARG, "natoms < 0");
  if (nlocal < 0 || nlocal > natoms) return fail(DP_ERR_ARG, "nlocal must be between 0 and natoms");
  if (!d_box || !d_energy || !d_virial || (natoms > 0 && (!d_coord || !d_atype || !d_force)))
    return fail(DP_ERR_ARG, "null device pointer");
  if (natoms > m->ws.cap) return fail(DP_ERR_CAPACITY, "natoms exceeds the reserved workspace (call dp_reserve)");
  CUDA_TRY(cudaSetDevice(m->device));
  return run_device(m, natoms, nlocal, d_coord, d_box, d_atype, d_energy, d_force, d_virial, d_atom_energy,
                    reinterpret_cast<cudaStream_t>(stream));
}

int dp_compute_device(dp_model* m, int natoms, const double* d_coord, const double* d_box, const int* d_atype,
                      double* d_energy, double* d_force, double* d_virial, double* d_atom_energy, void* stream) {
  return dp_compute_device_local(m, natoms, natoms, d_coord, d_box, d_atype, d_energy, d_force, d_virial,
                                 d_atom_energy, stream);
}

int dp_compute_local(dp_model* m, int natoms, int nlocal, const double* coord, const double* box, const int* atype,
                     double* energy, double* force, double* virial, double* atom_energy) {
  if (check_model(m)) return DP_ERR_ARG;
  if (natoms < 0) return fail(DP_ERR_ARG, "natoms < 0");
  if (nlocal < 0 || nlocal > natoms) return fail(DP_ERR_ARG, "nlocal must be between 0 and natoms");
  if (!box || !energy || !virial || (natoms > 0 && (!coord || !atype || !force)))
    return fail(DP_ERR_ARG, "null host pointer");
  int rc = check_box_host(box, m->rcut);
  if (rc != DP_OK) return rc;
  for (int i = 0; i < natoms; ++i)
    if (atype[i] < 0 || atype[i] >= m->nt) return fail(DP_ERR_ARG, "atom type out of range");
  for (long long i = 0; i < 3LL * natoms; ++i)
    if (!std::isfinite(coord[i])) return fail(DP_ERR_NAN, "non-finite coordinate");
  CUDA_TRY(cudaSetDevice(m->device));
  if (natoms > m->ws.cap && (rc = dp_reserve(m, natoms)) != DP_OK) return rc;
  Workspace& ws = m->ws;
  cudaStream_t st = m->stream;
  if (natoms > 0) {
    CUDA_TRY(cudaMemcpyAsync(ws.coord, coord, sizeof(double) * 3 * natoms, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(ws.atype, atype, sizeof(int) * natoms, cudaMemcpyHostToDevice, st));
  }
  CUDA_TRY(cudaMemcpyAsync(ws.box, box, sizeof(double) * 9, cudaMemcpyHostToDevice, st));
  rc = run_device(m, natoms, nlocal, ws.coord, ws.box, ws.atype, ws.energy, ws.force, ws.virial, ws.atom_energy, st);
  if (rc != DP_OK) return rc;
  CUDA_TRY(cudaMemcpyAsync(energy, ws.energy, sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(virial, ws.virial, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
  if (natoms > 0) {
    CUDA_TRY(cudaMemcpyAsync(force, ws.force, sizeof(double) * 3 * natoms, cudaMemcpyDeviceToHost, st));
    if (atom_energy)
      CUDA_TRY(cudaMemcpyAsync(atom_energy, ws.atom_energy, sizeof(double) * natoms, cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return read_status(m);
}

int dp_compute(dp_model* m, int natoms, const double* coord, const double* box, const int* atype, double* energy,
               double* force, double* virial, double* atom_energy) {
  return dp_compute_local(m, natoms, natoms, coord, box, atype, energy, force, virial, atom_energy);
}

int dp_compute_batch(dp_model* m, int nframes, const int* off, const double* coord, const double* box,
                     const int* atype, double* energy, double* force, double* virial) {
  if (check_model(m)) return DP_ERR_ARG;
  if (nframes < 0 || (nframes > 0 && (!off || !box || !energy || !virial))) return fail(DP_ERR_ARG, "bad batch arguments");
  if (nframes == 0) return DP_OK;
  // every frame is checked on the host before any of them runs
  int maxn = 0;
  for (int f = 0; f < nframes; ++f) {
    const int n = off[f + 1] - off[f];
    if (n < 0) return fail(DP_ERR_ARG, "atom_offsets must be non-decreasing");
    maxn = std::max(maxn, n);
    int rc = check_box_host(box + 9LL * f, m->rcut);
    if (rc != DP_OK) return rc;
  }
  const long long a0 = off[0], total = (long long)off[nframes] - a0;
  if (total > 0 && (!coord || !atype || !force)) return fail(DP_ERR_ARG, "null host pointer");
  for (long long i = 0; i < total; ++i)
    if (atype[a0 + i] < 0 || atype[a0 + i] >= m->nt) return fail(DP_ERR_ARG, "atom type out of range");
  for (long long i = 0; i < 3 * total; ++i)
    if (!std::isfinite(coord[3 * a0 + i])) return fail(DP_ERR_NAN, "non-finite coordinate");
  CUDA_TRY(cudaSetDevice(m->device));
  // The packed layout: frame f at slots [po[f], po[f+1]), its atom count
  // rounded up to whole force blocks, so that no block of the force kernel
  // holds atoms of two frames and every frame's sums run in the order of a
  // call on that frame alone.
  constexpr int PB = FORCE_BLOCK_ATOMS;
  auto padded = [](long long n) { return (n + PB - 1) / PB * PB; };
  std::vector<long long> po(nframes + 1, 0);
  for (int f = 0; f < nframes; ++f) po[f + 1] = po[f] + padded(off[f + 1] - off[f]);
  const long long P = po[nframes];
  if (P > (long long)INT_MAX) return fail(DP_ERR_CAPACITY, "batch too large");
  // One packed pass holds up to the workspace's atoms; the workspace grows to
  // min(P, BATCH_PACK_ATOMS) slots (at least the largest frame), and a larger
  // batch runs as several passes of consecutive frames.
  const long long want = std::max(padded(maxn), std::min(P, (long long)BATCH_PACK_ATOMS));
  int rc;
  if (want > m->ws.cap && (rc = dp_reserve(m, (int)want)) != DP_OK) {
    if (want == padded(maxn) || (rc = dp_reserve(m, (int)padded(maxn))) != DP_OK) return rc;
  }
  const long long cap = m->ws.cap;
  // host-side maps: pos[i] = the slot of atom i, frame of each slot (-1:
  // padding), and the first force block of each frame
  std::vector<int> pos((size_t)total), frame_of((size_t)P, -1), seg(nframes + 1);
  for (int f = 0; f < nframes; ++f) {
    const long long o = off[f] - a0;
    for (long long k = 0; k < off[f + 1] - off[f]; ++k) {
      pos[(size_t)(o + k)] = (int)(po[f] + k);
      frame_of[(size_t)(po[f] + k)] = f;
    }
  }
  for (int f = 0; f <= nframes; ++f) seg[f] = (int)(po[f] / PB);
  // Every frame's cell grid (cell edge >= rcut, as the device sets it up for
  // a single frame) and the first cell of each frame in a batch-wide count:
  // a pass searches all its frames at once when its cells fit the workspace.
  std::vector<CellGrid> grids(nframes);
  std::vector<long long> cum(nframes + 1, 0);
  std::vector<char> finite(nframes, 1);
  for (int f = 0; f < nframes; ++f) {
    CellGrid g{};
    g.ok = 1;
    for (int d = 0; d < 3; ++d) {
      const double L = box[9LL * f + 4 * d];
      g.L[d] = L;
      if (!std::isfinite(L)) finite[f] = 0;
      int nc = finite[f] ? (int)std::floor(L / (m->rcut * (1.0 + 1e-9))) : 1;
      if (nc < 3) nc = 1;
      if (nc > m->ws.cap_dim) nc = m->ws.cap_dim;
      g.nc[d] = nc;
    }
    g.ncells = g.nc[0] * g.nc[1] * g.nc[2];
    grids[f] = g;
    cum[f + 1] = cum[f] + g.ncells;
  }
  const bool cells_fit_int = cum[nframes] <= (long long)INT_MAX;
  std::vector<int> cbase(nframes + 1);
  for (int f = 0; f <= nframes; ++f) cbase[f] = cells_fit_int ? (int)cum[f] : 0;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t b_coord = up(sizeof(double) * 3 * total), b_type = up(sizeof(int) * total),
               b_box = up(sizeof(double) * 9 * nframes), b_e = up(sizeof(double) * nframes),
               b_coordP = up(sizeof(double) * 3 * P), b_typeP = up(sizeof(int) * P),
               b_grid = up(sizeof(CellGrid) * nframes), b_seg = up(sizeof(int) * (nframes + 1));
  const size_t need = 2 * b_coord + 2 * b_type + 2 * b_box + b_e + 2 * b_coordP + 2 * b_typeP + b_grid + 2 * b_seg;
  if (need > m->batch_cap) {
    if (m->batch_buf) CUDA_TRY(cudaFree(m->batch_buf));
    m->batch_buf = nullptr;
    m->batch_cap = 0;
    if (cudaMalloc(&m->batch_buf, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(DP_ERR_CUDA, "cudaMalloc of the batch buffer failed");
    }
    m->batch_cap = need;
  }
  char* p = reinterpret_cast<char*>(m->batch_buf);
  auto take = [&p](size_t b) { char* q = p; p += b; return q; };
  double* d_coord = reinterpret_cast<double*>(take(b_coord));
  double* d_force = reinterpret_cast<double*>(take(b_coord));
  int* d_type = reinterpret_cast<int*>(take(b_type));
  int* d_pos = reinterpret_cast<int*>(take(b_type));
  double* d_box = reinterpret_cast<double*>(take(b_box));
  double* d_vir = reinterpret_cast<double*>(take(b_box));
  double* d_e = reinterpret_cast<double*>(take(b_e));
  double* d_coordP = reinterpret_cast<double*>(take(b_coordP));
  double* d_forceP = reinterpret_cast<double*>(take(b_coordP));
  int* d_typeP = reinterpret_cast<int*>(take(b_typeP));
  int* d_frame = reinterpret_cast<int*>(take(b_typeP));
  CellGrid* d_grid = reinterpret_cast<CellGrid*>(take(b_grid));
  int* d_seg = reinterpret_cast<int*>(take(b_seg));
  int* d_cbase = reinterpret_cast<int*>(take(b_seg));
  cudaStream_t st = m->stream;
  Workspace& ws = m->ws;
  if (total > 0) {
    CUDA_TRY(cudaMemcpyAsync(d_coord, coord + 3 * a0, sizeof(double) * 3 * total, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d_type, atype + a0, sizeof(int) * total, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d_pos, pos.data(), sizeof(int) * total, cudaMemcpyHostToDevice, st));
    k_batch_pack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(d_coord, d_type, d_pos, total, d_coordP, d_typeP);
    note_launch();
  }
  if (P > 0) CUDA_TRY(cudaMemcpyAsync(d_frame, frame_of.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(d_seg, seg.data(), sizeof(int) * (nframes + 1), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(d_cbase, cbase.data(), sizeof(int) * (nframes + 1), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(d_grid, grids.data(), sizeof(CellGrid) * nframes, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(d_box, box, sizeof(double) * 9 * nframes, cudaMemcpyHostToDevice, st));
  for (int f0 = 0; f0 < nframes;) {
    int f1 = f0 + 1;
    while (f1 < nframes && po[f1 + 1] - po[f0] <= cap) ++f1;
    const long long P0 = po[f0];
    const int Pc = (int)(po[f1] - P0);
    m->last_stream = st;
    m->last_natoms = Pc;
    m->call_nlocal = Pc;  // every slot counts; padding is masked by its frame of -1
    prof_mark(m, "start", st);
    // a1-a2: every frame in its own box and cell grid, neighbour indices
    // relative to the pass; one search over the pass when its cells fit,
    // else one per frame
    bool packed = cells_fit_int && cum[f1] - cum[f0] <= (long long)m->ws.cell_cap;
    for (int f = f0; f < f1 && packed; ++f) packed = finite[f] != 0;
    if (packed) {
      NbrArgs a = nbr_args(m, Pc, d_coordP + 3 * P0, d_box, d_typeP + P0, d_grid, 0);
      launch_neighbors_packed(a, d_frame + P0, d_cbase, cbase[f0], (int)(cum[f1] - cum[f0]), st);
    } else {
      for (int f = f0; f < f1; ++f) {
        const int rel = (int)(po[f] - P0);
        NbrArgs a = nbr_args(m, off[f + 1] - off[f], d_coordP + 3 * po[f], d_box + 9LL * f, d_typeP + po[f],
                             d_grid + f, rel);
        a.n_out = (int)(po[f + 1] - po[f]);
        a.base = rel;
        launch_neighbors(a, st);
      }
    }
    prof_mark(m, "neighbors", st);
    rc = run_after_neighbors(m, Pc, d_coordP + 3 * P0, d_grid, d_frame + P0, d_seg + f0, f1 - f0, d_e + f0,
                             d_forceP + 3 * P0, d_vir + 9LL * f0, nullptr, st);
    if (rc != DP_OK) return rc;
    f0 = f1;
  }
  if (total > 0) {
    k_batch_unpack<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(d_forceP, d_pos, total, d_force);
    note_launch();
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(energy, d_e, sizeof(double) * nframes, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(virial, d_vir, sizeof(double) * 9 * nframes, cudaMemcpyDeviceToHost, st));
  if (total > 0) CUDA_TRY(cudaMemcpyAsync(force + 3 * a0, d_force, sizeof(double) * 3 * total, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return read_status(m);
}

int dp_get_status(dp_model* m) {
  if (check_model(m)) return DP_ERR_ARG;
  CUDA_TRY(cudaSetDevice(m->device));
  if (m->last_stream) CUDA_TRY(cudaStreamSynchronize(m->last_stream));
  CUDA_TRY(cudaDeviceSynchronize());
  return read_status(m);
}

int dp_nlist_device(dp_model* m, int natoms, const double* d_coord, const double* d_box, int* d_nlist, int* d_nnei,
                    void* stream) {
  if (check_model(m)) return DP_ERR_ARG;
  if (natoms < 0 || !d_box || (natoms > 0 && (!d_coord || !d_nlist || !d_nnei))) return fail(DP_ERR_ARG, "bad arguments");
  if (natoms > m->ws.cap) return fail(DP_ERR_CAPACITY, "natoms exceeds the reserved workspace (call dp_reserve)");
  CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // types are not needed for the list: pass a zero-type buffer of the workspace
  CUDA_TRY(cudaMemsetAsync(m->ws.atype, 0, sizeof(int) * (size_t)(natoms > 0 ? natoms : 1), st));
  run_neighbors(m, natoms, d_coord, d_box, m->ws.atype, st);
  if (natoms > 0) {
    CUDA_TRY(cudaMemcpyAsync(d_nlist, m->ws.nlist, sizeof(int) * (size_t)natoms * NP, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d_nnei, m->ws.nnei, sizeof(int) * (size_t)natoms, cudaMemcpyDeviceToDevice, st));
  }
  m->last_stream = st;
  m->last_natoms = natoms;
  return DP_OK;
}

int dp_stats(const dp_model* m, int* max_nnei, long long* n_truncated) {
  if (!m) return fail(DP_ERR_ARG, "model is null");
  const int n = m->last_natoms;
  std::vector<int> nc((size_t)(n > 0 ? n : 1), 0);
  if (n > 0 && cudaMemcpy(nc.data(), m->ws.ncand, sizeof(int) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(DP_ERR_CUDA, "cudaMemcpy failed");
  int mx = 0;
  long long tr = 0;
  for (int i = 0; i < n; ++i) {
    mx = std::max(mx, std::min(nc[i], m->sel));
    if (nc[i] > m->sel) ++tr;
  }
  if (max_nnei) *max_nnei = mx;
  if (n_truncated) *n_truncated = tr;
  return DP_OK;
}

int dp_debug_poison(dp_model* m) {
  if (check_model(m)) return DP_ERR_ARG;
  CUDA_TRY(cudaSetDevice(m->device));
  if (m->ws.mem) CUDA_TRY(cudaMemset(m->ws.mem, 0xFF, m->ws.bytes));
  CUDA_TRY(cudaDeviceSynchronize());
  return DP_OK;
}

long long dp_debug_copy(dp_model* m, const char* name, void* host_dst, size_t bytes) {
  if (check_model(m) || !name || !host_dst) return DP_ERR_ARG;
  Workspace& ws = m->ws;
  const size_t n = (size_t)m->last_natoms, rows = n * NP;
  const void* src = nullptr;
  size_t sz = 0;
  std::string s(name);
  if (s == "nlist") { src = ws.nlist; sz = rows * sizeof(int); }
  else if (s == "env") { src = ws.R; sz = rows * 4 * sizeof(float); }
  else if (s == "g") { src = ws.g; sz = rows * 4 * sizeof(float); }
  else if (s == "e") { src = ws.e; sz = n * sizeof(float); }
  else if (s == "D") { src = ws.X; sz = n * m->fit_in * sizeof(float); }
  else if (s.size() == 2 && s[0] == 'G' && s[1] >= '0' && s[1] - '0' <= m->nattn && !ws.G.empty()) {
    src = ws.G[s[1] - '0']; sz = rows * m->m1 * sizeof(float);
  }
  if (!src) return fail(DP_ERR_ARG, "unknown buffer name");
  sz = std::min(sz, bytes);
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(DP_ERR_CUDA, "sync failed");
  if (s[0] == 'G' && fused_tc_precision(m->precision)) {
    // the tensor-core path keeps G column-quad interleaved per atom: return it row-major
    const size_t m1 = (size_t)m->m1, full = rows * m1;
    std::vector<float> raw(full), out(full);
    if (cudaMemcpy(raw.data(), src, full * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(DP_ERR_CUDA, "copy failed");
    for (size_t atom = 0; atom < n; ++atom)
      for (int r = 0; r < NP; ++r)
        for (size_t c = 0; c < m1; ++c)
          out[(atom * NP + r) * m1 + c] = raw[atom * NP * m1 + cq_off(r, (int)c)];
    memcpy(host_dst, out.data(), sz);
    return (long long)sz;
  }
  if (cudaMemcpy(host_dst, src, sz, cudaMemcpyDeviceToHost) != cudaSuccess) return fail(DP_ERR_CUDA, "copy failed");
  return (long long)sz;
}

int dp_set_profiling(dp_model* m, int on) {
  if (check_model(m)) return DP_ERR_ARG;
  m->prof.on = on != 0;
  m->prof.count = 0;
  return DP_OK;
}

int dp_stage_times(dp_model* m, const char** names, float* ms, int max_stages) {
  if (check_model(m)) return DP_ERR_ARG;
  Profiler& p = m->prof;
  if (!p.on || p.count < 2) return 0;
  CUDA_TRY(cudaEventSynchronize(p.ev[p.count - 1]));
  int k = 0;
  for (int i = 1; i < p.count && k < max_stages; ++i) {
    if (strcmp(p.name[i], "start") == 0) continue;  // the gap between two calls
    float t = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&t, p.ev[i - 1], p.ev[i]));
    if (names) names[k] = p.name[i];
    if (ms) ms[k] = t;
    ++k;
  }
  return k;
}

long long dp_kernel_launches(void) { return g_launches.load(); }

// ------------------------------------------------------------------------
// Allocation-free neighbour list.  Its cell-list scratch is one file-scope
// device array per GPU instead of a model workspace, so the call works for
// callers that must not allocate (see dpa1.h).
namespace {
constexpr int NA_MAX_ATOMS = 65536;
constexpr int NA_CAP_DIM = 32;
constexpr int NA_MAX_CELLS = NA_CAP_DIM * NA_CAP_DIM * NA_CAP_DIM;
struct NoAllocScratch {
  CellGrid grid;
  int cell_count[NA_MAX_CELLS];
  int cell_start[NA_MAX_CELLS + 1];
  int cell_cursor[NA_MAX_CELLS];
  int cell_of[NA_MAX_ATOMS];
  int cell_atoms[NA_MAX_ATOMS];
  int ncand[NA_MAX_ATOMS];
  int types[NA_MAX_ATOMS];    // all zero: the list does not depend on types
  int types_c[NA_MAX_ATOMS];
  float4 coordf[NA_MAX_ATOMS];  // FP32 coordinates for the candidate screen
};
__device__ __align__(256) NoAllocScratch g_nbr_scratch;
constexpr int NA_MAX_DEVICES = 64;
NoAllocScratch* g_nbr_scratch_addr[NA_MAX_DEVICES] = {};
std::mutex g_nbr_scratch_mutex;
}  // namespace

int dp_nlist_noalloc(int natoms, const double* d_coord, const double* d_box, double rcut, int sel, int* d_nlist,
                     int* d_nnei, int* d_status, void* stream) {
  if (natoms < 0 || natoms > NA_MAX_ATOMS)
    return fail(DP_ERR_CAPACITY, "dp_nlist_noalloc: natoms must be between 0 and " + std::to_string(NA_MAX_ATOMS));
  if (!d_box || !d_status || (natoms > 0 && (!d_coord || !d_nlist || !d_nnei)))
    return fail(DP_ERR_ARG, "dp_nlist_noalloc: null device pointer");
  if (!(rcut > 0.0) || sel < 1 || sel > NP) return fail(DP_ERR_ARG, "dp_nlist_noalloc: need rcut > 0 and 1 <= sel <= 128");
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NA_MAX_DEVICES) return fail(DP_ERR_ARG, "dp_nlist_noalloc: device ordinal out of range");
  NoAllocScratch* s = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_nbr_scratch_mutex);
    if (!g_nbr_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_nbr_scratch);
      if (e != cudaSuccess || !p)
        return fail(DP_ERR_CUDA, std::string("dp_nlist_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      g_nbr_scratch_addr[dev] = reinterpret_cast<NoAllocScratch*>(p);
    }
    s = g_nbr_scratch_addr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  if (natoms > 0) CUDA_TRY(cudaMemsetAsync(s->types, 0, sizeof(int) * (size_t)natoms, st));
  NbrArgs a;
  a.coord = d_coord; a.box = d_box; a.atype = s->types;
  a.n = natoms; a.ntypes = 1; a.sel = sel; a.rcut = rcut;
  a.cap_dim = NA_CAP_DIM; a.cell_cap = NA_MAX_CELLS; a.grid = &s->grid;
  a.cell_of = s->cell_of; a.cell_count = s->cell_count; a.cell_start = s->cell_start;
  a.cell_cursor = s->cell_cursor; a.cell_atoms = s->cell_atoms;
  a.nlist = d_nlist; a.nnei = d_nnei; a.ncand = s->ncand; a.atype_c = s->types_c; a.coordf = s->coordf;
  a.err = d_status;
  launch_neighbors(a, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DP_ERR_CUDA, std::string("dp_nlist_noalloc: launch failed: ") + cudaGetErrorString(e));
  return DP_OK;
}

int dp_param_count(const dp_model* m) { return m ? m->ntheta : DP_ERR_ARG; }

int dp_get_params(dp_model* m, float* host, int count) {
  if (check_model(m) || !host || count != m->ntheta) return fail(DP_ERR_ARG, "dp_get_params: bad buffer");
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(host, m->theta, sizeof(float) * count, cudaMemcpyDeviceToHost));
  return DP_OK;
}

int dp_set_params(dp_model* m, const float* host, int count) {
  if (check_model(m) || !host || count != m->ntheta) return fail(DP_ERR_ARG, "dp_set_params: bad buffer");
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(m->theta, host, sizeof(float) * count, cudaMemcpyHostToDevice));
  refresh_derived(m, nullptr);
  CUDA_TRY(cudaDeviceSynchronize());
  return DP_OK;
}

int dp_get_grad(dp_model* m, float* host, int count) {
  if (check_model(m) || !host || count != m->ntheta) return fail(DP_ERR_ARG, "dp_get_grad: bad buffer");
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(host, m->grad, sizeof(float) * count, cudaMemcpyDeviceToHost));
  return DP_OK;
}

int dp_zero_grad(dp_model* m, void* stream) {
  if (check_model(m)) return DP_ERR_ARG;
  CUDA_TRY(cudaSetDevice(m->device));
  CUDA_TRY(cudaMemsetAsync(m->grad, 0, sizeof(float) * m->ntheta, reinterpret_cast<cudaStream_t>(stream)));
  return DP_OK;
}

int dp_train_frame(dp_model* m, int natoms, const double* d_coord, const double* d_box, const int* d_atype,
                   double e_ref, const double* d_force_ref, double pe, double pf, double* d_loss, void* stream) {
  if (check_model(m)) return DP_ERR_ARG;
  if ((m->precision != DP_PREC_FP32 && m->precision != DP_PREC_BF16X) || m->nattn != 0)
    return fail(DP_ERR_UNSUPPORTED,
                "dp_train_frame: training needs a model without attention layers in DP_PREC_FP32 or DP_PREC_BF16X");
  if (natoms < 1 || !d_coord || !d_box || !d_atype || !d_force_ref || !d_loss)
    return fail(DP_ERR_ARG, "dp_train_frame: bad arguments");
  if (natoms > m->ws.cap) return fail(DP_ERR_CAPACITY, "natoms exceeds the reserved workspace (call dp_reserve)");
  CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int cap = m->ws.cap, m1 = m->m1, nfit = m->nfit;
  const size_t rows = (size_t)cap * NP;
  int fmax = m->fit_in;
  for (int l = 0; l < nfit; ++l) fmax = std::max(fmax, m->fit[l]);
  struct TrainBufs {
    double *energy, *virial, *force, *v;
    float *gE, *Rd, *Gd, *dGd, *Td, *Xd, *dXd, *dH[2], *dHd[2], *dZ, *dZd, *Zd;
    std::vector<float*> Hd;
  } b;
  auto plan = [&](Arena& a) {
    b.energy = a.take<double>(1);
    b.virial = a.take<double>(9);
    b.force = a.take<double>((size_t)cap * 3);
    b.v = a.take<double>((size_t)cap * 3);
    b.gE = a.take<float>((size_t)m->ntheta);
    b.Rd = a.take<float>(rows * 4);
    b.Gd = a.take<float>(rows * m1);
    b.dGd = a.take<float>(rows * m1);
    b.Td = a.take<float>((size_t)cap * 4 * m1);
    b.Xd = a.take<float>((size_t)cap * m->fit_in);
    b.dXd = a.take<float>((size_t)cap * m->fit_in);
    b.Hd.assign(nfit, nullptr);
    for (int l = 0; l < nfit; ++l) b.Hd[l] = a.take<float>((size_t)cap * m->fit[l]);
    for (int k = 0; k < 2; ++k) {
      b.dH[k] = a.take<float>((size_t)cap * fmax);
      b.dHd[k] = a.take<float>((size_t)cap * fmax);
    }
    b.dZ = a.take<float>((size_t)cap * fmax);
    b.dZd = a.take<float>((size_t)cap * fmax);
    b.Zd = a.take<float>((size_t)cap * fmax);
  };
  Arena probe;
  plan(probe);
  if (m->t_cap != cap || !m->t_buf) {
    if (m->t_buf) CUDA_TRY(cudaFree(m->t_buf));
    m->t_buf = nullptr;
    m->t_cap = 0;
    if (cudaMalloc(&m->t_buf, probe.off) != cudaSuccess) {
      cudaGetLastError();
      return fail(DP_ERR_CUDA, "dp_train_frame: cudaMalloc of the training buffer failed");
    }
    m->t_cap = cap;
  }
  Arena real;
  real.base = reinterpret_cast<char*>(m->t_buf);
  real.cap = probe.off;
  plan(real);
  // 1. the energy evaluation, with dE/dtheta (unscaled) into gE
  CUDA_TRY(cudaMemsetAsync(b.gE, 0, sizeof(float) * (size_t)m->ntheta, st));
  float* grad_keep = m->grad;
  m->grad = b.gE;
  m->grad_scale = m->d_scales;  // 1
  int rc = run_device(m, natoms, natoms, d_coord, d_box, d_atype, b.energy, b.force, b.virial, nullptr, st);
  m->grad = grad_keep;
  m->grad_scale = nullptr;
  if (rc != DP_OK) return rc;
  // 2. loss, scales and v = F - F_ref; the energy term of the gradient
  launch_train_prep(natoms, b.energy, e_ref, b.force, d_force_ref, pe, pf, b.v, d_loss, m->d_scales, st);
  launch_axpy(m->grad, b.gE, m->ntheta, m->d_scales + 1, st);
  // 3. the force term: the tangent of dE/dtheta along v, scaled by -2 pf / 3N
  run_force_tangent(m, natoms, d_coord, b.v, b.Rd, b.Gd, b.dGd, b.Td, b.Xd, b.dXd, b.Hd, b.dH, b.dHd, b.dZ, b.dZd,
                    b.Zd, m->d_scales + 2, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DP_ERR_CUDA, std::string("dp_train_frame: launch failed: ") + cudaGetErrorString(e));
  return DP_OK;
}

int dp_adam_step(dp_model* m, double lr, double beta1, double beta2, double eps, void* stream) {
  if (check_model(m)) return DP_ERR_ARG;
  if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return fail(DP_ERR_ARG, "dp_adam_step: bad hyper-parameters");
  CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int t = ++m->adam_t;
  const float bc1 = (float)(1.0 - std::pow(beta1, t)), bc2 = (float)(1.0 - std::pow(beta2, t));
  launch_adam(m->theta, m->grad, m->adam_m, m->adam_v, m->ntheta, (float)lr, (float)beta1, (float)beta2, (float)eps,
              bc1, bc2, st);
  refresh_derived(m, st);
  return DP_OK;
}

int dp_md_run(dp_model* m, int natoms, double* d_coord, double* d_vel, const double* d_mass, const double* d_box,
              const int* d_atype, double dt, int nsteps, double* d_force, double* d_energy, double* d_virial,
              double* d_thermo, int use_graph, void* stream) {
  if (check_model(m)) return DP_ERR_ARG;
  if (natoms < 0 || nsteps < 0 || !(dt > 0.0)) return fail(DP_ERR_ARG, "dp_md_run: need natoms >= 0, nsteps >= 0, dt > 0");
  if (!d_box || !d_energy || !d_virial || !d_thermo ||
      (natoms > 0 && (!d_coord || !d_vel || !d_mass || !d_atype || !d_force)))
    return fail(DP_ERR_ARG, "dp_md_run: null device pointer");
  if (natoms > m->ws.cap) return fail(DP_ERR_CAPACITY, "natoms exceeds the reserved workspace (call dp_reserve)");
  CUDA_TRY(cudaSetDevice(m->device));
  cudaStream_t st = stream ? reinterpret_cast<cudaStream_t>(stream) : m->stream;
  if (!m->d_md_counter) {
    void* p = nullptr;
    CUDA_TRY(cudaMalloc(&p, sizeof(int)));
    m->d_md_counter = reinterpret_cast<int*>(p);
  }
  const int nb_cap = verlet_kick_blocks(m->ws.cap);
  if (!m->d_md_partial || m->md_partial_cap < nb_cap) {
    if (m->d_md_partial) cudaFree(m->d_md_partial);
    m->d_md_partial = nullptr;
    m->md_partial_cap = 0;
    void* p = nullptr;
    CUDA_TRY(cudaMalloc(&p, sizeof(double) * (size_t)(nb_cap > 0 ? nb_cap : 1)));
    m->d_md_partial = reinterpret_cast<double*>(p);
    m->md_partial_cap = nb_cap;
  }
  CUDA_TRY(cudaMemsetAsync(m->d_md_counter, 0, sizeof(int), st));
  // forces at the starting coordinates
  int rc = run_device(m, natoms, natoms, d_coord, d_box, d_atype, d_energy, d_force, d_virial, nullptr, st);
  if (rc != DP_OK) return rc;
  const bool prof = m->prof.on;
  auto one_step = [&]() -> int {
    launch_verlet_drift(natoms, dt, d_mass, d_force, d_vel, d_coord, st);
    int r = run_device(m, natoms, natoms, d_coord, d_box, d_atype, d_energy, d_force, d_virial, nullptr, st);
    launch_verlet_kick(natoms, dt, d_mass, d_force, d_vel, m->d_md_partial, d_energy, m->d_md_counter, d_thermo,
                       nsteps, st);
    return r;
  };
  if (!use_graph) {
    for (int s = 0; s < nsteps; ++s)
      if ((rc = one_step()) != DP_OK) return rc;
  } else if (nsteps > 0) {
    const double dtv = dt;
    const void* key_dt = nullptr;
    memcpy(&key_dt, &dtv, sizeof(dtv) < sizeof(key_dt) ? sizeof(dtv) : sizeof(key_dt));
    std::vector<const void*> key = {d_coord, d_vel, d_mass, d_box, d_atype, d_force, d_energy, d_virial, d_thermo,
                                    m->d_md_partial,
                                    reinterpret_cast<const void*>((intptr_t)natoms),
                                    reinterpret_cast<const void*>((intptr_t)nsteps),
                                    reinterpret_cast<const void*>((intptr_t)m->precision), key_dt};
    if (!m->md_exec || m->md_key != key) {
      if (m->md_exec) { cudaGraphExecDestroy(m->md_exec); m->md_exec = nullptr; }
      if (m->md_graph) { cudaGraphDestroy(m->md_graph); m->md_graph = nullptr; }
      m->prof.on = false;  // no event nodes inside the graph
      CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
      rc = one_step();
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(st, &g);
      m->prof.on = prof;
      if (rc != DP_OK) { if (g) cudaGraphDestroy(g); return rc; }
      if (e != cudaSuccess) return fail(DP_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(e));
      m->md_graph = g;
      CUDA_TRY(cudaGraphInstantiate(&m->md_exec, g, 0));
      m->md_key = key;
    }
    for (int s = 0; s < nsteps; ++s) CUDA_TRY(cudaGraphLaunch(m->md_exec, st));
  }
  if (!stream) CUDA_TRY(cudaStreamSynchronize(st));
  return DP_OK;
}

void dp_free(dp_model* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  free_workspace(m->ws);
  tc_free_weights(m);
  bf16x_free(m);
  for (void* p : m->allocations) cudaFree(p);
  if (m->d_err) cudaFree(m->d_err);
  if (m->stream) cudaStreamDestroy(m->stream);
  for (auto& e : m->prof.ev)
    if (e) cudaEventDestroy(e);
  if (m->md_exec) cudaGraphExecDestroy(m->md_exec);
  if (m->md_graph) cudaGraphDestroy(m->md_graph);
  if (m->d_md_counter) cudaFree(m->d_md_counter);
  if (m->d_md_partial) cudaFree(m->d_md_partial);
  if (m->batch_buf) cudaFree(m->batch_buf);
  if (m->t_buf) cudaFree(m->t_buf);
  delete m;
}

}  // extern "C"
