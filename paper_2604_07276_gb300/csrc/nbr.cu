// Stages a1-a2: cell binning and the full neighbour list (Sec. II-C: DP
// models need full lists; the O(N) cutoff search of Sec. II-A), plus the
// reverse list used by the deterministic force gather.
#include "common.cuh"
#include "kernels.h"

namespace dpa1 {

// One thread: validate the box and derive the cell grid.  Cell edges are
// >= rcut, so every neighbour of an atom lies in the 27 cells around it; an
// axis with fewer than 3 cells is treated as a single cell (no cell would
// otherwise be visited twice).
__global__ void k_cell_setup(const double* __restrict__ box, double rcut, int cap_dim,
                             CellGrid* __restrict__ cg, int* __restrict__ err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  CellGrid g;
  g.ok = 1;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b)
      if (a != b && box[3 * a + b] != 0.0) g.ok = 0;
    double L = box[4 * a];
    g.L[a] = L;
    if (!(L > 2.0 * rcut) || !isfinite(L)) g.ok = 0;
    int nc = g.ok ? (int)floor(L / (rcut * (1.0 + 1e-9))) : 1;
    if (nc < 3) nc = 1;
    if (nc > cap_dim) nc = cap_dim;
    g.nc[a] = nc;
  }
  g.ncells = g.nc[0] * g.nc[1] * g.nc[2];
  if (!g.ok) {
    set_err(err, ERR_BOX);
    g.nc[0] = g.nc[1] = g.nc[2] = 1;
    g.ncells = 1;
    g.L[0] = g.L[1] = g.L[2] = 1.0;
  }
  *cg = g;
}

__device__ __forceinline__ int cell_coord(double x, double L, int nc) {
  double w = x - L * floor(x / L);
  int c = (int)(w * (double)nc / L);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// frame non-null (packed batches): slot i belongs to frame frame[i] (-1:
// padding, no cell) with grid cgp[f] and cells from cell_base[f] - cb0 on.
__global__ void k_cell_count(const double* __restrict__ coord, const int* __restrict__ atype, int n,
                             int ntypes, const CellGrid* __restrict__ cgp, int* __restrict__ cell_of,
                             int* __restrict__ cell_count, int* __restrict__ atype_c, float4* __restrict__ coordf,
                             int* __restrict__ err, const int* __restrict__ frame, const int* __restrict__ cell_base,
                             int cb0) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int cbase = 0;
  const CellGrid* gp = cgp;
  if (frame) {
    const int f = frame[i];
    if (f < 0) {
      atype_c[i] = 0;
      cell_of[i] = -1;
      return;
    }
    gp = cgp + f;
    cbase = cell_base[f] - cb0;
  }
  const CellGrid g = *gp;
  double x = coord[3 * i], y = coord[3 * i + 1], z = coord[3 * i + 2];
  coordf[i] = make_float4((float)x, (float)y, (float)z, 0.f);
  int c = 0;
  if (!isfinite(x) || !isfinite(y) || !isfinite(z)) {
    set_err(err, ERR_NAN);
  } else {
    int cx = cell_coord(x, g.L[0], g.nc[0]);
    int cy = cell_coord(y, g.L[1], g.nc[1]);
    int cz = cell_coord(z, g.L[2], g.nc[2]);
    c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
  }
  c += cbase;
  int t = atype[i];
  if (t < 0 || t >= ntypes) {
    set_err(err, ERR_TYPE);
    t = t < 0 ? 0 : ntypes - 1;  // every later table lookup stays in bounds
  }
  atype_c[i] = t;
  cell_of[i] = c;
  atomicAdd(&cell_count[c], 1);
}

// Exclusive scan of the cell counts (one block).
__global__ void k_cell_scan(const int* __restrict__ cell_count, int* __restrict__ cell_start,
                            const CellGrid* __restrict__ cgp, int ncells_given) {
  __shared__ int part[1024];
  __shared__ int carry;
  const int ncells = ncells_given >= 0 ? ncells_given : cgp->ncells;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ncells; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < ncells ? cell_count[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < ncells) cell_start[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) cell_start[ncells] = carry;
}

__global__ void k_cell_fill(const int* __restrict__ cell_of, int n, const int* __restrict__ cell_start,
                            int* __restrict__ cell_cursor, int* __restrict__ cell_atoms) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell_of[i];
  if (c < 0) return;  // padding of a packed batch
  int pos = cell_start[c] + atomicAdd(&cell_cursor[c], 1);
  cell_atoms[pos] = i;
}

// Sort keys: the bit pattern of d^2 >= 0 (+0 or positive, never NaN) read as an
// unsigned integer orders like the value, so the sort needs no FP64 compare.
__device__ __forceinline__ bool key_gt(unsigned long long da, int ja, unsigned long long db, int jb) {
  return da > db || (da == db && ja > jb);
}

// mic() without its division when no image shift is possible: for |d| < L/2
// the rounded d / L lies in [-0.5, 0.5], rint gives 0 and mic returns d up to
// the sign of a zero, which the squared distance does not see.
__device__ __forceinline__ double mic_near(double d, double L) {
  return fabs(d) < 0.5 * L ? d : mic(d, L);
}

// One warp per centre atom: gather every candidate j != i with d^2 < rc^2 from
// the 27 surrounding cells (screened in FP32, decided in FP64 and
// bit-reproducible), then bitonic-sort the candidates by (d^2, j) and keep the
// first sel.  FP64 is slow on this part, so it is kept to the ~11 % of
// candidates that pass the screen.
constexpr int NBR_WARPS = 4;
// 10 blocks per SM (48 registers, no spills): the search is latency-bound and
// gains from the extra resident warps
__global__ void __launch_bounds__(32 * NBR_WARPS, 10)
k_neighbors(const double* __restrict__ coord, int n, int n_out, int base, const CellGrid* __restrict__ cgp,
            const int* __restrict__ cell_of, const int* __restrict__ cell_start,
            const int* __restrict__ cell_atoms, double rc2, int sel, int* __restrict__ nlist,
            int* __restrict__ nnei, int* __restrict__ ncand, int* __restrict__ atype_c,
            const float4* __restrict__ coordf, int* __restrict__ err, const int* __restrict__ frame,
            const int* __restrict__ cell_base, int cb0) {
  __shared__ unsigned long long skey[NBR_WARPS][NBR_CAP];
  __shared__ int sidx[NBR_WARPS][NBR_CAP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * NBR_WARPS + warp;
  const int fi = frame && i < n ? frame[i] : 0;
  if (i >= n || fi < 0) {
    // padding atoms of a packed batch: no neighbours, a valid type
    if (i < n_out || (i < n && fi < 0)) {
      for (int s = lane; s < NP; s += 32) nlist[(size_t)i * NP + s] = -1;
      if (lane == 0) {
        nnei[i] = 0;
        ncand[i] = 0;
        atype_c[i] = 0;
      }
    }
    return;
  }
  const CellGrid g = cgp[frame ? fi : 0];
  const int cbase = frame ? cell_base[fi] - cb0 : 0;  // the frame's first cell
  unsigned long long* key = skey[warp];
  int* idx = sidx[warp];
  const double xi = coord[3 * i], yi = coord[3 * i + 1], zi = coord[3 * i + 2];
  const float4 pi = coordf[i];
  const int ci = cell_of[i] - cbase;
  const int cx = ci % g.nc[0], cy = (ci / g.nc[0]) % g.nc[1], cz = ci / (g.nc[0] * g.nc[1]);
  const int ox = g.nc[0] >= 3 ? 1 : 0, oy = g.nc[1] >= 3 ? 1 : 0, oz = g.nc[2] >= 3 ? 1 : 0;
  const float Lf[3] = {(float)g.L[0], (float)g.L[1], (float)g.L[2]};
  const float iLf[3] = {1.0f / Lf[0], 1.0f / Lf[1], 1.0f / Lf[2]};
  const float rc2_screen = (float)rc2 * 1.0001f + 1e-4f;
  // pass 1: FP32 screen of every candidate in the 27 cells; survivors are
  // compacted into idx[] so that the FP64 decision below runs on full warps
  // (this part's FP64 rate is low, and a divergent FP64 branch costs the whole
  // warp)
  // a neighbouring cell's index along an axis, wrapped without a division
  // (offsets are -1, 0 or +1)
  auto wrap = [](int x, int nc) { return x < 0 ? x + nc : (x >= nc ? x - nc : x); };
  int ns = 0;
  for (int dz = -oz; dz <= oz; ++dz)
    for (int dy = -oy; dy <= oy; ++dy)
      for (int dx = -ox; dx <= ox; ++dx) {
        const int nx = wrap(cx + dx, g.nc[0]);
        const int ny = wrap(cy + dy, g.nc[1]);
        const int nz = wrap(cz + dz, g.nc[2]);
        int c = cbase + (nz * g.nc[1] + ny) * g.nc[0] + nx;
        int b = cell_start[c], e = cell_start[c + 1];
        for (int base = b; base < e; base += 32) {
          int t = base + lane;
          bool pass = false;
          int j = -1;
          if (t < e) {
            j = cell_atoms[t];
            // a component of the FP32 difference is off by at most ~1e-5 A
            // and the squared distance near rc^2 by ~1.3e-4 A^2, far inside
            // the margin, so a pair rejected here is never a neighbour (where
            // FP32 and FP64 pick different images, both distances exceed
            // L/2 > rcut)
            const float4 pj = coordf[j];
            float fx = pj.x - pi.x, fy = pj.y - pi.y, fz = pj.z - pi.z;
            fx -= Lf[0] * rintf(fx * iLf[0]);
            fy -= Lf[1] * rintf(fy * iLf[1]);
            fz -= Lf[2] * rintf(fz * iLf[2]);
            pass = j != i && fx * fx + fy * fy + fz * fz < rc2_screen;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, pass);
          const int pos = ns + __popc(bal & ((1u << lane) - 1u));
          if (pass && pos < NBR_CAP) idx[pos] = j;
          ns += __popc(bal);
        }
      }
  if (ns > NBR_CAP) {
    if (lane == 0) set_err(err, ERR_CAPACITY);
    ns = NBR_CAP;
  }
  __syncwarp();
  // pass 2: the exact FP64 decision on the survivors, compacted in place
  // (a write never reaches an entry that is still to be read)
  int cnt = 0;
  for (int base = 0; base < ns; base += 32) {
    const int t = base + lane;
    bool hit = false;
    double d2 = 0.0;
    int j = -1;
    if (t < ns) {
      j = idx[t];
      const double ddx = mic_near(__dsub_rn(coord[3 * j], xi), g.L[0]);
      const double ddy = mic_near(__dsub_rn(coord[3 * j + 1], yi), g.L[1]);
      const double ddz = mic_near(__dsub_rn(coord[3 * j + 2], zi), g.L[2]);
      d2 = sqdist(ddx, ddy, ddz);
      hit = d2 < rc2;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    const int pos = cnt + __popc(bal & ((1u << lane) - 1u));
    if (hit) {
      key[pos] = (unsigned long long)__double_as_longlong(d2);
      idx[pos] = j;
    }
    cnt += __popc(bal);
    __syncwarp();
  }
  if (lane == 0) ncand[i] = cnt;
  int P = 1;
  while (P < cnt) P <<= 1;
  for (int t = cnt + lane; t < P; t += 32) {
    key[t] = 0x7ff0000000000000ULL;  // +inf
    idx[t] = 0x7fffffff;
  }
  __syncwarp();
  // the bitonic network, a lane per compare-exchange pair (t, t + jj): pair
  // q has t = q with a zero bit inserted at jj
  for (int k = 2; k <= P; k <<= 1)
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      for (int q = lane; q < (P >> 1); q += 32) {
        const int t = ((q & ~(jj - 1)) << 1) | (q & (jj - 1)), o = t | jj;
        const bool asc = (t & k) == 0;
        const unsigned long long ka = key[t], kb = key[o];
        const int ia = idx[t], ib = idx[o];
        const bool sw = asc ? key_gt(ka, ia, kb, ib) : key_gt(kb, ib, ka, ia);
        if (sw) {
          key[t] = kb; key[o] = ka;
          idx[t] = ib; idx[o] = ia;
        }
      }
      __syncwarp();
    }
  const int keep = cnt < sel ? cnt : sel;
  for (int s = lane; s < NP; s += 32) nlist[(size_t)i * NP + s] = s < keep ? idx[s] + base : -1;
  if (lane == 0) nnei[i] = keep;
}

// Reverse list: for every kept pair (i, slot) -> j, record row i*NP+slot under j.
__global__ void k_rev_fill(const int* __restrict__ nlist, int n, int* __restrict__ rev_cnt,
                           int* __restrict__ rev_rows, int* __restrict__ err) {
  long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long long)n * NP) return;
  int j = nlist[row];
  if (j < 0) return;
  int pos = atomicAdd(&rev_cnt[j], 1);
  if (pos < REV_CAP)
    rev_rows[(size_t)j * REV_CAP + pos] = (int)row;
  else
    set_err(err, ERR_CAPACITY);
}

void launch_neighbors(const NbrArgs& a, cudaStream_t st) {
  cudaMemsetAsync(a.cell_count, 0, sizeof(int) * (size_t)a.cell_cap, st);
  cudaMemsetAsync(a.cell_cursor, 0, sizeof(int) * (size_t)a.cell_cap, st);
  k_cell_setup<<<1, 1, 0, st>>>(a.box, a.rcut, a.cap_dim, a.grid, a.err);
  note_launch();
  const int n_out = a.n_out > a.n ? a.n_out : a.n;
  if (n_out == 0) return;
  const int tb = 256;
  if (a.n > 0) {
    k_cell_count<<<(a.n + tb - 1) / tb, tb, 0, st>>>(a.coord, a.atype, a.n, a.ntypes, a.grid, a.cell_of,
                                                    a.cell_count, a.atype_c, a.coordf, a.err, nullptr, nullptr, 0);
    note_launch();
    k_cell_scan<<<1, 1024, 0, st>>>(a.cell_count, a.cell_start, a.grid, -1);
    note_launch();
    k_cell_fill<<<(a.n + tb - 1) / tb, tb, 0, st>>>(a.cell_of, a.n, a.cell_start, a.cell_cursor, a.cell_atoms);
    note_launch();
  }
  k_neighbors<<<(n_out + NBR_WARPS - 1) / NBR_WARPS, 32 * NBR_WARPS, 0, st>>>(
      a.coord, a.n, n_out, a.base, a.grid, a.cell_of, a.cell_start, a.cell_atoms, a.rcut * a.rcut, a.sel, a.nlist,
      a.nnei, a.ncand, a.atype_c, a.coordf, a.err, nullptr, nullptr, 0);
  note_launch();
}

void launch_neighbors_packed(const NbrArgs& a, const int* frame, const int* cell_base, int cb0, int ncells_total,
                             cudaStream_t st) {
  if (a.n == 0) return;
  cudaMemsetAsync(a.cell_count, 0, sizeof(int) * (size_t)ncells_total, st);
  cudaMemsetAsync(a.cell_cursor, 0, sizeof(int) * (size_t)ncells_total, st);
  const int tb = 256;
  k_cell_count<<<(a.n + tb - 1) / tb, tb, 0, st>>>(a.coord, a.atype, a.n, a.ntypes, a.grid, a.cell_of, a.cell_count,
                                                  a.atype_c, a.coordf, a.err, frame, cell_base, cb0);
  note_launch();
  k_cell_scan<<<1, 1024, 0, st>>>(a.cell_count, a.cell_start, a.grid, ncells_total);
  note_launch();
  k_cell_fill<<<(a.n + tb - 1) / tb, tb, 0, st>>>(a.cell_of, a.n, a.cell_start, a.cell_cursor, a.cell_atoms);
  note_launch();
  k_neighbors<<<(a.n + NBR_WARPS - 1) / NBR_WARPS, 32 * NBR_WARPS, 0, st>>>(
      a.coord, a.n, a.n, 0, a.grid, a.cell_of, a.cell_start, a.cell_atoms, a.rcut * a.rcut, a.sel, a.nlist, a.nnei,
      a.ncand, a.atype_c, a.coordf, a.err, frame, cell_base, cb0);
  note_launch();
}

void launch_reverse(const int* nlist, int n, int* rev_cnt, int* rev_rows, int* err, cudaStream_t st) {
  cudaMemsetAsync(rev_cnt, 0, sizeof(int) * (size_t)(n > 0 ? n : 1), st);
  if (n == 0) return;
  long long rows = (long long)n * NP;
  k_rev_fill<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(nlist, n, rev_cnt, rev_rows, err);
  note_launch();
}

}  // namespace dpa1
