// Stage a3 (smooth environment matrix), a14 (its adjoint: the per-pair
// gradient g_ij = dE/dr_ij) and a15 (forces and virial), plus the FP64
// energy reduction a9.
#include "common.cuh"
#include "kernels.h"

namespace dpa1 {

// Smooth environment matrix (Sec. II-B, DP-SE): s(r) = w(r)/r with the C2
// switch w, a row R_ij = (s, s x/r, s y/r, s z/r) normalised per centre type
// by (R - davg)/dstd.  Displacements come from the FP64 coordinates through
// the minimum image.  Real = double (the FP32 path) evaluates the row in FP64;
// Real = float (the 16-bit paths) rounds the FP64 displacement to FP32 and
// evaluates the rest in FP32, which keeps this part's error at ~1e-7
// relative, far below those paths' operand rounding.  Both store FP32.
template <typename Real>
__global__ void k_env(EnvArgs a) {
  long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long long)a.n * NP) return;
  const int i = (int)(row / NP);
  const int j = a.nlist[row];
  float4 R = make_float4(0.f, 0.f, 0.f, 0.f), rw = R, rv = R;
  double w64 = 0.0;
  if (j >= 0) {
    const CellGrid g = a.frame ? a.grid[a.frame[i]] : *a.grid;
    const double ex = a.coord[3 * j] - a.coord[3 * i];
    const double ey = a.coord[3 * j + 1] - a.coord[3 * i + 1];
    const double ez = a.coord[3 * j + 2] - a.coord[3 * i + 2];
    // no image shift inside half a box: skip the FP64 division of mic()
    const Real dx = (Real)(fabs(ex) < 0.5 * g.L[0] ? ex : mic(ex, g.L[0]));
    const Real dy = (Real)(fabs(ey) < 0.5 * g.L[1] ? ey : mic(ey, g.L[1]));
    const Real dz = (Real)(fabs(ez) < 0.5 * g.L[2] ? ez : mic(ez, g.L[2]));
    const Real d = sqrt(dx * dx + dy * dy + dz * dz);
    const Real rcs = a.rcs, rc = a.rc;
    Real sw;
    if (d < rcs) {
      sw = 1;
    } else if (d < rc) {
      const Real u = (d - rcs) / (rc - rcs);
      sw = u * u * u * ((Real)-6 * u * u + (Real)15 * u - (Real)10) + (Real)1;
    } else {
      sw = 0;
    }
    const Real inv_d = (Real)1 / d;
    const Real s = sw * inv_d;
    const Real hx = dx * inv_d, hy = dy * inv_d, hz = dz * inv_d;
    const int t = a.atype[i];
    const float* av = a.davg + 4 * t;
    const float* sv = a.dstd + 4 * t;
    R = make_float4((float)((s - (Real)av[0]) / (Real)sv[0]), (float)((s * hx - (Real)av[1]) / (Real)sv[1]),
                    (float)((s * hy - (Real)av[2]) / (Real)sv[2]), (float)((s * hz - (Real)av[3]) / (Real)sv[3]));
    rw = make_float4((float)hx, (float)hy, (float)hz, (float)sw);
    rv = make_float4((float)dx, (float)dy, (float)dz, (float)d);
    w64 = sw;
  }
  if (a.w64) a.w64[row] = w64;
  reinterpret_cast<float4*>(a.R)[row] = R;
  reinterpret_cast<float4*>(a.rw)[row] = rw;
  reinterpret_cast<float4*>(a.rv)[row] = rv;
}

void launch_env(const EnvArgs& a, cudaStream_t st) {
  long long rows = (long long)a.n * NP;
  if (rows == 0) return;
  if (a.fp64)
    k_env<double><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a);
  else
    k_env<float><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a);
  note_launch();
}

// Chain rule from dE/dR (4 columns), dE/dw and dE/drhat back to r_ij:
//   R0 = s(d), R1..3 = q(d) r with q = s/d, w = sw(d), rhat = r/d.
// Real = double recomputes r_ij from the FP64 coordinates (the FP32 path);
// Real = float uses the stored FP32 displacement.
template <typename Real>
__global__ void k_env_bwd(EnvBwdArgs a) {
  long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= (long long)a.n * NP) return;
  float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
  const int j = a.nlist[row];
  if (j >= 0) {
    const int i = (int)(row / NP);
    Real rx, ry, rz;
    if (sizeof(Real) == 8) {
      const CellGrid g = a.frame ? a.grid[a.frame[i]] : *a.grid;
      rx = (Real)mic(a.coord[3 * j] - a.coord[3 * i], g.L[0]);
      ry = (Real)mic(a.coord[3 * j + 1] - a.coord[3 * i + 1], g.L[1]);
      rz = (Real)mic(a.coord[3 * j + 2] - a.coord[3 * i + 2], g.L[2]);
    } else {
      const float4 rv = reinterpret_cast<const float4*>(a.rv)[row];
      rx = rv.x; ry = rv.y; rz = rv.z;
    }
    const float4 dR = reinterpret_cast<const float4*>(a.dR)[row];
    const float4 dg = reinterpret_cast<const float4*>(a.dgeo)[row];
    const int t = a.atype[i];
    const Real d = sqrt(rx * rx + ry * ry + rz * rz);
    const Real inv = Real(1) / d;
    const Real hx = rx * inv, hy = ry * inv, hz = rz * inv;
    const Real rcs = a.rcs, rc = a.rc;
    Real sw, dsw;
    if (d < rcs) {
      sw = 1; dsw = 0;
    } else if (d < rc) {
      const Real wdt = rc - rcs;
      const Real u = (d - rcs) / wdt;
      sw = u * u * u * (Real(-6) * u * u + Real(15) * u - Real(10)) + Real(1);
      dsw = Real(-30) * u * u * (u - Real(1)) * (u - Real(1)) / wdt;
    } else {
      sw = 0; dsw = 0;
    }
    const Real ds = dsw * inv - sw * inv * inv;  // d s / d d
    const Real q = sw * inv * inv;                // s / d
    const Real dq = dsw * inv * inv - Real(2) * sw * inv * inv * inv;
    const float* sv = a.dstd + 4 * t;
    const Real r0 = (Real)dR.x / sv[0], r1 = (Real)dR.y / sv[1], r2 = (Real)dR.z / sv[2], r3 = (Real)dR.w / sv[3];
    const Real vdotr = r1 * rx + r2 * ry + r3 * rz;
    const Real radial = r0 * ds + dq * vdotr + (Real)dg.w * dsw;  // coefficient of rhat
    const Real hdot = (Real)dg.x * hx + (Real)dg.y * hy + (Real)dg.z * hz;
    out.x = (float)(radial * hx + q * r1 + ((Real)dg.x - hdot * hx) * inv);
    out.y = (float)(radial * hy + q * r2 + ((Real)dg.y - hdot * hy) * inv);
    out.z = (float)(radial * hz + q * r3 + ((Real)dg.z - hdot * hz) * inv);
  }
  reinterpret_cast<float4*>(a.g)[row] = out;
}

void launch_env_bwd(const EnvBwdArgs& a, cudaStream_t st) {
  long long rows = (long long)a.n * NP;
  if (rows == 0) return;
  if (a.fp64)
    k_env_bwd<double><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a);
  else
    k_env_bwd<float><<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(a);
  note_launch();
}

// Forces F_k = sum_j g_kj - sum_{i: k in N(i)} g_ik (Eq. eq_forceAtomicEnergy
// with e_i depending on r_ij = x_j - x_i) and virial W = -sum r_ij (x) g_ij.
// One warp per atom; the reverse rows are sorted so that every sum runs in a
// fixed order (bitwise reproducible, no atomics).  A lane adds its few terms
// and the warp its 32 lane sums in FP32 (a fixed tree; the FP64 pipe of this
// GPU is narrow), the per-block virial and energy in FP64.
constexpr int FWARPS = FORCE_BLOCK_ATOMS;
__global__ void __launch_bounds__(32 * FWARPS) k_force(ForceArgs a) {
  __shared__ int srev[FWARPS][REV_CAP];
  __shared__ double sred[FWARPS][10];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k = blockIdx.x * FWARPS + warp;
  float f0 = 0.f, f1 = 0.f, f2 = 0.f;
  float v[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  double ek = 0;
  if (k < a.n) {
    const int nn = a.nnei[k];
    int cnt = a.rev_cnt[k];
    for (int s = lane; s < nn; s += 32) {
      const size_t row = (size_t)k * NP + s;
      const float4 g = reinterpret_cast<const float4*>(a.g)[row];
      const float4 r = reinterpret_cast<const float4*>(a.rv)[row];
      f0 += g.x; f1 += g.y; f2 += g.z;
      v[0] -= r.x * g.x; v[1] -= r.x * g.y; v[2] -= r.x * g.z;
      v[3] -= r.y * g.x; v[4] -= r.y * g.y; v[5] -= r.y * g.z;
      v[6] -= r.z * g.x; v[7] -= r.z * g.y; v[8] -= r.z * g.z;
    }
    if (cnt > REV_CAP) cnt = REV_CAP;
    int* rows = srev[warp];
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int t = lane; t < P; t += 32) rows[t] = t < cnt ? a.rev_rows[(size_t)k * REV_CAP + t] : 0x7fffffff;
    __syncwarp();
    for (int kk = 2; kk <= P; kk <<= 1)
      for (int jj = kk >> 1; jj > 0; jj >>= 1) {
        for (int t = lane; t < P; t += 32) {
          int o = t ^ jj;
          if (o > t) {
            bool asc = (t & kk) == 0;
            int x = rows[t], y = rows[o];
            if (asc ? x > y : x < y) { rows[t] = y; rows[o] = x; }
          }
        }
        __syncwarp();
      }
    for (int t = lane; t < cnt; t += 32) {
      const float4 g = reinterpret_cast<const float4*>(a.g)[rows[t]];
      f0 -= g.x; f1 -= g.y; f2 -= g.z;
    }
    f0 = warp_sum(f0); f1 = warp_sum(f1); f2 = warp_sum(f2);
    if (lane == 0) {
      a.force[3 * k] = f0; a.force[3 * k + 1] = f1; a.force[3 * k + 2] = f2;
      // ghost atoms: m_k = 0 (Eq. eq_forcesLocalGhost); padding of a packed batch: no atom
      ek = k < a.nlocal && (!a.frame || a.frame[k] >= 0) ? (double)a.e[k] : 0.0;
      if (a.atom_energy) a.atom_energy[k] = ek;
    }
  }
#pragma unroll
  for (int c = 0; c < 9; ++c) v[c] = warp_sum(v[c]);
  if (lane == 0) {
    for (int c = 0; c < 9; ++c) sred[warp][c] = v[c];
    sred[warp][9] = ek;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    double s = 0;
    for (int w = 0; w < FWARPS; ++w) s += sred[w][threadIdx.x];
    a.partials[(size_t)blockIdx.x * 10 + threadIdx.x] = s;
  }
}

// Sums the block partials in a fixed order: one block per frame of a packed
// batch (seg non-null: frame b owns partial rows [seg[b] - seg[0],
// seg[b+1] - seg[0])), else one block over rows [0, nblocks).
__global__ void k_finalize(const double* __restrict__ partials, int nblocks, const int* __restrict__ seg,
                           double* __restrict__ energy, double* __restrict__ virial) {
  __shared__ double red[10][32];
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;  // 10 warps, one per quantity
  int b0 = 0, cnt = nblocks;
  if (seg) {
    b0 = seg[blockIdx.x] - seg[0];
    cnt = seg[blockIdx.x + 1] - seg[blockIdx.x];
  }
  const double* p = partials + (size_t)b0 * 10 + c;
  // eight independent partial sums per lane (eight loads in flight), added
  // in a fixed order
  double s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int b = lane;
  for (; b + 7 * 32 < cnt; b += 8 * 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) s8[u] += p[(size_t)(b + 32 * u) * 10];
  }
  for (; b < cnt; b += 32) s8[0] += p[(size_t)b * 10];
  double s = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
  s = warp_sum_d(s);
  if (lane == 0) red[c][0] = s;
  __syncthreads();
  if (threadIdx.x < 9) virial[9 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
  if (threadIdx.x == 9) energy[blockIdx.x] = red[9][0];
}

void launch_force_virial(const ForceArgs& a, cudaStream_t st) {
  const int nb = a.n > 0 ? (a.n + FWARPS - 1) / FWARPS : 0;
  if (nb > 0) {
    k_force<<<nb, 32 * FWARPS, 0, st>>>(a);
    note_launch();
  }
  if (a.seg) {
    if (a.nseg > 0) {
      k_finalize<<<a.nseg, 320, 0, st>>>(a.partials, nb, a.seg, a.energy, a.virial);
      note_launch();
    }
  } else {
    k_finalize<<<1, 320, 0, st>>>(a.partials, nb, nullptr, a.energy, a.virial);
    note_launch();
  }
}

}  // namespace dpa1
