// Stage a16: velocity-Verlet integration of Newton's equations with the DPA-1
// forces (F = -grad E, Eq. eq_forceGradE; Sec. II-A integrates them with
// leap-frog or Verlet schemes).  Units: A, fs, amu, eV; an acceleration is
// F / m * 9.648533212e-3 A^2 fs^-2 per (eV / A / amu).
#include "common.cuh"
#include "kernels.h"

namespace dpa1 {

constexpr double EV_PER_AMU_A2_FS2 = 1.0 / 9.648533212e-3;  // (amu A^2 / fs^2) in eV
constexpr double ACC = 9.648533212e-3;                       // (eV / A / amu) in A / fs^2

// First half kick and drift: v += dt/2 F/m; x += dt v.
__global__ void k_verlet_drift(int n, double dt, const double* __restrict__ mass, const double* __restrict__ f,
                               double* __restrict__ v, double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * n) return;
  const double a = f[i] / mass[i / 3] * ACC;
  const double vi = v[i] + 0.5 * dt * a;
  v[i] = vi;
  x[i] += dt * vi;
}

constexpr int KICK_THREADS = 256;

int verlet_kick_blocks(int n) { return (3 * n + KICK_THREADS - 1) / KICK_THREADS; }

// Second half kick with the new forces: v += dt/2 F/m.  Each block's kinetic
// energy (a fixed warp tree, then its warps in order) goes to partial[block].
__global__ void __launch_bounds__(KICK_THREADS) k_verlet_kick(int n, double dt, const double* __restrict__ mass,
                                                                const double* __restrict__ f, double* __restrict__ v,
                                                                double* __restrict__ partial) {
  __shared__ double red[KICK_THREADS / 32];
  const int i = blockIdx.x * KICK_THREADS + threadIdx.x;
  double ke = 0.0;
  if (i < 3 * n) {
    const double m = mass[i / 3];
    const double vi = v[i] + 0.5 * dt * f[i] / m * ACC;
    v[i] = vi;
    ke = 0.5 * m * vi * vi;
  }
  ke = warp_sum_d(ke);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ke;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < KICK_THREADS / 32; ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

// The step's kinetic energy from the `nb` blocks' partial sums, reduced in
// FP64 in a fixed order (one block), and its record (E, kinetic, total).
__global__ void k_verlet_thermo(int nb, const double* __restrict__ partial, const double* __restrict__ energy,
                                int* __restrict__ counter, double* __restrict__ thermo, int nrec) {
  __shared__ double red[32];
  double ke = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) ke += partial[b];
  ke = warp_sum_d(ke);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ke;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    s *= EV_PER_AMU_A2_FS2;
    const int step = *counter;
    if (step < nrec) {
      thermo[3 * step] = *energy;
      thermo[3 * step + 1] = s;
      thermo[3 * step + 2] = *energy + s;
    }
    *counter = step + 1;
  }
}

void launch_verlet_drift(int n, double dt, const double* mass, const double* f, double* v, double* x, cudaStream_t st) {
  if (n == 0) return;
  k_verlet_drift<<<(3 * n + 255) / 256, 256, 0, st>>>(n, dt, mass, f, v, x);
  note_launch();
}

void launch_verlet_kick(int n, double dt, const double* mass, const double* f, double* v, double* partial,
                        const double* energy, int* counter, double* thermo, int nrec, cudaStream_t st) {
  const int nb = verlet_kick_blocks(n);
  if (nb > 0) {
    k_verlet_kick<<<nb, KICK_THREADS, 0, st>>>(n, dt, mass, f, v, partial);
    note_launch();
  }
  k_verlet_thermo<<<1, 1024, 0, st>>>(nb, partial, energy, counter, thermo, nrec);
  note_launch();
}

}  // namespace dpa1
