/*
 * dpa1.h - C ABI of the GB300 DPA-1 (se_atten) energy / force / virial engine.
 *
 * The calls follow the contract of the paper's DeepmdModel wrapper around
 * deepmd::compute() (Sec. IV-A): a model is loaded once with its type map,
 * cutoff and neighbour cap, and each call maps coordinates, box and atom
 * types to the total energy, per-atom forces and the virial.  The energy is
 * a sum of atomic energies e_i = Phi(D_i) of the descriptor D_i built from
 * the full neighbour list of atom i (Sec. II-B, Eq. eq_totE_singleAtomE),
 * and the forces are its exact negative gradient (Eq. eq_forceGradE,
 * Eq. eq_forceAtomicEnergy).
 *
 * Conventions shared by every call:
 *   - Units: Angstrom for lengths, eV for energies, eV/A for forces, eV for
 *     the virial.  Unit conversion for an MD engine is the caller's job.
 *   - The box is 9 doubles, row-major cell vectors; it must be orthorhombic
 *     (off-diagonal entries exactly 0) with every edge > 2 * rcut, else
 *     DP_ERR_BOX.
 *   - coord is [natoms][3] double, atype is [natoms] int in [0, ntypes).
 *   - Outputs: energy [1], force [natoms][3], virial [9] (row-major,
 *     W_ab = -sum_ij r_ij,a dE/dr_ij,b), atom_energy [natoms] (nullable).
 *   - The caller owns every array it passes.  The library owns the model and
 *     its device workspace.  No call keeps a pointer after it returns.
 *   - Every call returns a dp_status; no C++ exception crosses the ABI.  The
 *     text of the last error of the calling thread is dp_last_error().
 *   - One model is used by one host thread / stream at a time.
 */
#ifndef DPA1_H
#define DPA1_H

#include <stddef.h>

#if defined(__GNUC__)
#define DP_API __attribute__((visibility("default")))
#else
#define DP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dp_model dp_model; /* opaque, library-owned */

enum dp_status {
  DP_OK = 0,
  DP_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, type out of range) */
  DP_ERR_IO = -2,       /* weight file missing, truncated or of another format */
  DP_ERR_BOX = -3,      /* box not orthorhombic or an edge <= 2 * rcut */
  DP_ERR_CAPACITY = -4, /* natoms above the reserved size, or a device-side buffer overflowed */
  DP_ERR_CUDA = -5,     /* a CUDA runtime call failed */
  DP_ERR_TIMEOUT = -6,  /* a bounded device-side wait gave up */
  DP_ERR_NAN = -7,      /* non-finite coordinates */
  DP_ERR_UNSUPPORTED = -8 /* model shape this build has no kernel for */
};

enum dp_precision {
  DP_PREC_FP32 = 0,  /* every matrix product in FP32 SIMT arithmetic */
  DP_PREC_BF16 = 1,  /* attention-layer products on tcgen05 tensor cores (fused per-atom layer kernels):
                        BF16 operands, FP32 accumulation; attention width 128, embedding width <= 108 */
  DP_PREC_FP16X = 2, /* as DP_PREC_BF16 with FP16 operands and two-term (hi + lo) splits of the layer
                        input, the attention weights and [Wv Wo; bv Wo]; FP32 accumulation */
  DP_PREC_BF16X = 3  /* every product of the attention layers, the embedding net (25-50-100 and
                        32-64-128 nets) and the fitting net on tcgen05 tensor cores with BF16 operands,
                        both operands split in two terms (x = bf16(x) + bf16(x - bf16(x)), three
                        products), FP32 accumulation; attention width 128 or 256, embedding width <= 128 */
};

/* Load a model.
 *   weights_path : binary weight file (layout documented in synth/model.py).
 *   type_map     : ntypes element names; must equal the file's map, in order
 *                  (type id t of atype is type_map[t]).  May be NULL to accept
 *                  the file's map.
 *   rcut, rcut_smth, sel : must equal the file's values (Sec. II-C: the
 *                  cutoff of the full neighbour list and its cap), else
 *                  DP_ERR_ARG.  Pass a negative value to accept the file's.
 *   precision    : DP_PREC_FP32, DP_PREC_BF16, DP_PREC_FP16X or DP_PREC_BF16X
 *                  (DP_ERR_UNSUPPORTED for a model shape the mode has no
 *                  kernel for).
 *   device       : CUDA device ordinal; the model's memory lives there.
 * On success *out is a new model; release it with dp_free. */
DP_API int dp_init(dp_model** out, const char* weights_path, const char* const* type_map, int ntypes,
            double rcut, double rcut_smth, int sel, int precision, int device);

/* Energy, forces and virial of one frame from HOST arrays (Sec. IV-A,
 * deepmd::compute()).  Copies inputs to the device, runs the whole path on
 * the model's stream, copies results back and synchronises.  Grows the
 * workspace when natoms exceeds the reserved size.  natoms == 0 gives
 * zero energy and virial. */
DP_API int dp_compute(dp_model* m, int natoms, const double* coord, const double* box, const int* atype,
               double* energy, double* force, double* virial, double* atom_energy);

/* Same as dp_compute with DEVICE arrays on the caller's CUDA stream
 * (cudaStream_t passed as void*; NULL = the legacy default stream).  Never
 * synchronises the host and never allocates, so it can be captured in a
 * CUDA graph.  natoms must not exceed the size reserved with dp_reserve
 * (DP_ERR_CAPACITY otherwise, nothing launched).  Device-side failures (box
 * check, buffer overflow) are recorded in a device flag read by
 * dp_get_status; the outputs are then unspecified. */
DP_API int dp_compute_device(dp_model* m, int natoms, const double* d_coord, const double* d_box,
                      const int* d_atype, double* d_energy, double* d_force, double* d_virial,
                      double* d_atom_energy, void* cuda_stream);

/* Local and ghost atoms (Sec. II-C, Eq. eq_forcesLocalGhost): atoms
 * [0, nlocal) are local, atoms [nlocal, natoms) are ghost copies that a
 * domain-decomposed caller imports from its neighbours.  Neighbour lists run
 * over all natoms atoms, but only local atoms' energies count (m_j = 1 for
 * local j, 0 for ghosts): energy = sum of e_j over local j; force on every
 * atom k, local or ghost, = -d(energy)/dx_k (ghost forces are for the caller
 * to add to their owners); virial = -sum over local centres i of
 * sum_j r_ij (x) dE/dr_ij; atom_energy is e_j for local atoms and 0 for
 * ghosts.  0 <= nlocal <= natoms, else DP_ERR_ARG; nlocal == natoms is
 * dp_compute / dp_compute_device.  A caller with explicit ghost images
 * passes a box whose edges exceed the extent of all atoms plus rcut along
 * every non-periodic direction. */
DP_API int dp_compute_local(dp_model* m, int natoms, int nlocal, const double* coord, const double* box,
                            const int* atype, double* energy, double* force, double* virial,
                            double* atom_energy);
DP_API int dp_compute_device_local(dp_model* m, int natoms, int nlocal, const double* d_coord,
                                   const double* d_box, const int* d_atype, double* d_energy, double* d_force,
                                   double* d_virial, double* d_atom_energy, void* cuda_stream);

/* Several independent frames of uneven size from HOST arrays.  Frame f owns
 * atoms [atom_offsets[f], atom_offsets[f+1]) of coord / atype / force and
 * box[9f .. 9f+8], energy[f], virial[9f .. 9f+8].  Frames never interact.
 * Every frame's arguments are checked before any frame runs (DP_ERR_ARG /
 * DP_ERR_BOX / DP_ERR_NAN name the first bad one); the batch is then copied
 * to the device once and evaluated in packed passes: each frame's neighbour
 * list is built in its own box, and every later stage runs once over all the
 * frames of a pass (frames are padded to multiples of 4 atoms, so that each
 * frame's energy, forces and virial are bitwise those of a call on that frame
 * alone).  A pass holds as many atoms as the workspace; the call grows the
 * workspace to min(padded atoms, 65,536) atoms, at least the largest frame,
 * and runs a larger batch as several passes of consecutive frames.  The
 * results come back once.  A device-side error in any frame is returned for
 * the batch.  The library keeps a device buffer for the largest batch seen
 * until dp_free. */
DP_API int dp_compute_batch(dp_model* m, int nframes, const int* atom_offsets, const double* coord,
                     const double* box, const int* atype, double* energy, double* force,
                     double* virial);

/* Pre-size the device workspace for up to max_atoms atoms (needed before
 * dp_compute_device and before capturing it in a CUDA graph). */
DP_API int dp_reserve(dp_model* m, int max_atoms);

/* Switch the arithmetic of the network products (enum dp_precision). */
DP_API int dp_set_precision(dp_model* m, int precision);

/* Synchronise the model's last stream and return (then clear) the status
 * recorded by device-side checks of asynchronous calls. */
DP_API int dp_get_status(dp_model* m);

/* Full neighbour list of every atom (Sec. II-C): atoms j != i with
 * |mic(r_j - r_i)| < rcut, the sel nearest kept, sorted by (|r_ij|^2, j),
 * each row padded with -1 to 128 entries.  DEVICE arrays: d_nlist
 * [natoms][128] int, d_nnei [natoms] int (kept count).  Distances are
 * evaluated in FP64 without fused multiply-adds, so the list is exactly
 * reproducible on the host.  Same capacity and status rules as
 * dp_compute_device. */
DP_API int dp_nlist_device(dp_model* m, int natoms, const double* d_coord, const double* d_box,
                    int* d_nlist, int* d_nnei, void* cuda_stream);

/* Velocity-Verlet molecular dynamics with the model's forces (the MD loop the
 * paper couples the model to, Sec. II-A and Sec. IV-A), all on the device:
 * per step v += dt/2 F/m, x += dt v, forces at the new x (neighbour list
 * rebuilt), v += dt/2 F/m.  Units A, fs, amu, eV.  DEVICE arrays:
 *   d_coord [natoms][3], d_vel [natoms][3] (A/fs): updated in place;
 *   d_mass [natoms] (amu); d_box [9]; d_atype [natoms];
 *   d_force [natoms][3], d_energy [1], d_virial [9]: out, at the final step;
 *   d_thermo [nsteps][3]: out, (potential, kinetic, total) energy per step.
 * Forces are first evaluated at the starting coordinates.  With
 * use_graph != 0 one step is captured once into a CUDA graph (cached in the
 * model for the same pointers, sizes, dt and precision) and replayed nsteps
 * times.  Runs on cuda_stream (NULL: the model's own stream, then
 * synchronised).  natoms must not exceed the reserved size. */
DP_API int dp_md_run(dp_model* m, int natoms, double* d_coord, double* d_vel, const double* d_mass,
                     const double* d_box, const int* d_atype, double dt, int nsteps, double* d_force,
                     double* d_energy, double* d_virial, double* d_thermo, int use_graph, void* cuda_stream);

/* Training of a model without attention layers in FP32 (the distilled
 * student potential).  The trainable parameters form one FP32 vector:
 * embedding net (em_W0 em_b0 em_W1 em_b1 em_W2 em_b2), fitting layers
 * (fit_W fit_b per hidden layer), output layer (w, b) and per-type energy
 * bias, in the order and shapes of the weight file; the type embedding and
 * type-pair net stay fixed.  In the concat type-embedding mode (the
 * embedding net reads [s, T_j, T_i]) the vector holds the s row of em_W0
 * only: the type rows stay fixed with the type embedding, and the library
 * keeps their contribution plus em_b0 as a bias per type pair, refreshed
 * after every update.
 *   dp_param_count: number of entries.  dp_get_params / dp_set_params /
 *   dp_get_grad copy the vector / its gradient to or from host memory
 *   (count must equal dp_param_count).  dp_zero_grad clears the gradient.
 *   dp_train_frame: for one frame with reference energy e_ref (eV) and
 *   DEVICE reference forces d_force_ref [natoms][3], adds to the gradient
 *   dL/dtheta of L = pe ((E - e_ref)/N)^2 + pf mean |F - F_ref|^2 and writes
 *   (L, energy part, force part) to DEVICE d_loss [3].  Both parts are
 *   exact: the force part is -(2 pf / 3N) times the derivative of
 *   dE/dtheta along the displacement field v = F - F_ref (held fixed),
 *   evaluated in forward mode over the adjoint (one energy evaluation with
 *   its weight gradient, then one tangent pass).
 *   dp_adam_step: one Adam update of the vector with the accumulated
 *   gradient (then cleared). */
DP_API int dp_param_count(const dp_model* m);
DP_API int dp_get_params(dp_model* m, float* host, int count);
DP_API int dp_set_params(dp_model* m, const float* host, int count);
DP_API int dp_get_grad(dp_model* m, float* host, int count);
DP_API int dp_zero_grad(dp_model* m, void* cuda_stream);
DP_API int dp_train_frame(dp_model* m, int natoms, const double* d_coord, const double* d_box, const int* d_atype,
                          double e_ref, const double* d_force_ref, double pe, double pf, double* d_loss,
                          void* cuda_stream);
DP_API int dp_adam_step(dp_model* m, double lr, double beta1, double beta2, double eps, void* cuda_stream);

/* Largest neighbour count and number of atoms whose candidate set exceeded
 * sel in the last call (the sel cap is a property of the method, not an
 * error). */
DP_API int dp_stats(const dp_model* m, int* max_nnei, long long* n_truncated);

/* Parse the header of a weight file on the host only (no GPU needed).
 * ints16 receives the 16 header integers and dbls8 the 8 header doubles
 * described in synth/model.py; either may be NULL. */
DP_API int dp_inspect_weights(const char* weights_path, int* ints16, double* dbls8);

/* Diagnostics: copy the named internal device buffer of the last call to
 * host memory (at most bytes bytes).  Names: "nlist", "env", "G0", "G1",
 * "G2", "D", "e", "g".  "G<l>" is returned as [rows][m1] row-major whatever
 * the internal layout.  Returns the number of bytes copied, or a negative
 * dp_status. */
DP_API long long dp_debug_copy(dp_model* m, const char* name, void* host_dst, size_t bytes);

/* Diagnostics: fill the model's whole workspace (every intermediate buffer of
 * a call, not the weights) with 0xFF bytes, i.e. NaN in every floating-point
 * array and -1 in every integer one, and wait for it.  A later call must give
 * the same results bit for bit as before: no stage may depend on what an
 * earlier call left behind, nor on memory it never writes (e.g. the rows past
 * an atom's last neighbour, which the 16-bit paths neither read nor write).
 * Errors: DP_ERR_ARG for a null model, DP_ERR_CUDA. */
DP_API int dp_debug_poison(dp_model* m);

/* Profiling: dp_set_profiling(m, 1) clears the record and makes every later
 * call record a CUDA event on its stream after each stage (the per-region
 * timing of the paper's profiling setup, Sec. V-D); 0 switches it off.
 * dp_stage_times waits for the last recorded call and writes, for each
 * stage of every call since profiling was switched on, in launch order, its
 * name (static strings owned by the library) and device time in ms; it
 * returns the number of stages written (0 when profiling is off).  A stage
 * repeated per attention layer appears once per layer. */
DP_API int dp_set_profiling(dp_model* m, int on);
DP_API int dp_stage_times(dp_model* m, const char** names, float* ms, int max_stages);

/* Number of CUDA kernels this library has launched in this process. */
DP_API long long dp_kernel_launches(void);

/* Neighbour list without any allocation (this entry point has no counterpart
 * in the paper).  It builds the same list as dp_nlist_device (same rcut
 * rule, same order, rows padded with -1 to 128 entries), but needs no model
 * and never calls cudaMalloc, cudaFree or an allocating library: its cell-list
 * scratch is a fixed device array of about 2.7 MB that every GPU loading
 * this library holds until the process exits.  It is meant for callers that
 * cannot allocate device memory in the middle of their work: an MD engine
 * that hands the library only its own pooled buffers, code running inside a
 * host callback or a captured stream, or a real-time loop where the implicit
 * synchronisation of cudaMalloc would stall every other stream.
 *   natoms  : 0 .. 65536 atoms, else DP_ERR_CAPACITY and nothing is launched.
 *   d_coord : DEVICE [natoms][3] double; d_box: DEVICE [9] double (the box
 *             rules of every call: orthorhombic, edges > 2 * rcut).
 *   rcut, sel : cutoff (A, > 0) and neighbour cap (1 .. 128).
 *   d_nlist : DEVICE [natoms][128] int out; d_nnei: DEVICE [natoms] int out.
 *   d_status: DEVICE int out; zeroed, then ORed with device-side failure bits
 *             (1: bad box, 2: more than 256 candidates around an atom,
 *             4: non-finite coordinate).  Read it after the stream finishes.
 *   cuda_stream : the stream to run on (NULL = legacy default stream).
 * Asynchronous: returns once the work is queued.  The first call on a device
 * looks up the scratch array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls on a device share
 * the one scratch array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and corrupt each other's lists: order
 * them on one stream or synchronise in between. */
DP_API int dp_nlist_noalloc(int natoms, const double* d_coord, const double* d_box, double rcut, int sel,
                            int* d_nlist, int* d_nnei, int* d_status, void* cuda_stream);

/* Text of the calling thread's last error ("" if none). */
DP_API const char* dp_last_error(void);

/* Release the model and its device memory.  NULL is allowed. */
DP_API void dp_free(dp_model* m);

#ifdef __cplusplus
}
#endif

#endif /* DPA1_H */
