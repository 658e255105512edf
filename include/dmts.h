/*
 * dmts.h -- C ABI of the GB300 (sm_103a) distilled multi-time-step library.
 *
 * The library evaluates two neural-network potentials -- a "big" reference
 * model and a cheaper "small" distilled model with a shorter cutoff -- and
 * integrates Newton's equations with the multiple-time-step scheme of
 * Algorithm 1 of arXiv 2510.06562 (section "Integration scheme"): the small
 * model's forces drive every inner step, and every outer step a half-kick
 * with the difference F_big - F_small on each side restores the big model's
 * dynamics. The thermostat of Algorithm 1 is the identity here (NVE).
 *
 * Potential (both models; hyperparameters per model): invariant message
 * passing on the directed neighbour pairs within the cutoff rc,
 *   h0_i  = A[Z_i]
 *   per layer: u_i = h_i W_in; w_ij = fc(d_ij) (SiLU(e(d_ij) W1 + b1) W2 + b2);
 *              m_i = sum_j w_ij * u_j; h_i += SiLU(m_i U1 + c1) U2 + c2
 *   E_i   = SiLU(h_i R1 + d1) . R2 + d2 + e0[Z_i]
 *           + 1/2 sum_j rep_a exp(-d_ij/rep_rho) fc(d_ij; rep_cutoff),
 *   E     = sum_i E_i,
 * with the Bessel basis e_k(d) = sqrt(2/rc) sin(k pi d/rc)/d (k = 1..K) and
 * the cosine cutoff fc(d; r) = (cos(pi d/r) + 1)/2 (fc(d) = fc(d; rc)). The
 * last term is a fixed short-range pair repulsion (rep_a = 0 disables it).
 * Forces are F = -dE/dx.
 * The paper defers its architectures to its Supporting Information; this
 * family stands in for them (section "Neural Network Architectures").
 *
 * Units: positions in Angstrom, velocities in Angstrom/fs, masses in amu,
 * energies in eV, forces in eV/Angstrom, time in fs.
 *
 * Conventions for every call:
 *  - All arrays are owned by the caller; the library copies what it needs.
 *    A pointer may point to host memory or to CUDA device memory of the
 *    context's device; the library tells them apart itself.
 *  - Per-atom 3-vectors are arrays of N*3 doubles, atom-major
 *    (x[3*i + 0..2]), i.e. a C-contiguous [N][3] array.
 *  - Every call returns DMTS_OK (0) or a negative dmts_status and throws
 *    nothing. dmts_last_error() describes the last failure of the calling
 *    thread. After DMTS_ERR_ARG, DMTS_ERR_CAPACITY or DMTS_ERR_NONFINITE the
 *    context stays usable; after DMTS_ERR_CUDA it may not be, and later calls
 *    on it return DMTS_ERR_STATE.
 *  - All device work of a context runs on its own CUDA stream
 *    (dmts_stream); calls return after that work has completed.
 *  - A context is not thread-safe: one thread at a time per context.
 *    Different contexts may be used from different threads at the same
 *    time, also on one device; a context belongs to the device that is
 *    current when dmts_create is called.
 */
#ifndef DMTS_H
#define DMTS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported from libdmts.so (built with hidden default visibility). */
#if defined(__GNUC__)
#define DMTS_API __attribute__((visibility("default")))
#else
#define DMTS_API
#endif

typedef struct dmts_ctx dmts_ctx;

typedef enum {
    DMTS_OK = 0,
    DMTS_ERR_ARG = -1,        /* invalid argument (NULL, size, layout)            */
    DMTS_ERR_OOM = -2,        /* device or host allocation failed                 */
    DMTS_ERR_CUDA = -3,       /* CUDA runtime error (no device, launch failure)   */
    DMTS_ERR_CAPACITY = -4,   /* neighbour capacity could not be grown enough     */
    DMTS_ERR_NONFINITE = -5,  /* a position or velocity became NaN or infinite    */
    DMTS_ERR_TIMEOUT = -6,    /* a bounded device-side wait gave up               */
    DMTS_ERR_STATE = -7       /* context unusable, or no state set yet            */
} dmts_status;

/* Arithmetic of the multilayer perceptrons. DMTS_FP32: FP32 everywhere.
 * DMTS_BF16_MLP: dense layers on tensor cores with BF16 operands and FP32
 * accumulation; edge geometry, sums and forces stay FP32. */
enum { DMTS_FP32 = 0, DMTS_BF16_MLP = 1 };

/* Model selector for dmts_forces / dmts_neighbors / dmts_set_params. */
enum { DMTS_SMALL = 0, DMTS_BIG = 1 };

/* One potential. params: n_params doubles in the documented flat order
 *   A[S][F]; per layer: W_in[F][F], W1[K][F], b1[F], W2[F][F], b2[F],
 *   U1[F][F], c1[F], U2[F][F], c2[F]; then R1[F][F], d1[F], R2[F], d2[1],
 *   e0[S]
 * (matrices row-major, input index first: y = x W), so
 *   n_params = S F + n_layers (4 F^2 + K F + 4 F) + F^2 + 2 F + 1 + S.
 * Supported: 1 <= n_layers <= 4; n_feat in {32, 64}; 1 <= n_radial <= 16;
 * 1 <= n_species <= 16; cutoff > 0. Copied at dmts_create. */
typedef struct {
    double cutoff;       /* rc, Angstrom                                  */
    int n_radial;        /* K                                             */
    int n_layers;        /* message-passing layers                        */
    int n_feat;          /* F                                             */
    int n_species;       /* S                                             */
    const double* params;
    size_t n_params;
    int precision;       /* DMTS_FP32 or DMTS_BF16_MLP                    */
    double rep_a;        /* pair repulsion amplitude, eV (>= 0)           */
    double rep_rho;      /* its decay length, Angstrom (> 0 if rep_a > 0) */
    double rep_cutoff;   /* its cutoff, Angstrom (0 < rep_cutoff <= cutoff if rep_a > 0) */
} dmts_model_desc;

/* The simulated systems: n_systems independent systems stored back to back.
 * atom_offset[n_systems + 1] (atom_offset[0] = 0, non-decreasing), species
 * [N] in [0, n_species), mass [N] > 0 (amu), box [n_systems]: edge length of
 * a periodic cubic box (Angstrom, at least twice the largest cutoff), or
 * <= 0 for a non-periodic system. Atoms of different systems never interact.
 * Supported: any number of periodic systems sharing one box edge (replicas,
 * each with its own cells, integrated together in one graph), or any number
 * of non-periodic systems of at most 1024 atoms each; the two kinds are not
 * mixed in one context. */
typedef struct {
    int n_systems;
    const int* atom_offset;
    const int* species;
    const double* mass;
    const double* box;
} dmts_system_desc;

/* Create a context on the current CUDA device (Algorithm 1's two force
 * fields, masses and boxes). small may be NULL: then dmts_respa_step runs
 * single-time-step velocity Verlet with the big model. options: NULL, "" or
 * a flat JSON object of numbers and booleans (true = 1, false = 0); a key
 * other than those below, a repeated key, another kind of value or
 * malformed JSON is DMTS_ERR_ARG, checked before any device work.
 * Keys: "edge_capacity_factor" (default 1.5, the
 * neighbour-pair capacity relative to the uniform-density estimate),
 * "row_capacity" (initial per-atom neighbour capacity; it grows on demand),
 * "cell_capacity" (initial atoms per cell of the cell list with skin 0; it
 * grows on demand),
 * "autotune" (default 1: pick the kernels' work granularity by timing),
 * "atoms_per_cta_big" / "atoms_per_cta_small" (atoms per thread block of the
 * force kernels), "skin" (default 0, in [0, 10] Angstrom: Verlet-skin
 * neighbour lists; 0 builds the pair list from scratch at every evaluation,
 * which measured faster on liquid water at 3 fs outer steps).
 * With a skin, candidate rows of all j within rc + skin are kept from the
 * last rebuild and filtered with the exact cutoff test at every evaluation,
 * which yields the same pair set as a fresh build; both models' rows are
 * rebuilt, on the device, once some atom has moved by skin / 2 since then
 * (the model with the smaller cutoff filters its rows from the other's).
 * The paper does not describe its neighbour search; this is an
 * implementation choice that leaves every result unchanged up to the order
 * of floating-point additions.
 * "langevin_friction" (default 0 = NVE, in ps^-1; the paper uses 1),
 * "temperature" (K, default 300), "seed" (default 0): Algorithm 1's
 * thermostat step thermo(v, h) becomes the exact Ornstein-Uhlenbeck update
 * v <- c1 v + sqrt((1 - c1^2) k_B T / m) xi, c1 = exp(-gamma h), between the
 * two half-drifts of every inner step, and velocity Verlet (no small model)
 * becomes BAOAB. xi are standard normals from Philox-4x32-10 with counter
 * (atom index, inner-step counter low/high words, 0) and key (seed low/high
 * words), Box-Muller on the four uniforms (w + 1/2) 2^-32: (u0, u1) give the
 * x and y components, (u2, u3) the z component. The inner-step counter
 * starts at 0 at dmts_set_state and advances by n_inner per outer step.
 * A thermostatted run resumed from dmts_get_state (in this or a new
 * context) therefore needs a new seed: with the same seed the restarted
 * counter would draw the first segment's noise again. NVE runs resume
 * exactly.
 * "concurrent_models" (default 1): with fresh neighbour lists, the outer
 * step's large-model evaluation and the last inner step's small-model
 * evaluation (same positions, independent) run on two streams of the step
 * graph; results are identical either way.
 * "fallback_threshold" (eV/A, default 0 = off; the paper uses 150
 * kcal/mol/A = 6.505 eV/A): after each outer step of Algorithm 1, if some
 * atom's |F_big - F_small| exceeds it, the step is redone from its starting
 * state with n_inner single-time-step steps of dt / n_inner with the big
 * model (velocity Verlet, or BAOAB with the thermostat, drawing the noise of
 * the inner steps they replace), and the small model is evaluated at the end
 * (the paper's temporary reversion to the single-time-step integrator). The
 * monitor statistics (dmts_monitor) are gathered with or without it.
 * "atom_tensor_cores" (default 1): in DMTS_BF16_MLP mode, the per-atom MLPs
 * of models with F >= 64 run on the tensor cores with each operand split
 * into two BF16 parts (near-FP32 results); 0 keeps them on the FP32 kernels.
 * On success *out holds the new context; on failure *out is NULL. */
DMTS_API int dmts_create(const dmts_model_desc* small, const dmts_model_desc* big,
                const dmts_system_desc* sys, const char* options, dmts_ctx** out);

/* Set positions x[N*3] and velocities v[N*3] (NULL: zero velocities).
 * Periodic positions are wrapped into [0, L) as x - L floor(x / L).
 * If a wrapped position differs, bit for bit, from the context's current
 * one, the cached forces become invalid and the next dmts_respa_step
 * evaluates both models first (Algorithm 1's first_step). If every position
 * is unchanged (e.g. a caller that reads the state back after each call and
 * uploads it again, or changes only velocities), the forces cached at those
 * positions are kept: they depend on positions only, and every evaluation
 * is deterministic, so recomputing them would give the same bits. The
 * thermostat's inner-step counter restarts at 0 either way. n_atoms must
 * equal N. */
DMTS_API int dmts_set_state(dmts_ctx* ctx, const double* x, const double* v, int n_atoms);

/* Read back positions and velocities (either pointer may be NULL). */
DMTS_API int dmts_get_state(dmts_ctx* ctx, double* x, double* v);

/* Evaluate one model (DMTS_SMALL or DMTS_BIG) at the current positions.
 * f_out [N*3] forces F = -dE/dx (or NULL); energy_out [n_systems] potential
 * energies (or NULL); virial_out [n_systems*9] row-major 3x3 virial
 * W_ab = -sum_pairs r_ij,a dE/dr_ij,b (or NULL). */
DMTS_API int dmts_forces(dmts_ctx* ctx, int which, double* f_out, double* energy_out,
                double* virial_out);

/* n_outer steps of Algorithm 1 with outer step dt_outer_fs and n_inner inner
 * steps of dt_outer_fs / n_inner (n_inner = 1 without a small model: then
 * velocity Verlet with the big model). Positions of periodic systems are
 * wrapped after every drift. energies_out: NULL or [n_outer][n_systems][3]
 * holding, after each outer step, the big model's potential energy, the
 * kinetic energy and their sum. On neighbour overflow the call restores the
 * state it started from, grows the capacity and runs again. If the call
 * fails, the contents of energies_out are unspecified. */
DMTS_API int dmts_respa_step(dmts_ctx* ctx, int n_outer, double dt_outer_fs, int n_inner,
                    double* energies_out);

/* Destroy a context and free its device memory. NULL is a no-op. */
DMTS_API void dmts_destroy(dmts_ctx* ctx);

/* Message describing the calling thread's last error ("" if none).
 * DMTS_ERR_TIMEOUT: a bounded device-side wait (the tensor-core kernels'
 * completion waits) gave up. The kernel stopped early, so that call's
 * results are invalid; dmts_respa_step restores the state it started from.
 * If the work the kernel had in flight finished, the context stays usable
 * (the cached forces are invalidated); if that did not finish in time
 * either, later calls return DMTS_ERR_STATE. */
DMTS_API const char* dmts_last_error(void);

/* Neighbour pairs of one model at the current positions, in CSR form:
 * row_ptr [N+1] and col [capacity] (ascending within each row), directed
 * pairs (i, j) with j != i, same system, |r_ij|^2 < rc^2 evaluated in FP64
 * (r_ij = x_j - x_i - L rint((x_j - x_i)/L) when periodic, each operation
 * rounded, no fused multiply-add). *n_pairs receives the number of pairs;
 * DMTS_ERR_CAPACITY if it exceeds capacity (row_ptr is still written). */
DMTS_API int dmts_neighbors(dmts_ctx* ctx, int which, int* row_ptr, int* col,
                   long long capacity, long long* n_pairs);

/* Replace one model's parameters (same architecture, n_params doubles in the
 * flat order above). Invalidates the cached forces. */
DMTS_API int dmts_set_params(dmts_ctx* ctx, int which, const double* params, size_t n_params);

/* The cudaStream_t (as void*) on which the context launches its work. */
DMTS_API void* dmts_stream(dmts_ctx* ctx);

/* Number of the library's kernel launches since the context was created
 * (including launches inside CUDA graph replays). */
DMTS_API long long dmts_launch_count(dmts_ctx* ctx);

/* Force-difference monitor of dmts_respa_step (with a small model), since
 * the context was created or dmts_monitor_reset: the largest per-atom
 * |F_big - F_small| (eV/A) seen at the end of an outer step, the number of
 * outer steps redone by the fallback, the atom count above the threshold
 * summed over steps, and a histogram of log10 |dF| in bins of 1/8 decade
 * from 1e-3 eV/A (bin b: [10^(b/8 - 3), 10^((b+1)/8 - 3)); the first and the
 * last bins are open). hist receives min(n_bins, bin count) entries; any
 * output may be NULL. Returns the number of bins (48) or a negative status.
 * Synchronises the context's stream. */
DMTS_API int dmts_monitor(dmts_ctx* ctx, double* max_df, long long* n_fallback, long long* n_flagged,
                          long long* hist, int n_bins);
DMTS_API int dmts_monitor_reset(dmts_ctx* ctx);

/* Hydrogen mass repartitioning (the paper's HMR; the target mass is the
 * caller's choice, commonly 3.024 amu). Every atom lighter than 1.5 amu that
 * is bonded to an atom of at least 1.5 amu gets mass h_mass, and the
 * difference is taken from that bonded heavy atom (the first such partner in
 * bond order), so every molecule keeps its total mass. mass [n_atoms] in,
 * mass_out [n_atoms] out (may alias mass), bonds [n_bonds][2] atom indices.
 * Host-only; needs no context or GPU. DMTS_ERR_ARG if a bond index is out of
 * range or a mass would become <= 0 (mass_out is then not written). */
DMTS_API int dmts_hmr_masses(int n_atoms, const double* mass, int n_bonds, const int* bonds, double h_mass,
                             double* mass_out);

/* Verlet-skin statistics since the context was created: displacement checks
 * run (one per evaluation at new positions) and candidate-row rebuilds among
 * them. Both 0 when the skin is 0. Synchronises the context's stream. */
DMTS_API int dmts_neighbor_stats(dmts_ctx* ctx, long long* n_checks, long long* n_rebuilds);

/* Work granularity of one model's force kernels, forward and backward:
 * atoms per thread block (FP32), or persistent thread blocks per SM (BF16,
 * 0 = as many as fit; the tensor-core kernels cut the pair list into
 * 128-pair tiles, and the backward kernel keeps one or two tiles in flight
 * per CTA: dmts_get_bwd_tiles). The tuner (option "autotune", default 1)
 * times the candidates at the context's first force evaluation and keeps the
 * fastest for each pass. Results do not depend on the choice. Returns 1 if tuned, 0
 * if not yet, or a negative status. */
DMTS_API int dmts_get_tuning(dmts_ctx* ctx, int which, int* atoms_fwd, int* atoms_bwd);

/* Set one model's work granularity (as reported by dmts_get_tuning), clamped
 * to what the kernels support, and keep it: the tuner then leaves the context
 * alone. fwd, bwd >= 1; bwd_tiles: 128-pair tiles the tensor-core backward
 * kernel keeps in flight per CTA, 1 or 2 (two groups of 4 warps sharing one
 * copy of the weights), 0 to keep the current choice; ignored in FP32 mode.
 * Results do not depend on any of the choices. */
DMTS_API int dmts_set_tuning(dmts_ctx* ctx, int which, int fwd, int bwd, int bwd_tiles);

/* The tensor-core backward kernel's tiles in flight per CTA (1 or 2; the
 * tuner picks it with the CTAs per SM; 1 in FP32 mode), or a negative status. */
DMTS_API int dmts_get_bwd_tiles(dmts_ctx* ctx, int which);

/* Time one model's force evaluation at the current positions, stage by stage,
 * with CUDA events on the context's stream, averaged over reps (>= 1)
 * evaluations; each timed stage is bracketed by its own pair of events, whose
 * own cost (about 2 us on GB300) it includes, and stages without work read 0.
 * ms_out[n_out] receives milliseconds per evaluation for:
 *   [0] quantisation, cell list and neighbour list,
 *   [1] species embedding (no work: h^0 and u^0 depend only on species and
 *       parameters and are built once per parameter upload),
 *   [2 + l] forward edge pass of layer l (l < n_layers),
 *   [2 + n_layers + l] per-atom MLPs after it,
 *   [2 + 2 n_layers + l] backward edge pass of layer l,
 *   [2 + 3 n_layers + l] per-atom adjoint MLPs after it (0 for l = 0),
 *   [2 + 4 n_layers] energy reduction.
 * Returns the number of entries written (3 + 4 n_layers, at most n_out) or
 * a negative dmts_status. */
DMTS_API int dmts_time_stages(dmts_ctx* ctx, int which, int reps, double* ms_out, int n_out);

/* Force-matching distillation loss of the small model and its parameter
 * gradient (section "Training procedures": the distilled model is trained on
 * data labelled by the reference model):
 *   L(theta) = 1/(3 N M) sum_{m<M} sum_i |F_i(theta; x_m) - F_ref,m,i|^2,
 * with F = -dE/dx, so dL/dtheta involves second derivatives of the energy;
 * it is computed by hand-written adjoint kernels. Each frame's force and
 * energy come from the model in its precision setting (BF16 tensor-core
 * MLPs in DMTS_BF16_MLP mode: the gradient then carries that rounding); the
 * second-order adjoint passes are FP32. frames: [M][N*3] positions, f_ref: [M][N*3] reference
 * forces (host or device). loss_out: scalar; grad_out: n_params doubles in
 * the flat parameter order (gradients of d2 and e0 are exactly 0). Supported
 * for a single-layer small model with n_feat 32 and n_radial 8 or 16. The
 * context's positions and velocities are restored afterwards; the cached
 * forces are invalidated. */
DMTS_API int dmts_force_matching_grad(dmts_ctx* ctx, int n_frames, const double* frames,
                                      const double* f_ref, double* loss_out, double* grad_out);

/* Energy and force distillation loss of the small model and its parameter
 * gradient (section "Training procedures": the distilled model is trained on
 * the energies and forces the reference model gives for frames of a short
 * reference MD run):
 *   L(theta) = 1/M sum_{m<M} [ lambda_e ((E(theta; x_m) - E_ref,m) / N)^2
 *                              + 1/(3 N) sum_i |F_i(theta; x_m) - F_ref,m,i|^2 ],
 * E the frame's energy summed over the context's systems. The paper leaves
 * the weights to its Supporting Information; lambda_e >= 0 is the caller's
 * ((eV/atom)^-2 against (eV/A)^-2 for the force term; 0 gives
 * dmts_force_matching_grad). Arguments as dmts_force_matching_grad, plus
 * e_ref [M] reference energies (host or device); same support, FP32
 * adjoints, restored state and invalidated forces. The frames are enqueued
 * without host synchronisation between them; a neighbour overflow in any
 * frame grows the capacities and redoes the batch. */
DMTS_API int dmts_distill_grad(dmts_ctx* ctx, int n_frames, const double* frames, const double* f_ref,
                               const double* e_ref, double lambda_e, double* loss_out, double* grad_out);

/* One Adam step (Kingma and Ba, ICLR 2015) on one model's parameters:
 * with g = grad (n_params doubles, host or device), the caller's moment
 * estimates m1, m2 (n_params doubles each, host memory, zero before step 1)
 * become beta1 m1 + (1 - beta1) g and beta2 m2 + (1 - beta2) g^2, and the
 * parameters theta - lr (m1 / (1 - beta1^t)) / (sqrt(m2 / (1 - beta2^t)) + eps)
 * are uploaded as by dmts_set_params (t >= 1 is the step number). The update
 * of these few thousand numbers runs on the host inside the library. */
DMTS_API int dmts_adam_step(dmts_ctx* ctx, int which, const double* grad, double* m1, double* m2, long long t,
                            double lr, double beta1, double beta2, double eps);

/* The parameters of one model as last set (n_params doubles in the flat
 * order; host or device). */
DMTS_API int dmts_get_params(dmts_ctx* ctx, int which, double* params_out, size_t n_params);

/* ------------------------------------------------------------------------
 * Diagnostics (the paper has no counterpart).
 *
 * dmts_wait_selftest: one thread block on the context's stream allocates
 * tensor memory, waits on an mbarrier through the same bounded wait as the
 * tensor-core force kernels (at most max_polls polls, 1 <= max_polls <=
 * 2^22), frees the tensor memory and reports through the same device flag.
 * arrive = 1: a thread arrives first and the wait completes (DMTS_OK);
 * arrive = 0: nothing arrives, the wait gives up and the call returns
 * DMTS_ERR_TIMEOUT. No MMA is issued, so nothing is left in flight and the
 * context stays usable. It touches no state or cached force.
 *
 * dmts_philox4x32_10: the thermostat's noise generator (Philox-4x32 with 10
 * rounds; Salmon, Moraes, Dror and Shaw, SC 2011) run on the current device
 * for n counters ctr[n][4] under key[2] (host arrays of 32-bit words);
 * out[n][4] receives the raw output words, for comparison with the
 * generator's published known-answer vectors. Needs no context; allocates
 * and frees two small device buffers. */
DMTS_API int dmts_wait_selftest(dmts_ctx* ctx, int arrive, int max_polls);
DMTS_API int dmts_philox4x32_10(int n, const unsigned int* ctr, const unsigned int* key, unsigned int* out);

/* ------------------------------------------------------------------------
 * Allocation-free neighbour list. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- an MD engine
 * that owns all device memory through its own pool and hands plug-ins
 * pre-allocated buffers, or code running under a fixed memory budget, where
 * a cudaMalloc would synchronise the device or fail.
 *
 * Computes the same pair set and row order as dmts_neighbors for one system
 * without a context: directed pairs (i, j), j != i, |r_ij|^2 < cutoff^2 in
 * FP64 (minimum image when box > 0, which must be >= 2 cutoff; box <= 0 for a
 * non-periodic system), rows ascending by j.
 *   x        device pointer, n_atoms*3 doubles (atom-major), positions
 *   row_ptr  device pointer, n_atoms + 1 ints, output
 *   col      device pointer, capacity ints, output (may be NULL if capacity 0)
 *   n_pairs  host pointer, receives the number of pairs
 *   stream   cudaStream_t to run on (NULL: the legacy default stream); the
 *            call returns after its work on that stream has finished.
 * Its scratch (fixed-point positions, cell list, counts) is one static device
 * array of about 0.8 MB, reserved on every GPU that loads the library until
 * the process exits; no call allocates (no cudaMalloc, no cudaFree, no
 * allocating library routine). Limits: n_atoms <= DMTS_NOALLOC_MAX_ATOMS and
 * at most 256 neighbours per atom (else DMTS_ERR_ARG / DMTS_ERR_CAPACITY with
 * a message in dmts_last_error). DMTS_ERR_CAPACITY is also returned when the
 * pairs exceed capacity (row_ptr and *n_pairs are still written).
 * The call is synchronous: it waits for its stream and reads counts back to
 * the host. The first call on a device resolves the scratch array's device
 * address (cudaGetSymbolAddress) with that device current. The address is
 * kept for the life of the process, so do not reset a device
 * (cudaDeviceReset) on which this entry point has been called: the module
 * would be loaded again, possibly at another address. All calls share the
 * one array, so calls whose work overlaps on the GPU (other streams, other
 * host threads) race: issue them one at a time per device. */
#define DMTS_NOALLOC_MAX_ATOMS 16384

DMTS_API int dmts_neighbors_noalloc(const double* x, int n_atoms, double box, double cutoff,
                                    int* row_ptr, int* col, long long capacity,
                                    long long* n_pairs, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DMTS_H */
