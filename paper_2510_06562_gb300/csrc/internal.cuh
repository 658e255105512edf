// Internal declarations of the DMTS library (not part of the C ABI).
//
// Data layout in device memory (N atoms, F features, E directed pairs):
//   x, v           FP64 SoA [3][N]         integrator state
//   inv_mass       FP64 [N]
//   q              uint4 [N]               fixed-point positions {qx,qy,qz,system}
//                                          (coordinate = frame origin + q * Q/2^32)
//   row_ptr        int32 [N+1], col/recv int32 [E]   neighbour CSR (rows ascending)
//   h, u[l], z[l], gh, mbar   FP32 [N][F]  per-atom features and adjoints
//   force          FP32 SoA [3][N];  Ei FP64 [N];  vir6 FP32 [N][6]
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace dmts {

// Checked builds (compiled with -DDMTS_CHECK): the pair, row and cell indices
// the kernels gather and scatter with are tested against their array bounds
// before use. An index outside [0, n) records the source line in
// flags[kFlagCheck] (the largest line wins) and is replaced by 0, so the
// access stays inside the array; the call then fails with a message naming
// the line. Ordinary builds compile the check away. This stands in for a
// memory checker where none can be run.
#ifdef DMTS_CHECK
#define DMTS_IDX(i, n, flags) ::dmts::checked_index((i), (n), (flags), __LINE__)
#else
#define DMTS_IDX(i, n, flags) (i)
#endif

template <class I>
__device__ __forceinline__ I checked_index(I i, long long n, int* flags, int line) {
    if ((long long)i < 0 || (long long)i >= n) {
        if (flags) atomicMax(flags + 13, line);          // flags[kFlagCheck]
        return (I)0;
    }
    return i;
}

constexpr int kMaxLayers = 4;
constexpr int kThreads = 256;          // threads per CTA of the edge kernels
constexpr int kMaxMolAtoms = 1024;     // atoms per non-periodic system

// Offsets (in floats) of every parameter block inside the flat vector.
struct ModelOffsets {
    int A;
    int W_in[kMaxLayers], W1[kMaxLayers], b1[kMaxLayers], W2[kMaxLayers], b2[kMaxLayers];
    int U1[kMaxLayers], c1[kMaxLayers], U2[kMaxLayers], c2[kMaxLayers];
    int R1, d1, R2, d2, e0;
    int total;
};

ModelOffsets model_offsets(int S, int F, int K, int L);

// Per-system fixed-point frame: coordinate = origin + q * qscale.
struct Frame {
    double ox, oy, oz;   // origin (0 for periodic systems)
    double inv;          // 2^32 / Q
    float qscale;        // Q / 2^32 (exact power of two for non-periodic)
    float pad;
};

// Device flags word indices.
enum Flag {
    kFlagOverflow = 0,     // any neighbour capacity exceeded
    kFlagNonfinite = 1,    // NaN/Inf in x or v
    kFlagMaxRow0 = 2,      // max row length seen (small model)
    kFlagMaxRow1 = 3,      // (big model)
    kFlagMaxE0 = 4,        // max pair count seen (small)
    kFlagMaxE1 = 5,        // (big)
    kFlagStep = 6,         // energies ring index
    kFlagTimeout = 7,      // a bounded device-side wait gave up
    kFlagMaxVl0 = 8,       // max candidate (Verlet) row length seen (small model)
    kFlagMaxVl1 = 9,       // (big)
    kFlagMaxCell0 = 10,    // most atoms placed in one cell, when a cell overflowed (small model)
    kFlagMaxCell1 = 11,    // (big)
    kFlagMoved = 12,       // dmts_set_state: a position differs from the current one
    kFlagCheck = 13,       // checked builds: source line of an index outside its array
    kFlagCount = 14
};
static_assert(kFlagCheck == 13, "checked_index records into flags[13]");

// Verlet-skin bookkeeping (device memory, one per context). The candidate
// rows of both models were built at the positions x_ref; k_vl_check reduces
// max |x - x_ref|^2 into max_d2, and the last CTA to finish sets rebuild
// (read by the rebuild kernels as their gate) and clears max_d2 and done.
struct VerletState {
    unsigned long long max_d2;   // FP64 bits of the largest squared displacement
    unsigned int done;           // CTAs of the current check that have finished
    int rebuild;                 // gate of the rebuild kernels
    int force;                   // set by the host: rebuild at the next check
    int pad;
    long long n_checks, n_rebuilds;
};

// Algorithm 1's thermostat step as the exact Ornstein-Uhlenbeck update
// v <- c1 v + c2 sqrt(k_B T / m) xi (on = 0: the identity, NVE). The
// normals xi come from Philox-4x32-10 with counter (atom, t low, t high, 0)
// and key (seed low, seed high); t = *step + offset (offset k for inner step
// k of a captured outer step), and the step's closing kernel advances *step.
struct Langevin {
    int on;
    double c1, c2;
    double kT_accel;              // k_B T in eV times the eV/(A amu) -> A/fs^2 factor
    uint32_t key0, key1;
    unsigned long long* step;
    long long offset;
};

// Force-difference monitor (device memory, one per context), filled by the
// closing kernel of every outer step: per-atom |F_big - F_small| against the
// threshold, histogram of log10 |dF| in kMonitorBins bins of 1/8 decade from
// 1e-3 eV/A (first and last bins open), and the fallback decision of the step.
constexpr int kMonitorBins = 48;
struct ForceMonitor {
    unsigned long long max_bits;          // FP64 bits of the largest |dF| since the last reset
    unsigned long long step_max_bits;     // ... of the current outer step (cleared by the decision)
    unsigned long long n_flagged;         // atoms above the threshold, summed over steps
    unsigned long long n_fallback;        // outer steps redone with the single-time-step integrator
    unsigned long long hist[kMonitorBins];
    unsigned int done;                    // CTAs of the current step that have finished
    int pad;
};

struct MonitorArgs {
    ForceMonitor* mon;                    // nullptr: no monitoring
    double threshold;                     // eV/A; <= 0: no fallback decision
    cudaGraphConditionalHandle cond;      // set to 1 when the step falls back
    int use_cond;
};

// The small model's forces as the integrator kernels of a captured step
// read them: rows split across 128-pair tiles are summed from the tiles'
// carry slots (the order and sums of the separate fix-up pass, which the
// step then skips), rows without pairs read zero, other rows the force
// array. k_respa_post also writes the summed rows back, so the array is
// complete after the step. row_ptr == nullptr: the array is complete.
struct ForceFold {
    const int* row_ptr;
    long long e_cap;
    const float* carry;   // [tiles][2][carry_w]: slot 2t "first", 2t + 1 "last"
    int carry_w;
    int F;                // the force scalars follow the F vector values of a slot
};

// One system and no fallback: the closing kernel of a captured step also
// sums the kinetic energy and the large model's per-atom energies (each
// block's partial sums, then the last block adds the partials in block
// order) and writes the step's energy record, in place of two sum kernels
// and the record kernel. on == 0: those kernels run.
struct EnergyFuse {
    int on;
    const double* ei;        // the large model's per-atom energies E_i
    double* epot;            // [1] their sum
    double* ekin;            // [1] the kinetic energy
    double* part;            // [2 * blocks] block partials (kinetic, potential)
    unsigned int* ticket;    // zero between steps (the last block resets it)
    double* ring;            // energy record [ring_len][3] at flags[kFlagStep]
    int ring_len;
};

// A displacement check run inside a kernel that has just written x (the
// integrator) or by k_vl_check. st == nullptr: no check.
struct VerletCheck {
    const double* xref;
    VerletState* st;
    double thr2;
};

// Everything the neighbour builder needs for one model.
struct NbrArgs {
    int n_atoms;
    int n_sys;
    const uint4* q;
    const double* x;         // SoA [3][N] FP64 (exact band test)
    const int* atom_offset;  // [n_sys + 1]
    const double* box;       // [n_sys]
    const Frame* frame;      // [n_sys]
    double rc;               // cutoff
    float rc2_lo, rc2_hi;    // FP32 band around rc^2
    int nc;                  // cells per dimension (0: all pairs within system)
    const int* cell_start;   // [nc^3 + 1]
    const int* cell_atoms;   // [N] atoms in cell order
    const uint4* cell_q;     // [N] their fixed-point positions {qx, qy, qz, atom index}, in cell order
    const int* atom_pos;     // [N] each atom's place in cell order
    int row_cap;
    long long e_cap;
    int* nbr_tmp;            // [N][row_cap]
    int* nbr_cnt;            // [N]
    int* row_ptr;            // [N + 1]
    int* col;                // [e_cap]
    int* recv;               // [e_cap]
    int* flags;
    int which;
    // Verlet-skin mode
    const int* gate;         // non-null: the kernel runs only if *gate != 0
    int exact;               // 1: exact FP64 decision in the band; 0: keep every candidate with d^2 <= rc2_hi
    int flag_row;            // flags index receiving the longest row that exceeded row_cap
    double* xref;            // non-null: the builder records x here (positions of the rebuild)
    const int* src_rows;     // row filter input: candidate rows [N][src_cap], sorted by j
    const int* src_cnt;      // [N]
    int src_cap;
    // fresh lists (skin 0): cells of fixed capacity ccap > 0, slots
    // [n_cells][ccap] of cell_atoms / cell_q filled by atomic counters
    // cell_count (zero between builds: the compaction clears them)
    int ccap;
    int n_cells;
    int* cell_count;
    int placed;              // the atoms are already in the cells (placed by the integrator kernel)
    // fresh lists: the row scan folded into the compaction. The build adds each
    // block's pair count to block_sum [ceil(N / 8)] and chunk_sum
    // [ceil(N / 256)] (zero between builds: the compaction's last block clears
    // chunk_sum and its ticket)
    int* block_sum;
    int* chunk_sum;
    unsigned int* ticket;
};

// Fixed-capacity cells of one model, for the integrator kernel that moves the
// atoms to fill while it writes their fixed-point positions (nc = 0: none).
struct CellPlace {
    int nc, ccap;
    int* count;
    int* atoms;
    uint4* q;
    int* pos;
    int flag_cell;
};

// Arguments of the potential's kernels (one model, one layer).
struct PotArgs {
    int* check;              // checked builds: flags array receiving index violations
    const float* P;          // FP32 parameters, flat order
    ModelOffsets off;
    int layer;
    int n_layers;
    int n_atoms;
    int atoms_per_cta;
    const uint4* q;
    const Frame* frame;
    const int* species;
    const int* row_ptr;
    const int* col;
    const int* recv;
    long long e_cap;
    float rc;
    float pi_over_rc;
    float bessel_pref;       // sqrt(2 / rc)
    float rep_a;             // pair repulsion rep_a exp(-d / rho) fc(d; rep_rc); 0: off
    float rep_inv_rho;
    float rep_rc;
    float rep_pi_over_rc;
    float* erep;             // [N] per-atom repulsion energy (forward layer 0 writes)
    float* msg_out;          // [N][F] per-atom sums: messages m^l (forward) or ubar^l (backward)
    const unsigned char* wt; // BF16 operand tiles of the filter weights, per layer
    size_t wt_layer_bytes;
    const float* PT;         // FP32 transposed copies: W_in^T, U1^T, U2^T per layer, then R1^T
    // features
    const float* h_in;       // h entering the per-atom MLP of this layer (h^0 table for layer 0)
    float* h;
    const float* u;          // u^l (gathered)
    float* u_next;           // u^{l+1}
    float* z;                // z^l
    const float* z_prev;     // z^{l-1} (backward tail)
    float* gh;               // dE/dh
    const float* mbar;       // mbar^l (gathered)
    float* mbar_out;         // mbar^l (forward tail) or mbar^{l-1} (backward tail)
    // tensor-core backward: BF16 copies of u^l and mbar^l, interleaved per 16
    // features ([N][F/16][16 u | 16 mbar], F * 4 bytes per atom), gathered per pair
    const unsigned char* um; // layer l's rows (backward edge pass)
    unsigned char* um_u_out; // u half, written beside u_next (or u^0 by the embedding); may be null
    unsigned char* um_mbar_out;  // mbar half, written beside mbar_out; may be null
    const unsigned char* at; // tensor-core per-atom MLPs: BF16 hi/lo weight tiles (atom_tc.cu)
    double* Ei;              // [N]
    float* force;            // SoA [3][N]
    float* vir6;             // [N][6]
    int accumulate;          // backward: add to force/vir6 instead of overwrite
    int virial;              // backward: also the per-atom virial vir6 (tensor-core path; FP32 always)
    // tensor-core path: 128-pair tiles
    float* carry;            // [tiles][2][carry_w] partial sums of rows split across tiles
    int carry_w;             // F + 16
    int ctas_per_sm;         // persistent CTAs per SM (0: as many as fit)
    int bwd_tiles;           // tensor-core backward: 128-pair tiles in flight per CTA (1 or 2; 0: 2 at F = 64, else 1)
    int fused_fixup;         // tensor-core forward: the per-atom kernel after it sums the split rows itself
    int fold_fixup;          // tensor-core backward at layer 0: the integrator sums the split force rows
    int energy;              // 0: no per-atom energy is read (the forward pass skips the repulsion energy)
    int lean;                // 1: only the force is read afterwards (the per-atom kernel of a one-layer
                             // model stores neither z, h, dE/dh nor E_i)
};

// ---------------------------------------------------------------- launchers
// neighbours.cu
void launch_frames(int n_sys, const int* atom_offset, const double* x, int n_atoms,
                   const double* box, double rc_max, Frame* frame, cudaStream_t s);
void launch_quantize(int n_atoms, const double* x, const int* sys_of_atom, const Frame* frame,
                     uint4* q, cudaStream_t s);
void launch_neighbors(const NbrArgs& a, cudaStream_t s);
// Fresh pair list with fixed-capacity cells (a.ccap > 0; a.cell_count zero on
// entry, and again on exit): placement, row build, row scan, compaction.
// Verlet-skin lists: displacement check (sets st->rebuild), gated cell list,
// gated candidate build (a.nbr_tmp / a.nbr_cnt / a.row_cap = candidate rows),
// gated candidate-from-candidate filter, and the per-evaluation exact filter
// of candidate rows into the CSR.
void launch_vl_check(int n_atoms, const double* x, const int* sys_of_atom, const double* box,
                     const VerletCheck& vc, cudaStream_t s);
void launch_cells_gated(int n_atoms, const uint4* q, int nc, int* cell_count, int* cell_start,
                        int* cell_atoms, int* atom_cell, int* atom_slot, uint4* cell_q, int* atom_pos,
                        const int* gate, cudaStream_t s);
void launch_vl_build(const NbrArgs& a, cudaStream_t s);
void launch_row_filter(const NbrArgs& a, cudaStream_t s);
void launch_vl_filter(const NbrArgs& a, cudaStream_t s);

// potential_f32.cu
void launch_embed(const PotArgs& a, int F, cudaStream_t s);
void launch_edge_fwd_f32(const PotArgs& a, int F, int K, cudaStream_t s);
void launch_edge_bwd_f32(const PotArgs& a, int F, int K, cudaStream_t s);
int max_atoms_per_cta_f32(int F, int K, bool bwd);

// potential_bf16.cu (tensor cores; status receives 1 if a bounded wait gave up)
void launch_edge_fwd_bf16(const PotArgs& a, int F, int K, int* status, cudaStream_t s);
void launch_edge_bwd_bf16(const PotArgs& a, int F, int K, int* status, cudaStream_t s);
// Self-test of the bounded completion waits (no MMA): status bit 0 is set if
// the wait of at most `polls` polls gives up; with arrive = 0 nothing arrives.
void launch_wait_selftest(int arrive, unsigned int polls, int* status, cudaStream_t s);
size_t bf16_weight_tile_bytes(int F);
// CTAs per SM that fit for the forward (bwd = false) or backward kernel;
// tiles: the backward kernel's tiles in flight per CTA (1 or 2).
int bf16_max_ctas_per_sm(int F, bool bwd, int tiles = 0);
int bf16_default_bwd_tiles(int F);

// distill.cu: distillation (energy and force matching) gradient of a single-layer model
bool fm_supported(int F, int K, int L);
int fm_edge_ctas(int n_atoms);    // CTAs (= partial rows) of the gradient edge pass on the current device
int fm_atom_ctas(int n_atoms);    // blocks (= partial rows) of the per-atom adjoint pass
int fm_atom_rows(int n_atoms);    // rows of the per-atom passes' partial buffer
// Energy term of the distillation loss for one frame (e_ref null: none).
struct FmEnergy {
    const double* e_ref = nullptr;   // device scalar: the frame's reference energy
    const double* E = nullptr;       // device [n_sys]: the model's energies at the frame
    int n_sys = 0;
    double lambda = 0.0, inv_frames = 0.0;
    double* c_energy = nullptr;      // device scalar scratch: dL/dE of the frame
};
void launch_fm_frame(const PotArgs& p, int K, const double* f_ref, double c_loss, float* g, double* sq,
                     const float* m, float* mdot, float* mbar_psi, float* mdotbar_psi, float* ubar, float* partial_e,
                     float* partial_a, int n_params, double* grad, double* loss, const FmEnergy& en,
                     bool tensor_cores, int* status, cudaStream_t s);
// (tensor_cores: the filter-weight gradient sums over pairs on tcgen05 with
// BF16 operands; a bounded wait that gives up sets bit 0 of *status, bit 1
// as well if the tensor-core work in flight did not drain)

// atom_mlp.cu: per-atom MLPs after the edge passes
void launch_atom_fwd(const PotArgs& p, int F, const float* msg, cudaStream_t s);
void launch_atom_bwd(const PotArgs& p, int F, const float* ubar, cudaStream_t s);
// atom_tc.cu: the same passes on the tensor cores (BF16 precision mode)
void launch_atom_fwd_tc(const PotArgs& p, int F, const float* msg, int* status, cudaStream_t s);
void launch_atom_bwd_tc(const PotArgs& p, int F, const float* ubar, int* status, cudaStream_t s);
size_t atom_tile_bytes(int F, int L);
// Per-system FP64 sums (deterministic). With scratch (part: kSumMaxSplit x
// kSumChunks doubles, ctr: kSumMaxSplit counters, zero on entry and exit) a
// few large systems are split over many CTAs; calls that may run at the same
// time need separate scratch.
constexpr int kSumChunks = 48;
constexpr int kSumMaxSplit = 8;
struct SumScratch {
    double* part;
    unsigned int* ctr;
};
void launch_system_sum(int n_sys, const int* atom_offset, const double* per_atom, double* out,
                       int stride, const SumScratch& sc, cudaStream_t s);
void launch_virial_sum(int n_sys, const int* atom_offset, const float* vir6, double* out,
                       cudaStream_t s);

// integrate.cu
// Philox-4x32-10 words of n counters under key (k0, k1), as the thermostat draws them.
void launch_philox_words(int n, const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, cudaStream_t s);
// moved (or null): set to 1 if some wrapped position differs, bit for bit,
// from the position it replaces.
void launch_set_state(int n_atoms, const double* x_aos, const double* v_aos, const int* sys_of_atom,
                      const double* box, double* x, double* v, int* moved, cudaStream_t s);
void launch_get_state(int n_atoms, const double* x, const double* v, double* x_aos, double* v_aos,
                      cudaStream_t s);
void launch_forces_out(int n_atoms, const float* f, double* f_aos, cudaStream_t s);
// one inner step of Algorithm 1 before the small force: (outer half-kick with
// F - F_small | post-kick of the previous inner step), pre-kick, two half-drifts
// with wrapping, then quantisation of the new positions.
void launch_respa_pre(int n_atoms, int first, double c_outer, double c_inner, double half_h,
                      double* x, double* v, const double* inv_mass, const float* f_small,
                      const float* f_big, const int* sys_of_atom, const double* box,
                      const Frame* frame, uint4* q, int* flags, const VerletCheck& vc,
                      const Langevin& lg, const CellPlace& cp0, const CellPlace& cp1,
                      const ForceFold& fold, cudaStream_t s);
// after the big force: last inner post-kick and the outer half-kick.
// With a step counter: advances it by `advance` (the inner steps taken).
// With a monitor: the force-difference statistics and fallback decision.
// With fold.row_ptr: F_small's split rows are summed here and written back.
void launch_respa_post(int n_atoms, double c_outer, double c_inner, double* v,
                       const double* inv_mass, float* f_small, const float* f_big,
                       const double* x, double* ke, const double* mass, int* flags,
                       unsigned long long* step, int advance, const MonitorArgs& mon,
                       const ForceFold& fold, const EnergyFuse& ef, cudaStream_t s);
// Blocks of the closing kernels for n atoms (sizes EnergyFuse::part).
int integrator_blocks(int n_atoms);
// dst = src for the integrator state: x, v (FP64 [3][N]) and one force (FP32 [3][N]).
void launch_copy_state(int n_atoms, const double* x, const double* v, const float* f, double* x_out,
                       double* v_out, float* f_out, cudaStream_t s);
// velocity Verlet: half-kick + drift (with Langevin: half-drift, O-step,
// half-drift, i.e. BAOAB) + wrap + quantise; half-kick + kinetic energy.
void launch_vv_pre(int n_atoms, double c_half, double dt, double* x, double* v,
                   const double* inv_mass, const float* f, const int* sys_of_atom,
                   const double* box, const Frame* frame, uint4* q, int* flags, const VerletCheck& vc,
                   const Langevin& lg, cudaStream_t s);
void launch_vv_post(int n_atoms, double c_half, double* v, const double* inv_mass,
                    const float* f, const double* x, double* ke, const double* mass, int* flags,
                    unsigned long long* step, const EnergyFuse& ef, cudaStream_t s);
// energies ring: ring[step][sys] = {Epot, Ekin, Epot + Ekin}; step = flags[kFlagStep]++.
void launch_energy_record(int n_sys, const double* epot, const double* ekin, double* ring,
                          int ring_len, int* flags, cudaStream_t s);

// Sets the calling thread's message returned by dmts_last_error().
void set_error_message(const char* msg);

// Launch accounting (kernel launches issued, graph replays included).
extern thread_local long long* g_launch_counter;
inline void count_launch(long long n = 1) {
    if (g_launch_counter) *g_launch_counter += n;
}

// Raises kernel `kern`'s dynamic shared-memory limit to `bytes` on the calling
// thread's current device, once per kernel and device: the attribute belongs
// to the device, and the contexts of one process may use different devices.
// Thread-safe.
void smem_opt_in(const void* kern, int bytes);

}  // namespace dmts

// ------------------------------------------------------------ device helpers
#ifdef __CUDACC__
namespace dmts {

// Pair repulsion phi(d) = a exp(-d/rho) fc(d; r) and its derivative (0 beyond r).
__device__ __forceinline__ float rep_phi(float d, float a, float inv_rho, float r, float pi_over_r, float* dphi) {
    if (a == 0.f || d >= r) {
        if (dphi) *dphi = 0.f;
        return 0.f;
    }
    float s, c;
    sincospif(d * (pi_over_r * 0.31830988618379067f), &s, &c);
    float ex = a * expf(-d * inv_rho);
    float fc = 0.5f * (c + 1.0f);
    if (dphi) *dphi = ex * (-inv_rho * fc - 0.5f * pi_over_r * s);
    return ex * fc;
}

__device__ __forceinline__ float silu_f(float a, float& sig) {
    sig = 1.0f / (1.0f + __expf(-a));
    return a * sig;
}

// Squared displacement of one atom since the rebuild; periodic boxes take
// the nearest image (a move of L/2 or more trips the check either way).
// NaN counts as a large move.
__device__ __forceinline__ double vl_disp2(const double* __restrict__ x, const double* __restrict__ xref,
                                           size_t n, size_t i, double L, double thr2) {
    double d2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d = x[c * n + i] - xref[c * n + i];
        if (L > 0.0) {
            if (d > 0.5 * L) d -= L;
            else if (d < -0.5 * L) d += L;
        }
        d2 += d * d;
    }
    return (d2 <= thr2) ? d2 : fmax(d2, 2.0 * thr2 + 1.0);
}

// Reduce the block's largest squared displacement m into vc.st; the last
// block to finish sets the rebuild gate, clears the accumulator and counts.
// Every thread of every block must call it.
__device__ __forceinline__ void vl_block_decide(double m, const VerletCheck& vc) {
    __shared__ double vl_wmax[32];
    __shared__ bool vl_last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) vl_wmax[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)((blockDim.x + 31) >> 5); ++k) m = fmax(m, vl_wmax[k]);
        atomicMax(&vc.st->max_d2, (unsigned long long)__double_as_longlong(m));
        __threadfence();
        vl_last = atomicAdd(&vc.st->done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (vl_last && threadIdx.x == 0) {
        __threadfence();
        const double mx = __longlong_as_double((long long)atomicAdd(&vc.st->max_d2, 0ull));
        const int force = *(volatile int*)&vc.st->force;
        const int rb = (force || mx > vc.thr2) ? 1 : 0;
        vc.st->rebuild = rb;
        vc.st->force = 0;
        vc.st->max_d2 = 0ull;
        vc.st->done = 0u;
        vc.st->n_checks += 1;
        vc.st->n_rebuilds += rb;
    }
}

// Edge vector r_ij = x_j - x_i from fixed-point coordinates: the wrapped
// 32-bit difference is the minimum image for periodic systems.
__device__ __forceinline__ float3 edge_vec(uint4 qi, uint4 qj, float qscale) {
    float3 r;
    r.x = (float)(int)(qj.x - qi.x) * qscale;
    r.y = (float)(int)(qj.y - qi.y) * qscale;
    r.z = (float)(int)(qj.z - qi.z) * qscale;
    return r;
}

// Cell index along one axis of nc cells from a 32-bit fixed-point coordinate.
__device__ __forceinline__ int cell_coord(unsigned int qc, int nc) {
    return (int)(((unsigned long long)qc * (unsigned long long)nc) >> 32);
}

// Fixed-capacity cells (fresh lists): atom i, at fixed-point position p, takes
// the next free slot of its cell (atomic counter), with its position beside
// it; an atom beyond the capacity is not placed, and the overflow is flagged
// (the list is rebuilt with larger cells). The slot order varies from run to
// run; the builder sorts every row by j, so the list does not.
// Cell of a fixed-point position: periodic systems of one box edge, stored
// back to back, each own nc^3 cells (system p.w first).
__device__ __forceinline__ int cell_of(uint4 p, int nc) {
    return ((int)p.w * nc + cell_coord(p.z, nc)) * nc * nc + cell_coord(p.y, nc) * nc + cell_coord(p.x, nc);
}

__device__ __forceinline__ void place_in_cell(const CellPlace& cp, int i, uint4 p, int* __restrict__ flags) {
    const int nc = cp.nc;
    const int c = cell_of(p, nc);
    const int slot = atomicAdd(&cp.count[c], 1);
    if (slot < cp.ccap) {
        const int pos = c * cp.ccap + slot;
        cp.atoms[pos] = i;
        cp.q[pos] = make_uint4(p.x, p.y, p.z, (unsigned int)i);   // the atom index beside its position
        cp.pos[i] = pos;
    } else {
        cp.pos[i] = -1;
        atomicMax(&flags[cp.flag_cell], slot + 1);
        atomicOr(&flags[kFlagOverflow], 1);
    }
}

}  // namespace dmts
#endif
